// Slab-ordered matched adjoint (same operator as adjoint_scatter_kernel, Sec. 2.2 A^T): the exact
// transpose of the slab-staged forward projector's traversal.
//
// One CTA owns a 32 x 32 tile of detector pixels of one view (four rays per thread). It marches
// through the volume in slabs along the tile's dominant axis m, exactly like the forward projector:
// sample k of a ray belongs to slab s through integer boundaries computed by one FP32 formula, so
// every sample is scattered once. For each slab the CTA zeroes a shared-memory box (the tile's
// frustum in the slab, one voxel of margin), scatters y_r dt times the eight trilinear weights of
// every sample into it (weights accumulated in registers while a ray stays in one cell, flushed with
// shared-memory reductions), and then adds the box to the output volume with float4 global
// reductions, skipping all-zero groups.
//
// Precision: as in the brick adjoint, sample positions are formed relative to an anchor, here the
// centre X_s of each slab's box, from FP64 per-(tile, slab) constants (one lane per slab): the point
// where the tile's corner ray meets the plane through X_s, the per-pixel steps of that point, and
// the lattice phase of the corner ray at X_s. Each ray then needs only small FP32 quantities.
//
// Lanes of a warp take the 32 pixels of one tile row, so at a given step their samples lie along one
// line across the march direction. Where the tile marches along y or z that line runs along x: the
// lanes hit consecutive words of one box row, i.e. different banks. Where it marches along x, the lanes
// sit on different rows at nearly the same x; the box rows then get an odd pitch (one word more than
// the x extent, a multiple of four), which puts 32 consecutive rows on 32 different banks.
//
// Box accumulation: shared-memory FP32 reductions are a load / compare-and-swap sequence on this
// GPU, integer reductions a single operation (about 3.6x the throughput). Where a bound allows, a
// slab's box therefore holds int32 fixed-point sums: every cell contribution c (an FP32 register
// sum) enters as round(c 2^e), and the box value is converted back with 2^-e when it is added to
// the volume. The scale 2^e is chosen per (tile, slab) so that no single contribution exceeds 2^22
// (M 2^e < 2^22, which lets one FFMA with 1.5 2^23 do the rounding, see below) and no box value can
// exceed 2^30:
//   |box value| <= M * R * (1 / delta + 1)
// with M = max |y| dt over the tile, delta the index-space distance between consecutive samples
// (>= dt / max spacing; the sampled sum of the trilinear hat along one line is at most 1 / delta + 1
// because its line integral is at most 1), and R a bound on the tile rays that can pass through one
// voxel's support (-1, 1)^3: such a ray meets the plane through the voxel's centre inside the
// rectangle of half-widths 1 + |slope| of the tile's rays, and the pixels mapping there are counted
// through the tile's pixel-to-plane Jacobian on the slab's two end planes (10 % slack for the
// projective variation across a tile). Slabs whose bound H = R (1 / delta + 1) exceeds 128 (dense
// rays) keep FP32 reductions; below it the contribution bound is the binding one, so the quantum 2^-e
// lies in (2^-22 M, 2^-21 M] and each contribution is off by at most half of it.
// A contribution c with |c| <= 2^22 is rounded to the nearest integer (ties to even) by
// t = fma(w, a, 1.5 2^23), whose bits are 0x4B400000 + round(c): one full-rate FFMA and an integer
// add instead of a product and a conversion.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "device_common.cuh"
#include "host_rays.h"

namespace pyronn {

constexpr int AS_TU = 32, AS_TV = 32, AS_NT = 256, AS_RPT = 4;

struct AsTile {                 // per tile (FP64-derived)
    float D[3], Cu[3], Cv[3];   // corner-ray direction and its per-pixel steps
    float inv_nD, nD2;
    float dref[3];
};

struct AsSlab {                 // per (tile, slab), relative to the box centre X_s
    float A[3], Eu[3], Ev[3];   // corner-ray point on the plane through X_s, per-pixel steps
    float Xs[3];                // X_s - C (world mm)
    float o[3];                 // box-local index of X_s
    float f;                    // phase of the corner ray at X_s: (X_s - C) . dref = (K + f) dt
    int K;
    int lo[3], ext[3];          // box origin and extents (voxels); ext[0] == 0: empty slab
    int px;                     // row pitch of the box (words): ext[0], or ext[0] + 1 on x-march tiles
    float scale, inv_scale;     // fixed-point scale 2^e and 2^-e; scale == 0: FP32 box
};

// per-tile state in static shared memory; the slab table (one AsSlab per slab of the tile, at most
// cfg.max_slabs) lives in dynamic shared memory after the box
struct AsShared {
    float corner[5][6];
    AsTile tile;
    int srange[2];
    unsigned ymax;              // max |y| dt over the tile (FP32 bits)
    int nfixed;                 // slabs accumulated in fixed point
};

__device__ __forceinline__ void as_floor_frac(float q, int &i, float &f) {
    const float M = 12582912.0f;
    q = fminf(fmaxf(q, -1.0e6f), 1.0e6f);
    const float t = __fadd_rd(q, M);
    i = __float_as_int(t) - 0x4B400000;
    f = q - (t - M);
}

// no "memory" clobber: the box is read only after a barrier (a compiler fence), and a clobber would
// make the compiler reload every shared value after each reduction
__device__ __forceinline__ void as_red_shared(unsigned addr, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v));
}

__device__ __forceinline__ void as_red_shared_s32(unsigned addr, int v) {
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr), "r"(v));
}

// round(w a) (ties to even) for |w a| <= 2^22: the bits of w a + 1.5 2^23, formed by one FFMA with a
// single rounding, are 0x4B400000 + round(w a)
__device__ __forceinline__ int as_fix(float w, float a) {
    return (int)(__float_as_uint(fmaf(w, a, 12582912.0f)) - 0x4B400000u);
}

// Floor and fraction without the range clamp, for positions inside a slab box (|q| far below 2^22);
// a position outside that range gives an index outside the box, which the caller's bounds test routes
// to the checked global path.
__device__ __forceinline__ void as_floor_frac_unclamped(float q, int &i, float &f) {
    const float M = 12582912.0f;
    const float t = __fadd_rd(q, M);
    i = __float_as_int(t) - 0x4B400000;
    f = q - (t - M);
}

// Samples k0..k1 of a global FP32 ray (index coordinates) added straight to the volume with global
// atomics (rays nearly parallel to the slabs, and slabs whose box does not fit).
__device__ __noinline__ void as_scatter_global(const OpParams &p, float *vb, const RayIdx r, int k0, int k1, float y) {
    for (int k = k0; k <= k1; ++k) {
        const float t = fmaf((float)k, p.dt, 0.5f * p.dt);
        const float qx = fmaf(t, r.dx, r.cx), qy = fmaf(t, r.dy, r.cy), qz = fmaf(t, r.dz, r.cz);
        const float fx = floorf(qx), fy = floorf(qy), fz = floorf(qz);
        const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
        const float ax = qx - fx, ay = qy - fy, az = qz - fz;
        for (int c = 0; c < 8; ++c) {
            const int cx = ix + (c & 1), cy = iy + ((c >> 1) & 1), cz = iz + (c >> 2);
            if ((unsigned)cx < (unsigned)p.vol.nx && (unsigned)cy < (unsigned)p.vol.ny && (unsigned)cz < (unsigned)p.vol.nz) {
                const float w = ((c & 1) ? ax : 1.0f - ax) * (((c >> 1) & 1) ? ay : 1.0f - ay) * ((c >> 2) ? az : 1.0f - az);
                atomicAdd(vb + ((long long)cz * p.vol.ny + cy) * p.vol.nx + cx, y * w);
            }
        }
    }
}

// A cell whose 2 x 2 x 2 corner block (volume index of corner 0: gx, gy, gz) does not lie in the box:
// never expected (the box covers the tile's frustum); the corners inside the volume are added to
// global memory (values times unscale) and counted.
__device__ __noinline__ void as_out_of_box(const OpParams &p, float *vb, int gx, int gy, int gz, const float *vals,
                                           float unscale) {
    for (int c = 0; c < 8; ++c) {
        const int x = gx + (c & 1), y = gy + ((c >> 1) & 1), z = gz + (c >> 2);
        if ((unsigned)x < (unsigned)p.vol.nx && (unsigned)y < (unsigned)p.vol.ny && (unsigned)z < (unsigned)p.vol.nz) {
            atomicAdd(p.flags + FLAG_SLAB_OUT_OF_BOX, 1);
            atomicAdd(vb + ((long long)z * p.vol.ny + y) * p.vol.nx + x, vals[c] * unscale);
        }
    }
}

// Power-of-two scale for a box whose values are bounded by bound (> 0): bound 2^e <= 2^30.
__device__ __forceinline__ bool as_fixed_scale(float bound, float &scale, float &inv_scale) {
    if (!(bound >= 1.0e-30f) || !(bound < 3.0e38f)) return false;
    const int x = (int)((__float_as_uint(bound) >> 23) & 0xffu) - 126;   // bound = f 2^x, f in [0.5, 1)
    const int e = 30 - x;
    if (e < -120 || e > 120) return false;
    scale = __int_as_float((e + 127) << 23);
    inv_scale = __int_as_float((127 - e) << 23);
    return true;
}

// Bound on the tile rays that can pass through the support (-1, 1)^3 of one voxel of a slab whose
// box spans index planes planes[0] .. planes[1] along m (corner rays 0: (u0, v0), 1: (u1, v0),
// 2: (u0, v1), FP32 index coordinates). A ray with slopes s1, s2 (per unit of m) through the support
// meets the plane through the voxel centre inside the rectangle of half-widths 1 + |s1|, 1 + |s2|;
// the pixels whose rays meet the plane there lie in the preimage of that rectangle under the tile's
// pixel-to-plane Jacobian, whose bounding box holds at most (floor(extent) + 1) pixels per axis.
__device__ float as_ray_bound(const float (*corner)[6], int m, int a1, int a2, const float planes[2], int wu,
                              int wv) {
    const float cap = (float)(wu * wv);
    if (wu < 2 || wv < 2) return cap;
    // the count below treats the pixel-to-plane map as nearly affine over the tile; for tiles whose rays
    // spread by more than ~11 degrees from the centre ray (extreme fan angles) it falls back to all rays
    {
        const float *cc = corner[4];
        const float nc = sqrtf(cc[3] * cc[3] + cc[4] * cc[4] + cc[5] * cc[5]);
        for (int c = 0; c < 4; ++c) {
            const float *r = corner[c];
            const float dot = r[3] * cc[3] + r[4] * cc[4] + r[5] * cc[5];
            const float nr = sqrtf(r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
            if (!(dot > 0.98f * nr * nc)) return cap;
        }
    }
    float s1 = 0.0f, s2 = 0.0f;
    for (int c = 0; c < 4; ++c) {
        const float idm = 1.0f / corner[c][3 + m];
        s1 = fmaxf(s1, fabsf(corner[c][3 + a1] * idm));
        s2 = fmaxf(s2, fabsf(corner[c][3 + a2] * idm));
    }
    const float h1 = 1.0f + s1, h2 = 1.0f + s2;
    float best = 0.0f;
    for (int pl = 0; pl < 2; ++pl) {
        float q[3][2];
        for (int c = 0; c < 3; ++c) {
            const float t = (planes[pl] - corner[c][m]) / corner[c][3 + m];
            q[c][0] = fmaf(t, corner[c][3 + a1], corner[c][a1]);
            q[c][1] = fmaf(t, corner[c][3 + a2], corner[c][a2]);
        }
        const float iu = 1.0f / (float)(wu - 1), iv = 1.0f / (float)(wv - 1);
        const float ju0 = (q[1][0] - q[0][0]) * iu, ju1 = (q[1][1] - q[0][1]) * iu;
        const float jv0 = (q[2][0] - q[0][0]) * iv, jv1 = (q[2][1] - q[0][1]) * iv;
        const float det = fabsf(ju0 * jv1 - ju1 * jv0);
        if (!(det > 1.0e-12f)) return cap;
        // 2.2 = two half-widths with 10 % slack for the projective variation across the tile
        const float ext_u = 2.2f * (h1 * fabsf(jv1) + h2 * fabsf(jv0)) / det;
        const float ext_v = 2.2f * (h1 * fabsf(ju1) + h2 * fabsf(ju0)) / det;
        const float nu = fminf((float)wu, floorf(fminf(ext_u, 1.0e6f)) + 1.0f);
        const float nv = fminf((float)wv, floorf(fminf(ext_v, 1.0e6f)) + 1.0f);
        best = fmaxf(best, nu * nv);
    }
    return best;
}

// FP64 constants of slab s (box lo / ext already set): plane through the box centre.
__device__ void as_slab_setup(const OpParams &p, int view, int u0, int v0, AsSlab &S) {
    const double *x = p.views64 + (size_t)view * VIEW64_STRIDE;
    const double sp[3] = {p.sx, p.sy, p.sz};
    const double hv3[3] = {0.5 * (p.vol.nx - 1), 0.5 * (p.vol.ny - 1), 0.5 * (p.vol.nz - 1)};
    double Xb[3];
    for (int a = 0; a < 3; ++a) {
        const double ci = S.lo[a] + 0.5 * (S.ext[a] - 1);   // box centre, volume index
        Xb[a] = (ci - hv3[a]) * sp[a];
        S.o[a] = (float)(0.5 * (S.ext[a] - 1));
        S.Xs[a] = (float)Xb[a];
    }
    double A[3], Eu[3], Ev[3], D[3];
    if (p.perspective) {
        const double *Sx = x + 12, *c0 = x + 15, *c1 = x + 18, *c2 = x + 21, *nrm = x + 24;
        const double lam = ((Xb[0] - Sx[0]) * nrm[0] + (Xb[1] - Sx[1]) * nrm[1] + (Xb[2] - Sx[2]) * nrm[2]) / x[27];
        for (int i = 0; i < 3; ++i) {
            D[i] = c2[i] + u0 * c0[i] + v0 * c1[i];
            A[i] = Sx[i] + lam * D[i] - Xb[i];
            Eu[i] = lam * c0[i];
            Ev[i] = lam * c1[i];
        }
    } else {
        const double *Dc = x, *eu = x + 3, *ev = x + 6, *d = x + 9;
        const double hu = 0.5 * (p.det.nu - 1), hvv = 0.5 * (p.det.nv - 1);
        const double su = (u0 - hu) * p.du + p.ou, sv = (v0 - hvv) * p.dv + p.ov;
        double a0[3], du_[3], dv_[3];
        for (int i = 0; i < 3; ++i) {
            a0[i] = Dc[i] + su * eu[i] + sv * ev[i] - Xb[i];
            du_[i] = p.du * eu[i];
            dv_[i] = p.dv * ev[i];
            D[i] = d[i];
        }
        const double pa = a0[0] * d[0] + a0[1] * d[1] + a0[2] * d[2];
        const double pu = du_[0] * d[0] + du_[1] * d[1] + du_[2] * d[2];
        const double pv = dv_[0] * d[0] + dv_[1] * d[1] + dv_[2] * d[2];
        for (int i = 0; i < 3; ++i) {
            A[i] = a0[i] - pa * d[i];
            Eu[i] = du_[i] - pu * d[i];
            Ev[i] = dv_[i] - pv * d[i];
        }
    }
    const double nD = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    const double T = (Xb[0] * D[0] + Xb[1] * D[1] + Xb[2] * D[2]) / nD / (double)p.dt;
    for (int i = 0; i < 3; ++i) {
        S.A[i] = (float)A[i];
        S.Eu[i] = (float)Eu[i];
        S.Ev[i] = (float)Ev[i];
    }
    const double Kd = floor(T);
    S.K = (int)Kd;
    S.f = (float)(T - Kd);
}

__device__ void as_tile_setup(const OpParams &p, int view, int u0, int v0, AsTile &t) {
    const double *x = p.views64 + (size_t)view * VIEW64_STRIDE;
    double D[3], Cu[3], Cv[3];
    if (p.perspective) {
        const double *c0 = x + 15, *c1 = x + 18, *c2 = x + 21;
        for (int i = 0; i < 3; ++i) {
            D[i] = c2[i] + u0 * c0[i] + v0 * c1[i];
            Cu[i] = c0[i];
            Cv[i] = c1[i];
        }
    } else {
        for (int i = 0; i < 3; ++i) {
            D[i] = x[9 + i];
            Cu[i] = 0.0;
            Cv[i] = 0.0;
        }
    }
    const double nD2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
    const double nD = sqrt(nD2);
    for (int i = 0; i < 3; ++i) {
        t.D[i] = (float)D[i];
        t.Cu[i] = (float)Cu[i];
        t.Cv[i] = (float)Cv[i];
        t.dref[i] = (float)(D[i] / nD);
    }
    t.inv_nD = (float)(1.0 / nD);
    t.nD2 = (float)nD2;
}

// Ray (u0 + du, v0 + dv) of the tile: unit direction d and its change from the corner ray dd
// (formed without cancellation, as in the brick adjoint). as_ray_norm forms the ray's two scalars (the
// normalisation inv and the correction g: the divisions and the square root), as_ray_dir the vectors
// from them.
__device__ __forceinline__ void as_ray_norm(const AsTile &T, float fu, float fv, float &inv, float &g) {
    const float L0 = fmaf(fv, T.Cv[0], fu * T.Cu[0]);
    const float L1 = fmaf(fv, T.Cv[1], fu * T.Cu[1]);
    const float L2 = fmaf(fv, T.Cv[2], fu * T.Cu[2]);
    const float DL = fmaf(T.D[0], L0, fmaf(T.D[1], L1, T.D[2] * L2));
    const float LL = fmaf(L0, L0, fmaf(L1, L1, L2 * L2));
    const float eps = (2.0f * DL + LL) / T.nD2;
    const float sq = sqrtf(1.0f + eps);
    inv = T.inv_nD / sq;
    g = -eps / (sq * (1.0f + sq));
}

__device__ __forceinline__ void as_ray_dir(const AsTile &T, float fu, float fv, float inv, float g, float d[3],
                                           float dd[3]) {
    const float L0 = fmaf(fv, T.Cv[0], fu * T.Cu[0]);
    const float L1 = fmaf(fv, T.Cv[1], fu * T.Cu[1]);
    const float L2 = fmaf(fv, T.Cv[2], fu * T.Cu[2]);
    d[0] = (T.D[0] + L0) * inv;
    d[1] = (T.D[1] + L1) * inv;
    d[2] = (T.D[2] + L2) * inv;
    dd[0] = fmaf(T.dref[0], g, L0 * inv);
    dd[1] = fmaf(T.dref[1], g, L1 * inv);
    dd[2] = fmaf(T.dref[2], g, L2 * inv);
}

// a[j] for a runtime j < AS_RPT by a chain of selects: every access to a[] has a constant index, so the
// array stays in registers (a dynamically indexed array would live in local memory, whose loads miss
// the small L1 left beside the slab boxes and wait on L2)
template <typename V>
__device__ __forceinline__ V as_pick(const V (&a)[AS_RPT], int j) {
    V r = a[0];
#pragma unroll
    for (int i = 1; i < AS_RPT; ++i) r = j == i ? a[i] : r;
    return r;
}

// Zeroes the box (box_cap floats); as_tile expects a zero box and leaves it zero.
__device__ __forceinline__ void as_zero_box(float *box, int box_cap) {
    for (int e = 4 * threadIdx.x; e + 3 < box_cap; e += 4 * AS_NT)
        *reinterpret_cast<float4 *>(box + e) = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = (box_cap & ~3) + threadIdx.x; e < box_cap; e += AS_NT) box[e] = 0.0f;
}

// Detector tile (tile_x, tile_y) of one view of batch item b: adds y_scale A^T (sino - sino_b) (sino_b
// may be null) into the FP32 volume vol.
// CELL: the accumulation of fixed-point slabs fixed at compile time (AdjSlabCfg::cell_fixed: 0 one
// reduction per sample and corner, 1 cell sums), so that the default kernel's cell loop serves FP32
// boxes only; -1 reads it from cfg (persistent launches, whose volumes may differ).
template <typename T, int CELL>
__device__ __forceinline__ void as_tile(const OpParams &p, const AdjSlabCfg &cfg, const T *__restrict__ sino,
                                        const T *__restrict__ sino_b, float y_scale, float *__restrict__ vol,
                                        int view, int b, int tile_x, int tile_y, float *box, AsSlab *slabs,
                                        AsShared &sh) {
    const int depth = cfg.depth, guard = cfg.guard, box_cap = cfg.box_cap;
    const int allow_fixed = cfg.allow_fixed, cell_fixed = CELL >= 0 ? CELL : cfg.cell_fixed;
    const int tu0 = tile_x * AS_TU, tv0 = tile_y * AS_TV;
    const int tu1 = min(tu0 + AS_TU, p.det.nu) - 1, tv1 = min(tv0 + AS_TV, p.det.nv) - 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long s_off = (long long)b * p.sino_elems + (long long)view * p.det.nv * p.det.nu;
    const T *sb = sino + s_off;
    const T *sb2 = sino_b ? sino_b + s_off : nullptr;
    float *vb = vol + (long long)b * p.vol_elems;
    const FpRec &rec = p.fp[view];
    const float dt = p.dt;

    __syncthreads();   // every thread is done with the previous tile's shared state
    // corner and centre rays (FP32, global index coordinates) for the slab boxes
    if (tid < 5) {
        float cu, cv;
        if (tid < 4) {
            cu = (float)((tid & 1) ? tu1 : tu0);
            cv = (float)((tid & 2) ? tv1 : tv0);
        } else {
            cu = 0.5f * (float)(tu0 + tu1);
            cv = 0.5f * (float)(tv0 + tv1);
        }
        RayIdx c = ray_setup(rec, p.vol, cu, cv);
        sh.corner[tid][0] = c.cx; sh.corner[tid][1] = c.cy; sh.corner[tid][2] = c.cz;
        sh.corner[tid][3] = c.dx; sh.corner[tid][4] = c.dy; sh.corner[tid][5] = c.dz;
    }
    if (tid == 32) as_tile_setup(p, view, tu0, tv0, sh.tile);
    if (tid == 64) {
        sh.srange[0] = 1 << 30;
        sh.srange[1] = -(1 << 30);
        sh.ymax = 0u;
        sh.nfixed = 0;
    }
    __syncthreads();

    int m;
    {
        const float ax = fabsf(sh.corner[4][3]), ay = fabsf(sh.corner[4][4]), az = fabsf(sh.corner[4][5]);
        m = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    }
    const int a1 = (m == 0) ? 1 : 0, a2 = (m == 2) ? 1 : 2;
    const int dims[3] = {p.vol.nx, p.vol.ny, p.vol.nz};
    const int Nm = dims[m];
    const int D = depth, G = guard;
    const int base0 = -1;
    const int nslab_all = (Nm + 1 - base0 + D - 1) / D;

    // rays of this thread (pixel (u, v) of ray j): cfg.lanes 0: tile row warp * AS_RPT + j, lanes along u;
    // cfg.lanes 1: the warp's 32 x 4 pixel block taken so that in each pass j the lanes sit on every other
    // pixel of two rows two pixels apart (u = 2 (lane mod 16) + (j & 1), v = 2 (lane / 16) + (j >> 1)).
    // Neighbouring pixels are often less than a voxel apart in the volume, so lanes on adjacent pixels
    // share cells and their reductions hit the same word; two pixels apart they rarely do.
    const int lanes_mode = cfg.lanes;
    auto pixel = [&](int j, int &u, int &v) {
        if (lanes_mode) {
            u = tu0 + 2 * (lane & 15) + (j & 1);
            v = tv0 + warp * AS_RPT + 2 * (lane >> 4) + (j >> 1);
        } else {
            u = tu0 + lane;
            v = tv0 + warp * AS_RPT + j;
        }
    };
    // per-ray state kept across slabs (in registers, read through as_pick): value y dt (0: nothing to
    // scatter), and the global FP32 ray's march-axis coordinate, inverse step and sample range, which
    // define the slab partition; the precise direction is formed again per slab (as_ray_dir) from the
    // ray's normalisation scalars
    float yv[AS_RPT], rcm[AS_RPT], rinv[AS_RPT], rnrm[AS_RPT], rgc[AS_RPT];
    int rk0[AS_RPT], rk1[AS_RPT];
    unsigned ybits = 0u;
#pragma unroll
    for (int j = 0; j < AS_RPT; ++j) {
        int u, v;
        pixel(j, u, v);
        float yj = 0.0f;
        if (u <= tu1 && v <= tv1) {
            const long long o = (long long)v * p.det.nu + u;
            yj = ldg_f32(sb + o);
            if (sb2) yj -= ldg_f32(sb2 + o);   // fused residual of a gradient step
        }
        yv[j] = yj * (dt * y_scale);
        ybits = max(ybits, __float_as_uint(fabsf(yv[j])));
        rcm[j] = 0.0f;
        rinv[j] = 0.0f;
        rnrm[j] = 0.0f;
        rgc[j] = 0.0f;
        rk0[j] = 0;
        rk1[j] = -1;
    }
    ybits = __reduce_max_sync(0xffffffffu, ybits);
    if (lane == 0) atomicMax(&sh.ymax, ybits);
    // slab range of the tile from the rays' in-box sample ranges; rays barely advancing along m are
    // scattered straight to global memory here and take no part in the slab march
#pragma unroll
    for (int j = 0; j < AS_RPT; ++j) {
        if (yv[j] == 0.0f) continue;
        int u, v;
        pixel(j, u, v);
        const RayIdx r = ray_setup(rec, p.vol, (float)u, (float)v);
        int k0, k1;
        if (!ray_k_range(r, p.vol, dt, k0, k1)) {
            yv[j] = 0.0f;
            continue;
        }
        const float cm = m == 0 ? r.cx : (m == 1 ? r.cy : r.cz);
        const float dm = m == 0 ? r.dx : (m == 1 ? r.dy : r.dz);
        if (!(fabsf(dm) > 1e-3f * (fabsf(r.dx) + fabsf(r.dy) + fabsf(r.dz)))) {
            atomicAdd(p.flags + FLAG_SLAB_DIRECT_RAY, 1);
            as_scatter_global(p, vb, r, k0, k1, yv[j]);
            yv[j] = 0.0f;
            continue;
        }
        rcm[j] = cm;
        rinv[j] = 1.0f / (dt * dm);
        rk0[j] = k0;
        rk1[j] = k1;
        as_ray_norm(sh.tile, (float)(u - tu0), (float)(v - tv0), rnrm[j], rgc[j]);
        const float qa = fmaf(fmaf((float)k0, dt, 0.5f * dt), dm, cm);
        const float qb = fmaf(fmaf((float)k1, dt, 0.5f * dt), dm, cm);
        const float qlo = fmaxf(fminf(qa, qb), -1.0f), qhi = fminf(fmaxf(qa, qb), (float)Nm);
        int slo = ((int)floorf(qlo) - base0) / D, shi = ((int)floorf(qhi) - base0) / D;
        slo = max(min(slo, nslab_all - 1), 0);
        shi = max(min(shi, nslab_all - 1), 0);
        atomicMin(&sh.srange[0], slo);
        atomicMax(&sh.srange[1], shi);
    }
    // the box is all zero on entry; each flush zeroes what it added, so it is zero again for the next slab
    __syncthreads();
    const int s_first = sh.srange[0];
    const int nsl = sh.srange[1] >= s_first ? min(sh.srange[1] - s_first + 1, cfg.max_slabs) : 0;
    if (nsl <= 0) return;

    // slab boxes (FP32 from the corner rays, as in the forward projector) and FP64 anchors, one lane per slab
    for (int i = tid; i < nsl; i += AS_NT) {
        AsSlab &S = slabs[i];
        const int s = s_first + i;
        const int b_lo = base0 + s * D;
        const int b_hi = min(b_lo + D, Nm);
        int lo[3], hi[3];
        lo[m] = max(b_lo - G, -1 - G);
        hi[m] = min(b_hi + G, Nm + G);
        float mn1 = 3e38f, mx1 = -3e38f, mn2 = 3e38f, mx2 = -3e38f;
        const float planes[2] = {(float)(b_lo - G), (float)(b_hi + G)};
        for (int c = 0; c < 4; ++c) {
            const float *cr = sh.corner[c];
            const float idm = 1.0f / cr[3 + m];
            for (int pl = 0; pl < 2; ++pl) {
                const float t = (planes[pl] - cr[m]) * idm;
                const float q1 = fmaf(t, cr[3 + a1], cr[a1]);
                const float q2 = fmaf(t, cr[3 + a2], cr[a2]);
                mn1 = fminf(mn1, q1); mx1 = fmaxf(mx1, q1);
                mn2 = fminf(mn2, q2); mx2 = fmaxf(mx2, q2);
            }
        }
        const float gf = (float)(G + 2);
        mn1 = fmaxf(mn1, -gf); mx1 = fminf(mx1, (float)dims[a1] + gf);
        mn2 = fmaxf(mn2, -gf); mx2 = fminf(mx2, (float)dims[a2] + gf);
        lo[a1] = max((int)floorf(mn1) - 1, -1 - G);
        hi[a1] = min((int)floorf(mx1) + 2, dims[a1] + G);
        lo[a2] = max((int)floorf(mn2) - 1, -1 - G);
        hi[a2] = min((int)floorf(mx2) + 2, dims[a2] + G);
        // x origin on a 4-voxel boundary (float4 reductions into the volume)
        lo[0] = lo[0] >= 0 ? (lo[0] & ~3) : -(((-lo[0]) + 3) & ~3);
        int e0 = hi[0] - lo[0] + 1;
        e0 = (e0 + 3) & ~3;
        // x-march tiles: the lanes of a warp sit on different rows at nearly the same x, so the rows get
        // an odd pitch (where the configuration's box budget allows), which puts 32 consecutive rows on
        // 32 different banks
        // y- and z-march tiles: the lanes of a warp sit along x, so a row pitch that is a multiple of 32
        // words puts every voxel of a column (same x) on one bank whatever its row or plane; neighbouring
        // rays then collide only when they share a cell (where the padded box still fits the capacity)
        int px = m == 0 && cfg.xpad ? e0 + 1 : e0;
        if (m != 0 && cfg.ypad) {
            const int p32 = (e0 + 31) & ~31;
            if ((long long)p32 * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1) <= box_cap) px = p32;
        }
        const int e1 = hi[1] - lo[1] + 1, e2 = hi[2] - lo[2] + 1;
        const bool fits = e0 > 0 && e1 > 0 && e2 > 0 && (long long)px * e1 * e2 <= box_cap;
        for (int a = 0; a < 3; ++a) S.lo[a] = lo[a];
        S.ext[0] = fits ? e0 : 0;
        S.px = px;
        S.ext[1] = e1;
        S.ext[2] = e2;
        S.scale = 0.0f;
        S.inv_scale = 0.0f;
        if (fits) {
            as_slab_setup(p, view, tu0, tv0, S);
            if (allow_fixed) {
                const float R = as_ray_bound(sh.corner, m, a1, a2, planes, tu1 - tu0 + 1, tv1 - tv0 + 1);
                const float smax = (float)fmax(p.sx, fmax(p.sy, p.sz));
                const float H = R * (smax / dt + 1.0f);
                float sc, isc;
                // bound max(H, 2^8) M: box values below 2^30, single contributions below 2^22
                if (H <= 128.0f && as_fixed_scale(__uint_as_float(sh.ymax) * fmaxf(H, 256.0f), sc, isc)) {
                    S.scale = sc;
                    S.inv_scale = isc;
                    atomicAdd(&sh.nfixed, 1);
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        atomicAdd(p.flags + FLAG_ADJ_FIXED_SLABS, sh.nfixed);
        atomicAdd(p.flags + FLAG_ADJ_FLOAT_SLABS, nsl - sh.nfixed);
    }

    const unsigned box_base = (unsigned)__cvta_generic_to_shared(box);
    const float isx = p.vol.isx, isy = p.vol.isy, isz = p.vol.isz;
    const bool vec4 = (p.vol.nx & 3) == 0;

    for (int i = 0; i < nsl; ++i) {
        const AsSlab &S = slabs[i];
        const int s = s_first + i;
        if (S.ext[0] == 0) {
            // the tile's footprint in this slab does not fit the box: never expected (the host bound
            // covers every tile); counted, and the slab's samples go straight to global atomics
            if (tid == 0) atomicAdd(p.flags + FLAG_SLAB_OVERFLOW, 1);
        }
        const int Ex = S.ext[0], Ey = S.ext[1], Ez = S.ext[2];
        const float isc = S.inv_scale;
        const bool fx = S.scale != 0.0f;
        const float ysc = fx ? S.scale : 1.0f;
        const bool per_sample = fx && !cell_fixed;
        const int bo0 = S.lo[0], bo1 = S.lo[1], bo2 = S.lo[2];   // box origin
        const int Px = S.px;
        const unsigned sy4 = 4u * (unsigned)Px, sz4 = 4u * (unsigned)(Px * Ey);
        const int b_lo = base0 + s * D;
        const int b_hi = min(b_lo + D, Nm);
#pragma unroll 1
        for (int j = 0; j < AS_RPT; ++j) {
            const float y = as_pick(yv, j);
            if (y == 0.0f) continue;   // rays outside the detector or the volume, zero values, direct rays
            int u, v;
            pixel(j, u, v);
            // slab partition on the global FP32 ray (identical formula for the shared boundaries)
            const float cm = as_pick(rcm, j), inv_step = as_pick(rinv, j);
            int ka, kb;
            if (inv_step > 0.0f) {
                ka = (int)ceilf(fmaf((float)b_lo - cm, inv_step, -0.5f));
                kb = (int)ceilf(fmaf((float)b_hi - cm, inv_step, -0.5f)) - 1;
            } else {
                ka = (int)floorf(fmaf((float)b_hi - cm, inv_step, -0.5f)) + 1;
                kb = (int)floorf(fmaf((float)b_lo - cm, inv_step, -0.5f));
            }
            ka = max(ka, as_pick(rk0, j));
            kb = min(kb, as_pick(rk1, j));
            if (ka > kb) continue;
            if (Ex == 0) {
                as_scatter_global(p, vb, ray_setup(rec, p.vol, (float)u, (float)v), ka, kb, y);
                continue;
            }
            // precise local ray: point P on the plane through X_s, unit direction d, and the offset e
            // of (X_s + P) . d from the phase T dt of the tile's corner ray (K + f = T)
            const float fu = (float)(u - tu0), fv = (float)(v - tv0);
            float d[3], dd[3];
            as_ray_dir(sh.tile, fu, fv, as_pick(rnrm, j), as_pick(rgc, j), d, dd);
            const float P0 = fmaf(fv, S.Ev[0], fmaf(fu, S.Eu[0], S.A[0]));
            const float P1 = fmaf(fv, S.Ev[1], fmaf(fu, S.Eu[1], S.A[1]));
            const float P2 = fmaf(fv, S.Ev[2], fmaf(fu, S.Eu[2], S.A[2]));
            const float e = fmaf(S.Xs[0], dd[0], fmaf(S.Xs[1], dd[1], S.Xs[2] * dd[2])) +
                            fmaf(P0, d[0], fmaf(P1, d[1], P2 * d[2]));
            // sample k lies (k + 1/2) dt from the ray's point closest to the volume centre, which is
            // orthogonal to d, i.e. at s = (k + 1/2) dt - (X_s + P) . d = (k - K + 1/2 - f) dt - e from
            // X_s + P: sample ka has local index ka - K
            const float jf = (float)(ka - S.K);
            const float c_r = (0.5f - S.f) * dt - e;
            const float qP0 = fmaf(P0, isx, S.o[0]), qP1 = fmaf(P1, isy, S.o[1]), qP2 = fmaf(P2, isz, S.o[2]);
            const float qd0 = d[0] * isx, qd1 = d[1] * isy, qd2 = d[2] * isz;
            const float ys = y * ysc;   // fixed point: y dt 2^e; FP32 boxes: y dt
            if (per_sample) {
                // int32 boxes: every sample adds its eight corner weights, no cell bookkeeping
                const int n = kb - ka + 1;
                // Positions are monotone in the sample index along each axis (each is a chain of
                // correctly rounded FMAs of it), so when the first and the last sample's 2 x 2 x 2 blocks
                // lie in the box, every sample's does, and the segment needs no per-sample test. The
                // comparisons fail for NaN, which takes the checked loop.
                const float s_a = fmaf(jf, dt, c_r), s_b = fmaf(jf + (float)(n - 1), dt, c_r);
                const float pa0 = fmaf(s_a, qd0, qP0), pb0 = fmaf(s_b, qd0, qP0);
                const float pa1 = fmaf(s_a, qd1, qP1), pb1 = fmaf(s_b, qd1, qP1);
                const float pa2 = fmaf(s_a, qd2, qP2), pb2 = fmaf(s_b, qd2, qP2);
                const float ex0 = (float)(Ex - 1), ex1 = (float)(Ey - 1), ex2 = (float)(Ez - 1);
                if (pa0 >= 0.f && pb0 >= 0.f && pa0 < ex0 && pb0 < ex0 && pa1 >= 0.f && pb1 >= 0.f && pa1 < ex1 &&
                    pb1 < ex1 && pa2 >= 0.f && pb2 >= 0.f && pa2 < ex2 && pb2 < ex2) {
                    // floor(q) = bits(q + 1.5 2^23 rounded down) - 0x4B400000 for 0 <= q < 2^22; the
                    // constant is folded into the box base address (unsigned arithmetic mod 2^32)
                    const float Mg = 12582912.0f;
                    const unsigned abase = box_base - 0x4B400000u * (sz4 + sy4 + 4u);
                    // Packed FP32x2 forms of the scalar arithmetic (each lane rounds as the scalar instruction
                    // does, so the contributions are the same bit for bit): the (x, y) positions, floors and
                    // fractions in one pair, the weights of the two y rows, and the contributions of the y
                    // pairs of corners, rounded by the magic-number FFMA.
                    const f32x2 M2 = splat2(Mg), dt2 = splat2(dt), cr2 = splat2(c_r);
                    const f32x2 qd01 = pack2(qd0, qd1), qP01 = pack2(qP0, qP1);
                    auto fix_bits = [](float c) { return (int)(__float_as_uint(c) - 0x4B400000u); };
                    auto sample = [&](f32x2 jj2) {   // jj2 = (jj, jj)
                        const f32x2 sj2 = fma2(jj2, dt2, cr2);
                        const f32x2 q01 = fma2(sj2, qd01, qP01);
                        const float q2 = fmaf(lo2(sj2), qd2, qP2);
                        const f32x2 t01 = add2_rd(q01, M2);
                        const float t2 = __fadd_rd(q2, Mg);
                        const f32x2 a01 = sub2(q01, sub2(t01, M2));   // (ax, ay)
                        const float az = q2 - (t2 - Mg);
                        const unsigned a = abase + 4u * __float_as_uint(lo2(t01)) + sy4 * __float_as_uint(hi2(t01)) +
                                           sz4 * __float_as_uint(t2);
                        const float wz1 = ys * az, wz0 = ys - wz1;
                        const float ax = lo2(a01), ay = hi2(a01);
                        const f32x2 yy = pack2(1.f - ay, ay);
                        const f32x2 w0 = mul2(splat2(wz0), yy), w1 = mul2(splat2(wz1), yy);   // (w00, w01), (w10, w11)
                        const f32x2 ox = splat2(1.f - ax), xx = splat2(ax);
                        const f32x2 c0 = fma2(w0, ox, M2), c1 = fma2(w0, xx, M2);
                        const f32x2 c2 = fma2(w1, ox, M2), c3 = fma2(w1, xx, M2);
                        as_red_shared_s32(a, fix_bits(lo2(c0)));
                        as_red_shared_s32(a + 4u, fix_bits(lo2(c1)));
                        as_red_shared_s32(a + sy4, fix_bits(hi2(c0)));
                        as_red_shared_s32(a + sy4 + 4u, fix_bits(hi2(c1)));
                        as_red_shared_s32(a + sz4, fix_bits(lo2(c2)));
                        as_red_shared_s32(a + sz4 + 4u, fix_bits(lo2(c3)));
                        as_red_shared_s32(a + sz4 + sy4, fix_bits(hi2(c2)));
                        as_red_shared_s32(a + sz4 + sy4 + 4u, fix_bits(hi2(c3)));
                    };
                    // two independent samples per step
                    f32x2 jj2 = splat2(jf);
                    const f32x2 one2 = splat2(1.0f), two2 = splat2(2.0f);
                    int ii = 0;
                    for (; ii + 1 < n; ii += 2, jj2 = add2(jj2, two2)) {
                        sample(jj2);
                        sample(add2(jj2, one2));
                    }
                    if (ii < n) sample(jj2);
                    continue;
                }
                float jj = jf;
                for (int ii = 0; ii < n; ++ii, jj += 1.0f) {
                    const float sj = fmaf(jj, dt, c_r);
                    int ix, iy, iz;
                    float ax, ay, az;
                    as_floor_frac_unclamped(fmaf(sj, qd0, qP0), ix, ax);
                    as_floor_frac_unclamped(fmaf(sj, qd1, qP1), iy, ay);
                    as_floor_frac_unclamped(fmaf(sj, qd2, qP2), iz, az);
                    const float wz1 = ys * az, wz0 = ys - wz1;
                    const float oay = 1.f - ay, oax = 1.f - ax;
                    const float w00 = wz0 * oay, w01 = wz0 * ay, w10 = wz1 * oay, w11 = wz1 * ay;
                    if ((unsigned)ix < (unsigned)(Ex - 1) && (unsigned)iy < (unsigned)(Ey - 1) &&
                        (unsigned)iz < (unsigned)(Ez - 1)) {
                        const unsigned a = box_base + 4u * (unsigned)((iz * Ey + iy) * Px + ix);
                        as_red_shared_s32(a, __float2int_rn(w00 * oax));
                        as_red_shared_s32(a + 4u, __float2int_rn(w00 * ax));
                        as_red_shared_s32(a + sy4, __float2int_rn(w01 * oax));
                        as_red_shared_s32(a + sy4 + 4u, __float2int_rn(w01 * ax));
                        as_red_shared_s32(a + sz4, __float2int_rn(w10 * oax));
                        as_red_shared_s32(a + sz4 + 4u, __float2int_rn(w10 * ax));
                        as_red_shared_s32(a + sz4 + sy4, __float2int_rn(w11 * oax));
                        as_red_shared_s32(a + sz4 + sy4 + 4u, __float2int_rn(w11 * ax));
                    } else {
                        const float vals[8] = {w00 * oax, w00 * ax, w01 * oax, w01 * ax,
                                               w10 * oax, w10 * ax, w11 * oax, w11 * ax};
                        as_out_of_box(p, vb, ix + bo0, iy + bo1, iz + bo2, vals, isc);
                    }
                }
                continue;
            }
            // FP32 boxes (and fixed-point boxes in cell mode): a ray's weights are summed in registers while
            // it stays in one cell of the box and flushed with eight reductions when it moves on. A sample
            // whose 2 x 2 x 2 block is not in the box (where the corner rays do not bound the tile's rays:
            // extreme fan angles) flushes the pending cell and adds its corners inside the volume straight
            // to global memory.
            float a0 = 0.f, a1v = 0.f, a2v = 0.f, a3 = 0.f, a4 = 0.f, a5 = 0.f, a6 = 0.f, a7 = 0.f;
            int pcell = -1;   // box offset of the pending cell, -1: none
            float jj = jf;
            for (int k = ka; k <= kb + 1; ++k, jj += 1.0f) {
                int cell = -1, ix = 0, iy = 0, iz = 0;
                float ax = 0.f, ay = 0.f, az = 0.f;
                bool off_box = false;
                if (k <= kb) {
                    const float sj = fmaf(jj, dt, c_r);
                    as_floor_frac(fmaf(sj, qd0, qP0), ix, ax);
                    as_floor_frac(fmaf(sj, qd1, qP1), iy, ay);
                    as_floor_frac(fmaf(sj, qd2, qP2), iz, az);
                    if ((unsigned)ix < (unsigned)(Ex - 1) && (unsigned)iy < (unsigned)(Ey - 1) &&
                        (unsigned)iz < (unsigned)(Ez - 1))
                        cell = (iz * Ey + iy) * Px + ix;
                    else
                        off_box = true;
                }
                if (cell != pcell && pcell >= 0) {
                    // the cell's 2 x 2 x 2 block lies in the box: eight reductions (corners outside the volume
                    // land in the box margin and are dropped when the box is added)
                    const unsigned a = box_base + 4u * (unsigned)pcell;
                    if (CELL != 0 && fx) {   // fixed-point slabs reach this loop only in cell mode
                        as_red_shared_s32(a, __float2int_rn(a0));
                        as_red_shared_s32(a + 4u, __float2int_rn(a1v));
                        as_red_shared_s32(a + sy4, __float2int_rn(a2v));
                        as_red_shared_s32(a + sy4 + 4u, __float2int_rn(a3));
                        as_red_shared_s32(a + sz4, __float2int_rn(a4));
                        as_red_shared_s32(a + sz4 + 4u, __float2int_rn(a5));
                        as_red_shared_s32(a + sz4 + sy4, __float2int_rn(a6));
                        as_red_shared_s32(a + sz4 + sy4 + 4u, __float2int_rn(a7));
                    } else {
                        as_red_shared(a, a0);
                        as_red_shared(a + 4u, a1v);
                        as_red_shared(a + sy4, a2v);
                        as_red_shared(a + sy4 + 4u, a3);
                        as_red_shared(a + sz4, a4);
                        as_red_shared(a + sz4 + 4u, a5);
                        as_red_shared(a + sz4 + sy4, a6);
                        as_red_shared(a + sz4 + sy4 + 4u, a7);
                    }
                    a0 = a1v = a2v = a3 = a4 = a5 = a6 = a7 = 0.f;
                }
                pcell = cell;
                if (k > kb) break;
                const float wz1 = ys * az, wz0 = ys - wz1;
                const float w00 = wz0 * (1.f - ay), w01 = wz0 * ay, w10 = wz1 * (1.f - ay), w11 = wz1 * ay;
                if (off_box) {
                    const float vals[8] = {w00 * (1.f - ax), w00 * ax, w01 * (1.f - ax), w01 * ax,
                                           w10 * (1.f - ax), w10 * ax, w11 * (1.f - ax), w11 * ax};
                    as_out_of_box(p, vb, ix + bo0, iy + bo1, iz + bo2, vals, fx ? isc : 1.0f);
                    continue;
                }
                a0 = fmaf(w00, 1.f - ax, a0);
                a1v = fmaf(w00, ax, a1v);
                a2v = fmaf(w01, 1.f - ax, a2v);
                a3 = fmaf(w01, ax, a3);
                a4 = fmaf(w10, 1.f - ax, a4);
                a5 = fmaf(w10, ax, a5);
                a6 = fmaf(w11, 1.f - ax, a6);
                a7 = fmaf(w11, ax, a7);
            }
        }
        __syncthreads();
        // add the box to the volume (groups of four voxels along x, float4 reductions, all-zero groups
        // skipped) and zero it again; group indices advance by AS_NT groups per step without divisions.
        // Rows of odd pitch are read and cleared word by word.
        if (Ex > 0) {
            const bool vbox = (Px & 3) == 0;
            const int gx4 = Ex >> 2;
            const int ngroups = gx4 * Ey * Ez;
            const int srow = AS_NT / gx4;
            const int step_x = AS_NT - srow * gx4, step_y = srow % Ey, step_z = srow / Ey;
            int xg = tid % gx4;
            const int row0 = tid / gx4;
            int ly = row0 % Ey, lz = row0 / Ey;
            for (int gi = tid; gi < ngroups; gi += AS_NT) {
                float *pw = box + (4 * xg + Px * (ly + Ey * lz));
                float4 q = vbox ? *reinterpret_cast<const float4 *>(pw) : make_float4(pw[0], pw[1], pw[2], pw[3]);
                const int4 qi = *reinterpret_cast<const int4 *>(&q);
                // FP32 boxes: a group summing to -0 is left as is (adding to -0 is exact)
                const bool nz = fx ? (qi.x | qi.y | qi.z | qi.w) != 0
                                   : (q.x != 0.f || q.y != 0.f || q.z != 0.f || q.w != 0.f);
                if (nz) {
                    if (vbox) {
                        *reinterpret_cast<float4 *>(pw) = make_float4(0.f, 0.f, 0.f, 0.f);
                    } else {
                        pw[0] = 0.f; pw[1] = 0.f; pw[2] = 0.f; pw[3] = 0.f;
                    }
                    if (fx)
                        q = make_float4(__int2float_rn(qi.x) * isc, __int2float_rn(qi.y) * isc,
                                        __int2float_rn(qi.z) * isc, __int2float_rn(qi.w) * isc);
                    const int gx = bo0 + 4 * xg, gy = bo1 + ly, gz = bo2 + lz;
                    if ((unsigned)gy < (unsigned)p.vol.ny && (unsigned)gz < (unsigned)p.vol.nz) {
                        // 32-bit index: volumes hold fewer than 2^31 voxels (gx may be slightly negative)
                        float *dst = vb + ((gz * p.vol.ny + gy) * p.vol.nx + gx);
                        if (vec4 && gx >= 0 && gx + 3 < p.vol.nx) {
                            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(q.x),
                                         "f"(q.y), "f"(q.z), "f"(q.w)
                                         : "memory");
                        } else {
                            const float vv[4] = {q.x, q.y, q.z, q.w};
                            for (int c = 0; c < 4; ++c)
                                if ((unsigned)(gx + c) < (unsigned)p.vol.nx && vv[c] != 0.f) atomicAdd(dst + c, vv[c]);
                        }
                    }
                }
                xg += step_x;
                int carry = 0;
                if (xg >= gx4) {
                    xg -= gx4;
                    carry = 1;
                }
                ly += step_y + carry;
                lz += step_z;
                if (ly >= Ey) {
                    ly -= Ey;
                    lz += 1;
                }
            }
        }
        __syncthreads();   // the box is reused by the next slab
    }
}

template <typename T, int CELL>
__global__ void __launch_bounds__(AS_NT, 2) adjoint_slab_kernel(OpParams p, AdjSlabCfg cfg, const T *__restrict__ sino,
                                                                const T *__restrict__ sino_b, float y_scale,
                                                                float *__restrict__ vol) {
    extern __shared__ __align__(16) float box[];
    __shared__ AsShared sh;
    AsSlab *slabs = reinterpret_cast<AsSlab *>(box + ((cfg.box_cap + 3) & ~3));
    as_zero_box(box, cfg.box_cap);
    // grid (tile columns, views, tile rows x batch items), in the order that keeps the volume band of
    // one tile row in L2 while the resident CTAs reduce into it (see the launcher)
    const int ntv = (p.det.nv + AS_TV - 1) / AS_TV;
    as_tile<T, CELL>(p, cfg, sino, sino_b, y_scale, vol, blockIdx.y, blockIdx.z / ntv, blockIdx.x, blockIdx.z % ntv,
                     box, slabs, sh);
}

// Persistent launch over the (view, tile) items of several volumes (each with its own geometry and
// slab configuration, accumulating into its own FP32 volume): each CTA takes the next item from a
// device counter until all are done. Volumes are ordered by decreasing cost per item.
template <typename T>
__global__ void __launch_bounds__(AS_NT, 2) adjoint_slab_batched_kernel(const __grid_constant__ PlanLaunch L) {
    extern __shared__ __align__(16) float box[];
    __shared__ AsShared sh;
    __shared__ long long s_item;
    // one table position for every volume (after the largest box), so that no volume's table lands in
    // another volume's (zeroed) box
    int cap = 0;
    for (int i = 0; i < L.n; ++i) cap = max(cap, L.v[i].acfg.box_cap);
    AsSlab *slabs = reinterpret_cast<AsSlab *>(box + ((cap + 3) & ~3));
    as_zero_box(box, cap);
    const long long total = L.item_end[L.n - 1];
    for (;;) {
        __syncthreads();   // every thread has read the previous item number
        if (threadIdx.x == 0) s_item = atomicAdd(L.counter, 1);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        int i = 0;
        while (item >= L.item_end[i]) ++i;
        const PlanVolume &V = L.v[i];
        const long long local = item - (i ? L.item_end[i - 1] : 0);
        const int tiles = V.ntx * V.nty;
        const int view = (int)(local / tiles), t = (int)(local % tiles);
        as_tile<T, -1>(V.p, V.acfg, (const T *)V.in, (const T *)nullptr, 1.0f, V.acc, view, 0, t % V.ntx, t / V.ntx,
                   box, slabs, sh);
    }
}

template <typename T>
__global__ void adjoint_convert_kernel(const float *__restrict__ src, T *__restrict__ dst, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dst[i] = from_f32<T>(src[i]);
}

// ---------------------------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------------------------
namespace {

// Largest box (floats) of one 32 x 32 tile over its first and last slab (the box extent is convex in
// the slab position). Margins follow the kernel: lo = floor(min) - 1, hi = floor(max) + 2, x start
// rounded down to 4 and x extent up to 4, +1 for FP32 rounding.
long long as_tile_bound(const pyronn_geom *g, const FpRec &rec, int tu0, int tv0, int D, int G, int xpad) {
    const int tu1 = std::min(tu0 + AS_TU, g->nu) - 1, tv1 = std::min(tv0 + AS_TV, g->nv) - 1;
    RayD cr[4];
    for (int c = 0; c < 4; ++c) cr[c] = ray_setup_d(rec, g, (c & 1) ? tu1 : tu0, (c & 2) ? tv1 : tv0);
    const RayD ctr = ray_setup_d(rec, g, 0.5 * (tu0 + tu1), 0.5 * (tv0 + tv1));
    const int dims[3] = {g->nx, g->ny, g->nz};
    const double amax = std::max(std::fabs(ctr.d[0]), std::max(std::fabs(ctr.d[1]), std::fabs(ctr.d[2])));
    long long best = 0;
    for (int m = 0; m < 3; ++m) {
        if (std::fabs(ctr.d[m]) < 0.999 * amax) continue;
        const int a1 = (m == 0) ? 1 : 0, a2 = (m == 2) ? 1 : 2;
        const int Nm = dims[m];
        const int nslab = (Nm + 2 + D - 1) / D;
        for (int which = 0; which < 2; ++which) {
            const int s = which ? nslab - 1 : 0;
            const int b_lo = -1 + s * D, b_hi = std::min(b_lo + D, Nm);
            const double planes[2] = {(double)(b_lo - G), (double)(b_hi + G)};
            double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
            for (int c = 0; c < 4; ++c)
                for (int pl = 0; pl < 2; ++pl) {
                    const double t = (planes[pl] - cr[c].c[m]) / cr[c].d[m];
                    for (int a : {a1, a2}) {
                        const double q = cr[c].c[a] + t * cr[c].d[a];
                        mn[a] = std::min(mn[a], q);
                        mx[a] = std::max(mx[a], q);
                    }
                }
            long long e[3];
            bool bounded = true;
            for (int a = 0; a < 3; ++a) {
                if (a == m) e[a] = D + 2 * G + 1;
                else e[a] = box_extent(mx[a] - mn[a], 5, dims[a] + 2 * G + 2);
                bounded = bounded && e[a] >= 0;
                e[a] = std::min<long long>(e[a], dims[a] + 2 * G + 2);
            }
            if (!bounded) continue;
            e[0] = ((e[0] + 3 + 3) / 4) * 4;   // x start rounded down (<= 3 more), extent rounded up
            if (m == 0 && xpad) e[0] += 1;         // odd row pitch of x-march boxes
            best = std::max(best, e[0] * e[1] * e[2]);
        }
    }
    return best;
}

}  // namespace

static long long as_bound(const pyronn_geom *g, int depth, int guard, int xpad) {
    const int ntu = (g->nu + AS_TU - 1) / AS_TU, ntv = (g->nv + AS_TV - 1) / AS_TV;
    std::atomic<int> next(0);
    std::atomic<long long> best(0);
    auto work = [&]() {
        long long local = 0;
        for (int n = next.fetch_add(1); n < g->n_views; n = next.fetch_add(1))
            for (int j = 0; j < ntv; ++j)
                for (int i = 0; i < ntu; ++i)
                    local = std::max(local, as_tile_bound(g, g->fp_rec[n], i * AS_TU, j * AS_TV, depth, guard, xpad));
        long long cur = best.load();
        while (local > cur && !best.compare_exchange_weak(cur, local)) {
        }
    };
    const unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned i = 1; i < nt; ++i) th.emplace_back(work);
    work();
    for (auto &t : th) t.join();
    return best.load();
}

size_t adjoint_slab_smem_bytes(int box_cap, int max_slabs) {
    return sizeof(float) * (size_t)((box_cap + 3) & ~3) + sizeof(AsSlab) * (size_t)max_slabs;
}

// Deepest slab (8, 6, 5 or 4 planes; or the depth set by PYRONN_TUNE_ADJ_DEPTH) whose box and slab table
// let two CTAs share an SM (224 KB of shared memory, 1 KB reserved per CTA, the static tile state), first
// with the odd row pitch of x-march boxes, then without it; otherwise the last one tried (16-byte pitch)
// if its box fits in 160 KB (one CTA per SM).
AdjSlabCfg choose_adj_slab_cfg(const pyronn_geom *g) {
    AdjSlabCfg c{};
    if (g->ndim != 3) return c;
    const int nmax = std::max(g->nx, std::max(g->ny, g->nz));
    const double smin = std::min(g->sx, std::min(g->sy, g->sz));
    if (!(g->dt / smin < 65535.0)) return c;   // steps of 2^16 voxels or more: the brick adjoint
    c.guard = 1 + (int)std::floor(g->dt / smin);
    // two CTAs per SM: 224 KB of the SM's shared memory, 1 KB reserved per CTA, the static tile
    // state (the occupancy calculator on GB300 admits two CTAs of 114264 bytes each, not of 115152)
    const size_t soft = (224 * 1024) / 2 - 1024 - sizeof(AsShared) - 64;
    const long long hard = (160 * 1024) / 4;
    long long need = 0;
    bool fit = false;
    const int forced = g->tuning.adj_depth;
    const int depths[4] = {8, 6, 5, 4};
    const int ndepths = forced > 0 ? 1 : 4;
    for (int xpad = g->tuning.adj_pitch == 1 ? 0 : 1; xpad >= 0 && !fit; --xpad)   // 0 and 2: odd x-march pitch
        for (int di = 0; di < ndepths; ++di) {
            const int depth = forced > 0 ? forced : depths[di];
            need = as_bound(g, depth, c.guard, xpad);
            c.depth = depth;
            c.xpad = xpad;
            // slabs of a tile: planes -1 .. N, at most (N + 2 + depth - 1) / depth along any axis
            c.max_slabs = (nmax + 2 + depth - 1) / depth;
            if (need > 0 && adjoint_slab_smem_bytes((int)need, c.max_slabs) <= soft) {
                fit = true;
                break;
            }
        }
    c.box_cap = (int)std::min(need, hard);
    c.valid = need > 0 && need <= hard && adjoint_slab_smem_bytes(c.box_cap, c.max_slabs) <= 200 * 1024;
    c.allow_fixed = g->tuning.adj_accum != 1;
    c.cell_fixed = g->tuning.adj_accum == 2;
    c.lanes = g->tuning.adj_lanes == 2 ? 1 : 0;
    c.ypad = g->tuning.adj_pitch == 0;
    return c;
}

template <typename T>
__global__ void adjoint_widen_kernel(const T *__restrict__ src, float *__restrict__ dst, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dst[i] = to_f32<T>(src[i]);
}

// vol = y_scale A^T (sino - sino_b), or vol += ... when accumulate (sino_b may be null). acc: the FP32
// accumulation volume (vol itself for FP32; for BF16 / FP16 it is widened from vol first when
// accumulating and converted back at the end).
template <typename T>
static int launch_slab_t(const OpParams &p, const AdjSlabCfg &c, const void *sino, const void *sino_b, float y_scale,
                         bool accumulate, float *acc, void *vol, cudaStream_t st) {
    const long long n = p.vol_elems * p.batch;
    const int cblocks = stride_grid(n, 16);
    cudaError_t e = cudaSuccess;
    if (!accumulate) e = cudaMemsetAsync(acc, 0, sizeof(float) * (size_t)n, st);
    else if ((void *)acc != vol) adjoint_widen_kernel<T><<<cblocks, 256, 0, st>>>((const T *)vol, acc, n);
    if (e != cudaSuccess) return (int)e;
    const size_t smem = adjoint_slab_smem_bytes(c.box_cap, c.max_slabs);
    auto kern = c.cell_fixed ? adjoint_slab_kernel<T, 1> : adjoint_slab_kernel<T, 0>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    // Grid order: tile columns fastest, then views, then tile rows and batch items, so that the CTAs
    // resident at one time (the tiles of one tile row in consecutive views) reduce into one band of the
    // volume, which stays in L2 while they do; with views outermost every view's flushes would sweep the
    // whole volume, through DRAM once it exceeds L2. Views beyond the 65535 grid rows and batches beyond
    // 65535 tile rows are split into several launches.
    const int ntv = ceil_div(p.det.nv, AS_TV);
    const int per_launch = 65535 / ntv > 0 ? 65535 / ntv : 1;
    const long long view_elems = (long long)p.det.nv * p.det.nu;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        const int nb = p.batch - b0 < per_launch ? p.batch - b0 : per_launch;
        for (int v0 = 0; v0 < p.n_views; v0 += 65535) {
            const int nvw = p.n_views - v0 < 65535 ? p.n_views - v0 : 65535;
            OpParams q = p;
            q.fp = p.fp + v0;
            q.bp = p.bp ? p.bp + v0 : nullptr;
            q.views64 = p.views64 ? p.views64 + (size_t)v0 * VIEW64_STRIDE : nullptr;
            q.n_views = nvw;
            const long long so = b0 * p.sino_elems + v0 * view_elems;
            dim3 grid(ceil_div(p.det.nu, AS_TU), nvw, ntv * nb);
            kern<<<grid, AS_NT, smem, st>>>(
                q, c, (const T *)sino + so, sino_b ? (const T *)sino_b + so : (const T *)nullptr, y_scale,
                acc + b0 * p.vol_elems);
        }
    }
    if ((void *)acc != vol) adjoint_convert_kernel<T><<<cblocks, 256, 0, st>>>(acc, (T *)vol, n);
    return (int)cudaGetLastError();
}

template <typename T>
static int launch_slab_batched_t(const PlanLaunch &L, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(adjoint_slab_batched_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(adjoint_slab_batched_kernel<T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    for (int i = 0; i < L.n; ++i) {
        e = cudaMemsetAsync(L.v[i].acc, 0, sizeof(float) * (size_t)L.v[i].p.vol_elems, st);
        if (e != cudaSuccess) return (int)e;
    }
    e = cudaMemsetAsync(L.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return (int)e;
    adjoint_slab_batched_kernel<T><<<grid, AS_NT, smem, st>>>(L);
    for (int i = 0; i < L.n; ++i) {
        if ((void *)L.v[i].acc == L.v[i].out) continue;
        const long long n = L.v[i].p.vol_elems;
        const int blocks = stride_grid(n, 16);
        adjoint_convert_kernel<T><<<blocks, 256, 0, st>>>(L.v[i].acc, (T *)L.v[i].out, n);
    }
    return (int)cudaGetLastError();
}

// One persistent slab-ordered adjoint launch over a plan's volumes (each PlanVolume carries its slab
// configuration and FP32 accumulation volume, which is zeroed here; other element types are converted
// into the output afterwards). smem: the largest box of the plan, in bytes.
int launch_adjoint_slab_batched(const PlanLaunch &L, int dtype, int grid, size_t smem, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_slab_batched_t<float>(L, grid, smem, st);
        case PYRONN_BF16: return launch_slab_batched_t<__nv_bfloat16>(L, grid, smem, st);
        case PYRONN_F16: return launch_slab_batched_t<__half>(L, grid, smem, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

int adjoint_slab_batched_occupancy(size_t smem, int *blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(adjoint_slab_batched_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(adjoint_slab_batched_kernel<float>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, adjoint_slab_batched_kernel<float>, AS_NT,
                                                              smem);
}

int launch_adjoint_slab(const OpParams &p, const AdjSlabCfg &c, const void *sino, const void *sino_b, float y_scale,
                        bool accumulate, void *vol, float *acc32, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_slab_t<float>(p, c, sino, sino_b, y_scale, accumulate, (float *)vol, vol, st);
        case PYRONN_BF16:
            return launch_slab_t<__nv_bfloat16>(p, c, sino, sino_b, y_scale, accumulate, acc32, vol, st);
        case PYRONN_F16: return launch_slab_t<__half>(p, c, sino, sino_b, y_scale, accumulate, acc32, vol, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace pyronn
