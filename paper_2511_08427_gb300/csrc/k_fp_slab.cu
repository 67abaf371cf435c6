// Slab-staged ray-driven forward projector (same operator as fp_direct_kernel, Sec. 2.1).
//
// One CTA owns a TU x TV tile of detector pixels of one view (one ray per thread). The CTA
// marches through the volume along the axis m on which its central ray advances fastest, in
// slabs of D voxel planes. For every slab it stages, in shared memory, the box of voxels that
// the tile's rays can touch there (the frustum of the four corner rays, plus one voxel of
// margin and the interpolation neighbour), converted to FP32 and zero outside the volume. The
// rays then sample their part of the slab from shared memory.
//
// Sample partition. Slab s covers march-axis positions q_m in [b_s, b_{s+1}), b_s = -1 + s D.
// Ray r assigns sample k to slab s through integer boundaries K(b) computed by one FP32
// formula, so every sample of the ray is summed exactly once. A sample that FP32 places just
// across a boundary is at most one step (< 1 voxel) outside its slab; the staged box keeps G
// extra planes on both sides for it.
//
// The box size is bounded on the host (choose_fp_slab_cfg) over every tile and slab; a slab
// whose box would still not fit falls back to read-only-cache loads for that slab only.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

#include "device_common.cuh"
#include "host_rays.h"

namespace pyronn {

__device__ __forceinline__ float comp(const RayIdx &r, int a) { return a == 0 ? r.cx : (a == 1 ? r.cy : r.cz); }
__device__ __forceinline__ float dcomp(const RayIdx &r, int a) { return a == 0 ? r.dx : (a == 1 ? r.dy : r.dz); }

// First / last sample index of a ray whose march coordinate lies in [b_lo, b_hi).
__device__ __forceinline__ void slab_k_range(float cm, float inv_step, bool pos, float b_lo, float b_hi, int &ka,
                                             int &kb) {
    if (pos) {
        ka = (int)ceilf(fmaf(b_lo - cm, inv_step, -0.5f));
        kb = (int)ceilf(fmaf(b_hi - cm, inv_step, -0.5f)) - 1;
    } else {
        ka = (int)floorf(fmaf(b_hi - cm, inv_step, -0.5f)) + 1;
        kb = (int)floorf(fmaf(b_lo - cm, inv_step, -0.5f));
    }
}

template <typename T, int TU, int TV>
__global__ void __launch_bounds__(TU *TV) fp_slab_kernel(OpParams p, FpSlabCfg cfg, const T *__restrict__ vol,
                                                         T *__restrict__ sino) {
    constexpr int NT = TU * TV;
    extern __shared__ float sbox[];
    __shared__ float s_corner[5][6];

    const int view = blockIdx.z % p.n_views;
    const int b = blockIdx.z / p.n_views;
    const int tu0 = blockIdx.x * TU, tv0 = blockIdx.y * TV;
    const int tu1 = min(tu0 + TU, p.det.nu) - 1, tv1 = min(tv0 + TV, p.det.nv) - 1;
    const int tid = threadIdx.x;
    const int u = tu0 + tid % TU, v = tv0 + tid / TU;
    const bool active = (u <= tu1) && (v <= tv1);
    const T *vb = vol + (long long)b * p.vol_elems;
    const FpRec &rec = p.fp[view];

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
        s_corner[tid][0] = c.cx; s_corner[tid][1] = c.cy; s_corner[tid][2] = c.cz;
        s_corner[tid][3] = c.dx; s_corner[tid][4] = c.dy; s_corner[tid][5] = c.dz;
    }
    RayIdx r = ray_setup(rec, p.vol, (float)min(u, tu1), (float)min(v, tv1));
    int k0 = 0, k1 = -1;
    bool hit = active && ray_k_range(r, p.vol, p.dt, k0, k1);
    const int k0_all = k0, k1_all = k1;
    __syncthreads();

    // march axis: fastest-advancing index axis of the central ray
    int m;
    {
        float ax = fabsf(s_corner[4][3]), ay = fabsf(s_corner[4][4]), az = fabsf(s_corner[4][5]);
        m = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    }
    const int a1 = (m == 0) ? 1 : 0, a2 = (m == 2) ? 1 : 2;
    const int dims[3] = {p.vol.nx, p.vol.ny, p.vol.nz};
    const int Nm = dims[m];
    const float cm = comp(r, m), dm = dcomp(r, m);
    const bool pos = dm > 0.0f;
    // a ray that barely advances along m (never for tiles of ordinary size) is summed directly
    const bool marchable = fabsf(dm) > 1e-3f * (fabsf(r.dx) + fabsf(r.dy) + fabsf(r.dz));
    const bool direct_ray = hit && !marchable;
    if (direct_ray) hit = false;
    const float inv_step = marchable ? 1.0f / (p.dt * dm) : 0.0f;
    const int D = cfg.depth, G = cfg.guard;
    const int nslab = (Nm + 1 + D - 1) / D;
    const float hdt = 0.5f * p.dt;
    float acc = 0.0f;

    for (int s = 0; s < nslab; ++s) {
        const int b_lo = -1 + s * D;
        const int b_hi = min(b_lo + D, Nm);
        int ka = 0, kb = -1;
        if (hit) {
            slab_k_range(cm, inv_step, pos, (float)b_lo, (float)b_hi, ka, kb);
            ka = max(ka, k0);
            kb = min(kb, k1);
        }
        // staged box: march planes [b_lo - G, b_hi + G], cross axes from the corner rays
        int lo[3], hi[3];
        lo[m] = max(b_lo - G, -1 - G);
        hi[m] = min(b_hi + G, Nm + G);
        {
            float mn1 = 3e38f, mx1 = -3e38f, mn2 = 3e38f, mx2 = -3e38f;
            const float planes[2] = {(float)(b_lo - G), (float)(b_hi + G)};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float *cr = s_corner[c];
                float idm = 1.0f / cr[3 + m];
#pragma unroll
                for (int pl = 0; pl < 2; ++pl) {
                    float t = (planes[pl] - cr[m]) * idm;
                    float q1 = fmaf(t, cr[3 + a1], cr[a1]);
                    float q2 = fmaf(t, cr[3 + a2], cr[a2]);
                    mn1 = fminf(mn1, q1); mx1 = fmaxf(mx1, q1);
                    mn2 = fminf(mn2, q2); mx2 = fmaxf(mx2, q2);
                }
            }
            // clamp before the integer conversion (rays nearly parallel to the planes)
            const float gf = (float)(G + 2);
            mn1 = fmaxf(mn1, -gf); mx1 = fminf(mx1, (float)dims[a1] + gf);
            mn2 = fmaxf(mn2, -gf); mx2 = fminf(mx2, (float)dims[a2] + gf);
            lo[a1] = max((int)floorf(mn1) - 1, -1 - G);
            hi[a1] = min((int)floorf(mx1) + 2, dims[a1] + G);
            lo[a2] = max((int)floorf(mn2) - 1, -1 - G);
            hi[a2] = min((int)floorf(mx2) + 2, dims[a2] + G);
        }
        const int Ex = hi[0] - lo[0] + 1, Ey = hi[1] - lo[1] + 1, Ez = hi[2] - lo[2] + 1;
        // also acts as the barrier that ends the previous slab's reads of sbox
        if (!__syncthreads_or(ka <= kb)) continue;
        // an empty box (corner rays crossing the planes far outside the volume, as tiles of extreme fan
        // angles can) does not mean the tile's other rays miss it: such slabs take the global path too
        const bool staged = Ex > 0 && Ey > 0 && Ez > 0 && (long long)Ex * Ey * Ez <= cfg.smem_floats;
        if (staged) {
            // rows of the box (fixed y, z) are contiguous along x in memory and in shared memory
            const int rows = Ey * Ez;
            const float inv_ey = 1.0f / (float)Ey;
            const int lanes_x = Ex >= 32 ? 32 : (Ex > 16 ? 32 : (Ex > 8 ? 16 : (Ex > 4 ? 8 : 4)));
            const int rows_per_pass = NT / lanes_x;
            const int lx = tid % lanes_x;
            for (int row = tid / lanes_x; row < rows; row += rows_per_pass) {
                const int zz = (int)(((float)row + 0.5f) * inv_ey);
                const int yy = row - zz * Ey;
                const int gz = lo[2] + zz, gy = lo[1] + yy;
                const bool inyz = (unsigned)gz < (unsigned)p.vol.nz && (unsigned)gy < (unsigned)p.vol.ny;
                const T *grow = vb + ((long long)gz * p.vol.ny + gy) * p.vol.nx;
                float *srow = sbox + row * Ex;
                for (int x = lx; x < Ex; x += lanes_x) {
                    const int gx = lo[0] + x;
                    srow[x] = (inyz && (unsigned)gx < (unsigned)p.vol.nx) ? ldg_f32(grow + gx) : 0.0f;
                }
            }
            __syncthreads();
            const float fx0 = (float)lo[0], fy0 = (float)lo[1], fz0 = (float)lo[2];
            const int sy = Ex, sz = Ex * Ey;
            for (int k = ka; k <= kb; ++k) {
                float t = fmaf((float)k, p.dt, hdt);
                float qx = fmaf(t, r.dx, r.cx) - fx0;
                float qy = fmaf(t, r.dy, r.cy) - fy0;
                float qz = fmaf(t, r.dz, r.cz) - fz0;
                float fx = floorf(qx), fy = floorf(qy), fz = floorf(qz);
                float ax = qx - fx, ay = qy - fy, az = qz - fz;
                const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
                if ((unsigned)ix >= (unsigned)(Ex - 1) || (unsigned)iy >= (unsigned)(Ey - 1) ||
                    (unsigned)iz >= (unsigned)(Ez - 1)) {
                    // outside the staged box: never expected; counted and read from global memory
                    atomicAdd(p.flags + FLAG_SLAB_OUT_OF_BOX, 1);
                    acc += trilerp_zero(vb, p.vol, qx + fx0, qy + fy0, qz + fz0);
                    continue;
                }
                const float *s0 = sbox + (iz * sz + iy * sy + ix);
                float v000 = s0[0], v001 = s0[1], v010 = s0[sy], v011 = s0[sy + 1];
                float v100 = s0[sz], v101 = s0[sz + 1], v110 = s0[sz + sy], v111 = s0[sz + sy + 1];
                float c00 = fmaf(ax, v001 - v000, v000);
                float c01 = fmaf(ax, v011 - v010, v010);
                float c10 = fmaf(ax, v101 - v100, v100);
                float c11 = fmaf(ax, v111 - v110, v110);
                float c0 = fmaf(ay, c01 - c00, c00);
                float c1 = fmaf(ay, c11 - c10, c10);
                acc += fmaf(az, c1 - c0, c0);
            }
        } else {
            if (tid == 0) atomicAdd(p.flags + FLAG_SLAB_OVERFLOW, 1);
            for (int k = ka; k <= kb; ++k) {
                float t = fmaf((float)k, p.dt, hdt);
                acc += trilerp_zero(vb, p.vol, fmaf(t, r.dx, r.cx), fmaf(t, r.dy, r.cy), fmaf(t, r.dz, r.cz));
            }
        }
    }
    if (direct_ray) {
        atomicAdd(p.flags + FLAG_SLAB_DIRECT_RAY, 1);
        for (int k = k0_all; k <= k1_all; ++k) {
            float t = fmaf((float)k, p.dt, hdt);
            acc += trilerp_zero(vb, p.vol, fmaf(t, r.dx, r.cx), fmaf(t, r.dy, r.cy), fmaf(t, r.dz, r.cz));
        }
    }
    if (active)
        sino[(long long)b * p.sino_elems + ((long long)view * p.det.nv + v) * p.det.nu + u] = from_f32<T>(acc * p.dt);
}

// ---------------------------------------------------------------------------------------------
// host: box bound and launch
// ---------------------------------------------------------------------------------------------
namespace {


// Upper bound of the staged box (in elements) of one tile over all its slabs. The extent of a
// linear function's range over the corner rays is convex in the plane position, so the first
// and the last slab bound every slab in between.
long long tile_box_bound(const pyronn_geom *g, const FpRec &rec, int tu0, int tv0, int TU, int TV, int D, int G) {
    int tu1 = std::min(tu0 + TU, g->nu) - 1, tv1 = std::min(tv0 + TV, g->nv) - 1;
    RayD cr[4];
    for (int c = 0; c < 4; ++c)
        cr[c] = ray_setup_d(rec, g, (c & 1) ? tu1 : tu0, (c & 2) ? tv1 : tv0);
    RayD ctr = ray_setup_d(rec, g, 0.5 * (tu0 + tu1), 0.5 * (tv0 + tv1));
    const int dims[3] = {g->nx, g->ny, g->nz};
    double amax = std::max(std::fabs(ctr.d[0]), std::max(std::fabs(ctr.d[1]), std::fabs(ctr.d[2])));
    long long best = 0;
    for (int m = 0; m < 3; ++m) {
        if (std::fabs(ctr.d[m]) < 0.999 * amax) continue;   // the kernel may pick any near-tie axis
        int a1 = (m == 0) ? 1 : 0, a2 = (m == 2) ? 1 : 2;
        int Nm = dims[m];
        int nslab = (Nm + 1 + D - 1) / D;
        for (int which = 0; which < 2; ++which) {
            int s = which ? nslab - 1 : 0;
            int b_lo = -1 + s * D, b_hi = std::min(b_lo + D, Nm);
            double planes[2] = {(double)(b_lo - G), (double)(b_hi + G)};
            double mn1 = 1e300, mx1 = -1e300, mn2 = 1e300, mx2 = -1e300;
            for (int c = 0; c < 4; ++c)
                for (int pl = 0; pl < 2; ++pl) {
                    double t = (planes[pl] - cr[c].c[m]) / cr[c].d[m];
                    double q1 = cr[c].c[a1] + t * cr[c].d[a1], q2 = cr[c].c[a2] + t * cr[c].d[a2];
                    mn1 = std::min(mn1, q1); mx1 = std::max(mx1, q1);
                    mn2 = std::min(mn2, q2); mx2 = std::max(mx2, q2);
                }
            const long long e1 = box_extent(mx1 - mn1, 6, dims[a1] + 2 * G + 2);
            const long long e2 = box_extent(mx2 - mn2, 6, dims[a2] + 2 * G + 2);
            if (e1 < 0 || e2 < 0) continue;
            long long em = std::min<long long>(D + 2 * G + 1, Nm + 2 * G + 2);
            best = std::max(best, em * e1 * e2);
        }
    }
    return best;
}

}  // namespace

FpSlabCfg choose_fp_slab_cfg(const pyronn_geom *g) {
    FpSlabCfg cfg{};
    cfg.tu = 16;
    cfg.tv = 16;
    cfg.depth = 8;
    double smin = std::min(g->sx, std::min(g->sy, g->sz));
    double step_max = g->dt / smin;   // largest per-sample advance along any axis, in voxels
    // steps of 2^16 voxels or more (at most one sample per ray) go to the generic kernel; this keeps
    // the guard and the box arithmetic below in range
    if (!(step_max < 65535.0)) return cfg;
    cfg.guard = 1 + (int)std::floor(step_max);
    const int ntu = (g->nu + cfg.tu - 1) / cfg.tu, ntv = (g->nv + cfg.tv - 1) / cfg.tv;
    std::atomic<int> next(0);
    std::atomic<long long> best(0);
    auto work = [&]() {
        long long local = 0;
        for (int n = next.fetch_add(1); n < g->n_views; n = next.fetch_add(1))
            for (int j = 0; j < ntv; ++j)
                for (int i = 0; i < ntu; ++i)
                    local = std::max(local, tile_box_bound(g, g->fp_rec[n], i * cfg.tu, j * cfg.tv, cfg.tu, cfg.tv,
                                                           cfg.depth, cfg.guard));
        long long cur = best.load();
        while (local > cur && !best.compare_exchange_weak(cur, local)) {
        }
    };
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned i = 1; i < nt; ++i) th.emplace_back(work);
    work();
    for (auto &t : th) t.join();
    long long need = best.load();
    const long long cap = (200 * 1024) / 4;   // floats of dynamic shared memory we allow per CTA
    cfg.smem_floats = (int)std::min(need, cap);
    cfg.valid = need > 0 && need <= cap;
    return cfg;
}

template <typename T>
static int launch_slab_t(const OpParams &p, const FpSlabCfg &cfg, const void *vol, void *sino, cudaStream_t st) {
    constexpr int TU = 16, TV = 16;
    size_t smem = sizeof(float) * (size_t)cfg.smem_floats;
    cudaError_t e = cudaFuncSetAttribute(fp_slab_kernel<T, TU, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return (int)e;
    const int per_launch = 65535 / p.n_views > 0 ? 65535 / p.n_views : 1;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        int nb = p.batch - b0 < per_launch ? p.batch - b0 : per_launch;
        dim3 grid(ceil_div(p.det.nu, TU), ceil_div(p.det.nv, TV), p.n_views * nb);
        fp_slab_kernel<T, TU, TV><<<grid, TU * TV, smem, st>>>(p, cfg, (const T *)vol + b0 * p.vol_elems,
                                                               (T *)sino + b0 * p.sino_elems);
    }
    return (int)cudaGetLastError();
}

int launch_fp(const OpParams &p, const FpSlabCfg &cfg, const void *vol, void *sino, int dtype, void *stream) {
    if (!cfg.valid || cfg.tu != 16 || cfg.tv != 16) return launch_fp_direct(p, vol, sino, dtype, stream);
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_slab_t<float>(p, cfg, vol, sino, st);
        case PYRONN_BF16: return launch_slab_t<__nv_bfloat16>(p, cfg, vol, sino, st);
        case PYRONN_F16: return launch_slab_t<__half>(p, cfg, vol, sino, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace pyronn
