// Voxel-driven back-projector, brick form (same operator as bp_direct_kernel, Sec. 2.1).
//
// One CTA owns a 16 x 16 x BZ brick; each thread owns one z-column of BZ voxels and keeps its BZ
// sums in registers over every view. Detector coordinates are formed relative to the projection of
// the brick centre: per (brick, view), in FP64 (one lane per view of a chunk of 32 views),
//   (u0, v0, w0)  projection of the brick centre X_b,
//   Qa = Pa - u0 Pw, Qb = Pb - v0 Pw, Pw   (rows of P times the voxel spacing),
// so that for a voxel at index offset d from the centre u = u0 + (Qa . d) / w, v = v0 + (Qb . d) / w,
// w = w0 + Pw . d. Every FP32 quantity is of the size of the brick's footprint, so the bilinear
// weights carry ~1e-6-pixel errors instead of the ~1e-5 of absolute FP32 detector coordinates.
// When a view's u and w do not depend on z (circular orbits) only v is recomputed along a column;
// otherwise (tilted detectors, arbitrary trajectories) u, v and 1/w are formed per voxel. In both
// cases u and v are monotone along a column, so where every voxel of a warp's columns reads all four
// taps on the detector (each lane tests its column's end voxels, the warp votes) the warp reads them
// without bounds tests; other warps take the checked path, whose numerators advance by one addition
// per voxel.
#include "device_common.cuh"

namespace pyronn {

constexpr int BPB_X = 16, BPB_Y = 16, BPB_NT = BPB_X * BPB_Y, BPB_CHUNK = 32;

struct BpView {
    float Qa[3], Qb[3], Pw[3];   // per voxel-index step
    float w0;                    // depth ratio of the brick centre
    float fu, fv;                // fractional parts of u0, v0
    int U0, V0;                  // integer parts of u0, v0
    int flat;                    // 1: Qa_z == 0 and Pw_z == 0 (u, w constant along z)
    int valid;                   // 0: the brick centre is at or behind the source plane
};

__device__ void bp_view_setup(const OpParams &p, int view, const double Xb[3], BpView &o) {
    const double *x = p.views64 + (size_t)view * VIEW64_STRIDE;
    const double s[3] = {p.sx, p.sy, p.sz};
    double Pa[3], Pb[3], Pw[3], a0, b0, w0;
    if (p.perspective) {
        for (int i = 0; i < 3; ++i) {
            Pa[i] = x[i];
            Pb[i] = x[4 + i];
            Pw[i] = x[8 + i];
        }
        a0 = Pa[0] * Xb[0] + Pa[1] * Xb[1] + Pa[2] * Xb[2] + x[3];
        b0 = Pb[0] * Xb[0] + Pb[1] * Xb[1] + Pb[2] * Xb[2] + x[7];
        w0 = Pw[0] * Xb[0] + Pw[1] * Xb[1] + Pw[2] * Xb[2] + x[11];
    } else {
        const double *Dc = x, *eu = x + 3, *ev = x + 6;
        const double hu = 0.5 * (p.det.nu - 1), hv = 0.5 * (p.det.nv - 1);
        for (int i = 0; i < 3; ++i) {
            Pa[i] = eu[i] / p.du;
            Pb[i] = ev[i] / p.dv;
            Pw[i] = 0.0;
        }
        double Y[3] = {Xb[0] - Dc[0], Xb[1] - Dc[1], Xb[2] - Dc[2]};
        a0 = ((Y[0] * eu[0] + Y[1] * eu[1] + Y[2] * eu[2]) - p.ou) / p.du + hu;
        b0 = ((Y[0] * ev[0] + Y[1] * ev[1] + Y[2] * ev[2]) - p.ov) / p.dv + hv;
        w0 = 1.0;
    }
    o.valid = w0 > 0.0;
    if (!o.valid) w0 = 1.0;
    const double u0 = a0 / w0, v0 = b0 / w0;
    const double U = floor(u0), Vv = floor(v0);
    for (int i = 0; i < 3; ++i) {
        o.Qa[i] = (float)((Pa[i] - u0 * Pw[i]) * s[i]);
        o.Qb[i] = (float)((Pb[i] - v0 * Pw[i]) * s[i]);
        o.Pw[i] = (float)(Pw[i] * s[i]);
    }
    o.w0 = (float)w0;
    // clamp the integer parts far outside the detector (such views contribute nothing anyway)
    const double lim = 4.0e6;
    o.U0 = (int)fmin(fmax(U, -lim), lim);
    o.V0 = (int)fmin(fmax(Vv, -lim), lim);
    o.fu = (float)(u0 - U);
    o.fv = (float)(v0 - Vv);
    o.flat = (o.Qa[2] == 0.0f && o.Pw[2] == 0.0f);
}

// floor and fraction; q is clamped to +-1e6 first (the magic addition needs |q| < 2^22; detector
// coordinates that far out contribute nothing)
__device__ __forceinline__ void magic_floor(float q, int &i, float &f) {
    const float M = 12582912.0f;
    q = fminf(fmaxf(q, -1.0e6f), 1.0e6f);
    float t = __fadd_rd(q, M);
    i = __float_as_int(t) - 0x4B400000;
    f = q - (t - M);
}

template <typename T>
__device__ __forceinline__ float bilerp0(const T *__restrict__ q, int nu, int nv, int iu, int iv, float au, float av) {
    const bool u0 = (unsigned)iu < (unsigned)nu, u1 = (unsigned)(iu + 1) < (unsigned)nu;
    const bool v0 = (unsigned)iv < (unsigned)nv, v1 = (unsigned)(iv + 1) < (unsigned)nv;
    const int base = iv * nu + iu;   // one view holds fewer than 2^31 pixels
    const float q00 = (v0 && u0) ? ldg_f32(q + base) : 0.0f;
    const float q01 = (v0 && u1) ? ldg_f32(q + base + 1) : 0.0f;
    const float q10 = (v1 && u0) ? ldg_f32(q + base + nu) : 0.0f;
    const float q11 = (v1 && u1) ? ldg_f32(q + base + nu + 1) : 0.0f;
    const float r0 = fmaf(au, q01 - q00, q00);
    const float r1 = fmaf(au, q11 - q10, q10);
    return fmaf(av, r1 - r0, r0);
}

// Back-projection of one brick (block indices bxi, byi, bzi) of volume b.
template <typename T, int BZ, bool W2>
__device__ __forceinline__ void bp_brick(const OpParams &p, const T *__restrict__ sino, T *__restrict__ vol, int bxi,
                                         int byi, int bzi, int b, BpView *sv) {
    const int bx0 = bxi * BPB_X, by0 = byi * BPB_Y;
    const int bz0 = bzi * BZ;
    const int tid = threadIdx.x;
    const int lx = tid % BPB_X, ly = tid / BPB_X;
    const int i = bx0 + lx, j = by0 + ly;
    const T *sb = sino + (long long)b * p.sino_elems;
    const int nu = p.det.nu, nv = p.det.nv;

    // brick centre relative to the volume centre (world mm) and this thread's offset from it
    double Xb[3];
    Xb[0] = (bx0 + 0.5 * (BPB_X - 1) - 0.5 * (p.vol.nx - 1)) * p.sx;
    Xb[1] = (by0 + 0.5 * (BPB_Y - 1) - 0.5 * (p.vol.ny - 1)) * p.sy;
    Xb[2] = (bz0 + 0.5 * (BZ - 1) - 0.5 * (p.vol.nz - 1)) * p.sz;
    const float dx = (float)lx - 0.5f * (BPB_X - 1), dy = (float)ly - 0.5f * (BPB_Y - 1);
    const float dz0 = -0.5f * (BZ - 1);

    float acc[BZ];
#pragma unroll
    for (int z = 0; z < BZ; ++z) acc[z] = 0.0f;

    for (int n0 = 0; n0 < p.n_views; n0 += BPB_CHUNK) {
        const int nc = min(BPB_CHUNK, p.n_views - n0);
        __syncthreads();
        if (tid < nc) bp_view_setup(p, n0 + tid, Xb, sv[tid]);
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
            const BpView &V = sv[c];
            if (!V.valid) continue;
            const T *q = sb + (long long)(n0 + c) * nv * nu;
            float na = fmaf(V.Qa[0], dx, fmaf(V.Qa[1], dy, V.Qa[2] * dz0));
            float nb = fmaf(V.Qb[0], dx, fmaf(V.Qb[1], dy, V.Qb[2] * dz0));
            float w = fmaf(V.Pw[0], dx, fmaf(V.Pw[1], dy, fmaf(V.Pw[2], dz0, V.w0)));
            if (V.flat) {
                // Every lane of the warp is here (the view loop and the branches above are uniform): each
                // tests its own column, u fixed and v monotone in z (v_z = fma(z, Qb_z, nb) scaled by 1/w),
                // so the first and last voxel bound it; if all lanes' four taps lie on the detector, the
                // warp reads them without bounds tests
                const bool wpos = w > 0.0f;
                const float iw = wpos ? __frcp_rn(w) : 0.0f;
                const float qu = fmaf(na, iw, V.fu);
                const float qv0 = fmaf(nb, iw, V.fv), qv1 = fmaf(fmaf((float)(BZ - 1), V.Qb[2], nb), iw, V.fv);
                const float lu = -(float)V.U0, hu = (float)(nu - 1 - V.U0);
                const float lv = -(float)V.V0, hv = (float)(nv - 1 - V.V0);
                const bool ok = wpos && qu >= lu && qu < hu && qv0 >= lv && qv0 < hv && qv1 >= lv && qv1 < hv;
                const float om = W2 ? iw * iw : 1.0f;
                if (__all_sync(0xffffffffu, ok)) {
                    const float tu = __fadd_rd(qu, 12582912.0f);
                    const float au = qu - (tu - 12582912.0f);
                    const T *qc = q + (__float_as_int(tu) - 0x4B400000 + V.U0);
#pragma unroll
                    for (int z = 0; z < BZ; ++z) {
                        const float qv = fmaf(fmaf((float)z, V.Qb[2], nb), iw, V.fv);
                        const float t = __fadd_rd(qv, 12582912.0f);
                        const float av = qv - (t - 12582912.0f);
                        const T *r = qc + (__float_as_int(t) - 0x4B400000 + V.V0) * nu;
                        const float q00 = ldg_f32(r), q01 = ldg_f32(r + 1);
                        const float q10 = ldg_f32(r + nu), q11 = ldg_f32(r + nu + 1);
                        const float r0 = fmaf(au, q01 - q00, q00);
                        const float r1 = fmaf(au, q11 - q10, q10);
                        acc[z] = fmaf(om, fmaf(av, r1 - r0, r0), acc[z]);
                    }
                    continue;
                }
                if (!wpos) continue;
                int iu;
                float au;
                magic_floor(qu, iu, au);
                iu += V.U0;
                // the column iu and its bounds are shared by the brick's z voxels (32-bit detector
                // indices: one view holds fewer than 2^31 pixels)
                const bool u0 = (unsigned)iu < (unsigned)nu, u1 = (unsigned)(iu + 1) < (unsigned)nu;
#pragma unroll
                for (int z = 0; z < BZ; ++z) {
                    int iv;
                    float av;
                    magic_floor(fmaf(fmaf((float)z, V.Qb[2], nb), iw, V.fv), iv, av);
                    iv += V.V0;
                    const bool v0 = (unsigned)iv < (unsigned)nv, v1 = (unsigned)(iv + 1) < (unsigned)nv;
                    const T *r = q + (iv * nu + iu);
                    const float q00 = (v0 && u0) ? ldg_f32(r) : 0.0f;
                    const float q01 = (v0 && u1) ? ldg_f32(r + 1) : 0.0f;
                    const float q10 = (v1 && u0) ? ldg_f32(r + nu) : 0.0f;
                    const float q11 = (v1 && u1) ? ldg_f32(r + nu + 1) : 0.0f;
                    const float r0 = fmaf(au, q01 - q00, q00);
                    const float r1 = fmaf(au, q11 - q10, q10);
                    acc[z] = fmaf(om, fmaf(av, r1 - r0, r0), acc[z]);
                }
            } else {
                // General views (u and w vary along z: tilted detectors, arbitrary trajectories). Along a
                // column, u(z) = (na + z Qa_z) / (w + z Pw_z) and v(z) are ratios of linear functions whose
                // denominator stays positive when it is positive at both ends, hence monotone: the end
                // voxels bound the column. Lanes whose columns lie on the detector with a margin of 1e-3
                // pixel (far above the rounding of these small quantities) read their taps without bounds
                // tests when the whole warp does; positions are formed per z from the column's start.
                {
                    const float zl = (float)(BZ - 1);
                    const float w1 = fmaf(zl, V.Pw[2], w);
                    const bool wpos = w > 0.0f && w1 > 0.0f;
                    const float iw0 = wpos ? __frcp_rn(w) : 0.0f, iw1 = wpos ? __frcp_rn(w1) : 0.0f;
                    const float qu0 = fmaf(na, iw0, V.fu), qu1 = fmaf(fmaf(zl, V.Qa[2], na), iw1, V.fu);
                    const float qv0 = fmaf(nb, iw0, V.fv), qv1 = fmaf(fmaf(zl, V.Qb[2], nb), iw1, V.fv);
                    const float eps = 1e-3f;
                    const float lu = -(float)V.U0 + eps, hu = (float)(nu - 1 - V.U0) - eps;
                    const float lv = -(float)V.V0 + eps, hv = (float)(nv - 1 - V.V0) - eps;
                    const bool ok = wpos && qu0 >= lu && qu0 < hu && qu1 >= lu && qu1 < hu && qv0 >= lv && qv0 < hv &&
                                    qv1 >= lv && qv1 < hv;
                    if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
                        for (int z = 0; z < BZ; ++z) {
                            const float fz = (float)z;
                            const float iw = __frcp_rn(fmaf(fz, V.Pw[2], w));
                            const float qu = fmaf(fmaf(fz, V.Qa[2], na), iw, V.fu);
                            const float qv = fmaf(fmaf(fz, V.Qb[2], nb), iw, V.fv);
                            const float tu = __fadd_rd(qu, 12582912.0f), tv = __fadd_rd(qv, 12582912.0f);
                            const float au = qu - (tu - 12582912.0f), av = qv - (tv - 12582912.0f);
                            const T *r = q + ((__float_as_int(tv) - 0x4B400000 + V.V0) * nu +
                                              (__float_as_int(tu) - 0x4B400000 + V.U0));
                            const float q00 = ldg_f32(r), q01 = ldg_f32(r + 1);
                            const float q10 = ldg_f32(r + nu), q11 = ldg_f32(r + nu + 1);
                            const float r0 = fmaf(au, q01 - q00, q00);
                            const float r1 = fmaf(au, q11 - q10, q10);
                            const float om = W2 ? iw * iw : 1.0f;
                            acc[z] = fmaf(om, fmaf(av, r1 - r0, r0), acc[z]);
                        }
                        continue;
                    }
                }
#pragma unroll
                for (int z = 0; z < BZ; ++z) {
                    if (w > 0.0f) {
                        const float iw = __frcp_rn(w);
                        int iu, iv;
                        float au, av;
                        magic_floor(fmaf(na, iw, V.fu), iu, au);
                        magic_floor(fmaf(nb, iw, V.fv), iv, av);
                        const float om = W2 ? iw * iw : 1.0f;
                        acc[z] = fmaf(om, bilerp0(q, nu, nv, iu + V.U0, iv + V.V0, au, av), acc[z]);
                    }
                    na += V.Qa[2];
                    nb += V.Qb[2];
                    w += V.Pw[2];
                }
            }
        }
    }
    if (i < p.vol.nx && j < p.vol.ny) {
        T *vb = vol + (long long)b * p.vol_elems;
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            const int k = bz0 + z;
            if (k < p.vol.nz) vb[((long long)k * p.vol.ny + j) * p.vol.nx + i] = from_f32<T>(acc[z]);
        }
    }
}

// four CTAs per SM (64 registers) for columns of up to 8 voxels: the loop is latency-bound on its L1
// detector reads at three; three for 16-voxel columns (their 16 sums need more registers)
template <typename T, int BZ, bool W2>
__global__ void __launch_bounds__(BPB_NT, BZ > 8 ? 3 : 4) bp_brick_kernel(OpParams p, const T *__restrict__ sino,
                                                                       T *__restrict__ vol) {
    __shared__ BpView sv[BPB_CHUNK];
    const int nbz = (p.vol.nz + BZ - 1) / BZ;
    bp_brick<T, BZ, W2>(p, sino, vol, blockIdx.x, blockIdx.y, blockIdx.z % nbz, blockIdx.z / nbz, sv);
}

// Persistent launch over the bricks of several volumes.
template <typename T, bool W2>
__global__ void __launch_bounds__(BPB_NT, 4) bp_brick_batched_kernel(const __grid_constant__ PlanLaunch L) {
    __shared__ BpView sv[BPB_CHUNK];
    __shared__ int s_item;
    const long long total = L.item_end[L.n - 1];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(L.counter, 1);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        int i = 0;
        while (item >= L.item_end[i]) ++i;
        const PlanVolume &V = L.v[i];
        const int local = (int)(item - (i ? L.item_end[i - 1] : 0));
        const int bxi = local % V.ntx, byi = (local / V.ntx) % V.nty, bzi = local / (V.ntx * V.nty);
        if (W2 && V.p.perspective) bp_brick<T, 8, true>(V.p, (const T *)V.in, (T *)V.out, bxi, byi, bzi, 0, sv);
        else bp_brick<T, 8, false>(V.p, (const T *)V.in, (T *)V.out, bxi, byi, bzi, 0, sv);
    }
}

template <typename T, int BZ, bool W2>
static void launch_bpb(const OpParams &p, const void *sino, void *vol, cudaStream_t st) {
    const int nbx = ceil_div(p.vol.nx, BPB_X), nby = ceil_div(p.vol.ny, BPB_Y), nbz = ceil_div(p.vol.nz, BZ);
    const int per_launch = 65535 / nbz > 0 ? 65535 / nbz : 1;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        int nb = p.batch - b0 < per_launch ? p.batch - b0 : per_launch;
        dim3 grid(nbx, nby, nbz * nb);
        bp_brick_kernel<T, BZ, W2><<<grid, BPB_NT, 0, st>>>(p, (const T *)sino + b0 * p.sino_elems,
                                                           (T *)vol + b0 * p.vol_elems);
    }
}

// bz: voxels per thread along z of 3D volumes (4, 8 or 16; 0 = 8)
template <typename T>
static int launch_bpb_t(const OpParams &p, int bz, const void *sino, void *vol, cudaStream_t st) {
    const bool w2 = p.perspective && p.weight == PYRONN_BP_INV_W2;
    if (p.vol.nz == 1) {
        if (w2) launch_bpb<T, 1, true>(p, sino, vol, st);
        else launch_bpb<T, 1, false>(p, sino, vol, st);
    } else if (bz == 4) {
        if (w2) launch_bpb<T, 4, true>(p, sino, vol, st);
        else launch_bpb<T, 4, false>(p, sino, vol, st);
    } else if (bz == 16) {
        if (w2) launch_bpb<T, 16, true>(p, sino, vol, st);
        else launch_bpb<T, 16, false>(p, sino, vol, st);
    } else {
        if (w2) launch_bpb<T, 8, true>(p, sino, vol, st);
        else launch_bpb<T, 8, false>(p, sino, vol, st);
    }
    return (int)cudaGetLastError();
}

template <typename T>
static int launch_bp_batched_t(const PlanLaunch &L, int weight, int grid, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(L.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return (int)e;
    if (weight == PYRONN_BP_INV_W2) bp_brick_batched_kernel<T, true><<<grid, BPB_NT, 0, st>>>(L);
    else bp_brick_batched_kernel<T, false><<<grid, BPB_NT, 0, st>>>(L);
    return (int)cudaGetLastError();
}

// bricks of the batched back-projection are 16 x 16 x 8 (3D volumes only)
int launch_bp_brick_batched(const PlanLaunch &L, int dtype, int weight, int grid, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_bp_batched_t<float>(L, weight, grid, st);
        case PYRONN_BF16: return launch_bp_batched_t<__nv_bfloat16>(L, weight, grid, st);
        case PYRONN_F16: return launch_bp_batched_t<__half>(L, weight, grid, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

int bp_brick_batched_occupancy(int *blocks_per_sm) {
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, bp_brick_batched_kernel<float, true>,
                                                              BPB_NT, 0);
}

int launch_bp_brick(const OpParams &p, int bz, const void *sino, void *vol, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_bpb_t<float>(p, bz, sino, vol, st);
        case PYRONN_BF16: return launch_bpb_t<__nv_bfloat16>(p, bz, sino, vol, st);
        case PYRONN_F16: return launch_bpb_t<__half>(p, bz, sino, vol, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace pyronn
