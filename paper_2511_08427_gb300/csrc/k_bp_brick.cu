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
#include "bp_common.cuh"

namespace pyronn {

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
        if (tid < nc) bp_view_setup(p, n0 + tid, Xb, 0.5 * (BZ - 1), sv[tid]);
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
            const BpView &V = sv[c];
            if (!V.valid) continue;
            const T *q = sb + (long long)(n0 + c) * nv * nu;
            bp_view_global<T, BZ, W2>(V, q, nu, nv, dx, dy, dz0, acc);
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
