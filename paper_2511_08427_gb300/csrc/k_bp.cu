// Voxel-driven back-projector (Sec. 2.1: "projecting each voxel onto the detector and
// accumulating the measured line integrals"):
//
//   b_v = sum_views omega * sum_{u', v'} q[v', u'] hat(u - u') hat(v - v'),
//   (u w, v w, w) = P_view (voxel centre, 1),  omega = 1 or 1 / w^2,
//
// bilinear detector interpolation with zero outside the detector. A voxel at or behind the
// source plane of a view (w <= 0) receives nothing from that view.
//
// bp_direct_kernel: one thread per voxel, all views looped in registers; view matrices staged
// in shared memory per chunk of views.
#include "device_common.cuh"

namespace pyronn {

constexpr int BP_VIEW_CHUNK = 256;

template <typename T, bool PERSP, bool W2>
__global__ void __launch_bounds__(256) bp_direct_kernel(OpParams p, const T *__restrict__ sino, T *__restrict__ vol) {
    __shared__ float sP[BP_VIEW_CHUNK * 12];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z % p.vol.nz;
    const int b = blockIdx.z / p.vol.nz;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const float x = (float)i - p.vol.hx, y = (float)j - p.vol.hy, z = (float)k - p.vol.hz;
    const T *sb = sino + (long long)b * p.sino_elems;
    const int nu = p.det.nu, nv = p.det.nv;
    float acc = 0.0f;
    for (int n0 = 0; n0 < p.n_views; n0 += BP_VIEW_CHUNK) {
        const int nc = min(BP_VIEW_CHUNK, p.n_views - n0);
        __syncthreads();
        for (int e = tid; e < nc * 12; e += blockDim.x * blockDim.y) sP[e] = p.bp[n0 + e / 12].P[e % 12];
        __syncthreads();
        if (i < p.vol.nx && j < p.vol.ny) {
            for (int c = 0; c < nc; ++c) {
                const float *P = sP + 12 * c;
                float a = fmaf(P[0], x, fmaf(P[1], y, fmaf(P[2], z, P[3])));
                float bb = fmaf(P[4], x, fmaf(P[5], y, fmaf(P[6], z, P[7])));
                float iw = 1.0f;
                if (PERSP) {
                    float w = fmaf(P[8], x, fmaf(P[9], y, fmaf(P[10], z, P[11])));
                    if (!(w > 0.0f)) continue;
                    iw = __frcp_rn(w);
                }
                float u = fmaf(a, iw, p.det.hu), v = fmaf(bb, iw, p.det.hv);
                if (!(u > -1.0f && u < (float)nu && v > -1.0f && v < (float)nv)) continue;
                float fu = floorf(u), fv = floorf(v);
                float au = u - fu, av = v - fv;
                int iu = (int)fu, iv = (int)fv;
                bool u0 = iu >= 0, u1 = iu + 1 < nu, v0 = iv >= 0, v1 = iv + 1 < nv;
                const T *q = sb + ((long long)(n0 + c) * nv) * nu;
                const int base = iv * nu + iu;
                float q00 = (v0 && u0) ? ldg_f32(q + base) : 0.0f;
                float q01 = (v0 && u1) ? ldg_f32(q + base + 1) : 0.0f;
                float q10 = (v1 && u0) ? ldg_f32(q + base + nu) : 0.0f;
                float q11 = (v1 && u1) ? ldg_f32(q + base + nu + 1) : 0.0f;
                float r0 = fmaf(au, q01 - q00, q00);
                float r1 = fmaf(au, q11 - q10, q10);
                float val = fmaf(av, r1 - r0, r0);
                if (W2) val *= iw * iw;
                acc += val;
            }
        }
    }
    if (i < p.vol.nx && j < p.vol.ny)
        vol[(long long)b * p.vol_elems + ((long long)k * p.vol.ny + j) * p.vol.nx + i] = from_f32<T>(acc);
}

template <typename T, bool PERSP, bool W2>
static void launch_bp3(const OpParams &p, const void *sino, void *vol, cudaStream_t st) {
    dim3 block(32, 8);
    const int per_launch = 65535 / p.vol.nz > 0 ? 65535 / p.vol.nz : 1;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        int nb = p.batch - b0 < per_launch ? p.batch - b0 : per_launch;
        dim3 grid(ceil_div(p.vol.nx, 32), ceil_div(p.vol.ny, 8), p.vol.nz * nb);
        bp_direct_kernel<T, PERSP, W2><<<grid, block, 0, st>>>(p, (const T *)sino + b0 * p.sino_elems,
                                                              (T *)vol + b0 * p.vol_elems);
    }
}

template <typename T>
static int launch_t(const OpParams &p, const void *sino, void *vol, cudaStream_t st) {
    if (p.perspective) {
        if (p.weight == PYRONN_BP_INV_W2) launch_bp3<T, true, true>(p, sino, vol, st);
        else launch_bp3<T, true, false>(p, sino, vol, st);
    } else {
        launch_bp3<T, false, false>(p, sino, vol, st);
    }
    return (int)cudaGetLastError();
}

// Exact transpose of bp_direct_kernel: each voxel spreads x_v * omega with the bilinear weights
// of its projection over four detector pixels (FP32 atomic adds into a zeroed buffer).
template <typename T, bool PERSP, bool W2>
__global__ void __launch_bounds__(256) bp_transpose_kernel(OpParams p, const T *__restrict__ vol,
                                                           float *__restrict__ acc) {
    __shared__ float sP[BP_VIEW_CHUNK * 12];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z % p.vol.nz;
    const int b = blockIdx.z / p.vol.nz;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const bool inside = i < p.vol.nx && j < p.vol.ny;
    const float xv = inside ? ldg_f32(vol + (long long)b * p.vol_elems + ((long long)k * p.vol.ny + j) * p.vol.nx + i)
                            : 0.0f;
    const float x = (float)i - p.vol.hx, y = (float)j - p.vol.hy, z = (float)k - p.vol.hz;
    float *ab = acc + (long long)b * p.sino_elems;
    const int nu = p.det.nu, nv = p.det.nv;
    for (int n0 = 0; n0 < p.n_views; n0 += BP_VIEW_CHUNK) {
        const int nc = min(BP_VIEW_CHUNK, p.n_views - n0);
        __syncthreads();
        for (int e = tid; e < nc * 12; e += blockDim.x * blockDim.y) sP[e] = p.bp[n0 + e / 12].P[e % 12];
        __syncthreads();
        if (!inside || xv == 0.0f) continue;
        for (int c = 0; c < nc; ++c) {
            const float *P = sP + 12 * c;
            float a = fmaf(P[0], x, fmaf(P[1], y, fmaf(P[2], z, P[3])));
            float bb = fmaf(P[4], x, fmaf(P[5], y, fmaf(P[6], z, P[7])));
            float iw = 1.0f;
            if (PERSP) {
                float w = fmaf(P[8], x, fmaf(P[9], y, fmaf(P[10], z, P[11])));
                if (!(w > 0.0f)) continue;
                iw = __frcp_rn(w);
            }
            float u = fmaf(a, iw, p.det.hu), v = fmaf(bb, iw, p.det.hv);
            if (!(u > -1.0f && u < (float)nu && v > -1.0f && v < (float)nv)) continue;
            float fu = floorf(u), fv = floorf(v);
            float au = u - fu, av = v - fv;
            int iu = (int)fu, iv = (int)fv;
            bool u0 = iu >= 0, u1 = iu + 1 < nu, v0 = iv >= 0, v1 = iv + 1 < nv;
            float val = W2 ? xv * iw * iw : xv;
            float *q = ab + ((long long)(n0 + c) * nv) * nu + (iv * nu + iu);
            float wv0 = val * (1.0f - av), wv1 = val * av;
            if (v0 && u0) atomicAdd(q, wv0 * (1.0f - au));
            if (v0 && u1) atomicAdd(q + 1, wv0 * au);
            if (v1 && u0) atomicAdd(q + nu, wv1 * (1.0f - au));
            if (v1 && u1) atomicAdd(q + nu + 1, wv1 * au);
        }
    }
}

template <typename T>
__global__ void bp_convert_kernel(const float *__restrict__ src, T *__restrict__ dst, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dst[i] = from_f32<T>(src[i]);
}

template <typename T, bool PERSP, bool W2>
static void launch_bpt3(const OpParams &p, const void *vol, float *acc, cudaStream_t st) {
    dim3 block(32, 8);
    const int per_launch = 65535 / p.vol.nz > 0 ? 65535 / p.vol.nz : 1;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        int nb = p.batch - b0 < per_launch ? p.batch - b0 : per_launch;
        dim3 grid(ceil_div(p.vol.nx, 32), ceil_div(p.vol.ny, 8), p.vol.nz * nb);
        bp_transpose_kernel<T, PERSP, W2><<<grid, block, 0, st>>>(p, (const T *)vol + b0 * p.vol_elems,
                                                                 acc + b0 * p.sino_elems);
    }
}

template <typename T>
static int launch_t_transpose(const OpParams &p, const void *vol, float *acc, void *sino, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(float) * (size_t)p.sino_elems * p.batch, st);
    if (e != cudaSuccess) return (int)e;
    if (p.perspective) {
        if (p.weight == PYRONN_BP_INV_W2) launch_bpt3<T, true, true>(p, vol, acc, st);
        else launch_bpt3<T, true, false>(p, vol, acc, st);
    } else {
        launch_bpt3<T, false, false>(p, vol, acc, st);
    }
    if ((void *)acc != sino) {
        long long n = p.sino_elems * p.batch;
        int blocks = stride_grid(n, 16);
        bp_convert_kernel<T><<<blocks, 256, 0, st>>>(acc, (T *)sino, n);
    }
    return (int)cudaGetLastError();
}

int launch_bp_transpose(const OpParams &p, const void *vol, void *sino, float *acc32, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_t_transpose<float>(p, vol, (float *)sino, sino, st);
        case PYRONN_BF16: return launch_t_transpose<__nv_bfloat16>(p, vol, acc32, sino, st);
        case PYRONN_F16: return launch_t_transpose<__half>(p, vol, acc32, sino, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

int launch_bp(const OpParams &p, const void *sino, void *vol, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_t<float>(p, sino, vol, st);
        case PYRONN_BF16: return launch_t<__nv_bfloat16>(p, sino, vol, st);
        case PYRONN_F16: return launch_t<__half>(p, sino, vol, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace pyronn
