// Matched adjoint A^T of the ray-driven forward projector (Sec. 2.2: the system is the operator
// A with its adjoint A^T; Sec. 2.1: analytical gradients of every operator). This is the exact
// transpose of k_fp.cu's sampled operator:
//
//   (A^T y)_v = sum_r y_r dt sum_k prod_axes hat(q(r, k) - v),
//
// i.e. every sample of every ray spreads y_r dt with its eight trilinear weights.
//
// adjoint_scatter_kernel: one thread per ray, FP32 atomic adds into a zeroed FP32 buffer (the
// output itself for FP32 storage, a geometry-owned scratch buffer otherwise, converted at the end).
#include "device_common.cuh"

namespace pyronn {

template <typename T>
__global__ void __launch_bounds__(256) adjoint_scatter_kernel(OpParams p, const T *__restrict__ sino,
                                                              float *__restrict__ acc) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    const int view = blockIdx.z % p.n_views;
    const int b = blockIdx.z / p.n_views;
    if (u >= p.det.nu || v >= p.det.nv) return;
    float y = ldg_f32(sino + (long long)b * p.sino_elems + ((long long)view * p.det.nv + v) * p.det.nu + u) * p.dt;
    if (y == 0.0f) return;
    float *ab = acc + (long long)b * p.vol_elems;
    RayIdx r = ray_setup(p.fp[view], p.vol, (float)u, (float)v);
    int k0, k1;
    if (!ray_k_range(r, p.vol, p.dt, k0, k1)) return;
    const float hdt = 0.5f * p.dt;
    const int sy = p.vol.nx, sz = p.vol.nx * p.vol.ny;
    for (int k = k0; k <= k1; ++k) {
        float t = fmaf((float)k, p.dt, hdt);
        float qx = fmaf(t, r.dx, r.cx), qy = fmaf(t, r.dy, r.cy), qz = fmaf(t, r.dz, r.cz);
        float fx = floorf(qx), fy = floorf(qy), fz = floorf(qz);
        float ax = qx - fx, ay = qy - fy, az = qz - fz;
        int ix = (int)fx, iy = (int)fy, iz = (int)fz;
        bool x0 = (unsigned)ix < (unsigned)p.vol.nx, x1 = (unsigned)(ix + 1) < (unsigned)p.vol.nx;
        bool y0 = (unsigned)iy < (unsigned)p.vol.ny, y1 = (unsigned)(iy + 1) < (unsigned)p.vol.ny;
        bool z0 = (unsigned)iz < (unsigned)p.vol.nz, z1 = (unsigned)(iz + 1) < (unsigned)p.vol.nz;
        if (!((x0 || x1) && (y0 || y1) && (z0 || z1))) continue;
        const int base = iz * sz + iy * sy + ix;
        float wz1 = y * az, wz0 = y - wz1;
        float w00 = wz0 * (1.0f - ay), w01 = wz0 * ay, w10 = wz1 * (1.0f - ay), w11 = wz1 * ay;
        if (z0 && y0 && x0) atomicAdd(ab + base, w00 * (1.0f - ax));
        if (z0 && y0 && x1) atomicAdd(ab + base + 1, w00 * ax);
        if (z0 && y1 && x0) atomicAdd(ab + base + sy, w01 * (1.0f - ax));
        if (z0 && y1 && x1) atomicAdd(ab + base + sy + 1, w01 * ax);
        if (z1 && y0 && x0) atomicAdd(ab + base + sz, w10 * (1.0f - ax));
        if (z1 && y0 && x1) atomicAdd(ab + base + sz + 1, w10 * ax);
        if (z1 && y1 && x0) atomicAdd(ab + base + sz + sy, w11 * (1.0f - ax));
        if (z1 && y1 && x1) atomicAdd(ab + base + sz + sy + 1, w11 * ax);
    }
}

template <typename T>
__global__ void convert_from_f32_kernel(const float *__restrict__ src, T *__restrict__ dst, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dst[i] = from_f32<T>(src[i]);
}

template <typename T>
static int launch_t(const OpParams &p, const void *sino, float *acc, void *vol, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(float) * (size_t)p.vol_elems * p.batch, st);
    if (e != cudaSuccess) return (int)e;
    dim3 block(32, 8);
    const int per_launch = 65535 / p.n_views > 0 ? 65535 / p.n_views : 1;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        int nb = p.batch - b0 < per_launch ? p.batch - b0 : per_launch;
        dim3 grid(ceil_div(p.det.nu, 32), ceil_div(p.det.nv, 8), p.n_views * nb);
        adjoint_scatter_kernel<T><<<grid, block, 0, st>>>(p, (const T *)sino + b0 * p.sino_elems,
                                                          acc + b0 * p.vol_elems);
    }
    if ((void *)acc != vol) {
        long long n = p.vol_elems * p.batch;
        int blocks = stride_grid(n, 16);
        convert_from_f32_kernel<T><<<blocks, 256, 0, st>>>(acc, (T *)vol, n);
    }
    return (int)cudaGetLastError();
}

// Scatter into the caller-provided FP32 buffer acc (zeroed here), then write vol from it.
template <typename T>
static int launch_via_acc_t(const OpParams &p, const void *sino, float *acc, void *vol, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(float) * (size_t)p.vol_elems * p.batch, st);
    if (e != cudaSuccess) return (int)e;
    dim3 block(32, 8);
    const int per_launch = 65535 / p.n_views > 0 ? 65535 / p.n_views : 1;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        int nb = p.batch - b0 < per_launch ? p.batch - b0 : per_launch;
        dim3 grid(ceil_div(p.det.nu, 32), ceil_div(p.det.nv, 8), p.n_views * nb);
        adjoint_scatter_kernel<T><<<grid, block, 0, st>>>(p, (const T *)sino + b0 * p.sino_elems,
                                                          acc + b0 * p.vol_elems);
    }
    long long n = p.vol_elems * p.batch;
    int blocks = stride_grid(n, 16);
    convert_from_f32_kernel<T><<<blocks, 256, 0, st>>>(acc, (T *)vol, n);
    return (int)cudaGetLastError();
}

int launch_adjoint_scatter_acc(const OpParams &p, const void *sino, float *acc, void *vol, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_via_acc_t<float>(p, sino, acc, vol, st);
        case PYRONN_BF16: return launch_via_acc_t<__nv_bfloat16>(p, sino, acc, vol, st);
        case PYRONN_F16: return launch_via_acc_t<__half>(p, sino, acc, vol, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

int launch_adjoint(const OpParams &p, const void *sino, void *vol, float *acc32, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_t<float>(p, sino, (float *)vol, vol, st);
        case PYRONN_BF16: return launch_t<__nv_bfloat16>(p, sino, acc32, vol, st);
        case PYRONN_F16: return launch_t<__half>(p, sino, acc32, vol, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace pyronn
