// Element-wise helpers of the fused gradient-step entry point (pyronn_adjoint_update) for the adjoint
// kernels that do not fuse the residual and the update themselves: out = a - b, and vol += alpha w.
#include "device_common.cuh"

namespace pyronn {

template <typename T>
__global__ void residual_kernel(const T *__restrict__ a, const T *__restrict__ b, T *__restrict__ out, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) out[i] = from_f32<T>(to_f32<T>(a[i]) - to_f32<T>(b[i]));
}

template <typename T>
__global__ void axpy_kernel(T *__restrict__ vol, const T *__restrict__ w, float alpha, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += stride) vol[i] = from_f32<T>(fmaf(alpha, to_f32<T>(w[i]), to_f32<T>(vol[i])));
}

static int blocks_for(long long n) { return stride_grid(n, 16); }

int launch_residual(const void *a, const void *b, void *out, long long n, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32:
            residual_kernel<float><<<blocks_for(n), 256, 0, st>>>((const float *)a, (const float *)b, (float *)out, n);
            break;
        case PYRONN_BF16:
            residual_kernel<__nv_bfloat16><<<blocks_for(n), 256, 0, st>>>(
                (const __nv_bfloat16 *)a, (const __nv_bfloat16 *)b, (__nv_bfloat16 *)out, n);
            break;
        case PYRONN_F16:
            residual_kernel<__half><<<blocks_for(n), 256, 0, st>>>((const __half *)a, (const __half *)b, (__half *)out, n);
            break;
        default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

int launch_axpy(void *vol, const void *w, float alpha, long long n, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: axpy_kernel<float><<<blocks_for(n), 256, 0, st>>>((float *)vol, (const float *)w, alpha, n); break;
        case PYRONN_BF16:
            axpy_kernel<__nv_bfloat16><<<blocks_for(n), 256, 0, st>>>((__nv_bfloat16 *)vol, (const __nv_bfloat16 *)w,
                                                                       alpha, n);
            break;
        case PYRONN_F16:
            axpy_kernel<__half><<<blocks_for(n), 256, 0, st>>>((__half *)vol, (const __half *)w, alpha, n);
            break;
        default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

}  // namespace pyronn
