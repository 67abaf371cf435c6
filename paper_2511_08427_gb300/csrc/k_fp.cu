// Ray-driven forward projector (Sec. 2.1: "rays are cast through the volume for each detector
// pixel, accumulating absorption values along their path"), operator A of Sec. 2.2.
//
//   p_r = dt * sum_k I(c_r + (k + 1/2) dt d_r),   I = trilinear hat interpolant, zero outside.
//
// Two kernels:
//   fp_direct_kernel  one thread per ray, eight read-only-cache loads per sample (general
//                     fallback, and the reference the staged kernel is tested against);
//   fp_slab_kernel    (k_fp_slab.cu) one CTA per detector tile, volume slabs staged in
//                     shared memory.
#include "device_common.cuh"

namespace pyronn {

template <typename T>
__global__ void __launch_bounds__(256) fp_direct_kernel(OpParams p, const T *__restrict__ vol, T *__restrict__ sino) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    const int view = blockIdx.z % p.n_views;
    const int b = blockIdx.z / p.n_views;
    if (u >= p.det.nu || v >= p.det.nv) return;
    const T *vb = vol + (long long)b * p.vol_elems;
    RayIdx r = ray_setup(p.fp[view], p.vol, (float)u, (float)v);
    float acc = 0.0f;
    int k0, k1;
    if (ray_k_range(r, p.vol, p.dt, k0, k1)) {
        const float hdt = 0.5f * p.dt;
        for (int k = k0; k <= k1; ++k) {
            float t = fmaf((float)k, p.dt, hdt);
            acc += trilerp_zero(vb, p.vol, fmaf(t, r.dx, r.cx), fmaf(t, r.dy, r.cy), fmaf(t, r.dz, r.cz));
        }
    }
    sino[(long long)b * p.sino_elems + ((long long)view * p.det.nv + v) * p.det.nu + u] = from_f32<T>(acc * p.dt);
}

template <typename T>
static int launch_direct_t(const OpParams &p, const void *vol, void *sino, cudaStream_t st) {
    dim3 block(32, 8);
    const int per_launch = 65535 / p.n_views > 0 ? 65535 / p.n_views : 1;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        int nb = p.batch - b0 < per_launch ? p.batch - b0 : per_launch;
        dim3 grid(ceil_div(p.det.nu, 32), ceil_div(p.det.nv, 8), p.n_views * nb);
        fp_direct_kernel<T><<<grid, block, 0, st>>>(p, (const T *)vol + b0 * p.vol_elems,
                                                    (T *)sino + b0 * p.sino_elems);
    }
    return (int)cudaGetLastError();
}

int launch_fp_direct(const OpParams &p, const void *vol, void *sino, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_direct_t<float>(p, vol, sino, st);
        case PYRONN_BF16: return launch_direct_t<__nv_bfloat16>(p, vol, sino, st);
        case PYRONN_F16: return launch_direct_t<__half>(p, vol, sino, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace pyronn
