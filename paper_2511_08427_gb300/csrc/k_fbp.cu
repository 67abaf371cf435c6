// Filtered back-projection filter (Sec. 2.2: x = A^T F^T K F p; Listing 1's ramp filter and FDK
// weights): divergent-beam cosine pre-weighting, a ramp filter along detector rows and the scale that
// makes the 1/w^2-weighted (divergent) or plain (parallel) voxel-driven BP of the output the
// reconstruction. Same operator as the oracle's or_fbp_filter.
//
// The ramp is applied as a direct convolution with its taps (Ram-Lak or Shepp-Logan, unit spacing),
// organised like a matrix product with the Toeplitz tap matrix: a CTA filters 8 rows of one view,
// staged in shared memory column-major (the 8 rows of a column are one 32-byte load), and every
// thread accumulates 8 rows x 4 consecutive output bins. Per input column a thread needs one new
// tap (the other three slide along in registers) and one broadcast load of the 8 row values, for 32
// FMAs, so the kernel is bound by the FP32 pipe, not by shared memory.
#include "device_common.cuh"

namespace pyronn {

constexpr int FBP_ROWS = 8, FBP_OUT = 4;

__device__ __forceinline__ float ramp_tap_f(int k, int filter) {
    const float ipi2 = 0.10132118364233778f;   // 1 / pi^2
    if (filter == 1) return -2.0f * ipi2 / (4.0f * (float)k * (float)k - 1.0f);
    if (k == 0) return 0.25f;
    if ((k & 1) == 0) return 0.0f;
    return -ipi2 / ((float)k * (float)k);
}

// grid: (ceil(Nv / 8), V * batch); block: ceil(Nu / 4) threads rounded up to a warp; dynamic shared
// memory: 8 Nu (rows, column-major) + 2 Nu + 4 (taps h(-Nu .. Nu + 3)) floats.
template <typename T>
__global__ void fbp_filter_kernel(OpParams p, const FbpRec *__restrict__ rec, int filter, const T *__restrict__ in,
                                  T *__restrict__ out) {
    extern __shared__ __align__(16) float fsm[];
    const int Nu = p.det.nu, Nv = p.det.nv;
    float *rows = fsm;                       // rows[m * 8 + r]
    float *taps = fsm + FBP_ROWS * Nu;       // taps[k + Nu] = h(k), k in [-Nu, Nu + 4)
    const int view = blockIdx.y % p.n_views, b = blockIdx.y / p.n_views;
    const int v0 = blockIdx.x * FBP_ROWS;
    const FbpRec R = rec[view];
    const long long base = (long long)b * p.sino_elems + (long long)view * Nv * Nu;
    for (int k = threadIdx.x; k < 2 * Nu + 4; k += blockDim.x) taps[k] = ramp_tap_f(k - Nu, filter);
    for (int e = threadIdx.x; e < FBP_ROWS * Nu; e += blockDim.x) {
        const int r = e / Nu, m = e - r * Nu, v = v0 + r;
        float val = 0.0f;
        if (v < Nv) {
            val = to_f32<T>(in[base + (long long)v * Nu + m]);
            if (R.sdd > 0.0f) {   // divergent beam: cosine of the pixel's ray
                const float dx = fmaf((float)v, R.bv[0], fmaf((float)m, R.bu[0], R.b0[0]));
                const float dy = fmaf((float)v, R.bv[1], fmaf((float)m, R.bu[1], R.b0[1]));
                const float dz = fmaf((float)v, R.bv[2], fmaf((float)m, R.bu[2], R.b0[2]));
                val *= R.sdd * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            }
        }
        rows[m * FBP_ROWS + r] = val;
    }
    __syncthreads();
    const int u0 = threadIdx.x * FBP_OUT;
    float acc[FBP_ROWS][FBP_OUT];
#pragma unroll
    for (int r = 0; r < FBP_ROWS; ++r)
#pragma unroll
        for (int j = 0; j < FBP_OUT; ++j) acc[r][j] = 0.0f;
    // outputs u0 + j need h(u0 + j - m): at column m the window is h(u0 - m .. u0 + 3 - m); moving to
    // m + 1 shifts it by one tap. For u0 < Nu every index lies in [-Nu, Nu + 3).
    if (u0 < Nu) {
        float t0 = taps[u0 + Nu], t1 = taps[u0 + 1 + Nu], t2 = taps[u0 + 2 + Nu], t3 = taps[u0 + 3 + Nu];
        for (int m = 0; m < Nu; ++m) {
            const float4 a = *reinterpret_cast<const float4 *>(rows + m * FBP_ROWS);
            const float4 c = *reinterpret_cast<const float4 *>(rows + m * FBP_ROWS + 4);
            const float rv[FBP_ROWS] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
#pragma unroll
            for (int r = 0; r < FBP_ROWS; ++r) {
                acc[r][0] = fmaf(t0, rv[r], acc[r][0]);
                acc[r][1] = fmaf(t1, rv[r], acc[r][1]);
                acc[r][2] = fmaf(t2, rv[r], acc[r][2]);
                acc[r][3] = fmaf(t3, rv[r], acc[r][3]);
            }
            t3 = t2;
            t2 = t1;
            t1 = t0;
            t0 = taps[u0 - (m + 1) + Nu];
        }
#pragma unroll
        for (int r = 0; r < FBP_ROWS; ++r) {
            const int v = v0 + r;
            if (v >= Nv) continue;
#pragma unroll
            for (int j = 0; j < FBP_OUT; ++j)
                if (u0 + j < Nu) out[base + (long long)v * Nu + u0 + j] = from_f32<T>(R.scale * acc[r][j]);
        }
    }
}

template <typename T>
static int launch_fbp_t(const OpParams &p, const FbpRec *rec, int filter, const void *in, void *out, cudaStream_t st) {
    const int nu = p.det.nu;
    int threads = (nu + FBP_OUT - 1) / FBP_OUT;
    threads = ((threads + 31) / 32) * 32;
    const size_t smem = sizeof(float) * (size_t)(FBP_ROWS * nu + 2 * nu + 4);
    cudaError_t e = cudaFuncSetAttribute(fbp_filter_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    const int per_launch = 65535 / p.n_views > 0 ? 65535 / p.n_views : 1;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        const int nb = p.batch - b0 < per_launch ? p.batch - b0 : per_launch;
        dim3 grid(ceil_div(p.det.nv, FBP_ROWS), p.n_views * nb);
        fbp_filter_kernel<T><<<grid, threads, smem, st>>>(p, rec, filter, (const T *)in + b0 * p.sino_elems,
                                                          (T *)out + b0 * p.sino_elems);
    }
    return (int)cudaGetLastError();
}

int launch_fbp_filter(const OpParams &p, const FbpRec *rec, int filter, const void *in, void *out, int dtype,
                      void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_fbp_t<float>(p, rec, filter, in, out, st);
        case PYRONN_BF16: return launch_fbp_t<__nv_bfloat16>(p, rec, filter, in, out, st);
        case PYRONN_F16: return launch_fbp_t<__half>(p, rec, filter, in, out, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace pyronn
