// On-chip throughput micro-benchmarks used as roofline denominators for the projector kernels:
// shared-memory int32 and FP32 reductions (distinct addresses per lane), conflict-free 32-bit
// shared-memory loads, FP32 FMA issue, and 32-bit global loads (read-only path) and texture point
// fetches that hit in L1 (a 16 KB buffer read by every block, one cache line per warp request).
// Every index is masked into its array; there are no waits. Prints one JSON object: per-clock-per-SM
// rates at the SM clock reported by the device.
#include <cstdio>
#include <cuda_runtime.h>

namespace {

constexpr int NS = 2048, NG = 4096, ITER = 4096, THREADS = 256;

template <int MODE>
__global__ void probe(unsigned *out, const float *__restrict__ gsrc, cudaTextureObject_t tex) {
    __shared__ float sf[NS];
    __shared__ unsigned su[NS];
    for (int i = threadIdx.x; i < NS; i += blockDim.x) {
        sf[i] = 0.0f;
        su[i] = 0u;
    }
    __syncthreads();
    const float v = 1.0f + 1e-3f * threadIdx.x;
    float acc0 = v, acc1 = 2.0f * v, acc2 = 3.0f * v, acc3 = 4.0f * v;
    unsigned acc = 0u, accb = 0u, accc = 0u, accd = 0u;
    for (int i = 0; i < ITER; ++i) {
        const int idx = (threadIdx.x * 33 + i * 129) & (NS - 1);   // distinct banks within a warp
        if (MODE == 0) {
            const unsigned a = (unsigned)__cvta_generic_to_shared(su + idx);
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(3u));
        } else if (MODE == 1) {
            const unsigned a = (unsigned)__cvta_generic_to_shared(sf + idx);
            asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v));
        } else if (MODE == 2 || MODE == 4 || MODE == 5) {
            // four independent loads per iteration (one word per bank / one cache line per warp each), so
            // that a warp keeps several in flight
            const int j = (threadIdx.x & ~31) + i * 128 + (threadIdx.x & 31);
            float x0, x1, x2, x3;
            if (MODE == 2) {
                x0 = sf[j & (NS - 1)]; x1 = sf[(j + 32) & (NS - 1)];
                x2 = sf[(j + 64) & (NS - 1)]; x3 = sf[(j + 96) & (NS - 1)];
            } else if (MODE == 4) {
                x0 = __ldg(gsrc + (j & (NG - 1))); x1 = __ldg(gsrc + ((j + 32) & (NG - 1)));
                x2 = __ldg(gsrc + ((j + 64) & (NG - 1))); x3 = __ldg(gsrc + ((j + 96) & (NG - 1)));
            } else {
                x0 = tex1Dfetch<float>(tex, j & (NG - 1)); x1 = tex1Dfetch<float>(tex, (j + 32) & (NG - 1));
                x2 = tex1Dfetch<float>(tex, (j + 64) & (NG - 1)); x3 = tex1Dfetch<float>(tex, (j + 96) & (NG - 1));
            }
            acc += __float_as_uint(x0);
            accb += __float_as_uint(x1);
            accc += __float_as_uint(x2);
            accd += __float_as_uint(x3);
        } else {
            acc0 = fmaf(acc0, 0.999f, 1e-3f);
            acc1 = fmaf(acc1, 0.999f, 1e-3f);
            acc2 = fmaf(acc2, 0.999f, 1e-3f);
            acc3 = fmaf(acc3, 0.999f, 1e-3f);
        }
    }
    __syncthreads();
    acc += accb + accc + accd;
    if (threadIdx.x == 0) out[blockIdx.x] = su[1] + acc + __float_as_uint(sf[3] + acc0 + acc1 + acc2 + acc3);
    else if (acc == 0xffffffffu) out[blockIdx.x] = acc;   // keeps the loads live
}

template <int MODE>
double rate(int blocks, unsigned *out, const float *gsrc, cudaTextureObject_t tex, double sm_hz, int sms,
            int ops_per_iter) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.0f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(a);
        probe<MODE><<<blocks, THREADS>>>(out, gsrc, tex);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double ops = (double)blocks * THREADS * ITER * ops_per_iter;
    return ops / (ms * 1e-3) / (sms * sm_hz);
}

}  // namespace

int main() {
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, 0) != cudaSuccess) return 1;
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
    const int sms = pr.multiProcessorCount, blocks = sms * 4;
    unsigned *out = nullptr;
    float *gsrc = nullptr;
    if (cudaMalloc(&out, sizeof(unsigned) * blocks) != cudaSuccess) return 1;
    if (cudaMalloc(&gsrc, sizeof(float) * NG) != cudaSuccess) return 1;
    cudaMemset(gsrc, 0, sizeof(float) * NG);
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypeLinear;
    rd.res.linear.devPtr = gsrc;
    rd.res.linear.desc = cudaCreateChannelDesc<float>();
    rd.res.linear.sizeInBytes = sizeof(float) * NG;
    cudaTextureDesc td{};
    td.readMode = cudaReadModeElementType;
    cudaTextureObject_t tex = 0;
    if (cudaCreateTextureObject(&tex, &rd, &td, nullptr) != cudaSuccess) return 1;
    const double hz = clk_khz * 1e3;
    const double red_u32 = rate<0>(blocks, out, gsrc, tex, hz, sms, 1);
    const double red_f32 = rate<1>(blocks, out, gsrc, tex, hz, sms, 1);
    const double lds = rate<2>(blocks, out, gsrc, tex, hz, sms, 4);
    const double ffma = rate<3>(blocks, out, gsrc, tex, hz, sms, 4);
    const double ldg = rate<4>(blocks, out, gsrc, tex, hz, sms, 4);
    const double texf = rate<5>(blocks, out, gsrc, tex, hz, sms, 4);
    const cudaError_t e = cudaDeviceSynchronize();
    cudaDestroyTextureObject(tex);
    cudaFree(gsrc);
    cudaFree(out);
    printf("{\"device\": \"%s\", \"sms\": %d, \"clock_mhz\": %.0f, \"red_shared_u32_per_clk_sm\": %.2f, "
           "\"red_shared_f32_per_clk_sm\": %.2f, \"ld_shared_f32_per_clk_sm\": %.2f, \"ffma_per_clk_sm\": %.2f, "
           "\"ld_global_l1_f32_per_clk_sm\": %.2f, \"tex_fetch_f32_per_clk_sm\": %.2f, \"status\": \"%s\"}\n",
           pr.name, sms, hz / 1e6, red_u32, red_f32, lds, ffma, ldg, texf, cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
