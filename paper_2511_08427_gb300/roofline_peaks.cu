// On-chip throughput of the units that bound the projector kernels, measured on the device the
// library runs on: these are the denominators of the roofline fractions the benchmark reports.
//
//   0  int32 shared-memory reductions (red.shared.add.s32), one distinct bank per lane
//   1  FP32 shared-memory reductions (red.shared.add.f32), one distinct bank per lane
//   2  32-bit shared-memory loads, one distinct bank per lane, four independent loads in flight
//   3  FP32 fused multiply-adds, four independent chains per thread
//   4  32-bit global loads through the read-only path that hit in L1 (a 16 KB buffer, one cache line
//      per warp request), four in flight
//   5  texture point fetches (tex1Dfetch of FP32), four in flight
//   6  trilinear filtered fetches of a 3D FP32 texture (hardware interpolation), four in flight, the
//      lanes of a warp on neighbouring texels of a 32^3 array that stays in the texture cache
//
// Each probe launches 4 CTAs of 256 threads per SM. Thread 0 of every CTA records its SM and that SM's
// cycle counter after a barrier at the start and at the end of its loop; per SM, the operations of its
// CTAs over the span from the first start to the last end give a rate per SM clock cycle, independent
// of the clock the GPU runs at and of how the CTAs were distributed (the median over SMs is reported,
// with the clock itself: cycles / elapsed time).
// Every index is masked into its array and no thread waits on another outside a barrier.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

namespace {

constexpr int NS = 2048, NG = 4096, ITER = 4096, THREADS = 256, CTAS_PER_SM = 4, TEX3 = 32;

template <int MODE>
__global__ void __launch_bounds__(THREADS) probe(unsigned *out, long long *cycles, const float *__restrict__ gsrc,
                                                 cudaTextureObject_t tex1, cudaTextureObject_t tex3) {
    // cycles[3 b .. 3 b + 2]: the SM this CTA ran on, its cycle counter after the opening barrier and
    // after the closing barrier
    __shared__ float sf[NS];
    __shared__ unsigned su[NS];
    for (int i = threadIdx.x; i < NS; i += blockDim.x) {
        sf[i] = 0.0f;
        su[i] = 0u;
    }
    __syncthreads();
    long long t0 = clock64();
    const float v = 1.0f + 1e-3f * threadIdx.x;
    float acc0 = v, acc1 = 2.0f * v, acc2 = 3.0f * v, acc3 = 4.0f * v;
    unsigned acc = 0u, accb = 0u, accc = 0u, accd = 0u;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < ITER; ++i) {
        if (MODE == 0 || MODE == 1) {
            const int idx = (threadIdx.x * 33 + i * 129) & (NS - 1);   // distinct banks within a warp
            if (MODE == 0) {
                const unsigned a = (unsigned)__cvta_generic_to_shared(su + idx);
                asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(3));
            } else {
                const unsigned a = (unsigned)__cvta_generic_to_shared(sf + idx);
                asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(a), "f"(v));
            }
        } else if (MODE == 2 || MODE == 4 || MODE == 5) {
            const int j = (threadIdx.x & ~31) + i * 128 + lane;
            float x0, x1, x2, x3;
            if (MODE == 2) {
                x0 = sf[j & (NS - 1)]; x1 = sf[(j + 32) & (NS - 1)];
                x2 = sf[(j + 64) & (NS - 1)]; x3 = sf[(j + 96) & (NS - 1)];
            } else if (MODE == 4) {
                x0 = __ldg(gsrc + (j & (NG - 1))); x1 = __ldg(gsrc + ((j + 32) & (NG - 1)));
                x2 = __ldg(gsrc + ((j + 64) & (NG - 1))); x3 = __ldg(gsrc + ((j + 96) & (NG - 1)));
            } else {
                x0 = tex1Dfetch<float>(tex1, j & (NG - 1)); x1 = tex1Dfetch<float>(tex1, (j + 32) & (NG - 1));
                x2 = tex1Dfetch<float>(tex1, (j + 64) & (NG - 1)); x3 = tex1Dfetch<float>(tex1, (j + 96) & (NG - 1));
            }
            acc += __float_as_uint(x0);
            accb += __float_as_uint(x1);
            accc += __float_as_uint(x2);
            accd += __float_as_uint(x3);
        } else if (MODE == 6) {
            // a warp samples 32 points 0.75 texel apart along x (as adjacent rays do), in a plane that
            // moves with the iteration; coordinates stay inside the array
            const float x = 2.0f + 0.75f * (float)lane;
            const float y = 2.0f + (float)((warp * 3 + i) & 15) + 0.37f;
            const float z = 2.0f + (float)((i * 5 + warp) & 15) + 0.61f;
            const float x0 = tex3D<float>(tex3, x, y, z);
            const float x1 = tex3D<float>(tex3, x + 0.5f, y + 1.0f, z);
            const float x2 = tex3D<float>(tex3, x, y + 2.0f, z + 1.0f);
            const float x3 = tex3D<float>(tex3, x + 0.25f, y + 3.0f, z + 2.0f);
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
    // every thread stores its results to shared memory before the closing barrier, so no part of the
    // loop (the FMA chains in particular) can be scheduled after the second clock read
    __syncwarp();
    acc += accb + accc + accd;
    su[threadIdx.x] = acc + __float_as_uint(acc0 + acc1 + acc2 + acc3);
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        cycles[3 * blockIdx.x] = smid;
        cycles[3 * blockIdx.x + 1] = t0;
        cycles[3 * blockIdx.x + 2] = t1;
        out[blockIdx.x] = su[1] + su[255] + __float_as_uint(sf[3]);
    }
}

struct Probe {
    int blocks, sms;
    unsigned *out;
    long long *cycles;
    const float *gsrc;
    cudaTextureObject_t tex1, tex3;
};

// Runs one probe three times. From the last run: per SM, the operations of the CTAs that ran on it over
// the cycles from the first CTA's start to the last CTA's end (the cycle counter is per SM); returns the
// median over SMs of operations per cycle, and the SM clock in MHz (median cycles / event time), or a
// negative rate on a CUDA error.
template <int MODE>
double rate(const Probe &P, int ops_per_iter, double *mhz) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.0;
    }
    float ms = 0.0f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(a);
        probe<MODE><<<P.blocks, THREADS>>>(P.out, P.cycles, P.gsrc, P.tex1, P.tex3);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    std::vector<long long> rec(3 * (size_t)P.blocks);
    if (cudaMemcpy(rec.data(), P.cycles, sizeof(long long) * rec.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1.0;
    const int nsm_max = 1024;
    std::vector<long long> lo(nsm_max, -1), hi(nsm_max, -1);
    std::vector<int> n(nsm_max, 0);
    for (int b = 0; b < P.blocks; ++b) {
        const long long sm = rec[3 * b], t0 = rec[3 * b + 1], t1 = rec[3 * b + 2];
        if (sm < 0 || sm >= nsm_max) return -1.0;
        lo[sm] = (lo[sm] < 0 || t0 < lo[sm]) ? t0 : lo[sm];
        hi[sm] = t1 > hi[sm] ? t1 : hi[sm];
        ++n[sm];
    }
    const double ops_per_cta = (double)THREADS * ITER * ops_per_iter;
    std::vector<double> r, cyc;
    for (int sm = 0; sm < nsm_max; ++sm)
        if (n[sm] > 0 && hi[sm] > lo[sm]) {
            r.push_back(n[sm] * ops_per_cta / (double)(hi[sm] - lo[sm]));
            cyc.push_back((double)(hi[sm] - lo[sm]));
        }
    if (r.empty()) return -1.0;
    std::sort(r.begin(), r.end());
    std::sort(cyc.begin(), cyc.end());
    *mhz = cyc[cyc.size() / 2] / (ms * 1e-3) / 1e6;
    return r[r.size() / 2];
}

}  // namespace

// out[0..9]: SM count, SM clock (MHz, median of the probes), then per SM clock cycle: int32 shared
// reductions, FP32 shared reductions, 32-bit shared loads, FP32 FMAs (instructions, not FLOP), L1-hit
// 32-bit global loads, texture point fetches, trilinear 3D texture fetches; out[9] 0 on success.
// Returns 0, or a CUDA error code.
extern "C" __attribute__((visibility("default"))) int pyronn_roofline_measure(double *out, int n_out) {
    if (!out || n_out < 10) return (int)cudaErrorInvalidValue;
    std::memset(out, 0, sizeof(double) * (size_t)n_out);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    Probe P{};
    P.sms = sms;
    P.blocks = sms * CTAS_PER_SM;
    unsigned *dout = nullptr;
    long long *dcyc = nullptr;
    float *gsrc = nullptr;
    cudaArray_t arr = nullptr;
    cudaTextureObject_t t1 = 0, t3 = 0;
    int rc = 0;
    do {
        if ((e = cudaMalloc(&dout, sizeof(unsigned) * P.blocks)) != cudaSuccess) break;
        if ((e = cudaMalloc(&dcyc, 3 * sizeof(long long) * P.blocks)) != cudaSuccess) break;
        if ((e = cudaMalloc(&gsrc, sizeof(float) * NG)) != cudaSuccess) break;
        if ((e = cudaMemset(gsrc, 0, sizeof(float) * NG)) != cudaSuccess) break;
        cudaResourceDesc rd{};
        rd.resType = cudaResourceTypeLinear;
        rd.res.linear.devPtr = gsrc;
        rd.res.linear.desc = cudaCreateChannelDesc<float>();
        rd.res.linear.sizeInBytes = sizeof(float) * NG;
        cudaTextureDesc td{};
        td.readMode = cudaReadModeElementType;
        if ((e = cudaCreateTextureObject(&t1, &rd, &td, nullptr)) != cudaSuccess) break;
        const cudaChannelFormatDesc cd = cudaCreateChannelDesc<float>();
        if ((e = cudaMalloc3DArray(&arr, &cd, make_cudaExtent(TEX3, TEX3, TEX3))) != cudaSuccess) break;
        std::vector<float> host((size_t)TEX3 * TEX3 * TEX3);
        for (size_t i = 0; i < host.size(); ++i) host[i] = (float)(i % 97) * 0.01f;
        cudaMemcpy3DParms cp{};
        cp.srcPtr = make_cudaPitchedPtr(host.data(), TEX3 * sizeof(float), TEX3, TEX3);
        cp.dstArray = arr;
        cp.extent = make_cudaExtent(TEX3, TEX3, TEX3);
        cp.kind = cudaMemcpyHostToDevice;
        if ((e = cudaMemcpy3D(&cp)) != cudaSuccess) break;
        cudaResourceDesc rd3{};
        rd3.resType = cudaResourceTypeArray;
        rd3.res.array.array = arr;
        cudaTextureDesc td3{};
        td3.readMode = cudaReadModeElementType;
        td3.filterMode = cudaFilterModeLinear;
        for (int a = 0; a < 3; ++a) td3.addressMode[a] = cudaAddressModeBorder;
        if ((e = cudaCreateTextureObject(&t3, &rd3, &td3, nullptr)) != cudaSuccess) break;
        P.out = dout;
        P.cycles = dcyc;
        P.gsrc = gsrc;
        P.tex1 = t1;
        P.tex3 = t3;
        double mhz[7] = {};
        const double r[7] = {rate<0>(P, 1, &mhz[0]), rate<1>(P, 1, &mhz[1]), rate<2>(P, 4, &mhz[2]),
                             rate<3>(P, 4, &mhz[3]), rate<4>(P, 4, &mhz[4]), rate<5>(P, 4, &mhz[5]),
                             rate<6>(P, 4, &mhz[6])};
        bool ok = true;
        for (int i = 0; i < 7; ++i) ok = ok && r[i] > 0.0;
        if (!ok) {
            e = cudaGetLastError();
            rc = e != cudaSuccess ? (int)e : (int)cudaErrorUnknown;
            break;
        }
        std::sort(mhz, mhz + 7);
        out[0] = sms;
        out[1] = mhz[3];
        for (int i = 0; i < 7; ++i) out[2 + i] = r[i];
        out[9] = 0.0;
    } while (false);
    if (t3) cudaDestroyTextureObject(t3);
    if (t1) cudaDestroyTextureObject(t1);
    if (arr) cudaFreeArray(arr);
    if (gsrc) cudaFree(gsrc);
    if (dcyc) cudaFree(dcyc);
    if (dout) cudaFree(dout);
    if (rc) return rc;
    return e == cudaSuccess ? 0 : (int)e;
}
