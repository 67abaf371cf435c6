// Acquisition-artifact simulation on sinograms (Sec. 2.4: detector jitter, Gaussian noise, ring
// artifacts, gantry motion blur). Every random quantity is an input (shifts, noise samples, chosen
// columns), so these are deterministic transforms; sinograms are [batch][V][Nv][Nu], u fastest.
#include "device_common.cuh"

namespace pyronn {

static int ew_blocks(long long n) { return stride_grid(n, 32); }

// out[v][u] = in[v][u - s] (axis 0, one shift per row) or in[v - s][u] (axis 1, one shift per column).
template <typename T>
__global__ void jitter_kernel(const T *__restrict__ in, T *__restrict__ out, const int *__restrict__ shifts, int axis,
                              int nu, int nv, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(i % nu);
        const long long row = i / nu;             // (item, view, v)
        const int v = (int)(row % nv);
        const long long img = row / nv;           // (item, view)
        float val = 0.0f;
        if (axis == 0) {
            const int src = u - shifts[row];
            if (src >= 0 && src < nu) val = to_f32<T>(in[row * nu + src]);
        } else {
            const int src = v - shifts[img * nu + u];
            if (src >= 0 && src < nv) val = to_f32<T>(in[(img * nv + src) * nu + u]);
        }
        out[i] = from_f32<T>(val);
    }
}

template <typename T>
__global__ void noise_kernel(const T *__restrict__ in, T *__restrict__ out, const float *__restrict__ noise, float mean,
                             float sd, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = from_f32<T>(to_f32<T>(in[i]) + fmaf(sd, noise[i], mean));
}

// element (item, view in [v0, v1), v, column index c): out = in * gains[c] at u = columns[c]
template <typename T>
__global__ void ring_kernel(const T *__restrict__ in, T *__restrict__ out, const int *__restrict__ cols,
                            const float *__restrict__ gains, int ncol, int nu, int nv, int n_views, int v0, int v1,
                            long long n) {
    const int nsel = v1 - v0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % ncol);
        long long r = i / ncol;
        const int v = (int)(r % nv);
        r /= nv;
        const int view = v0 + (int)(r % nsel);
        const long long item = r / nsel;
        const int u = cols[c];
        if (u < 0 || u >= nu) continue;
        const long long o = ((item * n_views + view) * nv + v) * nu + u;
        out[o] = from_f32<T>(to_f32<T>(in[o]) * gains[c]);
    }
}

// out(u, v) of view n = (1 / L) sum_j bilinear(in, u + t_j cos a_n, v + t_j sin a_n), t_j = j - (L - 1) / 2
template <typename T>
__global__ void blur_kernel(const T *__restrict__ in, T *__restrict__ out, const float *__restrict__ angles, int length,
                            int nu, int nv, int n_views, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(i % nu);
        const long long row = i / nu;
        const int v = (int)(row % nv);
        const long long img = row / nv;
        const int view = (int)(img % n_views);
        const T *src = in + img * (long long)nv * nu;
        float ca, sa;
        sincosf(angles[view], &sa, &ca);
        float acc = 0.0f;
        for (int j = 0; j < length; ++j) {
            const float t = (float)j - 0.5f * (float)(length - 1);
            const float x = fmaf(t, ca, (float)u), y = fmaf(t, sa, (float)v);
            const float fx = floorf(x), fy = floorf(y);
            const int x0 = (int)fx, y0 = (int)fy;
            const float ax = x - fx, ay = y - fy;
            float s = 0.0f;
            if (y0 >= 0 && y0 < nv) {
                if (x0 >= 0 && x0 < nu) s += (1.0f - ax) * (1.0f - ay) * to_f32<T>(src[(long long)y0 * nu + x0]);
                if (x0 + 1 >= 0 && x0 + 1 < nu) s += ax * (1.0f - ay) * to_f32<T>(src[(long long)y0 * nu + x0 + 1]);
            }
            if (y0 + 1 >= 0 && y0 + 1 < nv) {
                if (x0 >= 0 && x0 < nu) s += (1.0f - ax) * ay * to_f32<T>(src[(long long)(y0 + 1) * nu + x0]);
                if (x0 + 1 >= 0 && x0 + 1 < nu) s += ax * ay * to_f32<T>(src[(long long)(y0 + 1) * nu + x0 + 1]);
            }
            acc += s;
        }
        out[i] = from_f32<T>(acc / (float)length);
    }
}

#define PYRONN_DISPATCH(dtype, CALL)                                   \
    switch (dtype) {                                                   \
        case PYRONN_F32: { using T = float; CALL; break; }             \
        case PYRONN_BF16: { using T = __nv_bfloat16; CALL; break; }    \
        case PYRONN_F16: { using T = __half; CALL; break; }            \
        default: return (int)cudaErrorInvalidValue;                    \
    }

int launch_sim_jitter(const void *in, void *out, const int *shifts, int axis, int nu, int nv, long long n, int dtype,
                      void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    PYRONN_DISPATCH(dtype, (jitter_kernel<T><<<ew_blocks(n), 256, 0, st>>>((const T *)in, (T *)out, shifts, axis, nu,
                                                                            nv, n)));
    return (int)cudaGetLastError();
}

int launch_sim_noise(const void *in, void *out, const float *noise, float mean, float sd, long long n, int dtype,
                     void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    PYRONN_DISPATCH(dtype, (noise_kernel<T><<<ew_blocks(n), 256, 0, st>>>((const T *)in, (T *)out, noise, mean, sd, n)));
    return (int)cudaGetLastError();
}

int launch_sim_ring(const void *in, void *out, const int *cols, const float *gains, int ncol, int nu, int nv, int n_views,
                    int v0, int v1, int batch, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)batch * (v1 - v0) * nv * ncol;
    if (n <= 0) return 0;
    PYRONN_DISPATCH(dtype, (ring_kernel<T><<<ew_blocks(n), 256, 0, st>>>((const T *)in, (T *)out, cols, gains, ncol, nu,
                                                                          nv, n_views, v0, v1, n)));
    return (int)cudaGetLastError();
}

int launch_sim_blur(const void *in, void *out, const float *angles, int length, int nu, int nv, int n_views, long long n,
                    int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    PYRONN_DISPATCH(dtype, (blur_kernel<T><<<ew_blocks(n), 256, 0, st>>>((const T *)in, (T *)out, angles, length, nu, nv,
                                                                          n_views, n)));
    return (int)cudaGetLastError();
}

#undef PYRONN_DISPATCH

}  // namespace pyronn
