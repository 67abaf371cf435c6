// Hardware-filtered texture forward projector (opt-in FP variant 5): the paper's "texture
// interpolation" option (Sec. 2.1: faster than kernel interpolation, but it needs an extra copy of the
// volume) with the texture unit doing the trilinear interpolation.
//
// The volume is copied into a geometry-owned 3D texture array (FP32, or half floats for FP16 storage)
// with border addressing (texels outside the grid read zero) and linear filtering; sample k of a ray at
// index position q reads tex3D(q + 1/2), texel i having its centre at coordinate i + 1/2. That is the
// library's hat-function interpolant with zero padding, except that the texture unit weighs the eight
// texels with fractions of 8 fractional bits: each weight is off by up to 2^-9, so projections carry a
// relative error of the order of 1e-3 (measured against the FP64 oracle in the tests) instead of the
// FP32 path's 1e-6. It computes only the forward projection; the autograd backward of a projection is
// the matched adjoint of the exact operator whichever projector ran.
//
// One thread per ray, samples unrolled by four so that four fetches are in flight per thread. Grid:
// tile columns fastest, then views, then tile rows (the tiles of one detector row band in consecutive
// views read one band of the volume, which stays in the texture cache and L2).
#include <algorithm>

#include "device_common.cuh"

namespace pyronn {

constexpr int TXF_TU = 32, TXF_TV = 8, TXF_NT = TXF_TU * TXF_TV;

template <typename T>
__global__ void __launch_bounds__(TXF_NT) fp_texf_kernel(OpParams p, cudaTextureObject_t tex, T *__restrict__ sino) {
    const int view = blockIdx.y;
    const int u = blockIdx.x * TXF_TU + (threadIdx.x & (TXF_TU - 1));
    const int v = blockIdx.z * TXF_TV + threadIdx.x / TXF_TU;
    if (u >= p.det.nu || v >= p.det.nv) return;
    const RayIdx r = ray_setup(p.fp[view], p.vol, (float)u, (float)v);
    int k0, k1;
    float acc = 0.0f;
    if (ray_k_range(r, p.vol, p.dt, k0, k1)) {
        const float hdt = 0.5f * p.dt;
        // texture coordinates of sample k: index position + 1/2
        const float c0x = fmaf(hdt, r.dx, r.cx) + 0.5f, c0y = fmaf(hdt, r.dy, r.cy) + 0.5f;
        const float c0z = fmaf(hdt, r.dz, r.cz) + 0.5f;
        const float stx = p.dt * r.dx, sty = p.dt * r.dy, stz = p.dt * r.dz;
        float kf = (float)k0;
        const int n = k1 - k0 + 1;
        int i = 0;
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
        for (; i + 3 < n; i += 4, kf += 4.0f) {
            const float k1f = kf + 1.0f, k2f = kf + 2.0f, k3f = kf + 3.0f;
            a0 += tex3D<float>(tex, fmaf(kf, stx, c0x), fmaf(kf, sty, c0y), fmaf(kf, stz, c0z));
            a1 += tex3D<float>(tex, fmaf(k1f, stx, c0x), fmaf(k1f, sty, c0y), fmaf(k1f, stz, c0z));
            a2 += tex3D<float>(tex, fmaf(k2f, stx, c0x), fmaf(k2f, sty, c0y), fmaf(k2f, stz, c0z));
            a3 += tex3D<float>(tex, fmaf(k3f, stx, c0x), fmaf(k3f, sty, c0y), fmaf(k3f, stz, c0z));
        }
        for (; i < n; ++i, kf += 1.0f) a0 += tex3D<float>(tex, fmaf(kf, stx, c0x), fmaf(kf, sty, c0y), fmaf(kf, stz, c0z));
        acc = (a0 + a1) + (a2 + a3);
    }
    sino[(long long)view * p.det.nv * p.det.nu + (long long)v * p.det.nu + u] = from_f32<T>(acc * p.dt);
}

bool fp_texf_usable(const pyronn_geom *g, int dtype) {
    if (g->ndim != 3 || (dtype != PYRONN_F32 && dtype != PYRONN_F16)) return false;
    int dev = 0, w = 0, h = 0, d = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&w, cudaDevAttrMaxTexture3DWidth, dev);
    cudaDeviceGetAttribute(&h, cudaDevAttrMaxTexture3DHeight, dev);
    cudaDeviceGetAttribute(&d, cudaDevAttrMaxTexture3DDepth, dev);
    return g->nx <= w && g->ny <= h && g->nz <= d;
}

// (Re)creates the geometry's filtered 3D texture for element type dtype (caller holds g->mu).
static int ensure_texf(pyronn_geom *g, int dtype) {
    if (g->texf_obj && g->texf_dtype == dtype) return 0;
    if (g->texf_obj) cudaDestroyTextureObject((cudaTextureObject_t)g->texf_obj);
    if (g->texf_arr) cudaFreeArray((cudaArray_t)g->texf_arr);
    g->texf_obj = 0;
    g->texf_arr = nullptr;
    g->texf_dtype = -1;
    const cudaChannelFormatDesc ch = dtype == PYRONN_F16 ? cudaCreateChannelDescHalf() : cudaCreateChannelDesc<float>();
    cudaArray_t arr = nullptr;
    cudaError_t e = cudaMalloc3DArray(&arr, &ch, make_cudaExtent(g->nx, g->ny, g->nz));
    if (e != cudaSuccess) return (int)e;
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = arr;
    cudaTextureDesc td{};
    for (int a = 0; a < 3; ++a) td.addressMode[a] = cudaAddressModeBorder;
    td.filterMode = cudaFilterModeLinear;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    cudaTextureObject_t obj = 0;
    e = cudaCreateTextureObject(&obj, &rd, &td, nullptr);
    if (e != cudaSuccess) {
        cudaFreeArray(arr);
        return (int)e;
    }
    g->texf_arr = arr;
    g->texf_obj = (unsigned long long)obj;
    g->texf_dtype = dtype;
    return 0;
}

// Copies each volume of the batch into the texture and projects it (caller holds g->mu). The copy of
// item b + 1 is ordered after the projection of item b on the stream.
int launch_fp_texf(pyronn_geom *g, const OpParams &p, const void *vol, void *sino, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_texf(g, dtype);
    if (rc) return rc;
    const size_t es = dtype_size(dtype);
    const int ntv = ceil_div(p.det.nv, TXF_TV);
    const long long view_elems = (long long)p.det.nv * p.det.nu;
    for (int b = 0; b < p.batch; ++b) {
        cudaMemcpy3DParms cp{};
        cp.srcPtr = make_cudaPitchedPtr(const_cast<char *>((const char *)vol + es * (size_t)b * p.vol_elems),
                                        es * (size_t)g->nx, g->nx, g->ny);
        cp.dstArray = (cudaArray_t)g->texf_arr;
        cp.extent = make_cudaExtent(g->nx, g->ny, g->nz);
        cp.kind = cudaMemcpyDeviceToDevice;
        cudaError_t e = cudaMemcpy3DAsync(&cp, st);
        if (e != cudaSuccess) return (int)e;
        for (int v0 = 0; v0 < p.n_views; v0 += 65535) {
            const int nvw = std::min(p.n_views - v0, 65535);
            OpParams q = p;
            q.fp = p.fp + v0;
            q.n_views = nvw;
            dim3 grid(ceil_div(p.det.nu, TXF_TU), nvw, ntv);
            const long long off = (long long)b * p.sino_elems + v0 * view_elems;
            if (dtype == PYRONN_F16)
                fp_texf_kernel<__half><<<grid, TXF_NT, 0, st>>>(q, (cudaTextureObject_t)g->texf_obj,
                                                               (__half *)sino + off);
            else
                fp_texf_kernel<float><<<grid, TXF_NT, 0, st>>>(q, (cudaTextureObject_t)g->texf_obj,
                                                              (float *)sino + off);
        }
    }
    return (int)cudaGetLastError();
}

}  // namespace pyronn
