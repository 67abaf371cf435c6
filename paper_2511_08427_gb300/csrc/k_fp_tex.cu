// Texture-gather forward projector (same operator as fp_direct_kernel, Sec. 2.1). This is the
// paper's "texture interpolation" option (Sec. 2.1: faster, at the cost of an extra copy of the
// volume into a texture) without hardware filtering, whose 8-bit weight fractions would miss FP32
// parity: the texture unit only gathers texels, and the interpolation stays in FP32.
//
// Layout: every z plane of every batch item is a tile of (Nx + 2) x (Ny + 2) texels of one 2D gather
// texture (CUDA allows gathers on plain 2D arrays only); the two extra columns and rows of a tile are
// zero, and each item has an all-zero tile before and after its planes. A sample at index position
// (x, y, z) with floor (ix, iy, iz) needs texels ix .. ix + 1, iy .. iy + 1 of planes iz and iz + 1:
// two gathers at the tile origins of those planes. Samples of the conservative k range lie at most
// one index unit outside the support box (ix >= -2, ix <= Nx), so their texels are zero columns,
// zero rows, zero tiles or the texture border, never another plane's data.
//
// One thread per ray; no shared-memory staging, no block-wide synchronisation in the sample loop.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"

namespace pyronn {

constexpr int TEX_TU = 32, TEX_TV = 8, TEX_NT = TEX_TU * TEX_TV;

__device__ __forceinline__ void tex_floor_frac(float q, int &i, float &fl, float &f) {
    const float M = 12582912.0f;
    const float t = __fadd_rd(q, M);
    i = __float_as_int(t) - 0x4B400000;
    fl = t - M;
    f = q - fl;
}

// org[t] = gather coordinate of texel (0, 0) of tile t plus one (a gather at (X + 1, Y + 1) returns
// texels X .. X + 1, Y .. Y + 1), for the Nz + 2 tiles of batch item b_first + blockIdx.z / V.
template <typename T>
__global__ void __launch_bounds__(TEX_NT) fp_tex_kernel(OpParams p, cudaTextureObject_t tex,
                                                        const float2 *__restrict__ org, int b_first,
                                                        T *__restrict__ sino) {
    extern __shared__ float2 s_org[];
    const int view = blockIdx.z % p.n_views, b = blockIdx.z / p.n_views;
    const int ntile = p.vol.nz + 2;
    for (int t = threadIdx.x; t < ntile; t += TEX_NT) s_org[t] = org[(long long)(b_first + b) * ntile + t];
    __syncthreads();
    const int u = blockIdx.x * TEX_TU + (threadIdx.x & (TEX_TU - 1));
    const int v = blockIdx.y * TEX_TV + threadIdx.x / TEX_TU;
    if (u >= p.det.nu || v >= p.det.nv) return;
    const RayIdx r = ray_setup(p.fp[view], p.vol, (float)u, (float)v);
    int k0, k1;
    float acc = 0.0f;
    if (ray_k_range(r, p.vol, p.dt, k0, k1)) {
        const float hdt = 0.5f * p.dt;
        const float c0x = fmaf(hdt, r.dx, r.cx), c0y = fmaf(hdt, r.dy, r.cy), c0z = fmaf(hdt, r.dz, r.cz);
        const float stx = p.dt * r.dx, sty = p.dt * r.dy, stz = p.dt * r.dz;
        const int tmax = ntile - 1;
        float kf = (float)k0;
        for (int k = k0; k <= k1; ++k, kf += 1.0f) {
            const float qx = fmaf(kf, stx, c0x), qy = fmaf(kf, sty, c0y), qz = fmaf(kf, stz, c0z);
            int ix, iy, iz;
            float fx, fy, fz, ax, ay, az;
            tex_floor_frac(qx, ix, fx, ax);
            tex_floor_frac(qy, iy, fy, ay);
            tex_floor_frac(qz, iz, fz, az);
            const float2 o0 = s_org[min(max(iz + 1, 0), tmax)];
            const float2 o1 = s_org[min(max(iz + 2, 0), tmax)];
            const float4 g0 = tex2Dgather<float4>(tex, fx + o0.x, fy + o0.y, 0);
            const float4 g1 = tex2Dgather<float4>(tex, fx + o1.x, fy + o1.y, 0);
            // gather order: (x0, y1), (x1, y1), (x1, y0), (x0, y0)
            const float c00 = fmaf(ax, g0.z - g0.w, g0.w);
            const float c01 = fmaf(ax, g0.y - g0.x, g0.x);
            const float c10 = fmaf(ax, g1.z - g1.w, g1.w);
            const float c11 = fmaf(ax, g1.y - g1.x, g1.x);
            const float c0 = fmaf(ay, c01 - c00, c00);
            const float c1 = fmaf(ay, c11 - c10, c10);
            acc += fmaf(az, c1 - c0, c0);
        }
    }
    sino[(long long)b * p.sino_elems + ((long long)view * p.det.nv + v) * p.det.nu + u] = from_f32<T>(acc * p.dt);
}

// ---------------------------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------------------------

namespace {

struct TexLayout {
    int tw, th;        // tile width / height (texels)
    int cols, rows;    // tiles per row / rows of tiles
    int ntile;         // tiles (batch x (Nz + 2))
};

TexLayout tex_layout(const pyronn_geom *g, int batch) {
    TexLayout L{};
    L.tw = g->nx + 2;
    L.th = g->ny + 2;
    L.ntile = batch * (g->nz + 2);
    L.cols = std::max(1, (int)std::ceil(std::sqrt((double)L.ntile * L.th / L.tw)));
    L.rows = (L.ntile + L.cols - 1) / L.cols;
    return L;
}

}  // namespace

// The texture path applies to 3D FP32 volumes whose tiled array fits the device's gather limits.
bool fp_tex_usable(const pyronn_geom *g, int batch, int dtype) {
    if (dtype != PYRONN_F32 || g->ndim != 3) return false;
    static int maxw = -1, maxh = -1;
    if (maxw < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture2DGatherWidth, dev);
        cudaDeviceGetAttribute(&maxh, cudaDevAttrMaxTexture2DGatherHeight, dev);
    }
    const TexLayout L = tex_layout(g, batch);
    return (long long)L.cols * L.tw <= maxw && (long long)L.rows * L.th <= maxh;
}

// (Re)creates the geometry's tiled gather texture for `batch` FP32 volumes (all texels zero).
static int ensure_tex(pyronn_geom *g, int batch, cudaStream_t st) {
    if (g->tex_obj && g->tex_batch == batch) return 0;
    if (g->tex_obj) cudaDestroyTextureObject((cudaTextureObject_t)g->tex_obj);
    if (g->tex_arr) cudaFreeArray((cudaArray_t)g->tex_arr);
    if (g->d_tex_org) cudaFree(g->d_tex_org);
    g->tex_obj = 0;
    g->tex_arr = nullptr;
    g->d_tex_org = nullptr;
    g->tex_batch = 0;
    const TexLayout L = tex_layout(g, batch);
    const size_t W = (size_t)L.cols * L.tw, H = (size_t)L.rows * L.th;
    cudaChannelFormatDesc ch = cudaCreateChannelDesc<float>();
    cudaArray_t arr = nullptr;
    cudaError_t e = cudaMallocArray(&arr, &ch, W, H, cudaArrayTextureGather);
    if (e != cudaSuccess) return (int)e;
    float *zeros = nullptr;
    e = cudaMallocAsync(&zeros, sizeof(float) * W * H, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(zeros, 0, sizeof(float) * W * H, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DToArrayAsync(arr, 0, 0, zeros, sizeof(float) * W, sizeof(float) * W, H,
                                     cudaMemcpyDeviceToDevice, st);
    if (zeros) cudaFreeAsync(zeros, st);
    std::vector<float2> org((size_t)L.ntile);
    for (int t = 0; t < L.ntile; ++t)
        org[t] = make_float2((float)((t % L.cols) * L.tw + 1), (float)((t / L.cols) * L.th + 1));
    float2 *d_org = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d_org, sizeof(float2) * org.size());
    if (e == cudaSuccess) e = cudaMemcpy(d_org, org.data(), sizeof(float2) * org.size(), cudaMemcpyHostToDevice);
    cudaTextureObject_t obj = 0;
    if (e == cudaSuccess) {
        cudaResourceDesc rd{};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = arr;
        cudaTextureDesc td{};
        td.addressMode[0] = cudaAddressModeBorder;
        td.addressMode[1] = cudaAddressModeBorder;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        e = cudaCreateTextureObject(&obj, &rd, &td, nullptr);
    }
    if (e != cudaSuccess) {
        cudaFree(d_org);
        cudaFreeArray(arr);
        return (int)e;
    }
    g->tex_arr = arr;
    g->tex_obj = (unsigned long long)obj;
    g->d_tex_org = d_org;
    g->tex_batch = batch;
    return 0;
}

// Copies the volumes into their tiles and launches the projector (caller holds g->mu).
int launch_fp_tex(pyronn_geom *g, const OpParams &p, const void *vol, void *sino, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_tex(g, p.batch, st);
    if (rc) return rc;
    const TexLayout L = tex_layout(g, p.batch);
    const float *v = (const float *)vol;
    for (int b = 0; b < p.batch; ++b)
        for (int z = 0; z < g->nz; ++z) {
            const int t = b * (g->nz + 2) + 1 + z;
            cudaError_t e = cudaMemcpy2DToArrayAsync(
                (cudaArray_t)g->tex_arr, sizeof(float) * (size_t)(t % L.cols) * L.tw, (size_t)(t / L.cols) * L.th,
                v + (size_t)b * p.vol_elems + (size_t)z * g->nx * g->ny, sizeof(float) * g->nx, sizeof(float) * g->nx,
                g->ny, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return (int)e;
        }
    const size_t smem = sizeof(float2) * (size_t)(g->nz + 2);
    const int per_launch = 65535 / p.n_views > 0 ? 65535 / p.n_views : 1;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        const int nb = std::min(p.batch - b0, per_launch);
        dim3 grid(ceil_div(p.det.nu, TEX_TU), ceil_div(p.det.nv, TEX_TV), p.n_views * nb);
        fp_tex_kernel<float><<<grid, TEX_NT, smem, st>>>(p, (cudaTextureObject_t)g->tex_obj,
                                                          (const float2 *)g->d_tex_org, b0,
                                                          (float *)sino + (size_t)b0 * p.sino_elems);
    }
    return (int)cudaGetLastError();
}

}  // namespace pyronn
