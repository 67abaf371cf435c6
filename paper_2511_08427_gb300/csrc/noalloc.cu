// Matched adjoint that allocates no device memory.
//
// Some callers cannot let a library allocate device memory: code running inside a restricted
// allocator (a memory pool that owns the whole device), a framework that forbids allocation in a
// region, or real-time pipelines that must never call cudaMalloc after start-up. The regular entry
// points allocate on first use (per-geometry view tables; FP32 accumulation buffers for reduced
// precision storage). pyronn_adjoint_noalloc instead runs the atomic-scatter adjoint with its
// per-view ray table and its FP32 accumulator in the file-scope device arrays below, whose size is
// fixed when the library is loaded: every GPU that loads the library holds them until the process
// exits.
//
// All calls on a device share these arrays, and each call leaves its results in them: the
// accumulator is cleared at the start of every call. Calls whose work overlaps on the GPU (other
// streams, other threads) race on the arrays; serialise them, for example on one stream.
#include <cuda_runtime.h>

#include <mutex>

#include "device_common.cuh"

namespace pyronn {

constexpr int NOALLOC_MAX_VIEWS = 4096;
constexpr long long NOALLOC_MAX_ELEMS = 8LL * 1024 * 1024;   // FP32 accumulator: 32 MiB

static __device__ __align__(256) FpRec g_noalloc_views[NOALLOC_MAX_VIEWS];
static __device__ __align__(256) float g_noalloc_acc[NOALLOC_MAX_ELEMS];

namespace {

struct NoallocDevice {
    bool ready = false;
    FpRec *views = nullptr;   // device addresses of the arrays above on this device
    float *acc = nullptr;
};

constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[MAX_DEVICES];

// Once per device, with that device current: the host-side names of the arrays are stand-ins, not
// device addresses, so ask the runtime for their addresses on this device.
int noalloc_setup(int dev, NoallocDevice **out) {
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(PYRONN_INVALID_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoallocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        void *pv = nullptr, *pa = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&pv, g_noalloc_views);
        if (e != cudaSuccess)
            return set_error(PYRONN_CUDA_ERROR, "cudaGetSymbolAddress(view table): %s", cudaGetErrorString(e));
        e = cudaGetSymbolAddress(&pa, g_noalloc_acc);
        if (e != cudaSuccess)
            return set_error(PYRONN_CUDA_ERROR, "cudaGetSymbolAddress(accumulator): %s", cudaGetErrorString(e));
        d.views = (FpRec *)pv;
        d.acc = (float *)pa;
        d.ready = true;
    }
    *out = &d;
    return PYRONN_OK;
}

}  // namespace
}  // namespace pyronn

using namespace pyronn;

extern "C" PYRONN_API int pyronn_adjoint_noalloc(pyronn_geom_t g, const void *sino, void *vol, int dtype, int batch,
                                                 void *stream) {
    clear_error();
    if (!g) return set_error(PYRONN_INVALID_ARG, "null geometry");
    if (!sino || !vol) return set_error(PYRONN_INVALID_ARG, "null buffer");
    if ((((uintptr_t)sino) | ((uintptr_t)vol)) & 15u) return set_error(PYRONN_MISALIGNED, "buffers must be 16-byte aligned");
    if (dtype_size(dtype) == 0) return set_error(PYRONN_UNSUPPORTED_DTYPE, "unsupported dtype %d", dtype);
    if (batch < 1) return set_error(PYRONN_INVALID_ARG, "batch must be >= 1 (got %d)", batch);
    const long long nvox = (long long)g->nx * g->ny * g->nz;
    if (g->n_views > NOALLOC_MAX_VIEWS)
        return set_error(PYRONN_INVALID_ARG, "pyronn_adjoint_noalloc supports at most %d views (geometry has %d)",
                         NOALLOC_MAX_VIEWS, g->n_views);
    if (nvox * batch > NOALLOC_MAX_ELEMS)
        return set_error(PYRONN_INVALID_ARG,
                         "pyronn_adjoint_noalloc supports at most %lld voxels in total (volume %lld x batch %d)",
                         NOALLOC_MAX_ELEMS, nvox, batch);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(PYRONN_CUDA_ERROR, "cudaGetDevice: %s", cudaGetErrorString(e));
    NoallocDevice *d = nullptr;
    int rc = noalloc_setup(dev, &d);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemcpyAsync(d->views, g->fp_rec.data(), sizeof(FpRec) * (size_t)g->n_views, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_error(PYRONN_CUDA_ERROR, "view table copy: %s", cudaGetErrorString(e));
    OpParams p = make_params(g, batch);
    p.fp = d->views;
    p.bp = nullptr;
    p.flags = nullptr;
    p.views64 = nullptr;
    e = (cudaError_t)launch_adjoint_scatter_acc(p, sino, d->acc, vol, dtype, stream);
    if (e != cudaSuccess) return set_error(PYRONN_CUDA_ERROR, "adjoint launch: %s", cudaGetErrorString(e));
    return PYRONN_OK;
}
