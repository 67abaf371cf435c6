// Batched plans: several volumes, each with its own size and geometry, processed by one persistent
// launch per operator (items taken from a device work counter, larger items first).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "pyronn_internal.h"

using namespace pyronn;

struct pyronn_plan {
    int n = 0;
    int dtype = 0;
    int device = -1;
    std::vector<pyronn_geom *> geoms;   // caller order
    std::vector<FpTmaBox> cfg;          // per geometry, for dtype
    std::vector<int> order_fp, order_brick;
    int *d_counter = nullptr;           // three counters: FP, adjoint, BP
    int fp_grid = 0, adj_grid = 0, bp_grid = 0;
    size_t fp_smem = 0;
    // adjoint: slab-ordered (persistent, shared-memory boxes) where every geometry has a slab
    // configuration, else output-stationary bricks
    bool adj_slab = false;
    size_t adj_smem = 0;
    std::vector<AdjSlabCfg> acfg;
    float *d_acc = nullptr;             // FP32 accumulation volumes (BF16 / FP16 plans)
    std::vector<size_t> acc_off;
    unsigned char *d_vt = nullptr;      // y-fastest copies of the volumes whose x-march FP boxes use one
    std::vector<size_t> vt_off;         // byte offsets into d_vt (per geometry; unused without a copy)
};

namespace {

int cuda_err(cudaError_t e, const char *what) {
    return set_error(PYRONN_CUDA_ERROR, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

extern "C" {

int pyronn_plan_create(int n, const pyronn_geom_t *geoms, int dtype, pyronn_plan_t *out) {
    clear_error();
    if (!out || !geoms) return set_error(PYRONN_INVALID_ARG, "null argument");
    if (n < 1 || n > PLAN_MAX) return set_error(PYRONN_INVALID_ARG, "a plan holds 1 to %d geometries (got %d)", PLAN_MAX, n);
    if (dtype_size(dtype) == 0) return set_error(PYRONN_UNSUPPORTED_DTYPE, "unsupported dtype %d", dtype);
    pyronn_plan *P = new pyronn_plan();
    P->n = n;
    P->dtype = dtype;
    int rc = PYRONN_OK;
    for (int i = 0; i < n && !rc; ++i) {
        pyronn_geom *g = geoms[i];
        if (!g) rc = set_error(PYRONN_INVALID_ARG, "geometry %d is null", i);
        else if (g->ndim != 3) rc = set_error(PYRONN_INVALID_ARG, "geometry %d: batched plans take 3D geometries", i);
        else if ((long long)g->nx * g->ny * g->nz >= (1LL << 31))
            rc = set_error(PYRONN_INVALID_ARG, "geometry %d: volume too large", i);
        else if ((rc = ensure_device(g)) == PYRONN_OK) {
            // volumes whose rows are not a multiple of 16 bytes (depth 0) cannot use tensor copies; the
            // forward projection runs them through the per-geometry projector on the same stream
            FpTmaBox c = choose_fp_tma_box(g, dtype_size(dtype), g->tuning.fp_depth, g->tuning.fp_nbuf,
                                           g->tuning.fp_minb, g->tuning.fp_transpose == 0);
            c.packed = g->tuning.fp_packed == 1 ? 0 : (g->tuning.fp_packed == 2 ? 1 : 2);
            P->geoms.push_back(g);
            P->cfg.push_back(c);
        }
    }
    if (!rc) {
        for (int i = 1; i < n; ++i)
            if (P->geoms[i]->device != P->geoms[0]->device)
                rc = set_error(PYRONN_INVALID_ARG, "all geometries of a plan must live on one device");
    }
    if (rc) {
        delete P;
        return rc;
    }
    P->device = P->geoms[0]->device;
    // processing order: the longest rays (FP) / the most views per brick (adjoint, BP) first
    std::vector<double> cost_fp(n), cost_brick(n);
    for (int i = 0; i < n; ++i) {
        const pyronn_geom *g = P->geoms[i];
        cost_fp[i] = std::sqrt((g->nx * g->sx) * (g->nx * g->sx) + (g->ny * g->sy) * (g->ny * g->sy) +
                               (g->nz * g->sz) * (g->nz * g->sz)) / g->dt;
        cost_brick[i] = (double)g->n_views * (double)g->nu * g->nv / ((double)g->nx * g->ny);
    }
    P->order_fp.resize(n);
    P->order_brick.resize(n);
    std::iota(P->order_fp.begin(), P->order_fp.end(), 0);
    std::iota(P->order_brick.begin(), P->order_brick.end(), 0);
    std::stable_sort(P->order_fp.begin(), P->order_fp.end(), [&](int a, int b) { return cost_fp[a] > cost_fp[b]; });
    std::stable_sort(P->order_brick.begin(), P->order_brick.end(),
                     [&](int a, int b) { return cost_brick[a] > cost_brick[b]; });
    // persistent grids from the occupancy of each kernel
    for (int i = 0; i < n; ++i)
        if (P->cfg[i].depth > 0)
            P->fp_smem = std::max(P->fp_smem,
                                  (size_t)P->cfg[i].nbuf * dtype_size(dtype) * (size_t)P->cfg[i].buf_elems + 128);
    int sms = 0, occ = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
    if (e != cudaSuccess) {
        delete P;
        return cuda_err(e, "device attributes");
    }
    if (P->fp_smem == 0) P->fp_smem = 128;
    if ((e = (cudaError_t)fp_tma_batched_occupancy(dtype, P->fp_smem, &occ)) != cudaSuccess) {
        delete P;
        return cuda_err(e, "forward-projector occupancy");
    }
    P->fp_grid = sms * std::max(occ, 1);
    if ((e = (cudaError_t)adjoint_brick_batched_occupancy(&occ)) != cudaSuccess) {
        delete P;
        return cuda_err(e, "adjoint occupancy");
    }
    P->adj_grid = sms * std::max(occ, 1);
    if ((e = (cudaError_t)bp_brick_batched_occupancy(&occ)) != cudaSuccess) {
        delete P;
        return cuda_err(e, "back-projector occupancy");
    }
    P->bp_grid = sms * std::max(occ, 1);
    // slab-ordered adjoint for the whole plan if every geometry has a valid slab configuration
    P->adj_slab = true;
    size_t acc_total = 0;
    int max_box = 0, max_slabs = 0;
    for (int i = 0; i < n; ++i) {
        const AdjSlabCfg &c = geom_adj_cfg(P->geoms[i]);
        P->acfg.push_back(c);
        P->acc_off.push_back(acc_total);
        acc_total += (size_t)P->geoms[i]->nx * P->geoms[i]->ny * P->geoms[i]->nz;
        if (!c.valid || (P->geoms[i]->adj_variant != 0 && P->geoms[i]->adj_variant != 3)) P->adj_slab = false;
        max_box = std::max(max_box, c.box_cap);
        max_slabs = std::max(max_slabs, c.max_slabs);
    }
    // the batched kernel puts every volume's slab table after the largest box
    P->adj_smem = adjoint_slab_smem_bytes(max_box, max_slabs);
    if (P->adj_slab) {
        if ((e = (cudaError_t)adjoint_slab_batched_occupancy(P->adj_smem, &occ)) != cudaSuccess) {
            delete P;
            return cuda_err(e, "slab adjoint occupancy");
        }
        P->adj_grid = sms * std::max(occ, 1);
        if (dtype != PYRONN_F32) {
            e = cudaMalloc(&P->d_acc, sizeof(float) * acc_total);
            if (e != cudaSuccess) {
                delete P;
                return set_error(PYRONN_OOM, "adjoint accumulation volumes: %s", cudaGetErrorString(e));
            }
        }
    }
    // y-fastest copies for the forward projector (256-byte aligned, one per volume that uses one)
    size_t vt_total = 0;
    for (int i = 0; i < n; ++i) {
        P->vt_off.push_back(vt_total);
        const pyronn_geom *g = P->geoms[i];
        if (P->cfg[i].depth > 0 && P->cfg[i].xt)
            vt_total += (dtype_size(dtype) * (size_t)g->nx * g->ny * g->nz + 255) / 256 * 256;
    }
    if (vt_total > 0) {
        e = cudaMalloc(&P->d_vt, vt_total);
        if (e != cudaSuccess) {
            if (P->d_acc) cudaFree(P->d_acc);
            delete P;
            return set_error(PYRONN_OOM, "transposed volumes: %s", cudaGetErrorString(e));
        }
    }
    e = cudaMalloc(&P->d_counter, 4 * sizeof(int));
    if (e != cudaSuccess) {
        if (P->d_acc) cudaFree(P->d_acc);
        if (P->d_vt) cudaFree(P->d_vt);
        delete P;
        return set_error(PYRONN_OOM, "work counters: %s", cudaGetErrorString(e));
    }
    *out = P;
    return PYRONN_OK;
}

int pyronn_plan_destroy(pyronn_plan_t P) {
    clear_error();
    if (!P) return PYRONN_OK;
    if (P->d_counter) cudaFree(P->d_counter);
    if (P->d_acc) cudaFree(P->d_acc);
    if (P->d_vt) cudaFree(P->d_vt);
    delete P;
    return PYRONN_OK;
}

int pyronn_plan_info(pyronn_plan_t P, int *n, int64_t *items_fp, int64_t *items_brick, int *grids) {
    clear_error();
    if (!P) return set_error(PYRONN_INVALID_ARG, "null plan");
    if (n) *n = P->n;
    long long ifp = 0, ib = 0;
    for (int i = 0; i < P->n; ++i) {
        const pyronn_geom *g = P->geoms[i];
        ifp += (long long)g->n_views * ((g->nu + FP_TILE_U - 1) / FP_TILE_U) * ((g->nv + FP_TILE_V - 1) / FP_TILE_V);
        ib += (long long)((g->nx + 15) / 16) * ((g->ny + 15) / 16) * ((g->nz + 15) / 16);
    }
    if (items_fp) *items_fp = ifp;
    if (items_brick) *items_brick = ib;
    if (grids) {
        grids[0] = P->fp_grid;
        grids[1] = P->adj_grid;
        grids[2] = P->bp_grid;
    }
    return PYRONN_OK;
}

static int check_ptrs(const pyronn_plan *P, const void *const *a, const void *const *b) {
    if (!a || !b) return set_error(PYRONN_INVALID_ARG, "null pointer array");
    for (int i = 0; i < P->n; ++i) {
        if (!a[i] || !b[i]) return set_error(PYRONN_INVALID_ARG, "buffer %d is null", i);
        if ((((uintptr_t)a[i]) | ((uintptr_t)b[i])) & 15u)
            return set_error(PYRONN_MISALIGNED, "buffer %d is not 16-byte aligned", i);
    }
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != P->device) return set_error(PYRONN_INVALID_ARG, "the plan lives on device %d, current is %d", P->device, dev);
    return PYRONN_OK;
}

int pyronn_plan_fp(pyronn_plan_t P, const void *const *vols, void *const *sinos, void *stream) {
    clear_error();
    if (!P) return set_error(PYRONN_INVALID_ARG, "null plan");
    int rc = check_ptrs(P, vols, (const void *const *)sinos);
    if (rc) return rc;
    PlanLaunch L{};
    L.n = 0;
    L.counter = P->d_counter + 0;
    long long acc = 0;
    for (int k = 0; k < P->n; ++k) {
        const int i = P->order_fp[k];
        pyronn_geom *g = P->geoms[i];
        if (P->cfg[i].depth <= 0) {
            rc = pyronn_fp(g, vols[i], sinos[i], P->dtype, 1, stream);
            if (rc) return rc;
            continue;
        }
        PlanVolume &V = L.v[L.n];
        V.p = make_params(g, 1);
        V.cfg = P->cfg[i];
        V.in = vols[i];
        V.out = sinos[i];
        V.vt = V.cfg.xt ? (void *)(P->d_vt + P->vt_off[i]) : nullptr;
        V.ntx = (g->nu + FP_TILE_U - 1) / FP_TILE_U;
        V.nty = (g->nv + FP_TILE_V - 1) / FP_TILE_V;
        V.ntz = 1;
        acc += (long long)g->n_views * V.ntx * V.nty;
        L.item_end[L.n++] = acc;
    }
    if (L.n == 0) return PYRONN_OK;
    int e = launch_fp_tma_batched(L, P->dtype, P->fp_grid, P->fp_smem, stream);
    return e ? cuda_err((cudaError_t)e, "batched forward projection") : PYRONN_OK;
}

static int brick_launch(pyronn_plan_t P, const void *const *sinos, void *const *vols, int weight, void *stream,
                        int op) {
    clear_error();
    if (!P) return set_error(PYRONN_INVALID_ARG, "null plan");
    int rc = check_ptrs(P, sinos, (const void *const *)vols);
    if (rc) return rc;
    if (op == 2 && weight != PYRONN_BP_PLAIN && weight != PYRONN_BP_INV_W2)
        return set_error(PYRONN_INVALID_ARG, "unknown back-projection weight %d", weight);
    PlanLaunch L{};
    L.n = P->n;
    L.counter = P->d_counter + op;
    const int bz = op == 1 ? 16 : 8;   // adjoint bricks 16^3, back-projection bricks 16 x 16 x 8
    long long acc = 0;
    for (int k = 0; k < P->n; ++k) {
        const int i = P->order_brick[k];
        const pyronn_geom *g = P->geoms[i];
        PlanVolume &V = L.v[k];
        V.p = make_params(g, 1);
        V.p.weight = weight;
        V.in = sinos[i];
        V.out = vols[i];
        V.ntx = (g->nx + 15) / 16;
        V.nty = (g->ny + 15) / 16;
        V.ntz = (g->nz + bz - 1) / bz;
        acc += (long long)V.ntx * V.nty * V.ntz;
        L.item_end[k] = acc;
    }
    int e = op == 1 ? launch_adjoint_brick_batched(L, P->dtype, P->adj_grid, stream)
                    : launch_bp_brick_batched(L, P->dtype, weight, P->bp_grid, stream);
    return e ? cuda_err((cudaError_t)e, op == 1 ? "batched adjoint" : "batched back-projection") : PYRONN_OK;
}

int pyronn_plan_adjoint(pyronn_plan_t P, const void *const *sinos, void *const *vols, void *stream) {
    if (!P || !P->adj_slab) return brick_launch(P, sinos, vols, PYRONN_BP_PLAIN, stream, 1);
    clear_error();
    int rc = check_ptrs(P, sinos, (const void *const *)vols);
    if (rc) return rc;
    // items (view, 32 x 32 detector tile), volumes with the longest rays first
    PlanLaunch L{};
    L.n = P->n;
    L.counter = P->d_counter + 1;
    long long acc = 0;
    for (int k = 0; k < P->n; ++k) {
        const int i = P->order_fp[k];
        pyronn_geom *g = P->geoms[i];
        PlanVolume &V = L.v[k];
        V.p = make_params(g, 1);
        V.acfg = P->acfg[i];
        V.in = sinos[i];
        V.out = vols[i];
        V.acc = P->dtype == PYRONN_F32 ? (float *)vols[i] : P->d_acc + P->acc_off[i];
        V.ntx = (g->nu + 31) / 32;
        V.nty = (g->nv + 31) / 32;
        V.ntz = 1;
        acc += (long long)g->n_views * V.ntx * V.nty;
        L.item_end[k] = acc;
    }
    const int e = launch_adjoint_slab_batched(L, P->dtype, P->adj_grid, P->adj_smem, stream);
    return e ? cuda_err((cudaError_t)e, "batched adjoint") : PYRONN_OK;
}

int pyronn_plan_bp(pyronn_plan_t P, const void *const *sinos, void *const *vols, int weight, void *stream) {
    return brick_launch(P, sinos, vols, weight, stream, 2);
}

}  // extern "C"
