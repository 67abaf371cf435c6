// Autotuner (the batched-launch pattern's "tile and brick shapes chosen by measurement"): times the
// candidate configurations of one operator of a geometry on the device with CUDA events and applies
// the fastest through the geometry's tuning knobs. Every candidate computes the same operator.
#include <cuda_runtime.h>

#include <cstring>

#include "pyronn_internal.h"

using namespace pyronn;

namespace {

struct Candidate {
    int a, b;   // op 0: slab depth, buffers; op 1: slab depth, pitch mode; op 2: brick depth, kernel variant
};

const Candidate FP_CANDIDATES[] = {{8, 2}, {8, 1}, {4, 2}, {4, 1}, {12, 1}, {16, 1}, {6, 1}};
const Candidate ADJ_CANDIDATES[] = {{8, 0}, {6, 0}, {5, 0}, {4, 0}, {6, 1}, {4, 1}, {3, 0}};
const Candidate BP_CANDIDATES[] = {{8, 2}, {4, 2}, {16, 2}, {8, 3}, {16, 3}};

int apply(pyronn_geom_t g, int op, const Candidate &c) {
    int rc = PYRONN_OK;
    if (op == 0) {
        if ((rc = pyronn_geom_set_tuning(g, PYRONN_TUNE_FP_DEPTH, c.a))) return rc;
        return pyronn_geom_set_tuning(g, PYRONN_TUNE_FP_BUFFERS, c.b);
    }
    if (op == 1) {
        if ((rc = pyronn_geom_set_tuning(g, PYRONN_TUNE_ADJ_DEPTH, c.a))) return rc;
        return pyronn_geom_set_tuning(g, PYRONN_TUNE_ADJ_PITCH, c.b);
    }
    if ((rc = pyronn_geom_set_tuning(g, PYRONN_TUNE_BP_BRICK_Z, c.a))) return rc;
    return pyronn_geom_set_variant(g, 2, c.b);
}

// Whether the candidate runs on the kernel it tunes (a depth whose boxes do not fit makes the library
// fall back to another kernel, which is not a candidate).
bool applicable(pyronn_geom_t g, int op, int dtype) {
    int cfg[20];
    if (op == 0) return pyronn_geom_fp_config(g, dtype, cfg) == PYRONN_OK && cfg[0] == 3;
    if (op == 1) return pyronn_geom_adjoint_config(g, cfg) == PYRONN_OK && cfg[0] == 3;
    return g->ndim == 3 && pyronn_geom_bp_config(g, dtype, cfg) == PYRONN_OK && cfg[0] == g->bp_variant;
}

int run(pyronn_geom_t g, int op, const void *in, void *out, int dtype, void *stream) {
    if (op == 0) return pyronn_fp(g, in, out, dtype, 1, stream);
    if (op == 1) return pyronn_adjoint(g, in, out, dtype, 1, stream);
    return pyronn_bp(g, in, out, dtype, 1, PYRONN_BP_PLAIN, stream);
}

}  // namespace

extern "C" PYRONN_API int pyronn_autotune(pyronn_geom_t g, int op, const void *in, void *out, int dtype, int repeats,
                                          void *stream, double *result) {
    clear_error();
    if (!g || !in || !out || !result) return set_error(PYRONN_INVALID_ARG, "null argument");
    if (op < 0 || op > 2) return set_error(PYRONN_INVALID_ARG, "unknown operator %d", op);
    if (repeats < 1 || repeats > 1000) return set_error(PYRONN_INVALID_ARG, "repeats %d out of [1, 1000]", repeats);
    if (dtype_size(dtype) == 0) return set_error(PYRONN_UNSUPPORTED_DTYPE, "unsupported dtype %d", dtype);
    for (int i = 0; i < 4; ++i) result[i] = 0.0;
    const Candidate *cand = op == 0 ? FP_CANDIDATES : (op == 1 ? ADJ_CANDIDATES : BP_CANDIDATES);
    const int n = op == 0 ? (int)(sizeof(FP_CANDIDATES) / sizeof(Candidate))
                          : (op == 1 ? (int)(sizeof(ADJ_CANDIDATES) / sizeof(Candidate))
                                     : (int)(sizeof(BP_CANDIDATES) / sizeof(Candidate)));
    // the knobs as they were: restored if no candidate applies
    Tuning before;
    int before_bp_variant = 0;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        before = g->tuning;
        before_bp_variant = g->bp_variant;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return set_error(PYRONN_CUDA_ERROR, "event creation failed");
    }
    int best = -1, timed = 0, rc = PYRONN_OK;
    float best_ms = 0.0f;
    for (int i = 0; i < n && rc == PYRONN_OK; ++i) {
        if ((rc = apply(g, op, cand[i]))) break;
        if (!applicable(g, op, dtype)) continue;
        if ((rc = run(g, op, in, out, dtype, stream))) break;   // warm-up (and first-use set-up)
        cudaEventRecord(e0, st);
        for (int r = 0; r < repeats && rc == PYRONN_OK; ++r) rc = run(g, op, in, out, dtype, stream);
        if (rc) break;
        cudaEventRecord(e1, st);
        cudaError_t ce = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce != cudaSuccess) {
            rc = set_error(PYRONN_CUDA_ERROR, "autotune timing: %s", cudaGetErrorString(ce));
            break;
        }
        ms /= (float)repeats;
        ++timed;
        if (best < 0 || ms < best_ms) {
            best = i;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != PYRONN_OK || best < 0) {
        std::lock_guard<std::mutex> lk(g->mu);
        g->tuning = before;
        g->bp_variant = before_bp_variant;
        g->adj_cfg_ready = 0;
        g->tma_ready[0] = g->tma_ready[1] = g->tma_ready[2] = 0;
        if (rc != PYRONN_OK) return rc;
        return set_error(PYRONN_INVALID_ARG, "no candidate configuration applies to this geometry and operator");
    }
    if ((rc = apply(g, op, cand[best]))) return rc;
    result[0] = best_ms;
    result[1] = cand[best].a;
    result[2] = cand[best].b;
    result[3] = timed;
    return PYRONN_OK;
}
