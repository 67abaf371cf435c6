// C ABI of the operators: argument validation, lazy device set-up and dispatch to the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "pyronn_internal.h"

using namespace pyronn;

namespace pyronn {

const AdjSlabCfg &geom_adj_cfg(pyronn_geom *g) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (!g->adj_cfg_ready) {
        g->adj_cfg = choose_adj_slab_cfg(g);
        g->adj_cfg_ready = 1;
    }
    return g->adj_cfg;
}

}  // namespace pyronn

namespace {

int check_ptr(const void *p, const char *what) {
    if (!p) return set_error(PYRONN_INVALID_ARG, "%s is null", what);
    if (((uintptr_t)p) & 15u) return set_error(PYRONN_MISALIGNED, "%s is not 16-byte aligned", what);
    return PYRONN_OK;
}

int common_checks(pyronn_geom_t g, int dtype, int batch) {
    if (!g) return set_error(PYRONN_INVALID_ARG, "null geometry");
    if (dtype_size(dtype) == 0) return set_error(PYRONN_UNSUPPORTED_DTYPE, "unsupported dtype %d", dtype);
    if (batch < 1) return set_error(PYRONN_INVALID_ARG, "batch must be >= 1 (got %d)", batch);
    long long nvox = (long long)g->nx * g->ny * g->nz;
    long long nsino = (long long)g->nu * g->nv * g->n_views;
    if (nvox >= (1LL << 31) || (long long)g->nu * g->nv >= (1LL << 31))
        return set_error(PYRONN_INVALID_ARG, "volume or detector too large for 32-bit in-volume indexing");
    if (nsino * batch <= 0 || nvox * batch <= 0) return set_error(PYRONN_INVALID_ARG, "empty operand");
    return PYRONN_OK;   // the device tables are set up by the caller once every argument has been checked
}

int cuda_rc(int e, const char *what) {
    if (e == 0) return PYRONN_OK;
    return set_error(PYRONN_CUDA_ERROR, "%s: %s", what, cudaGetErrorString((cudaError_t)e));
}

int ensure_scratch(pyronn_geom_t g, size_t bytes) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->scratch_bytes >= bytes) return PYRONN_OK;
    if (g->d_scratch) cudaFree(g->d_scratch);
    g->d_scratch = nullptr;
    g->scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&g->d_scratch, bytes);
    if (e != cudaSuccess) return set_error(PYRONN_OOM, "scratch allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
    g->scratch_bytes = bytes;
    return PYRONN_OK;
}

// Grows a geometry-owned device buffer to at least `bytes`.
int ensure_buffer(pyronn_geom_t g, void **buf, size_t *cur, size_t bytes, const char *what) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (*cur >= bytes) return PYRONN_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *cur = 0;
    cudaError_t e = cudaMalloc(buf, bytes);
    if (e != cudaSuccess) return set_error(PYRONN_OOM, "%s allocation of %zu bytes: %s", what, bytes, cudaGetErrorString(e));
    *cur = bytes;
    return PYRONN_OK;
}

int ensure_stage(pyronn_geom_t g, size_t in_bytes, size_t out_bytes) {
    std::lock_guard<std::mutex> lk(g->mu);
    cudaError_t e = cudaSuccess;
    if (g->stage_in_bytes < in_bytes) {
        cudaFree(g->d_stage_in);
        g->d_stage_in = nullptr;
        g->stage_in_bytes = 0;
        e = cudaMalloc(&g->d_stage_in, in_bytes);
        if (e != cudaSuccess) return set_error(PYRONN_OOM, "staging allocation: %s", cudaGetErrorString(e));
        g->stage_in_bytes = in_bytes;
    }
    if (g->stage_out_bytes < out_bytes) {
        cudaFree(g->d_stage_out);
        g->d_stage_out = nullptr;
        g->stage_out_bytes = 0;
        e = cudaMalloc(&g->d_stage_out, out_bytes);
        if (e != cudaSuccess) return set_error(PYRONN_OOM, "staging allocation: %s", cudaGetErrorString(e));
        g->stage_out_bytes = out_bytes;
    }
    return PYRONN_OK;
}

const FpSlabCfg &fp_cfg(pyronn_geom_t g) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (!g->fp_cfg_ready) {
        g->fp_cfg = choose_fp_slab_cfg(g);
        g->fp_cfg_ready = 1;
    }
    return g->fp_cfg;
}

const AdjSlabCfg &adj_cfg(pyronn_geom_t g) { return geom_adj_cfg(g); }

const FpTmaBox &tma_cfg(pyronn_geom_t g, int dtype) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (!g->tma_ready[dtype]) {
        g->tma_cfg[dtype] = choose_fp_tma_box(g, dtype_size(dtype), g->tuning.fp_depth, g->tuning.fp_nbuf,
                                              g->tuning.fp_minb, g->tuning.fp_transpose == 0);
        g->tma_cfg[dtype].packed = g->tuning.fp_packed == 1 ? 0 : (g->tuning.fp_packed == 2 ? 1 : 2);
        g->tma_ready[dtype] = 1;
    }
    return g->tma_cfg[dtype];
}

}  // namespace

extern "C" {

int pyronn_fp(pyronn_geom_t g, const void *vol, void *sino, int dtype, int batch, void *stream) {
    clear_error();
    int rc = common_checks(g, dtype, batch);
    if (rc) return rc;
    if ((rc = check_ptr(vol, "vol")) || (rc = check_ptr(sino, "sino"))) return rc;
    if ((rc = ensure_device(g))) return rc;
    OpParams p = make_params(g, batch);
    if (g->fp_variant == 1)
        return cuda_rc(launch_fp_direct(p, vol, sino, dtype, stream), "forward projection launch");
    if (g->fp_variant == 4 && fp_tex_usable(g, batch, dtype)) {
        std::lock_guard<std::mutex> lk(g->mu);
        return cuda_rc(launch_fp_tex(g, p, vol, sino, stream), "forward projection launch");
    }
    if (g->fp_variant == 5 && fp_texf_usable(g, dtype)) {
        std::lock_guard<std::mutex> lk(g->mu);
        return cuda_rc(launch_fp_texf(g, p, vol, sino, dtype, stream), "forward projection launch");
    }
    if (g->fp_variant == 0 || g->fp_variant >= 3) {
        const FpTmaBox &tb = tma_cfg(g, dtype);
        if (tb.depth > 0) {
            if (tb.xt) {
                const size_t bytes = dtype_size(dtype) * (size_t)p.vol_elems * (size_t)batch;
                if ((rc = ensure_buffer(g, &g->d_vol_t, &g->vol_t_bytes, bytes, "transposed volume"))) return rc;
            }
            return cuda_rc(launch_fp_tma(p, tb, vol, g->d_vol_t, sino, dtype, stream), "forward projection launch");
        }
    }
    return cuda_rc(launch_fp(p, fp_cfg(g), vol, sino, dtype, stream), "forward projection launch");
}

int pyronn_geom_fp_config(pyronn_geom_t g, int dtype, int *out) {
    clear_error();
    if (!g || !out) return set_error(PYRONN_INVALID_ARG, "null argument");
    if (dtype_size(dtype) == 0) return set_error(PYRONN_UNSUPPORTED_DTYPE, "unsupported dtype %d", dtype);
    for (int i = 0; i < 20; ++i) out[i] = 0;
    const FpTmaBox &tb = tma_cfg(g, dtype);
    const FpSlabCfg &sc = fp_cfg(g);
    int kernel = 1;
    if (g->fp_variant == 1) kernel = 1;
    else if (g->fp_variant == 4 && fp_tex_usable(g, 1, dtype)) kernel = 4;
    else if (g->fp_variant == 5 && fp_texf_usable(g, dtype)) kernel = 5;
    else if ((g->fp_variant == 0 || g->fp_variant >= 3) && tb.depth > 0) kernel = 3;
    else if (sc.valid) kernel = 2;
    out[0] = kernel;
    out[1] = kernel == 3 ? tb.depth : sc.depth;
    out[2] = kernel == 3 ? tb.guard : sc.guard;
    out[3] = tb.slab0;
    for (int m = 0; m < 3; ++m) {
        out[4 + 3 * m] = tb.bx[m];
        out[5 + 3 * m] = tb.by[m];
        out[6 + 3 * m] = tb.bz[m];
    }
    out[13] = tb.buf_elems;
    out[14] = kernel == 3 ? (int)((size_t)tb.nbuf * dtype_size(dtype) * (size_t)tb.buf_elems + 128)
                          : (kernel == 2 ? (int)(sizeof(float) * (size_t)sc.smem_floats) : 0);
    out[15] = sc.smem_floats;
    out[16] = kernel == 3 ? tb.xt : 0;
    return PYRONN_OK;
}

int pyronn_geom_adjoint_config(pyronn_geom_t g, int *out) {
    clear_error();
    if (!g || !out) return set_error(PYRONN_INVALID_ARG, "null argument");
    const AdjSlabCfg &ac = adj_cfg(g);
    int kernel = g->adj_variant == 1 ? 1 : 2;
    if ((g->adj_variant == 0 || g->adj_variant == 3) && ac.valid) kernel = 3;
    for (int i = 0; i < 8; ++i) out[i] = 0;
    out[0] = kernel;
    out[1] = ac.depth;
    out[2] = ac.guard;
    out[3] = ac.box_cap;
    out[4] = ac.xpad;
    out[5] = ac.max_slabs;
    out[6] = ac.ypad;
    return PYRONN_OK;
}

int pyronn_geom_bp_config(pyronn_geom_t g, int dtype, int *out) {
    clear_error();
    if (!g || !out) return set_error(PYRONN_INVALID_ARG, "null argument");
    if (dtype_size(dtype) == 0) return set_error(PYRONN_UNSUPPORTED_DTYPE, "unsupported dtype %d", dtype);
    for (int i = 0; i < 8; ++i) out[i] = 0;
    int kernel = g->bp_variant == 1 ? 1 : 2;
    if ((g->bp_variant == 3 || g->bp_variant == 0) && bp_tma_usable(g, dtype)) kernel = 3;
    out[0] = kernel;
    out[1] = kernel == 3 ? g->bpt_cfg[dtype][0] : 0;
    out[2] = kernel == 3 ? g->bpt_cfg[dtype][1] : 0;
    out[3] = g->ndim == 2 ? 1 : (kernel == 3 ? g->bpt_cfg[dtype][5] : bp_brick_depth(g->tuning.bp_brick_z, g->nz));
    out[4] = kernel == 3 ? g->bpt_cfg[dtype][3] : 0;
    out[5] = kernel == 3 ? g->bpt_cfg[dtype][4] : 0;
    return PYRONN_OK;
}

int pyronn_geom_set_tuning(pyronn_geom_t g, int param, int value) {
    clear_error();
    if (!g) return set_error(PYRONN_INVALID_ARG, "null geometry");
    std::lock_guard<std::mutex> lk(g->mu);
    switch (param) {
        case PYRONN_TUNE_FP_DEPTH:
            if (value < 0 || value > 64) return set_error(PYRONN_INVALID_ARG, "slab depth %d out of [0, 64]", value);
            g->tuning.fp_depth = value;
            break;
        case PYRONN_TUNE_FP_BUFFERS:
            if (value < 0 || value > 2) return set_error(PYRONN_INVALID_ARG, "buffer count %d out of [0, 2]", value);
            g->tuning.fp_nbuf = value;
            break;
        case PYRONN_TUNE_FP_CTAS_PER_SM:
            if (value != 0 && value != 2 && value != 3 && value != 4)
                return set_error(PYRONN_INVALID_ARG, "CTAs per SM must be 0 (automatic), 2, 3 or 4 (got %d)", value);
            g->tuning.fp_minb = value;
            break;
        case PYRONN_TUNE_ADJ_PITCH:
            if (value < 0 || value > 2) return set_error(PYRONN_INVALID_ARG, "pitch mode %d out of [0, 2]", value);
            g->tuning.adj_pitch = value;
            g->adj_cfg_ready = 0;
            break;
        case PYRONN_TUNE_FP_TRANSPOSE:
            if (value < 0 || value > 1) return set_error(PYRONN_INVALID_ARG, "transpose mode %d out of [0, 1]", value);
            g->tuning.fp_transpose = value;
            break;
        case PYRONN_TUNE_ADJ_ACCUM:
            if (value < 0 || value > 2) return set_error(PYRONN_INVALID_ARG, "accumulation mode %d out of [0, 2]", value);
            g->tuning.adj_accum = value;
            g->adj_cfg_ready = 0;
            break;
        case PYRONN_TUNE_ADJ_DEPTH:
            if (value != 0 && (value < 2 || value > 16))
                return set_error(PYRONN_INVALID_ARG, "adjoint slab depth must be 0 (automatic) or in [2, 16] (got %d)", value);
            g->tuning.adj_depth = value;
            g->adj_cfg_ready = 0;
            break;
        case PYRONN_TUNE_ADJ_LANES:
            if (value < 0 || value > 2) return set_error(PYRONN_INVALID_ARG, "lane mapping %d out of [0, 2]", value);
            g->tuning.adj_lanes = value;
            g->adj_cfg_ready = 0;
            break;
        case PYRONN_TUNE_FP_PACKED:
            if (value < 0 || value > 3) return set_error(PYRONN_INVALID_ARG, "packed mode %d out of [0, 3]", value);
            g->tuning.fp_packed = value;
            break;
        case PYRONN_TUNE_BP_BRICK_Z:
            if (value != 0 && value != 4 && value != 8 && value != 16)
                return set_error(PYRONN_INVALID_ARG, "brick depth must be 0 (automatic), 4, 8 or 16 (got %d)", value);
            g->tuning.bp_brick_z = value;
            break;
        default:
            return set_error(PYRONN_INVALID_ARG, "unknown tuning parameter %d", param);
    }
    g->tma_ready[0] = g->tma_ready[1] = g->tma_ready[2] = 0;
    return PYRONN_OK;
}

int pyronn_geom_set_variant(pyronn_geom_t g, int op, int variant) {
    clear_error();
    if (!g) return set_error(PYRONN_INVALID_ARG, "null geometry");
    if (op < 0 || op > 2) return set_error(PYRONN_INVALID_ARG, "unknown operator %d", op);
    const int vmax = op == 0 ? 5 : 3;
    if (variant < 0 || variant > vmax) return set_error(PYRONN_INVALID_ARG, "unknown variant %d", variant);
    if (op == 0) g->fp_variant = variant;
    else if (op == 1) g->adj_variant = variant;
    else g->bp_variant = variant;
    return PYRONN_OK;
}

int pyronn_adjoint(pyronn_geom_t g, const void *sino, void *vol, int dtype, int batch, void *stream) {
    clear_error();
    int rc = common_checks(g, dtype, batch);
    if (rc) return rc;
    if ((rc = check_ptr(vol, "vol")) || (rc = check_ptr(sino, "sino"))) return rc;
    if ((rc = ensure_device(g))) return rc;
    OpParams p = make_params(g, batch);
    if (g->adj_variant == 0 || g->adj_variant == 3) {
        const AdjSlabCfg &ac = adj_cfg(g);
        if (ac.valid) {
            float *acc = nullptr;
            if (dtype != PYRONN_F32) {
                if ((rc = ensure_scratch(g, sizeof(float) * (size_t)p.vol_elems * batch))) return rc;
                acc = (float *)g->d_scratch;
            }
            return cuda_rc(launch_adjoint_slab(p, ac, sino, nullptr, 1.0f, false, vol, acc, dtype, stream),
                           "adjoint launch");
        }
    }
    if (g->adj_variant != 1) return cuda_rc(launch_adjoint_brick(p, sino, vol, dtype, stream), "adjoint launch");
    float *acc = nullptr;
    if (dtype != PYRONN_F32) {
        if ((rc = ensure_scratch(g, sizeof(float) * (size_t)p.vol_elems * batch))) return rc;
        acc = (float *)g->d_scratch;
    }
    return cuda_rc(launch_adjoint(p, sino, vol, acc, dtype, stream), "adjoint launch");
}

int pyronn_adjoint_update(pyronn_geom_t g, const void *sino, const void *sino_b, double alpha, void *vol, int dtype,
                          int batch, void *stream) {
    clear_error();
    int rc = common_checks(g, dtype, batch);
    if (rc) return rc;
    if ((rc = check_ptr(vol, "vol")) || (rc = check_ptr(sino, "sino"))) return rc;
    if (sino_b && (rc = check_ptr(sino_b, "sino_b"))) return rc;
    if (!std::isfinite(alpha)) return set_error(PYRONN_INVALID_ARG, "alpha must be finite");
    if ((rc = ensure_device(g))) return rc;
    OpParams p = make_params(g, batch);
    if (g->adj_variant == 0 || g->adj_variant == 3) {
        const AdjSlabCfg &ac = adj_cfg(g);
        if (ac.valid) {
            float *acc = nullptr;
            if (dtype != PYRONN_F32) {
                if ((rc = ensure_scratch(g, sizeof(float) * (size_t)p.vol_elems * batch))) return rc;
                acc = (float *)g->d_scratch;
            }
            return cuda_rc(launch_adjoint_slab(p, ac, sino, sino_b, (float)alpha, true, vol, acc, dtype, stream),
                           "adjoint update launch");
        }
    }
    // kernels without the fused form: residual into a work sinogram, adjoint into a work volume, axpy
    const size_t es = dtype_size(dtype);
    const long long ns = p.sino_elems * batch, nv = p.vol_elems * batch;
    const void *y = sino;
    if (sino_b) {
        if ((rc = ensure_buffer(g, &g->d_upd_sino, &g->upd_sino_bytes, es * (size_t)ns, "update sinogram"))) return rc;
        if ((rc = cuda_rc(launch_residual(sino, sino_b, g->d_upd_sino, ns, dtype, stream), "residual launch"))) return rc;
        y = g->d_upd_sino;
    }
    if ((rc = ensure_buffer(g, &g->d_upd_vol, &g->upd_vol_bytes, es * (size_t)nv, "update volume"))) return rc;
    if ((rc = pyronn_adjoint(g, y, g->d_upd_vol, dtype, batch, stream))) return rc;
    return cuda_rc(launch_axpy(vol, g->d_upd_vol, (float)alpha, nv, dtype, stream), "update launch");
}

int pyronn_fbp_filter(pyronn_geom_t g, const void *sino, void *out, int filter, int dtype, int batch, void *stream) {
    clear_error();
    int rc = common_checks(g, dtype, batch);
    if (rc) return rc;
    if ((rc = check_ptr(sino, "sino")) || (rc = check_ptr(out, "out"))) return rc;
    if (filter != PYRONN_FILTER_RAM_LAK && filter != PYRONN_FILTER_SHEPP_LOGAN)
        return set_error(PYRONN_INVALID_ARG, "unknown filter %d", filter);
    if (g->nu > 4096) return set_error(PYRONN_INVALID_ARG, "FBP rows longer than 4096 pixels are not supported");
    if ((rc = ensure_device(g)) || (rc = ensure_fbp(g))) return rc;
    OpParams p = make_params(g, batch);
    return cuda_rc(launch_fbp_filter(p, g->d_fbp, filter, sino, out, dtype, stream), "FBP filter launch");
}

// ---------------------------------------------------------------------------------------------
// acquisition artifacts (Sec. 2.4)
// ---------------------------------------------------------------------------------------------

int pyronn_sim_detector_jitter(pyronn_geom_t g, const void *sino, void *out, const int32_t *shifts, int axis, int dtype,
                               int batch, void *stream) {
    clear_error();
    int rc = common_checks(g, dtype, batch);
    if (rc) return rc;
    if ((rc = check_ptr(sino, "sino")) || (rc = check_ptr(out, "out"))) return rc;
    if (!shifts) return set_error(PYRONN_INVALID_ARG, "null shifts");
    if (axis != 0 && axis != 1) return set_error(PYRONN_INVALID_ARG, "axis must be 0 (rows) or 1 (columns)");
    if (sino == out) return set_error(PYRONN_INVALID_ARG, "jitter cannot run in place");
    const long long n = (long long)batch * g->n_views * g->nv * g->nu;
    if ((rc = ensure_device(g))) return rc;
    return cuda_rc(launch_sim_jitter(sino, out, shifts, axis, g->nu, g->nv, n, dtype, stream), "jitter launch");
}

int pyronn_sim_gaussian_noise(pyronn_geom_t g, const void *sino, void *out, const float *noise, double mean, double sd,
                              int dtype, int batch, void *stream) {
    clear_error();
    int rc = common_checks(g, dtype, batch);
    if (rc) return rc;
    if ((rc = check_ptr(sino, "sino")) || (rc = check_ptr(out, "out"))) return rc;
    if (!noise) return set_error(PYRONN_INVALID_ARG, "null noise");
    if (!std::isfinite(mean) || !std::isfinite(sd)) return set_error(PYRONN_INVALID_ARG, "mean and std must be finite");
    const long long n = (long long)batch * g->n_views * g->nv * g->nu;
    if ((rc = ensure_device(g))) return rc;
    return cuda_rc(launch_sim_noise(sino, out, noise, (float)mean, (float)sd, n, dtype, stream), "noise launch");
}

int pyronn_sim_ring(pyronn_geom_t g, const void *sino, void *out, const int32_t *columns, const float *gains,
                    int n_columns, int view_begin, int view_end, int dtype, int batch, void *stream) {
    clear_error();
    int rc = common_checks(g, dtype, batch);
    if (rc) return rc;
    if ((rc = check_ptr(sino, "sino")) || (rc = check_ptr(out, "out"))) return rc;
    if (n_columns < 0 || (n_columns > 0 && (!columns || !gains)))
        return set_error(PYRONN_INVALID_ARG, "columns / gains missing");
    if (view_begin < 0 || view_end > g->n_views || view_begin > view_end)
        return set_error(PYRONN_INVALID_ARG, "view range [%d, %d) outside [0, %d]", view_begin, view_end, g->n_views);
    if ((rc = ensure_device(g))) return rc;
    const size_t bytes = dtype_size(dtype) * (size_t)batch * g->n_views * g->nv * g->nu;
    if (out != sino) {
        cudaError_t e = cudaMemcpyAsync(out, sino, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_rc((int)e, "ring copy");
    }
    if (n_columns == 0 || view_end == view_begin) return PYRONN_OK;
    return cuda_rc(launch_sim_ring(out, out, columns, gains, n_columns, g->nu, g->nv, g->n_views, view_begin, view_end,
                                   batch, dtype, stream),
                   "ring launch");
}

int pyronn_sim_motion_blur(pyronn_geom_t g, const void *sino, void *out, const float *angles, int length, int dtype,
                           int batch, void *stream) {
    clear_error();
    int rc = common_checks(g, dtype, batch);
    if (rc) return rc;
    if ((rc = check_ptr(sino, "sino")) || (rc = check_ptr(out, "out"))) return rc;
    if (!angles) return set_error(PYRONN_INVALID_ARG, "null angles");
    if (length < 1 || length > 1024) return set_error(PYRONN_INVALID_ARG, "kernel length %d out of [1, 1024]", length);
    if (sino == out) return set_error(PYRONN_INVALID_ARG, "motion blur cannot run in place");
    const long long n = (long long)batch * g->n_views * g->nv * g->nu;
    if ((rc = ensure_device(g))) return rc;
    return cuda_rc(launch_sim_blur(sino, out, angles, length, g->nu, g->nv, g->n_views, n, dtype, stream), "blur launch");
}

int pyronn_bp(pyronn_geom_t g, const void *sino, void *vol, int dtype, int batch, int weight, void *stream) {
    clear_error();
    int rc = common_checks(g, dtype, batch);
    if (rc) return rc;
    if ((rc = check_ptr(vol, "vol")) || (rc = check_ptr(sino, "sino"))) return rc;
    if (weight != PYRONN_BP_PLAIN && weight != PYRONN_BP_INV_W2)
        return set_error(PYRONN_INVALID_ARG, "unknown back-projection weight %d", weight);
    if ((rc = ensure_device(g))) return rc;
    OpParams p = make_params(g, batch);
    p.weight = weight;
    if (g->bp_variant == 1) return cuda_rc(launch_bp(p, sino, vol, dtype, stream), "back-projection launch");
    if ((g->bp_variant == 3 || g->bp_variant == 0) && bp_tma_usable(g, dtype))
        return cuda_rc(launch_bp_tma(g, p, sino, vol, dtype, stream), "back-projection launch");
    return cuda_rc(launch_bp_brick(p, bp_brick_depth(g->tuning.bp_brick_z, g->nz), sino, vol, dtype, stream),
                   "back-projection launch");
}

int pyronn_bp_transpose(pyronn_geom_t g, const void *vol, void *sino, int dtype, int batch, int weight,
                        void *stream) {
    clear_error();
    int rc = common_checks(g, dtype, batch);
    if (rc) return rc;
    if ((rc = check_ptr(vol, "vol")) || (rc = check_ptr(sino, "sino"))) return rc;
    if (weight != PYRONN_BP_PLAIN && weight != PYRONN_BP_INV_W2)
        return set_error(PYRONN_INVALID_ARG, "unknown back-projection weight %d", weight);
    if ((rc = ensure_device(g))) return rc;
    OpParams p = make_params(g, batch);
    p.weight = weight;
    float *acc = nullptr;
    if (dtype != PYRONN_F32) {
        if ((rc = ensure_scratch(g, sizeof(float) * (size_t)p.sino_elems * batch))) return rc;
        acc = (float *)g->d_scratch;
    }
    return cuda_rc(launch_bp_transpose(p, vol, sino, acc, dtype, stream), "back-projection transpose launch");
}

// Views v0 .. v0 + n - 1 of p: per-view tables move by v0; the per-volume sinogram stride (sino_elems)
// stays that of all views, so the caller offsets the sinogram pointer by v0 views.
static OpParams view_range(const OpParams &p, int v0, int n) {
    OpParams pc = p;
    pc.n_views = n;
    pc.fp += v0;
    pc.bp += v0;
    pc.views64 += (size_t)v0 * VIEW64_STRIDE;
    return pc;
}

// The stream and events of the overlapped host copies (created once per geometry, on its device).
static int ensure_pipe(pyronn_geom_t g) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->copy_stream) return PYRONN_OK;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (int i = 0; e == cudaSuccess && i < 9; ++i) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        g->pipe_ev[i] = ev;
    }
    if (e != cudaSuccess) {
        for (void *&ev : g->pipe_ev)
            if (ev) cudaEventDestroy((cudaEvent_t)ev), ev = nullptr;
        if (s) cudaStreamDestroy(s);
        return cuda_rc((int)e, "copy stream");
    }
    g->copy_stream = s;
    return PYRONN_OK;
}

// Forward projection of host buffers with the download of the sinogram overlapped: the views are
// projected in up to 8 chunks on `stream` (the volume's y-fastest copy is made once, by the first), and
// each chunk's sinogram rows go back to the host on the geometry's copy stream as soon as the chunk is
// done. Every view needs the whole volume, so its upload comes first. Only for the TMA projector.
static int fp_host_overlapped(pyronn_geom_t g, const FpTmaBox &tb, const void *in_host, void *out_host, int dtype,
                              int batch, cudaStream_t st) {
    int rc;
    if ((rc = ensure_pipe(g))) return rc;
    const size_t es = dtype_size(dtype);
    const size_t vol_bytes = es * (size_t)g->nx * g->ny * g->nz * batch;
    const size_t view_bytes = es * (size_t)g->nu * g->nv;
    const size_t sino_item = view_bytes * (size_t)g->n_views;   // one volume's sinogram
    if (tb.xt && (rc = ensure_buffer(g, &g->d_vol_t, &g->vol_t_bytes, vol_bytes, "transposed volume"))) return rc;
    cudaStream_t cs = (cudaStream_t)g->copy_stream;
    cudaError_t e = cudaMemcpyAsync(g->d_stage_in, in_host, vol_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_rc((int)e, "host-to-device copy");
    const OpParams p = make_params(g, batch);
    const int nchunk = std::min(8, g->n_views);
    for (int k = 0; k < nchunk; ++k) {
        const int v0 = (int)((long long)g->n_views * k / nchunk), v1 = (int)((long long)g->n_views * (k + 1) / nchunk);
        const OpParams pc = view_range(p, v0, v1 - v0);
        unsigned char *dev_k = (unsigned char *)g->d_stage_out + (size_t)v0 * view_bytes;
        e = (cudaError_t)launch_fp_tma(pc, tb, g->d_stage_in, g->d_vol_t, dev_k, dtype, st, k == 0);
        if (e == cudaSuccess) e = cudaEventRecord((cudaEvent_t)g->pipe_ev[k], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, (cudaEvent_t)g->pipe_ev[k], 0);
        for (int b = 0; e == cudaSuccess && b < batch; ++b)
            e = cudaMemcpyAsync((unsigned char *)out_host + b * sino_item + (size_t)v0 * view_bytes,
                                dev_k + b * sino_item, (size_t)(v1 - v0) * view_bytes, cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(cs);
            return cuda_rc((int)e, "forward projection with overlapped download");
        }
    }
    e = cudaEventRecord((cudaEvent_t)g->pipe_ev[8], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, (cudaEvent_t)g->pipe_ev[8], 0);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(cs);
        return cuda_rc((int)e, "copy stream join");
    }
    return cuda_rc((int)cudaStreamSynchronize(st), "stream synchronise");
}

static int host_op(pyronn_geom_t g, const void *in_host, void *out_host, int dtype, int batch, void *stream, int fp) {
    clear_error();
    int rc = common_checks(g, dtype, batch);
    if (rc) return rc;
    if (!in_host || !out_host) return set_error(PYRONN_INVALID_ARG, "null host buffer");
    if ((rc = ensure_device(g))) return rc;
    size_t es = dtype_size(dtype);
    size_t vol_bytes = es * (size_t)g->nx * g->ny * g->nz * batch;
    size_t sino_bytes = es * (size_t)g->nu * g->nv * g->n_views * batch;
    size_t in_bytes = fp ? vol_bytes : sino_bytes, out_bytes = fp ? sino_bytes : vol_bytes;
    if ((rc = ensure_stage(g, in_bytes, out_bytes))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (fp && (g->fp_variant == 0 || g->fp_variant == 3)) {
        const FpTmaBox &tb = tma_cfg(g, dtype);
        if (tb.depth > 0) return fp_host_overlapped(g, tb, in_host, out_host, dtype, batch, st);
    }
    cudaError_t e = cudaMemcpyAsync(g->d_stage_in, in_host, in_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_rc((int)e, "host-to-device copy");
    rc = fp ? pyronn_fp(g, g->d_stage_in, g->d_stage_out, dtype, batch, stream)
            : pyronn_adjoint(g, g->d_stage_in, g->d_stage_out, dtype, batch, stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(out_host, g->d_stage_out, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_rc((int)e, "device-to-host copy");
    return cuda_rc((int)cudaStreamSynchronize(st), "stream synchronise");
}

int pyronn_fp_host(pyronn_geom_t g, const void *vol_host, void *sino_host, int dtype, int batch, void *stream) {
    return host_op(g, vol_host, sino_host, dtype, batch, stream, 1);
}

int pyronn_adjoint_host(pyronn_geom_t g, const void *sino_host, void *vol_host, int dtype, int batch, void *stream) {
    return host_op(g, sino_host, vol_host, dtype, batch, stream, 0);
}

}  // extern "C"
