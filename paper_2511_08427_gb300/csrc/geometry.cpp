// Host-side geometry: projection matrices (FP64) and the per-view FP32 device tables.
//
// Sec. 2.4 ("Flexible Trajectory Modeling"): projection matrices are generated from the source
// position, the detector position and the detector directions; circular trajectories are
// produced by rotating an initial configuration view by view, arbitrary ones use the given
// positions directly. Sec. 2.1: calibrated projection matrices can be used for cone beam.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <thread>

#include "pyronn_internal.h"

namespace pyronn {

int stride_grid(long long n, int ctas_per_sm) {
    static std::mutex mu;
    static int sms[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = -1;
    int count = 0;
    if (dev >= 0) {
        std::lock_guard<std::mutex> lk(mu);
        if (sms[dev] == 0 && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms[dev] = 0;
        count = sms[dev];
    }
    if (count <= 0) count = 1;
    const long long need = (n + 255) / 256;
    const long long cap = (long long)count * ctas_per_sm;
    return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

}  // namespace pyronn

namespace pyronn {

static thread_local std::string g_last_error;

int set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

void clear_error() { g_last_error.clear(); }

size_t dtype_size(int dtype) {
    switch (dtype) {
        case PYRONN_F32: return 4;
        case PYRONN_BF16: return 2;
        case PYRONN_F16: return 2;
        default: return 0;
    }
}

namespace {

struct M3 {
    double a[9];
    double operator()(int r, int c) const { return a[3 * r + c]; }
};

bool inverse3(const M3 &m, M3 &out) {
    const double *x = m.a;
    double c00 = x[4] * x[8] - x[5] * x[7];
    double c01 = x[5] * x[6] - x[3] * x[8];
    double c02 = x[3] * x[7] - x[4] * x[6];
    double det = x[0] * c00 + x[1] * c01 + x[2] * c02;
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
    double id = 1.0 / det;
    double adj[9] = {c00, x[2] * x[7] - x[1] * x[8], x[1] * x[5] - x[2] * x[4],
                     c01, x[0] * x[8] - x[2] * x[6], x[2] * x[3] - x[0] * x[5],
                     c02, x[1] * x[6] - x[0] * x[7], x[0] * x[4] - x[1] * x[3]};
    for (int i = 0; i < 9; ++i) out.a[i] = adj[i] * id;
    return true;
}

void cross(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// The device tables hold spacings and their reciprocals in FP32.
bool fp32_spacing(double s) {
    return s > 0 && std::isfinite((float)s) && (float)s > 0.0f && std::isfinite((float)(1.0 / s));
}

// Sample indices and counts stay far inside 32-bit and FP32-exact ranges: the diagonal of the support
// box ((-1, N) on every axis) spans at most 2^22 steps; the step and its reciprocal are finite in FP32.
int check_step(const pyronn_geom *g, double dt) {
    if (!(dt > 0) || !std::isfinite((float)dt) || !std::isfinite((float)(1.0 / dt)))
        return set_error(PYRONN_INVALID_ARG, "step %g mm must be positive, with it and its reciprocal finite in FP32",
                         dt);
    const double ex = (g->nx + 1) * g->sx, ey = (g->ny + 1) * g->sy;
    const double ez = g->ndim == 3 ? (g->nz + 1) * g->sz : 0.0;
    const double diag = std::sqrt(ex * ex + ey * ey + ez * ez);
    if (!(diag / dt <= 4194304.0))
        return set_error(PYRONN_INVALID_ARG, "step %g mm: the volume's diagonal (%g mm) spans more than 2^22 steps",
                         dt, diag);
    return PYRONN_OK;
}

int check_descs(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views, int want_ndim) {
    if (!vol || !det) return set_error(PYRONN_INVALID_ARG, "null descriptor");
    if (vol->ndim != 2 && vol->ndim != 3) return set_error(PYRONN_INVALID_ARG, "vol.ndim must be 2 or 3");
    if (want_ndim && vol->ndim != want_ndim)
        return set_error(PYRONN_INVALID_ARG, "this geometry needs a %dD volume descriptor", want_ndim);
    for (int i = 0; i < 3; ++i)
        if (vol->shape[i] < 1 || vol->shape[i] > 16384)
            return set_error(PYRONN_INVALID_ARG, "vol.shape[%d] = %d out of range [1, 16384]", i, vol->shape[i]);
    if (vol->ndim == 2 && vol->shape[0] != 1) return set_error(PYRONN_INVALID_ARG, "2D volume needs shape[0] == 1");
    for (int i = (vol->ndim == 2 ? 1 : 0); i < 3; ++i) {
        if (!fp32_spacing(vol->spacing[i]))
            return set_error(PYRONN_INVALID_ARG, "vol.spacing[%d] must be positive, with it and its reciprocal "
                             "finite in FP32", i);
        if (!std::isfinite(vol->offset[i])) return set_error(PYRONN_INVALID_ARG, "vol.offset[%d] must be finite", i);
    }
    for (int i = 0; i < 2; ++i) {
        if (det->shape[i] < 1 || det->shape[i] > 65536)
            return set_error(PYRONN_INVALID_ARG, "det.shape[%d] = %d out of range", i, det->shape[i]);
        if (!fp32_spacing(det->spacing[i]))
            return set_error(PYRONN_INVALID_ARG, "det.spacing[%d] must be positive, with it and its reciprocal "
                             "finite in FP32", i);
        if (!std::isfinite(det->offset[i])) return set_error(PYRONN_INVALID_ARG, "det.offset[%d] must be finite", i);
    }
    if (vol->ndim == 2 && det->shape[0] != 1) return set_error(PYRONN_INVALID_ARG, "2D detector needs shape[0] == 1");
    if (n_views < 1 || n_views > (1 << 20)) return set_error(PYRONN_INVALID_ARG, "n_views = %d out of range", n_views);
    return PYRONN_OK;
}

pyronn_geom *new_geom(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views) {
    pyronn_geom *g = new pyronn_geom();
    g->ndim = vol->ndim;
    g->nz = vol->shape[0]; g->ny = vol->shape[1]; g->nx = vol->shape[2];
    if (vol->ndim == 2) {
        g->sz = 1.0; g->oz = 0.0;
    } else {
        g->sz = vol->spacing[0]; g->oz = vol->offset[0];
    }
    g->sy = vol->spacing[1]; g->sx = vol->spacing[2];
    g->oy = vol->offset[1]; g->ox = vol->offset[2];
    g->nv = det->shape[0]; g->nu = det->shape[1];
    g->dv = det->spacing[0]; g->du = det->spacing[1];
    g->ov = det->offset[0]; g->ou = det->offset[1];
    g->n_views = n_views;
    double smin = std::min(g->sx, g->sy);
    if (g->ndim == 3) smin = std::min(smin, g->sz);
    g->dt = 0.5 * smin;
    g->views.assign((size_t)n_views * 12, 0.0);
    return g;
}

// P = M^-1 [I | -S] with M = [du eu | dv ev | D0 - S] (Sec. 2.4).
bool pmat_from_frame(const double S[3], const double Dc[3], const double eu_in[3], const double ev_in[3],
                     const pyronn_geom *g, double P[12]) {
    double eu[3], ev[3];
    double nu_ = std::sqrt(dot3(eu_in, eu_in)), nv_ = std::sqrt(dot3(ev_in, ev_in));
    if (!(nu_ > 0) || !(nv_ > 0)) return false;
    for (int i = 0; i < 3; ++i) { eu[i] = eu_in[i] / nu_; ev[i] = ev_in[i] / nv_; }
    double D0[3];
    for (int i = 0; i < 3; ++i)
        D0[i] = Dc[i] + (g->ou - 0.5 * (g->nu - 1) * g->du) * eu[i] + (g->ov - 0.5 * (g->nv - 1) * g->dv) * ev[i];
    M3 M, Mi;
    for (int i = 0; i < 3; ++i) {
        M.a[3 * i + 0] = g->du * eu[i];
        M.a[3 * i + 1] = g->dv * ev[i];
        M.a[3 * i + 2] = D0[i] - S[i];
    }
    if (!inverse3(M, Mi)) return false;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) P[4 * r + c] = Mi(r, c);
        P[4 * r + 3] = -(Mi(r, 0) * S[0] + Mi(r, 1) * S[1] + Mi(r, 2) * S[2]);
    }
    return true;
}

// Rescale a 3 x 4 matrix so that |inv(P[:, :3]) e0| = du and w(C) > 0.
bool normalise_pmat(const double *Pin, const pyronn_geom *g, double *Pout) {
    M3 M, Mi;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M.a[3 * r + c] = Pin[4 * r + c];
    if (!inverse3(M, Mi)) return false;
    double l = std::sqrt(Mi(0, 0) * Mi(0, 0) + Mi(1, 0) * Mi(1, 0) + Mi(2, 0) * Mi(2, 0));
    double w = Pin[8] * g->ox + Pin[9] * g->oy + Pin[10] * g->oz + Pin[11];
    if (!(l > 0) || w == 0.0 || !std::isfinite(w)) return false;
    double kappa = l / g->du;
    if (w < 0) kappa = -kappa;
    for (int i = 0; i < 12; ++i) Pout[i] = kappa * Pin[i];
    return true;
}

void circular_frame(int n, int n_views, double range, double sid, double sdd, double pitch, double S[3],
                    double Dc[3], double eu[3], double ev[3]) {
    double step = range / n_views;
    double t = n * step;
    double c = std::cos(t), s = std::sin(t);
    double z = pitch * (n - 0.5 * (n_views - 1)) * step / (2.0 * M_PI);
    S[0] = sid * c; S[1] = sid * s; S[2] = z;
    Dc[0] = -(sdd - sid) * c; Dc[1] = -(sdd - sid) * s; Dc[2] = z;
    eu[0] = -s; eu[1] = c; eu[2] = 0.0;
    ev[0] = 0.0; ev[1] = 0.0; ev[2] = 1.0;
}

int finish(pyronn_geom *g, pyronn_geom_t *out) {
    int rc = finalize_geometry(g);
    if (rc) {
        delete g;
        return rc;
    }
    *out = g;
    return PYRONN_OK;
}

}  // namespace

// Build the FP32 device records from the FP64 views.
// Per-view FBP constants (see or_fbp_filter for the definitions): perspective views give the source
// -> pixel basis inv(M') (columns du eu, dv ev, D0 - S), sdd = 1 / |P_3| (P's third row spans w = 0 at
// the source to w = 1 on the detector), r = w(volume centre) and tau = r |du eu|.
int ensure_fbp(pyronn_geom *g) {
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->d_fbp) return PYRONN_OK;
    const int V = g->n_views;
    const double pi = 3.14159265358979323846;
    std::vector<FbpRec> rec(V);
    for (int n = 0; n < V; ++n) {
        FbpRec &f = rec[n];
        double scale;
        if (g->kind == 1) {
            const double *r = &g->views[12 * (size_t)n];
            const double *x = &g->views_ext[(size_t)n * VIEW64_STRIDE];
            const double nn = std::sqrt(r[8] * r[8] + r[9] * r[9] + r[10] * r[10]);
            const double ratio = x[11];   // w at the volume centre
            const double pu = std::sqrt(x[15] * x[15] + x[16] * x[16] + x[17] * x[17]);
            const double tau = ratio * pu;
            scale = pi / V * ratio * ratio / tau;
            f.sdd = (float)(1.0 / nn);
            for (int i = 0; i < 3; ++i) {
                f.bu[i] = (float)x[15 + i];
                f.bv[i] = (float)x[18 + i];
                f.b0[i] = (float)x[21 + i];
            }
        } else {
            scale = pi / V / g->du;
            f.sdd = 0.0f;
            for (int i = 0; i < 3; ++i) f.b0[i] = f.bu[i] = f.bv[i] = 0.0f;
        }
        f.scale = (float)scale;
    }
    cudaError_t e = cudaMalloc(&g->d_fbp, sizeof(FbpRec) * (size_t)V);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_fbp, rec.data(), sizeof(FbpRec) * (size_t)V, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(g->d_fbp);
        g->d_fbp = nullptr;
        return set_error(PYRONN_CUDA_ERROR, "FBP constants: %s", cudaGetErrorString(e));
    }
    return PYRONN_OK;
}

int finalize_geometry(pyronn_geom *g) {
    if (int rc = check_step(g, g->dt)) return rc;
    const int V = g->n_views;
    g->fp_rec.assign(V, FpRec{});
    g->bp_rec.assign(V, BpRec{});
    g->views_ext.assign((size_t)V * VIEW64_STRIDE, 0.0);
    const double C[3] = {g->ox, g->oy, g->oz};
    const double s[3] = {g->sx, g->sy, g->sz};
    const double hu = 0.5 * (g->nu - 1), hv = 0.5 * (g->nv - 1);
    for (int n = 0; n < V; ++n) {
        const double *r = &g->views[12 * (size_t)n];
        double R0[3], Ru[3], Rv[3], B0[3], Bu[3], Bv[3], Pc[12];
        if (g->kind == 1) {
            M3 Mp, M;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Mp.a[3 * i + j] = r[4 * i + j];
            if (!inverse3(Mp, M)) return set_error(PYRONN_SINGULAR, "view %d: singular projection matrix", n);
            double S[3], col0[3], col1[3], col2[3];
            for (int i = 0; i < 3; ++i) {
                S[i] = -(M(i, 0) * r[3] + M(i, 1) * r[7] + M(i, 2) * r[11]);
                col0[i] = M(i, 0); col1[i] = M(i, 1); col2[i] = M(i, 2);
            }
            double nrm[3];
            cross(col0, col1, nrm);
            double den = dot3(col2, nrm);
            if (den == 0.0) return set_error(PYRONN_SINGULAR, "view %d: source lies in the detector plane", n);
            double CS[3] = {C[0] - S[0], C[1] - S[1], C[2] - S[2]};
            double lam = dot3(CS, nrm) / den;
            for (int i = 0; i < 3; ++i) {
                R0[i] = (S[i] - C[i]) + lam * col2[i];
                Ru[i] = lam * col0[i];
                Rv[i] = lam * col1[i];
                B0[i] = col2[i]; Bu[i] = col0[i]; Bv[i] = col1[i];
            }
            double *x = &g->views_ext[(size_t)n * VIEW64_STRIDE];
            for (int row = 0; row < 3; ++row) {
                for (int a = 0; a < 3; ++a) x[4 * row + a] = r[4 * row + a];
                x[4 * row + 3] = r[4 * row + 0] * C[0] + r[4 * row + 1] * C[1] + r[4 * row + 2] * C[2] + r[4 * row + 3];
            }
            for (int i = 0; i < 3; ++i) {
                x[12 + i] = S[i] - C[i];
                x[15 + i] = col0[i]; x[18 + i] = col1[i]; x[21 + i] = col2[i]; x[24 + i] = nrm[i];
            }
            x[27] = den;
            // BP: centred voxel index -> centred detector coordinate times w
            for (int row = 0; row < 3; ++row) {
                for (int a = 0; a < 3; ++a) Pc[4 * row + a] = r[4 * row + a] * s[a];
                Pc[4 * row + 3] = r[4 * row + 0] * C[0] + r[4 * row + 1] * C[1] + r[4 * row + 2] * C[2] + r[4 * row + 3];
            }
            for (int a = 0; a < 4; ++a) {
                Pc[a] -= hu * Pc[8 + a];
                Pc[4 + a] -= hv * Pc[8 + a];
            }
        } else {
            const double *Dc = r, *eu = r + 3, *ev = r + 6, *d = r + 9;
            for (int i = 0; i < 3; ++i) {
                R0[i] = Dc[i] - C[i] + (g->ou - hu * g->du) * eu[i] + (g->ov - hv * g->dv) * ev[i];
                Ru[i] = g->du * eu[i];
                Rv[i] = g->dv * ev[i];
                B0[i] = d[i]; Bu[i] = 0.0; Bv[i] = 0.0;
            }
            double *x = &g->views_ext[(size_t)n * VIEW64_STRIDE];
            for (int i = 0; i < 3; ++i) {
                x[i] = Dc[i] - C[i]; x[3 + i] = eu[i]; x[6 + i] = ev[i]; x[9 + i] = d[i];
            }
            double CD[3] = {C[0] - Dc[0], C[1] - Dc[1], C[2] - Dc[2]};
            for (int a = 0; a < 3; ++a) {
                Pc[a] = eu[a] * s[a] / g->du;
                Pc[4 + a] = ev[a] * s[a] / g->dv;
                Pc[8 + a] = 0.0;
            }
            Pc[3] = (dot3(CD, eu) - g->ou) / g->du;
            Pc[7] = (dot3(CD, ev) - g->ov) / g->dv;
            Pc[11] = 1.0;
        }
        FpRec &f = g->fp_rec[n];
        for (int i = 0; i < 3; ++i) {
            f.R0[i] = (float)R0[i]; f.Ru[i] = (float)Ru[i]; f.Rv[i] = (float)Rv[i];
            f.B0[i] = (float)B0[i]; f.Bu[i] = (float)Bu[i]; f.Bv[i] = (float)Bv[i];
        }
        for (int i = 0; i < 12; ++i) g->bp_rec[n].P[i] = (float)Pc[i];
        bool finite = true;
        for (int i = 0; i < 3; ++i)
            finite = finite && std::isfinite(f.R0[i]) && std::isfinite(f.Ru[i]) && std::isfinite(f.Rv[i]) &&
                     std::isfinite(f.B0[i]) && std::isfinite(f.Bu[i]) && std::isfinite(f.Bv[i]);
        for (int i = 0; i < 12; ++i) finite = finite && std::isfinite(g->bp_rec[n].P[i]);
        for (int i = 0; i < VIEW64_STRIDE; ++i) finite = finite && std::isfinite(g->views_ext[(size_t)n * VIEW64_STRIDE + i]);
        if (!finite)
            return set_error(PYRONN_INVALID_ARG, "view %d: the geometry does not fit the FP32 device tables "
                             "(a non-finite entry)", n);
    }
    g->sample_count = -1;
    g->fp_cfg_ready = 0;
    g->tma_ready[0] = g->tma_ready[1] = g->tma_ready[2] = 0;
    g->adj_cfg_ready = 0;
    return PYRONN_OK;
}

int ensure_device(pyronn_geom *g) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(PYRONN_CUDA_ERROR, "cudaGetDevice: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->d_fp && g->device == dev) return PYRONN_OK;
    if (g->d_fp && g->device != dev)
        return set_error(PYRONN_INVALID_ARG, "geometry tables live on device %d, current device is %d", g->device, dev);
    size_t nf = sizeof(FpRec) * g->n_views, nb = sizeof(BpRec) * g->n_views;
    void *pf = nullptr, *pb = nullptr, *pg = nullptr;
    e = cudaMalloc(&pg, sizeof(int) * N_FLAGS);
    if (e != cudaSuccess) return set_error(PYRONN_OOM, "cudaMalloc(flags): %s", cudaGetErrorString(e));
    e = cudaMemset(pg, 0, sizeof(int) * N_FLAGS);
    if (e != cudaSuccess) {
        cudaFree(pg);
        return set_error(PYRONN_CUDA_ERROR, "cudaMemset(flags): %s", cudaGetErrorString(e));
    }
    e = cudaMalloc(&pf, nf);
    if (e != cudaSuccess) {
        cudaFree(pg);
        return set_error(PYRONN_OOM, "cudaMalloc(view tables): %s", cudaGetErrorString(e));
    }
    e = cudaMalloc(&pb, nb);
    if (e != cudaSuccess) {
        cudaFree(pg);
        cudaFree(pf);
        return set_error(PYRONN_OOM, "cudaMalloc(view tables): %s", cudaGetErrorString(e));
    }
    e = cudaMemcpy(pf, g->fp_rec.data(), nf, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pb, g->bp_rec.data(), nb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(pg);
        cudaFree(pf);
        cudaFree(pb);
        return set_error(PYRONN_CUDA_ERROR, "upload of view tables: %s", cudaGetErrorString(e));
    }
    void *pv = nullptr;
    e = cudaMalloc(&pv, sizeof(double) * g->views_ext.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(pv, g->views_ext.data(), sizeof(double) * g->views_ext.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(pv);
        cudaFree(pg);
        cudaFree(pf);
        cudaFree(pb);
        return set_error(PYRONN_CUDA_ERROR, "upload of FP64 views: %s", cudaGetErrorString(e));
    }
    g->d_views64 = (double *)pv;
    g->d_flags = (int *)pg;
    g->d_fp = (FpRec *)pf;
    g->d_bp = (BpRec *)pb;
    g->device = dev;
    return PYRONN_OK;
}

OpParams make_params(const pyronn_geom *g, int batch) {
    OpParams p{};
    p.vol.nx = g->nx; p.vol.ny = g->ny; p.vol.nz = g->nz;
    p.vol.hx = 0.5f * (g->nx - 1); p.vol.hy = 0.5f * (g->ny - 1); p.vol.hz = 0.5f * (g->nz - 1);
    p.vol.isx = (float)(1.0 / g->sx); p.vol.isy = (float)(1.0 / g->sy); p.vol.isz = (float)(1.0 / g->sz);
    p.det.nu = g->nu; p.det.nv = g->nv;
    p.det.hu = 0.5f * (g->nu - 1); p.det.hv = 0.5f * (g->nv - 1);
    p.n_views = g->n_views;
    p.batch = batch;
    p.perspective = g->kind;
    p.weight = 0;
    p.dt = (float)g->dt;
    p.fp = g->d_fp;
    p.bp = g->d_bp;
    p.flags = g->d_flags;
    p.views64 = g->d_views64;
    p.sx = g->sx; p.sy = g->sy; p.sz = g->sz;
    p.du = g->du; p.dv = g->dv; p.ou = g->ou; p.ov = g->ov;
    p.vol_elems = (long long)g->nx * g->ny * g->nz;
    p.sino_elems = (long long)g->nu * g->nv * g->n_views;
    return p;
}

}  // namespace pyronn

using namespace pyronn;

extern "C" {

int pyronn_geom_create_parallel2d(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                                  double angular_range, pyronn_geom_t *out) {
    clear_error();
    if (!out) return set_error(PYRONN_INVALID_ARG, "out is null");
    int rc = check_descs(vol, det, n_views, 2);
    if (rc) return rc;
    if (!std::isfinite(angular_range)) return set_error(PYRONN_INVALID_ARG, "angular_range must be finite");
    pyronn_geom *g = new_geom(vol, det, n_views);
    g->kind = 0;
    for (int n = 0; n < n_views; ++n) {
        double t = n * (angular_range / n_views);
        double c = std::cos(t), s = std::sin(t);
        double *r = &g->views[12 * (size_t)n];
        r[0] = r[1] = r[2] = 0.0;
        r[3] = -s; r[4] = c; r[5] = 0.0;
        r[6] = 0.0; r[7] = 0.0; r[8] = 1.0;
        r[9] = -c; r[10] = -s; r[11] = 0.0;
    }
    return finish(g, out);
}

static int create_circular(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views, double range,
                           double sid, double sdd, double pitch, int ndim, pyronn_geom_t *out) {
    clear_error();
    if (!out) return set_error(PYRONN_INVALID_ARG, "out is null");
    int rc = check_descs(vol, det, n_views, ndim);
    if (rc) return rc;
    if (!(sid > 0) || !(sdd > sid) || !std::isfinite(sdd) || !std::isfinite(range) || !std::isfinite(pitch))
        return set_error(PYRONN_INVALID_ARG, "need 0 < sid < sdd (got sid=%g sdd=%g)", sid, sdd);
    pyronn_geom *g = new_geom(vol, det, n_views);
    g->kind = 1;
    for (int n = 0; n < n_views; ++n) {
        double S[3], Dc[3], eu[3], ev[3];
        circular_frame(n, n_views, range, sid, sdd, pitch, S, Dc, eu, ev);
        if (!pmat_from_frame(S, Dc, eu, ev, g, &g->views[12 * (size_t)n])) {
            delete g;
            return set_error(PYRONN_SINGULAR, "view %d: singular detector frame", n);
        }
    }
    return finish(g, out);
}

int pyronn_geom_create_fan2d(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                             double angular_range, double sid, double sdd, pyronn_geom_t *out) {
    return create_circular(vol, det, n_views, angular_range, sid, sdd, 0.0, 2, out);
}

int pyronn_geom_create_cone_circular(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                                     double angular_range, double sid, double sdd, double helical_pitch_mm,
                                     pyronn_geom_t *out) {
    return create_circular(vol, det, n_views, angular_range, sid, sdd, helical_pitch_mm, 3, out);
}

int pyronn_geom_create_from_positions(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                                      const double *src, const double *det_centre, const double *eu,
                                      const double *ev, pyronn_geom_t *out) {
    clear_error();
    if (!out || !src || !det_centre || !eu || !ev) return set_error(PYRONN_INVALID_ARG, "null argument");
    int rc = check_descs(vol, det, n_views, 3);
    if (rc) return rc;
    pyronn_geom *g = new_geom(vol, det, n_views);
    g->kind = 1;
    for (int n = 0; n < n_views; ++n) {
        if (!pmat_from_frame(src + 3 * n, det_centre + 3 * n, eu + 3 * n, ev + 3 * n, g, &g->views[12 * (size_t)n])) {
            delete g;
            return set_error(PYRONN_SINGULAR, "view %d: singular detector frame", n);
        }
    }
    return finish(g, out);
}

int pyronn_geom_create_cone_matrices(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                                     const double *P, pyronn_geom_t *out) {
    clear_error();
    if (!out || !P) return set_error(PYRONN_INVALID_ARG, "null argument");
    int rc = check_descs(vol, det, n_views, 3);
    if (rc) return rc;
    pyronn_geom *g = new_geom(vol, det, n_views);
    g->kind = 1;
    for (int n = 0; n < n_views; ++n) {
        for (int i = 0; i < 12; ++i)
            if (!std::isfinite(P[12 * (size_t)n + i])) {
                delete g;
                return set_error(PYRONN_INVALID_ARG, "view %d: non-finite matrix entry", n);
            }
        if (!normalise_pmat(P + 12 * (size_t)n, g, &g->views[12 * (size_t)n])) {
            delete g;
            return set_error(PYRONN_SINGULAR, "view %d: matrix is singular or w = 0 at the volume centre", n);
        }
    }
    return finish(g, out);
}

int pyronn_geom_create_matrices2d(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                                  const double *P, pyronn_geom_t *out) {
    clear_error();
    if (!out || !P) return set_error(PYRONN_INVALID_ARG, "null argument");
    int rc = check_descs(vol, det, n_views, 2);
    if (rc) return rc;
    int n_affine = 0;
    for (int n = 0; n < n_views; ++n) {
        const double *p = P + 6 * (size_t)n;
        for (int i = 0; i < 6; ++i)
            if (!std::isfinite(p[i])) return set_error(PYRONN_INVALID_ARG, "view %d: non-finite matrix entry", n);
        n_affine += (p[3] == 0.0 && p[4] == 0.0 && p[5] != 0.0);
    }
    if (n_affine != 0 && n_affine != n_views)
        return set_error(PYRONN_INVALID_ARG, "mix of affine (parallel) and perspective (fan) matrices");
    pyronn_geom *g = new_geom(vol, det, n_views);
    if (n_affine) {
        g->kind = 0;
        for (int n = 0; n < n_views; ++n) {
            const double *p = P + 6 * (size_t)n;
            double a = p[0] / p[5], b = p[1] / p[5], c = p[2] / p[5];
            double sigma = std::sqrt(a * a + b * b);
            if (!(sigma > 0) || std::fabs(sigma * g->du - 1.0) > 1e-6) {
                delete g;
                return set_error(PYRONN_INVALID_ARG,
                                 "view %d: affine row scale 1/%g does not match detector spacing %g", n, 1.0 / sigma,
                                 g->du);
            }
            double eu[2] = {a / sigma, b / sigma};
            double t = g->du * (0.5 * (g->nu - 1) - c) - g->ou;  // Dc = t eu reproduces u = P[0] . (x, y, 1)
            double *r = &g->views[12 * (size_t)n];
            r[0] = t * eu[0]; r[1] = t * eu[1]; r[2] = 0.0;
            r[3] = eu[0]; r[4] = eu[1]; r[5] = 0.0;
            r[6] = 0.0; r[7] = 0.0; r[8] = 1.0;
            r[9] = -eu[1]; r[10] = eu[0]; r[11] = 0.0;
        }
    } else {
        g->kind = 1;
        for (int n = 0; n < n_views; ++n) {
            const double *p = P + 6 * (size_t)n;
            // embed: (x, y, z, 1) -> (u w, v w, w) with the v row (0, 0, 1 / dv, 0)
            double P3[12] = {p[0], p[1], 0.0, p[2], 0.0, 0.0, 1.0 / g->dv, 0.0, p[3], p[4], 0.0, p[5]};
            double *out_p = &g->views[12 * (size_t)n];
            if (!normalise_pmat(P3, g, out_p)) {
                delete g;
                return set_error(PYRONN_SINGULAR, "view %d: matrix is singular or w = 0 at the image centre", n);
            }
            // the v row only maps z to the single detector row; keep it scale-free
            out_p[4] = 0.0; out_p[5] = 0.0; out_p[6] = 1.0 / g->dv; out_p[7] = 0.0;
        }
    }
    return finish(g, out);
}

int pyronn_geom_destroy(pyronn_geom_t g) {
    clear_error();
    if (!g) return PYRONN_OK;
    // device buffers are freed on the device they were allocated on
    if (g->d_fp || g->d_scratch || g->d_stage_in || g->d_stage_out || g->d_upd_sino || g->d_upd_vol || g->d_fbp ||
        g->d_vol_t || g->copy_stream || g->tex_arr || g->texf_arr) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (g->device >= 0 && g->device != cur) cudaSetDevice(g->device);
        cudaFree(g->d_fp);
        cudaFree(g->d_bp);
        cudaFree(g->d_flags);
        cudaFree(g->d_views64);
        cudaFree(g->d_scratch);
        cudaFree(g->d_stage_in);
        cudaFree(g->d_stage_out);
        cudaFree(g->d_upd_sino);
        cudaFree(g->d_upd_vol);
        cudaFree(g->d_fbp);
        cudaFree(g->d_vol_t);
        for (void *ev : g->pipe_ev)
            if (ev) cudaEventDestroy((cudaEvent_t)ev);
        if (g->copy_stream) cudaStreamDestroy((cudaStream_t)g->copy_stream);
        if (g->tex_obj) cudaDestroyTextureObject((cudaTextureObject_t)g->tex_obj);
        if (g->tex_arr) cudaFreeArray((cudaArray_t)g->tex_arr);
        cudaFree(g->d_tex_org);
        if (g->texf_obj) cudaDestroyTextureObject((cudaTextureObject_t)g->texf_obj);
        if (g->texf_arr) cudaFreeArray((cudaArray_t)g->texf_arr);
        if (g->device >= 0 && cur >= 0 && g->device != cur) cudaSetDevice(cur);
    }
    delete g;
    return PYRONN_OK;
}

int pyronn_geom_set_step(pyronn_geom_t g, double dt_mm) {
    clear_error();
    if (!g) return set_error(PYRONN_INVALID_ARG, "null geometry");
    if (int rc = check_step(g, dt_mm)) return rc;
    g->dt = dt_mm;
    g->sample_count = -1;
    g->fp_cfg_ready = 0;
    g->tma_ready[0] = g->tma_ready[1] = g->tma_ready[2] = 0;
    g->adj_cfg_ready = 0;
    return PYRONN_OK;
}

int pyronn_geom_get_step(pyronn_geom_t g, double *dt_mm) {
    clear_error();
    if (!g || !dt_mm) return set_error(PYRONN_INVALID_ARG, "null argument");
    *dt_mm = g->dt;
    return PYRONN_OK;
}

int pyronn_geom_info(pyronn_geom_t g, int *n_views, int *kind, int *ndim) {
    clear_error();
    if (!g) return set_error(PYRONN_INVALID_ARG, "null geometry");
    if (n_views) *n_views = g->n_views;
    if (kind) *kind = g->kind;
    if (ndim) *ndim = g->ndim;
    return PYRONN_OK;
}

int pyronn_geom_get_views(pyronn_geom_t g, double *out) {
    clear_error();
    if (!g || !out) return set_error(PYRONN_INVALID_ARG, "null argument");
    std::memcpy(out, g->views.data(), sizeof(double) * g->views.size());
    return PYRONN_OK;
}

int pyronn_geom_count_samples(pyronn_geom_t g, int64_t *total) {
    clear_error();
    if (!g || !total) return set_error(PYRONN_INVALID_ARG, "null argument");
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if (g->sample_count >= 0) {
            *total = g->sample_count;
            return PYRONN_OK;
        }
    }
    // FP64 ray setup from the FP64 views (same construction as the device tables, unrounded)
    const int V = g->n_views;
    std::vector<double> rec((size_t)V * 18);
    {
        const double C[3] = {g->ox, g->oy, g->oz};
        for (int n = 0; n < V; ++n) {
            const double *r = &g->views[12 * (size_t)n];
            double *o = &rec[18 * (size_t)n];
            if (g->kind == 1) {
                M3 Mp, M;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) Mp.a[3 * i + j] = r[4 * i + j];
                inverse3(Mp, M);
                for (int i = 0; i < 3; ++i) {
                    o[i] = -(M(i, 0) * r[3] + M(i, 1) * r[7] + M(i, 2) * r[11]) - C[i];  // S - C
                    o[3 + i] = 0.0; o[6 + i] = 0.0;
                    o[9 + i] = M(i, 2); o[12 + i] = M(i, 0); o[15 + i] = M(i, 1);
                }
            } else {
                const double hu = 0.5 * (g->nu - 1), hv = 0.5 * (g->nv - 1);
                for (int i = 0; i < 3; ++i) {
                    o[i] = r[i] - C[i] + (g->ou - hu * g->du) * r[3 + i] + (g->ov - hv * g->dv) * r[6 + i];
                    o[3 + i] = g->du * r[3 + i];
                    o[6 + i] = g->dv * r[6 + i];
                    o[9 + i] = r[9 + i]; o[12 + i] = 0.0; o[15 + i] = 0.0;
                }
            }
        }
    }
    const double s[3] = {g->sx, g->sy, g->sz};
    const double h[3] = {0.5 * (g->nx - 1), 0.5 * (g->ny - 1), 0.5 * (g->nz - 1)};
    const double N[3] = {(double)g->nx, (double)g->ny, (double)g->nz};
    const double dt = g->dt;
    std::atomic<int> next(0);
    std::atomic<long long> sum(0);
    auto work = [&]() {
        long long local = 0;
        for (int n = next.fetch_add(1); n < V; n = next.fetch_add(1)) {
            const double *o = &rec[18 * (size_t)n];
            for (int v = 0; v < g->nv; ++v)
                for (int u = 0; u < g->nu; ++u) {
                    double Y[3], D[3];
                    for (int i = 0; i < 3; ++i) {
                        Y[i] = o[i] + u * o[3 + i] + v * o[6 + i];
                        D[i] = o[9 + i] + u * o[12 + i] + v * o[15 + i];
                    }
                    double nd = std::sqrt(dot3(D, D));
                    for (int i = 0; i < 3; ++i) D[i] /= nd;
                    double tau = -dot3(Y, D);
                    double lo = -INFINITY, hi = INFINITY;
                    bool empty = false;
                    for (int a = 0; a < 3; ++a) {
                        double c = (Y[a] + tau * D[a]) / s[a] + h[a];
                        double d = D[a] / s[a];
                        if (d == 0.0) {
                            if (!(c > -1.0 && c < N[a])) empty = true;
                            continue;
                        }
                        double t1 = (-1.0 - c) / d, t2 = (N[a] - c) / d;
                        lo = std::max(lo, std::min(t1, t2));
                        hi = std::min(hi, std::max(t1, t2));
                    }
                    if (empty || !(hi > lo)) continue;
                    // integers k with lo < (k + 1/2) dt < hi; hi - lo is at most the support box's
                    // diagonal, at most 2^22 steps, so the count is exact in double
                    const double k0 = std::floor(lo / dt - 0.5) + 1, k1 = std::ceil(hi / dt - 0.5) - 1;
                    if (k1 >= k0) local += (long long)(k1 - k0 + 1);
                }
        }
        sum.fetch_add(local);
    };
    unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned i = 1; i < nt; ++i) th.emplace_back(work);
    work();
    for (auto &t : th) t.join();
    const long long count = sum.load();
    {
        std::lock_guard<std::mutex> lk(g->mu);
        g->sample_count = count;
    }
    *total = count;
    return PYRONN_OK;
}

int pyronn_geom_read_flags(pyronn_geom_t g, int *out, int reset) {
    clear_error();
    if (!g || !out) return set_error(PYRONN_INVALID_ARG, "null argument");
    for (int i = 0; i < N_FLAGS; ++i) out[i] = 0;
    if (!g->d_flags) return PYRONN_OK;
    cudaError_t e = cudaMemcpy(out, g->d_flags, sizeof(int) * N_FLAGS, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reset) e = cudaMemset(g->d_flags, 0, sizeof(int) * N_FLAGS);
    if (e != cudaSuccess) return set_error(PYRONN_CUDA_ERROR, "reading device flags: %s", cudaGetErrorString(e));
    return PYRONN_OK;
}

const char *pyronn_last_error(void) { return g_last_error.c_str(); }

int pyronn_version(void) { return 100; }

}  // extern "C"
