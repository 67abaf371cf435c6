/*
 * FP64 CPU oracle for the ray-driven forward projector, its exact transpose and the
 * voxel-driven back-projector of "An update to PYRO-NN" (Sec. 2.1 and Sec. 2.2).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load this file:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it. It shares no
 * code with the CUDA library; both follow the same written definition.
 *
 * Plain, slow, obviously correct: one loop per definition, FP64 everywhere, no blocking,
 * no fusion, no incremental stepping. OpenMP only splits independent rays / voxels.
 *
 * Definition followed (Sec. 2.1: "rays are cast through the volume for each detector pixel,
 * accumulating absorption values along their path"; "projecting each voxel onto the detector
 * and accumulating"; Sec. 2.2: A and its adjoint A^T; Sec. 2.4: projection matrices built
 * from source / detector positions and detector directions). Where the paper is silent, the
 * readings below are the project's:
 *   - voxel (i,j,k) has its centre at ((i-(Nx-1)/2) sx + ox, (j-(Ny-1)/2) sy + oy, (k-(Nz-1)/2) sz + oz);
 *   - a ray is sampled at t_k = (k + 1/2) dt (mm) from its point closest to the volume centre;
 *   - the volume is the hat-function (trilinear, zero outside the grid) interpolant;
 *   - FP:  p_r = dt * sum_k I(c_r + t_k d_r);
 *   - A^T: (A^T y)_v = sum_r y_r dt sum_k prod_a hat(q_a(r,k) - v_a)   (exact transpose of FP);
 *   - BP:  b_v = sum_views omega * sum_{u',v'} q[v',u'] hat(u - u') hat(v - v'), with (u, v, w)
 *          the projection of the voxel centre, omega = 1 or 1/w^2; views with w <= 0 (voxel at or
 *          behind the source plane) contribute nothing.
 *
 * Parity status: every function here is pinned by tests that do not reuse this code
 * (closed forms, invariants, brute force on tiny grids); see tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Geometry description handed in by the caller. */
typedef struct {
    int nx, ny, nz;        /* volume shape (x fastest in memory: index (k*ny + j)*nx + i) */
    double sx, sy, sz;     /* voxel spacing, mm */
    double ox, oy, oz;     /* world position of the volume centre, mm */
    int nu, nv;            /* detector shape (u fastest in memory) */
    double du, dv;         /* pixel spacing, mm (used by parallel views) */
    double ou, ov;         /* detector centre offset along eu / ev, mm (parallel views) */
    int n_views;
    int kind;              /* 0 = parallel: view record = Dc[3] eu[3] ev[3] d[3]; 1 = perspective: P (3x4) */
    const double *views;   /* n_views x 12 doubles */
    double dt;             /* sampling step along rays, mm */
} og_t;

static double hat(double s) { double a = 1.0 - fabs(s); return a > 0.0 ? a : 0.0; }

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------------------
 * Geometry (Sec. 2.4, projection matrices from source / detector positions and directions).
 * ------------------------------------------------------------------------------------------- */

static int inv3(const double m[9], double out[9]) {
    double c00 = m[4] * m[8] - m[5] * m[7];
    double c01 = m[5] * m[6] - m[3] * m[8];
    double c02 = m[3] * m[7] - m[4] * m[6];
    double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    if (det == 0.0 || !isfinite(det)) return -1;
    double id = 1.0 / det;
    out[0] = c00 * id; out[1] = (m[2] * m[7] - m[1] * m[8]) * id; out[2] = (m[1] * m[5] - m[2] * m[4]) * id;
    out[3] = c01 * id; out[4] = (m[0] * m[8] - m[2] * m[6]) * id; out[5] = (m[2] * m[3] - m[0] * m[5]) * id;
    out[6] = c02 * id; out[7] = (m[1] * m[6] - m[0] * m[7]) * id; out[8] = (m[0] * m[4] - m[1] * m[3]) * id;
    return 0;
}

/* Circular (pitch = 0) or helical source orbit, Listing 1 parameters (sdd, sid, angular range):
 * view n at angle t = n * range / V; source sid (cos t, sin t, z_n); detector centre
 * -(sdd - sid) (cos t, sin t, 0) + (0, 0, z_n); eu = (-sin t, cos t, 0); ev = (0, 0, 1);
 * z_n = pitch * (n - (V-1)/2) * (range / V) / (2 pi). Arrays are V x 3. */
void or_frames_circular(int n_views, double angular_range, double sid, double sdd, double pitch,
                        double *src, double *det, double *eu, double *ev) {
    for (int n = 0; n < n_views; ++n) {
        double step = angular_range / n_views;
        double t = n * step;
        double c = cos(t), s = sin(t);
        double z = pitch * (n - 0.5 * (n_views - 1)) * step / (2.0 * M_PI);
        src[3 * n + 0] = sid * c;            src[3 * n + 1] = sid * s;            src[3 * n + 2] = z;
        det[3 * n + 0] = -(sdd - sid) * c;   det[3 * n + 1] = -(sdd - sid) * s;   det[3 * n + 2] = z;
        eu[3 * n + 0] = -s;                  eu[3 * n + 1] = c;                   eu[3 * n + 2] = 0.0;
        ev[3 * n + 0] = 0.0;                 ev[3 * n + 1] = 0.0;                 ev[3 * n + 2] = 1.0;
    }
}

/* P = M^{-1} [I | -S], M = [du eu | dv ev | D0 - S], D0 the centre of pixel (0, 0):
 * D0 = Dc + (ou - (nu-1)/2 du) eu + (ov - (nv-1)/2 dv) ev. P maps world (x, y, z, 1) to
 * (u w, v w, w) with (u, v) pixel indices and w the depth ratio to the detector plane.
 * Returns 0, or -1 if some view's M is singular. P is V x 12 (row-major 3 x 4). */
int or_pmat_from_frames(int n_views, const double *src, const double *det, const double *eu, const double *ev,
                        int nu, int nv, double du, double dv, double ou, double ov, double *P) {
    for (int n = 0; n < n_views; ++n) {
        const double *S = src + 3 * n, *Dc = det + 3 * n, *a = eu + 3 * n, *b = ev + 3 * n;
        double D0[3], M[9], Mi[9];
        for (int i = 0; i < 3; ++i)
            D0[i] = Dc[i] + (ou - 0.5 * (nu - 1) * du) * a[i] + (ov - 0.5 * (nv - 1) * dv) * b[i];
        for (int i = 0; i < 3; ++i) {
            M[3 * i + 0] = du * a[i];
            M[3 * i + 1] = dv * b[i];
            M[3 * i + 2] = D0[i] - S[i];
        }
        if (inv3(M, Mi)) return -1;
        double *p = P + 12 * n;
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) p[4 * r + c] = Mi[3 * r + c];
            p[4 * r + 3] = -(Mi[3 * r + 0] * S[0] + Mi[3 * r + 1] * S[1] + Mi[3 * r + 2] * S[2]);
        }
    }
    return 0;
}

/* Normalise user-supplied projection matrices (Sec. 2.1: "calibrated projection matrices from
 * real systems can be used"). P is defined up to a scale; the scale is fixed so that the first
 * column of inv(P[:, :3]) has length du (it is du * eu up to the scale) and w > 0 at the point
 * (cx, cy, cz). Returns -1 if a left 3x3 block is singular or w vanishes there. */
int or_normalise_pmat(int n_views, const double *Pin, double du, double cx, double cy, double cz, double *Pout) {
    for (int n = 0; n < n_views; ++n) {
        const double *p = Pin + 12 * n;
        double M[9], Mi[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) M[3 * r + c] = p[4 * r + c];
        if (inv3(M, Mi)) return -1;
        double l = sqrt(Mi[0] * Mi[0] + Mi[3] * Mi[3] + Mi[6] * Mi[6]);
        double w = p[8] * cx + p[9] * cy + p[10] * cz + p[11];
        if (l == 0.0 || w == 0.0) return -1;
        /* inv(kappa P) = inv(P) / kappa: |col0| / kappa = du  ->  kappa = l / du */
        double kappa = l / du;
        if (w < 0) kappa = -kappa;
        for (int i = 0; i < 12; ++i) Pout[12 * n + i] = kappa * p[i];
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Rays (Sec. 2.1, one ray per detector pixel).
 * ------------------------------------------------------------------------------------------- */

/* Ray of pixel (u, v) of view n: origin a and unit direction d in world mm. Perspective:
 * a = S = -inv(M') p4 and d = normalise(inv(M') (u, v, 1)) for P = [M' | p4] (normalised so the
 * direction points from the source to the detector). Parallel: a is the pixel centre on the
 * detector plane and d the view's direction. Returns -1 for a singular matrix. */
static int ray_of(const og_t *g, int n, double u, double v, double a[3], double d[3]) {
    const double *r = g->views + 12 * n;
    if (g->kind == 1) {
        double M[9], Mi[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[3 * i + j] = r[4 * i + j];
        if (inv3(M, Mi)) return -1;
        for (int i = 0; i < 3; ++i) {
            a[i] = -(Mi[3 * i + 0] * r[3] + Mi[3 * i + 1] * r[7] + Mi[3 * i + 2] * r[11]);
            d[i] = Mi[3 * i + 0] * u + Mi[3 * i + 1] * v + Mi[3 * i + 2];
        }
    } else {
        const double *Dc = r, *eu = r + 3, *ev = r + 6, *dir = r + 9;
        double su = (u - 0.5 * (g->nu - 1)) * g->du + g->ou;
        double sv = (v - 0.5 * (g->nv - 1)) * g->dv + g->ov;
        for (int i = 0; i < 3; ++i) {
            a[i] = Dc[i] + su * eu[i] + sv * ev[i];
            d[i] = dir[i];
        }
    }
    double nrm = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (nrm == 0.0) return -1;
    for (int i = 0; i < 3; ++i) d[i] /= nrm;
    return 0;
}

/* Index-space position of the k-th sample of a ray: the ray's point closest to the volume
 * centre C is c = a + ((C - a) . d) d; sample k sits at c + (k + 1/2) dt d (world mm), and its
 * index coordinate along each axis is (X - o) / s + (N - 1) / 2. */
typedef struct { double c[3], d[3]; } oray_t;

static void ray_ref(const og_t *g, const double a[3], const double d[3], oray_t *out) {
    double C[3] = {g->ox, g->oy, g->oz};
    double tau = (C[0] - a[0]) * d[0] + (C[1] - a[1]) * d[1] + (C[2] - a[2]) * d[2];
    for (int i = 0; i < 3; ++i) { out->c[i] = a[i] + tau * d[i]; out->d[i] = d[i]; }
}

static void sample_index(const og_t *g, const oray_t *ray, long k, double q[3]) {
    double t = (k + 0.5) * g->dt;
    double X[3];
    for (int i = 0; i < 3; ++i) X[i] = ray->c[i] + t * ray->d[i];
    q[0] = (X[0] - g->ox) / g->sx + 0.5 * (g->nx - 1);
    q[1] = (X[1] - g->oy) / g->sy + 0.5 * (g->ny - 1);
    q[2] = (X[2] - g->oz) / g->sz + 0.5 * (g->nz - 1);
}

/* Every sample inside the support box lies within |t| <= R of c, R the half-diagonal of the
 * box (-1, N_a) in each axis; a sample range covering [-R, R] is therefore complete. */
static long k_bound(const og_t *g) {
    double hx = 0.5 * (g->nx + 1) * g->sx, hy = 0.5 * (g->ny + 1) * g->sy, hz = 0.5 * (g->nz + 1) * g->sz;
    double R = sqrt(hx * hx + hy * hy + hz * hz);
    return (long)ceil(R / g->dt) + 2;
}

static int in_box(const og_t *g, const double q[3]) {
    return q[0] > -1.0 && q[0] < g->nx && q[1] > -1.0 && q[1] < g->ny && q[2] > -1.0 && q[2] < g->nz;
}

/* Hat-function interpolant I(q) = sum_v f_v prod_a hat(q_a - v_a), zero outside the grid. */
static double interp(const og_t *g, const double *vol, const double q[3]) {
    long i0 = (long)floor(q[0]), j0 = (long)floor(q[1]), k0 = (long)floor(q[2]);
    double s = 0.0;
    for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                long i = i0 + di, j = j0 + dj, k = k0 + dk;
                if (i < 0 || i >= g->nx || j < 0 || j >= g->ny || k < 0 || k >= g->nz) continue;
                double w = hat(q[0] - i) * hat(q[1] - j) * hat(q[2] - k);
                s += w * vol[((size_t)k * g->ny + j) * g->nx + i];
            }
    return s;
}

static double fp_one(const og_t *g, const double *vol, long ray_id) {
    int u = (int)(ray_id % g->nu);
    int v = (int)((ray_id / g->nu) % g->nv);
    int n = (int)(ray_id / ((long)g->nu * g->nv));
    double a[3], d[3], q[3];
    oray_t ray;
    if (ray_of(g, n, u, v, a, d)) return NAN;
    ray_ref(g, a, d, &ray);
    long K = k_bound(g);
    double acc = 0.0;
    for (long k = -K - 1; k <= K; ++k) {
        sample_index(g, &ray, k, q);
        if (!in_box(g, q)) continue;
        acc += interp(g, vol, q);
    }
    return g->dt * acc;
}

/* Forward projection of every ray; sino is [V][nv][nu]. */
void or_fp(const og_t *g, const double *vol, double *sino) {
    long nr = (long)g->n_views * g->nv * g->nu;
#pragma omp parallel for schedule(dynamic, 64)
    for (long r = 0; r < nr; ++r) sino[r] = fp_one(g, vol, r);
}

/* Forward projection of the listed rays only (ray id = (view * nv + v) * nu + u). */
void or_fp_rays(const og_t *g, const double *vol, long n, const int64_t *ids, double *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < n; ++i) out[i] = fp_one(g, vol, (long)ids[i]);
}

/* Number of samples of each view that lie inside the open support box (-1, N_a) on every axis. */
void or_count_samples(const og_t *g, int64_t *per_view) {
    long K = k_bound(g);
    for (int n = 0; n < g->n_views; ++n) {
        int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
        for (long p = 0; p < (long)g->nu * g->nv; ++p) {
            double a[3], d[3], q[3];
            oray_t ray;
            if (ray_of(g, n, (double)(p % g->nu), (double)(p / g->nu), a, d)) continue;
            ray_ref(g, a, d, &ray);
            for (long k = -K - 1; k <= K; ++k) {
                sample_index(g, &ray, k, q);
                total += in_box(g, q);
            }
        }
        per_view[n] = total;
    }
}

/* Exact transpose of the forward projector, scattering y_r * dt * prod hat into vol for the
 * listed rays (serial; vol is accumulated into, not cleared). */
static void adj_one(const og_t *g, long ray_id, double y, double *vol) {
    if (y == 0.0) return;
    int u = (int)(ray_id % g->nu);
    int v = (int)((ray_id / g->nu) % g->nv);
    int n = (int)(ray_id / ((long)g->nu * g->nv));
    double a[3], d[3], q[3];
    oray_t ray;
    if (ray_of(g, n, u, v, a, d)) return;
    ray_ref(g, a, d, &ray);
    long K = k_bound(g);
    for (long k = -K - 1; k <= K; ++k) {
        sample_index(g, &ray, k, q);
        if (!in_box(g, q)) continue;
        long i0 = (long)floor(q[0]), j0 = (long)floor(q[1]), k0 = (long)floor(q[2]);
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    long i = i0 + di, j = j0 + dj, kk = k0 + dk;
                    if (i < 0 || i >= g->nx || j < 0 || j >= g->ny || kk < 0 || kk >= g->nz) continue;
                    double w = hat(q[0] - i) * hat(q[1] - j) * hat(q[2] - kk);
                    vol[((size_t)kk * g->ny + j) * g->nx + i] += y * g->dt * w;
                }
    }
}

void or_adjoint_rays(const og_t *g, long n, const int64_t *ids, const double *y, double *vol) {
    for (long i = 0; i < n; ++i) adj_one(g, (long)ids[i], y[i], vol);
}

/* Full transpose: vol = A^T sino. Threads scatter into private buffers that are summed in a
 * fixed order at the end. Returns -1 if a buffer cannot be allocated. */
int or_adjoint(const og_t *g, const double *sino, double *vol) {
    size_t nvox = (size_t)g->nx * g->ny * g->nz;
    long nr = (long)g->n_views * g->nv * g->nu;
    int nt = or_max_threads();
    double *buf = (double *)calloc((size_t)nt * nvox, sizeof(double));
    if (!buf) return -1;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = buf + (size_t)tid * nvox;
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < nr; ++r) adj_one(g, r, sino[r], mine);
    }
    memset(vol, 0, nvox * sizeof(double));
    for (int t = 0; t < nt; ++t)
        for (size_t i = 0; i < nvox; ++i) vol[i] += buf[(size_t)t * nvox + i];
    free(buf);
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Voxel-driven back-projection (Sec. 2.1: project each voxel onto the detector, accumulate).
 * ------------------------------------------------------------------------------------------- */

/* Detector coordinates (u, v) and depth ratio w of world point X in view n. */
static void project(const og_t *g, int n, const double X[3], double *u, double *v, double *w) {
    const double *r = g->views + 12 * n;
    if (g->kind == 1) {
        double a = r[0] * X[0] + r[1] * X[1] + r[2] * X[2] + r[3];
        double b = r[4] * X[0] + r[5] * X[1] + r[6] * X[2] + r[7];
        double c = r[8] * X[0] + r[9] * X[1] + r[10] * X[2] + r[11];
        *u = a / c; *v = b / c; *w = c;
    } else {
        const double *Dc = r, *eu = r + 3, *ev = r + 6;
        double Y[3] = {X[0] - Dc[0], X[1] - Dc[1], X[2] - Dc[2]};
        *u = ((Y[0] * eu[0] + Y[1] * eu[1] + Y[2] * eu[2]) - g->ou) / g->du + 0.5 * (g->nu - 1);
        *v = ((Y[0] * ev[0] + Y[1] * ev[1] + Y[2] * ev[2]) - g->ov) / g->dv + 0.5 * (g->nv - 1);
        *w = 1.0;
    }
}

static double bp_one(const og_t *g, const double *sino, int weight_mode, long vox) {
    int i = (int)(vox % g->nx);
    int j = (int)((vox / g->nx) % g->ny);
    int k = (int)(vox / ((long)g->nx * g->ny));
    double X[3] = {(i - 0.5 * (g->nx - 1)) * g->sx + g->ox,
                   (j - 0.5 * (g->ny - 1)) * g->sy + g->oy,
                   (k - 0.5 * (g->nz - 1)) * g->sz + g->oz};
    double acc = 0.0;
    for (int n = 0; n < g->n_views; ++n) {
        double u, v, w;
        project(g, n, X, &u, &v, &w);
        /* reading: a voxel at or behind the source plane (w <= 0) receives nothing from the view */
        if (g->kind == 1 && !(w > 0.0)) continue;
        long u0 = (long)floor(u), v0 = (long)floor(v);
        const double *q = sino + (size_t)n * g->nu * g->nv;
        double s = 0.0;
        for (int dv = 0; dv < 2; ++dv)
            for (int du = 0; du < 2; ++du) {
                long uu = u0 + du, vv = v0 + dv;
                if (uu < 0 || uu >= g->nu || vv < 0 || vv >= g->nv) continue;
                s += q[(size_t)vv * g->nu + uu] * hat(u - uu) * hat(v - vv);
            }
        double omega = (weight_mode == 1) ? 1.0 / (w * w) : 1.0;
        acc += omega * s;
    }
    return acc;
}

/* vol = BP(sino); weight_mode 0: omega = 1, 1: omega = 1 / w^2. */
void or_bp(const og_t *g, const double *sino, int weight_mode, double *vol) {
    long nvox = (long)g->nx * g->ny * g->nz;
#pragma omp parallel for schedule(dynamic, 256)
    for (long x = 0; x < nvox; ++x) vol[x] = bp_one(g, sino, weight_mode, x);
}

/* BP at the listed voxels only (voxel id = (k * ny + j) * nx + i). */
void or_bp_voxels(const og_t *g, const double *sino, int weight_mode, long n, const int64_t *ids, double *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < n; ++i) out[i] = bp_one(g, sino, weight_mode, (long)ids[i]);
}

/* ---------------------------------------------------------------------------------------------
 * Filtered back-projection (Sec. 2.2: x = A^T F^T K F p with a ramp K; Listing 1 builds it from a
 * ramp filter, a Fourier transform and the cone back-projection). The filter is applied here as a
 * direct convolution with the ramp's taps along each detector row, after the cosine pre-weighting
 * of divergent beams (FDK), and scaled so that the 1/w^2-weighted (divergent) or plain (parallel)
 * voxel-driven BP of the result is the reconstruction.
 * ------------------------------------------------------------------------------------------- */

/* Ramp taps for unit detector spacing at offset k. filter 0 (Ram-Lak): the ramp band-limited to the
 * detector's Nyquist frequency, sampled (1/4 at 0, 0 at even offsets, -1/(pi k)^2 at odd ones);
 * filter 1 (Shepp-Logan): the ramp times a sinc window, -2 / (pi^2 (4 k^2 - 1)). */
static double ramp_tap(long k, int filter) {
    const double pi = 3.14159265358979323846;
    if (filter == 1) return -2.0 / (pi * pi * (4.0 * (double)k * (double)k - 1.0));
    if (k == 0) return 0.25;
    if (k % 2 == 0) return 0.0;
    return -1.0 / (pi * pi * (double)k * (double)k);
}

/* out = scale (1 / tau) sum_m h(u - m) c(m, v) p(m, v) per detector row, with, per view:
 *   perspective: the detector plane is w = 1 and the source plane w = 0 (P's third row gives w),
 *     so the source-detector distance is sdd = 1 / |n| (n the row's first three entries); the
 *     ratio r = w(volume centre) = sid / sdd; pixel (u, v) lies at S + inv(M')(u, v, 1), at distance
 *     L(u, v) from the source, and c = sdd / L is the cosine of its ray; tau = r |inv(M') e_u| is the
 *     detector pitch scaled to the volume centre;
 *   parallel: c = 1, r = 1, tau = du;
 *   scale = (pi / V) r^2 (the angular step of a [0, pi) parallel or [0, 2 pi) divergent scan with the
 *   1/2 of the full scan, and the FDK distance factor that turns the 1/w^2 weight into (sid/U)^2).
 * Returns -1 for a singular view. */
int or_fbp_filter(const og_t *g, int filter, const double *sino, double *out) {
    const double pi = 3.14159265358979323846;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int n = 0; n < g->n_views; ++n) {
        const double *r = g->views + 12 * n;
        double tau = g->du, ratio = 1.0, sdd = 1.0, Mi[9] = {0};
        if (g->kind == 1) {
            double M[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) M[3 * i + j] = r[4 * i + j];
            if (inv3(M, Mi)) {
#pragma omp atomic write
                bad = 1;
                continue;
            }
            const double nn = sqrt(r[8] * r[8] + r[9] * r[9] + r[10] * r[10]);
            sdd = 1.0 / nn;
            ratio = r[8] * g->ox + r[9] * g->oy + r[10] * g->oz + r[11];
            const double pu = sqrt(Mi[0] * Mi[0] + Mi[3] * Mi[3] + Mi[6] * Mi[6]);
            tau = ratio * pu;
        }
        const double scale = pi / g->n_views * ratio * ratio / tau;
        double *pw = (double *)malloc(sizeof(double) * (size_t)g->nu);
        for (int v = 0; v < g->nv; ++v) {
            const double *row = sino + ((size_t)n * g->nv + v) * g->nu;
            double *orow = out + ((size_t)n * g->nv + v) * g->nu;
            for (int m = 0; m < g->nu; ++m) {
                double c = 1.0;
                if (g->kind == 1) {
                    double d[3];
                    for (int i = 0; i < 3; ++i) d[i] = Mi[3 * i + 0] * m + Mi[3 * i + 1] * v + Mi[3 * i + 2];
                    c = sdd / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                }
                pw[m] = c * row[m];
            }
            for (int u = 0; u < g->nu; ++u) {
                double s = 0.0;
                for (int m = 0; m < g->nu; ++m) s += ramp_tap((long)u - m, filter) * pw[m];
                orow[u] = scale * s;
            }
        }
        free(pw);
    }
    return bad ? -1 : 0;
}
