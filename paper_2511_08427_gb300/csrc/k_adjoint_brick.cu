// Output-stationary matched adjoint (same operator as adjoint_scatter_kernel, Sec. 2.2 A^T).
//
// One CTA owns a BX x BY x BZ brick of the output volume and accumulates it in shared memory over
// every view; the brick is written once at the end, so there are no global atomics. For each
// view the CTA enumerates the detector pixels whose rays can reach the brick (the bounding
// rectangle of the projected, one-voxel-extended brick), walks each such ray through the brick
// and scatters y_r dt times the eight trilinear weights of every sample into the brick with
// shared-memory atomics (only corners inside the brick; the neighbouring bricks take the rest).
//
// Precision. A sample's position is computed relative to the brick centre, so every FP32
// quantity in the sample loop is of the size of the brick:
//   - per (brick, view), in FP64 (one lane per view): the point A where the footprint-corner ray
//     meets the plane through the brick centre (parallel to the detector; orthogonal to the rays
//     for parallel beams), the per-pixel steps of that point and of the ray direction, and the
//     lattice phase T = (X_b - C) . d_ref = (K + f) dt of the corner ray;
//   - per ray, in FP32 on small quantities: its point P on that plane, its unit direction d,
//     the change of direction from the corner ray (formed without cancellation), and
//     e = (X_b - C) . (d - d_ref) + P . d, so that sample k = K + j sits at
//     P + ((j + 1/2 - f) dt - e) d.
// This keeps the sample positions within ~1e-6 voxel of the FP64 definition, which the
// random-cotangent parity tests need (the adjoint of a noise cotangent is itself a random-walk
// sum, so relative position errors are not averaged away).
#include "device_common.cuh"

namespace pyronn {

struct BrickView {
    int u_lo, v_lo, nu_r, nv_r;     // footprint rectangle (nu_r == 0: empty)
    float A[3];                     // corner-ray point on the brick plane, relative to the brick centre
    float Eu[3], Ev[3];             // per-pixel steps of that point
    float D[3];                     // corner-ray direction (unnormalised)
    float Cu[3], Cv[3];             // per-pixel steps of the direction (zero for parallel beams)
    float inv_nD, nD2;              // 1 / |D|, |D|^2
    float dref[3];                  // D / |D|
    float f;                        // phase: (X_b - C) . dref = (K + f) dt, 0 <= f < 1
    int pad;
};

constexpr int ADJ_VIEW_CHUNK = 32;

// floor / fraction by the round-down magic-number addition; q is clamped to +-64 (brick-local
// positions of in-brick samples are within [-1, 16]; anything beyond contributes nothing)
__device__ __forceinline__ void floor_frac_clamped(float q, int &i, float &f) {
    const float M = 12582912.0f;
    q = fminf(fmaxf(q, -64.0f), 64.0f);
    const float t = __fadd_rd(q, M);
    i = __float_as_int(t) - 0x4B400000;
    f = q - (t - M);
}

// no "memory" clobber: the accumulator is read only after a barrier (a compiler fence), and a clobber
// would make the compiler reload shared values after each reduction
__device__ __forceinline__ void red_add_shared(unsigned addr, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v));
}

// add the eight corner weights of cell (ix, iy, iz) to the brick accumulator (corners inside only)
template <int BX, int BY, int BZ>
__device__ __forceinline__ void flush_cell(unsigned acc_base, int ix, int iy, int iz, float a0, float a1, float a2,
                                           float a3, float a4, float a5, float a6, float a7) {
    const bool x0 = (unsigned)ix < (unsigned)BX, x1 = (unsigned)(ix + 1) < (unsigned)BX;
    const bool y0 = (unsigned)iy < (unsigned)BY, y1 = (unsigned)(iy + 1) < (unsigned)BY;
    const bool z0 = (unsigned)iz < (unsigned)BZ, z1 = (unsigned)(iz + 1) < (unsigned)BZ;
    const unsigned base = acc_base + 4u * (unsigned)((iz * BY + iy) * BX + ix);
    constexpr unsigned SY = 4u * BX, SZ = 4u * BX * BY;
    if (z0 && y0 && x0) red_add_shared(base, a0);
    if (z0 && y0 && x1) red_add_shared(base + 4u, a1);
    if (z0 && y1 && x0) red_add_shared(base + SY, a2);
    if (z0 && y1 && x1) red_add_shared(base + SY + 4u, a3);
    if (z1 && y0 && x0) red_add_shared(base + SZ, a4);
    if (z1 && y0 && x1) red_add_shared(base + SZ + 4u, a5);
    if (z1 && y1 && x0) red_add_shared(base + SZ + SY, a6);
    if (z1 && y1 && x1) red_add_shared(base + SZ + SY + 4u, a7);
}

// FP64 per-(brick, view) set-up. Xb: brick centre relative to the volume centre (world mm);
// ext_lo / ext_hi: the extended brick (one voxel around it) relative to the volume centre.
__device__ void brick_view_setup(const OpParams &p, int view, const double Xb[3], const double ext_lo[3],
                                 const double ext_hi[3], BrickView &bv) {
    const double *x = p.views64 + (size_t)view * VIEW64_STRIDE;
    const int nu = p.det.nu, nv = p.det.nv;
    const double hu = 0.5 * (nu - 1), hv = 0.5 * (nv - 1);
    // footprint: project the eight corners of the extended brick
    double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
    bool behind = false;
    for (int c = 0; c < 8; ++c) {
        double X[3] = {(c & 1) ? ext_hi[0] : ext_lo[0], (c & 2) ? ext_hi[1] : ext_lo[1],
                       (c & 4) ? ext_hi[2] : ext_lo[2]};
        double u, v;
        if (p.perspective) {
            double a = x[0] * X[0] + x[1] * X[1] + x[2] * X[2] + x[3];
            double b = x[4] * X[0] + x[5] * X[1] + x[6] * X[2] + x[7];
            double w = x[8] * X[0] + x[9] * X[1] + x[10] * X[2] + x[11];
            if (!(w > 0.0)) {
                behind = true;
                continue;
            }
            u = a / w;
            v = b / w;
        } else {
            double Y[3] = {X[0] - x[0], X[1] - x[1], X[2] - x[2]};
            u = ((Y[0] * x[3] + Y[1] * x[4] + Y[2] * x[5]) - p.ou) / p.du + hu;
            v = ((Y[0] * x[6] + Y[1] * x[7] + Y[2] * x[8]) - p.ov) / p.dv + hv;
        }
        umin = fmin(umin, u); umax = fmax(umax, u);
        vmin = fmin(vmin, v); vmax = fmax(vmax, v);
    }
    int u_lo, u_hi, v_lo, v_hi;
    if (behind) {
        u_lo = 0; u_hi = nu - 1; v_lo = 0; v_hi = nv - 1;
    } else {
        umin = fmax(umin, -2.0); umax = fmin(umax, (double)nu + 1.0);
        vmin = fmax(vmin, -2.0); vmax = fmin(vmax, (double)nv + 1.0);
        u_lo = max((int)ceil(umin) - 1, 0); u_hi = min((int)floor(umax) + 1, nu - 1);
        v_lo = max((int)ceil(vmin) - 1, 0); v_hi = min((int)floor(vmax) + 1, nv - 1);
    }
    bv.u_lo = u_lo; bv.v_lo = v_lo;
    bv.nu_r = (u_hi >= u_lo && v_hi >= v_lo) ? u_hi - u_lo + 1 : 0;
    bv.nv_r = (u_hi >= u_lo && v_hi >= v_lo) ? v_hi - v_lo + 1 : 0;
    if (bv.nu_r == 0) return;

    double A[3], Eu[3], Ev[3], D[3], Cu[3], Cv[3];
    if (p.perspective) {
        const double *S = x + 12, *c0 = x + 15, *c1 = x + 18, *c2 = x + 21, *nrm = x + 24;
        double den = x[27];
        double lam = ((Xb[0] - S[0]) * nrm[0] + (Xb[1] - S[1]) * nrm[1] + (Xb[2] - S[2]) * nrm[2]) / den;
        for (int i = 0; i < 3; ++i) {
            D[i] = c2[i] + u_lo * c0[i] + v_lo * c1[i];
            A[i] = S[i] + lam * D[i] - Xb[i];
            Eu[i] = lam * c0[i];
            Ev[i] = lam * c1[i];
            Cu[i] = c0[i];
            Cv[i] = c1[i];
        }
    } else {
        const double *Dc = x, *eu = x + 3, *ev = x + 6, *d = x + 9;
        double su = (u_lo - hu) * p.du + p.ou, sv = (v_lo - hv) * p.dv + p.ov;
        double a0[3], du_[3], dv_[3];
        for (int i = 0; i < 3; ++i) {
            a0[i] = Dc[i] + su * eu[i] + sv * ev[i] - Xb[i];   // corner-ray origin relative to X_b
            du_[i] = p.du * eu[i];
            dv_[i] = p.dv * ev[i];
        }
        double pa = a0[0] * d[0] + a0[1] * d[1] + a0[2] * d[2];
        double pu = du_[0] * d[0] + du_[1] * d[1] + du_[2] * d[2];
        double pv = dv_[0] * d[0] + dv_[1] * d[1] + dv_[2] * d[2];
        for (int i = 0; i < 3; ++i) {
            A[i] = a0[i] - pa * d[i];
            Eu[i] = du_[i] - pu * d[i];
            Ev[i] = dv_[i] - pv * d[i];
            D[i] = d[i];
            Cu[i] = 0.0;
            Cv[i] = 0.0;
        }
    }
    double nD2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
    double nD = sqrt(nD2);
    double dref[3] = {D[0] / nD, D[1] / nD, D[2] / nD};
    double T = (Xb[0] * dref[0] + Xb[1] * dref[1] + Xb[2] * dref[2]) / (double)p.dt;
    double K = floor(T);
    for (int i = 0; i < 3; ++i) {
        bv.A[i] = (float)A[i]; bv.Eu[i] = (float)Eu[i]; bv.Ev[i] = (float)Ev[i];
        bv.D[i] = (float)D[i]; bv.Cu[i] = (float)Cu[i]; bv.Cv[i] = (float)Cv[i];
        bv.dref[i] = (float)dref[i];
    }
    bv.inv_nD = (float)(1.0 / nD);
    bv.nD2 = (float)nD2;
    bv.f = (float)(T - K);
}

template <int BX, int BY, int BZ>
struct AdjShared {
    float acc[BX * BY * BZ];
    BrickView sv[ADJ_VIEW_CHUNK];
    int s_off[ADJ_VIEW_CHUNK + 1];
};

// Adjoint of one brick (block indices bxi, byi, bzi) of volume b: accumulates every view in shared
// memory and writes the brick once.
template <typename T, int BX, int BY, int BZ>
__device__ __forceinline__ void adjoint_brick(const OpParams &p, const T *__restrict__ sino, T *__restrict__ vol,
                                              int bxi, int byi, int bzi, int b, AdjShared<BX, BY, BZ> &S) {
    constexpr int NT = 256;
    constexpr int NB = BX * BY * BZ;
    float *acc = S.acc;
    BrickView *sv = S.sv;
    int *s_off = S.s_off;
    const int bx0 = bxi * BX, by0 = byi * BY;
    const int bz0 = bzi * BZ;
    const int tid = threadIdx.x;
    const T *sb = sino + (long long)b * p.sino_elems;

    __syncthreads();   // the previous brick's write-back is done with the accumulator
    for (int i = tid; i < NB; i += NT) acc[i] = 0.0f;
    const unsigned acc_base = (unsigned)__cvta_generic_to_shared(acc);

    // brick centre and extended brick, relative to the volume centre (world mm)
    const double sp[3] = {p.sx, p.sy, p.sz};
    const double hv3[3] = {0.5 * (p.vol.nx - 1), 0.5 * (p.vol.ny - 1), 0.5 * (p.vol.nz - 1)};
    const int b0[3] = {bx0, by0, bz0};
    const int Bd[3] = {BX, BY, BZ};
    double Xb[3], elo[3], ehi[3];
    for (int a = 0; a < 3; ++a) {
        Xb[a] = (b0[a] + 0.5 * (Bd[a] - 1) - hv3[a]) * sp[a];
        elo[a] = (b0[a] - 1 - hv3[a]) * sp[a];
        ehi[a] = (b0[a] + Bd[a] - hv3[a]) * sp[a];
    }
    const float Xbf[3] = {(float)Xb[0], (float)Xb[1], (float)Xb[2]};
    const float isx = p.vol.isx, isy = p.vol.isy, isz = p.vol.isz;
    const float hbx = 0.5f * (BX - 1), hby = 0.5f * (BY - 1), hbz = 0.5f * (BZ - 1);
    const float dt = p.dt;
    const int nu = p.det.nu, nv = p.det.nv;

    for (int n0 = 0; n0 < p.n_views; n0 += ADJ_VIEW_CHUNK) {
        const int nc = min(ADJ_VIEW_CHUNK, p.n_views - n0);
        __syncthreads();   // previous chunk's readers of sv are done
        if (tid < nc) brick_view_setup(p, n0 + tid, Xb, elo, ehi, sv[tid]);
        __syncthreads();
        if (tid == 0) {
            // rectangles padded to multiples of 3: rays are visited in nine interleaved 3 x 3 phases,
            // so the rays of consecutive lanes are 3 pixels apart and rarely share a voxel
            int o = 0;
            for (int c = 0; c < nc; ++c) {
                s_off[c] = o;
                o += 9 * ((sv[c].nu_r + 2) / 3) * ((sv[c].nv_r + 2) / 3);
            }
            s_off[nc] = o;
        }
        __syncthreads();
        const int total = s_off[nc];
        int c = 0;
        for (int r = tid; r < total; r += NT) {
            while (r >= s_off[c + 1]) ++c;
            const BrickView &V = sv[c];
            const int lr = r - s_off[c];
            const int nu3 = (V.nu_r + 2) / 3, nv3 = (V.nv_r + 2) / 3;
            const int cls = nu3 * nv3;
            const int ph = lr / cls, qq = lr - ph * cls;
            const int dv3 = qq / nu3;
            const int du_ = (ph % 3) + 3 * (qq - dv3 * nu3), dv_ = (ph / 3) + 3 * dv3;
            if (du_ >= V.nu_r || dv_ >= V.nv_r) continue;
            const int u = V.u_lo + du_, v = V.v_lo + dv_;
            float y = ldg_f32(sb + ((long long)(n0 + c) * nv + v) * nu + u);
            if (y == 0.0f) continue;
            y *= dt;
            const float fu = (float)du_, fv = (float)dv_;
            // ray point on the brick plane and direction
            float P0 = fmaf(fv, V.Ev[0], fmaf(fu, V.Eu[0], V.A[0]));
            float P1 = fmaf(fv, V.Ev[1], fmaf(fu, V.Eu[1], V.A[1]));
            float P2 = fmaf(fv, V.Ev[2], fmaf(fu, V.Eu[2], V.A[2]));
            float L0 = fmaf(fv, V.Cv[0], fu * V.Cu[0]);
            float L1 = fmaf(fv, V.Cv[1], fu * V.Cu[1]);
            float L2 = fmaf(fv, V.Cv[2], fu * V.Cu[2]);
            // |D + L|^2 = |D|^2 (1 + eps)
            float DL = fmaf(V.D[0], L0, fmaf(V.D[1], L1, V.D[2] * L2));
            float LL = fmaf(L0, L0, fmaf(L1, L1, L2 * L2));
            float eps = (2.0f * DL + LL) / V.nD2;
            float sq = sqrtf(1.0f + eps);
            float inv = V.inv_nD / sq;
            float d0 = (V.D[0] + L0) * inv, d1 = (V.D[1] + L1) * inv, d2 = (V.D[2] + L2) * inv;
            // d - dref, without cancellation
            float g = -eps / (sq * (1.0f + sq));
            float dd0 = fmaf(V.dref[0], g, L0 * inv);
            float dd1 = fmaf(V.dref[1], g, L1 * inv);
            float dd2 = fmaf(V.dref[2], g, L2 * inv);
            float e = fmaf(Xbf[0], dd0, fmaf(Xbf[1], dd1, Xbf[2] * dd2)) + fmaf(P0, d0, fmaf(P1, d1, P2 * d2));
            // sample j at s_j = j dt + c_r along d from P; brick-local index q = (P + s d) / s + hb
            const float c_r = (0.5f - V.f) * dt - e;
            const float qP0 = fmaf(P0, isx, hbx), qP1 = fmaf(P1, isy, hby), qP2 = fmaf(P2, isz, hbz);
            const float qd0 = d0 * isx, qd1 = d1 * isy, qd2 = d2 * isz;
            // s-range where the sample lies in the extended brick [-1, B) on every axis
            float slo = -3.0e38f, shi = 3.0e38f;
            bool empty = false;
            clip_axis(qP0, qd0, BX, slo, shi, empty);
            clip_axis(qP1, qd1, BY, slo, shi, empty);
            clip_axis(qP2, qd2, BZ, slo, shi, empty);
            if (empty || !(shi > slo)) continue;
            const float idt = 1.0f / dt;
            const int j0 = (int)floorf((slo - c_r) * idt);
            const int j1 = (int)ceilf((shi - c_r) * idt);
            // the eight weights accumulate in registers while the sample stays in one cell and are
            // flushed to the brick (no-return shared-memory reductions) when it moves on
            float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f, a4 = 0.0f, a5 = 0.0f, a6 = 0.0f, a7 = 0.0f;
            int pix = 0, piy = 0, piz = 0, pkey = -1;
            for (int j = j0; j <= j1 + 1; ++j) {
                int key = -2, ix = 0, iy = 0, iz = 0;
                float ax = 0.0f, ay = 0.0f, az = 0.0f;
                if (j <= j1) {
                    const float s = fmaf((float)j, dt, c_r);
                    const float qx = fmaf(s, qd0, qP0), qy = fmaf(s, qd1, qP1), qz = fmaf(s, qd2, qP2);
                    floor_frac_clamped(qx, ix, ax);
                    floor_frac_clamped(qy, iy, ay);
                    floor_frac_clamped(qz, iz, az);
                    key = ((iz + 8) << 20) | ((iy + 8) << 10) | (ix + 8);
                }
                if (key != pkey) {
                    if (pkey >= 0) flush_cell<BX, BY, BZ>(acc_base, pix, piy, piz, a0, a1, a2, a3, a4, a5, a6, a7);
                    a0 = a1 = a2 = a3 = a4 = a5 = a6 = a7 = 0.0f;
                    pkey = key;
                    pix = ix; piy = iy; piz = iz;
                }
                if (j <= j1) {
                    const float wz1 = y * az, wz0 = y - wz1;
                    const float w00 = wz0 * (1.0f - ay), w01 = wz0 * ay, w10 = wz1 * (1.0f - ay), w11 = wz1 * ay;
                    a0 = fmaf(w00, 1.0f - ax, a0);
                    a1 = fmaf(w00, ax, a1);
                    a2 = fmaf(w01, 1.0f - ax, a2);
                    a3 = fmaf(w01, ax, a3);
                    a4 = fmaf(w10, 1.0f - ax, a4);
                    a5 = fmaf(w10, ax, a5);
                    a6 = fmaf(w11, 1.0f - ax, a6);
                    a7 = fmaf(w11, ax, a7);
                }
            }
        }
    }
    __syncthreads();
    T *vb = vol + (long long)b * p.vol_elems;
    for (int i = tid; i < NB; i += NT) {
        const int lx = i % BX, ly = (i / BX) % BY, lz = i / (BX * BY);
        const int gx = bx0 + lx, gy = by0 + ly, gz = bz0 + lz;
        if (gx < p.vol.nx && gy < p.vol.ny && gz < p.vol.nz)
            vb[((long long)gz * p.vol.ny + gy) * p.vol.nx + gx] = from_f32<T>(acc[i]);
    }
}

template <typename T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(256, 4) adjoint_brick_kernel(OpParams p, const T *__restrict__ sino,
                                                            T *__restrict__ vol) {
    __shared__ AdjShared<BX, BY, BZ> S;
    const int nbz = (p.vol.nz + BZ - 1) / BZ;
    adjoint_brick<T, BX, BY, BZ>(p, sino, vol, blockIdx.x, blockIdx.y, blockIdx.z % nbz, blockIdx.z / nbz, S);
}

// Persistent launch over the bricks of several volumes (items = bricks, largest volumes first).
template <typename T, int BX, int BY, int BZ>
__global__ void __launch_bounds__(256, 4) adjoint_brick_batched_kernel(const __grid_constant__ PlanLaunch L) {
    __shared__ AdjShared<BX, BY, BZ> S;
    __shared__ int s_item;
    const long long total = L.item_end[L.n - 1];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(L.counter, 1);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        int i = 0;
        while (item >= L.item_end[i]) ++i;
        const PlanVolume &V = L.v[i];
        const int local = (int)(item - (i ? L.item_end[i - 1] : 0));
        const int bxi = local % V.ntx, byi = (local / V.ntx) % V.nty, bzi = local / (V.ntx * V.nty);
        adjoint_brick<T, BX, BY, BZ>(V.p, (const T *)V.in, (T *)V.out, bxi, byi, bzi, 0, S);
    }
}

template <typename T, int BX, int BY, int BZ>
static int launch_brick_t(const OpParams &p, const void *sino, void *vol, cudaStream_t st) {
    const int nbx = ceil_div(p.vol.nx, BX), nby = ceil_div(p.vol.ny, BY), nbz = ceil_div(p.vol.nz, BZ);
    const int per_launch = 65535 / nbz > 0 ? 65535 / nbz : 1;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        int nb = p.batch - b0 < per_launch ? p.batch - b0 : per_launch;
        dim3 grid(nbx, nby, nbz * nb);
        adjoint_brick_kernel<T, BX, BY, BZ><<<grid, 256, 0, st>>>(p, (const T *)sino + b0 * p.sino_elems,
                                                                   (T *)vol + b0 * p.vol_elems);
    }
    return (int)cudaGetLastError();
}

template <typename T>
static int launch_brick_dims(const OpParams &p, const void *sino, void *vol, cudaStream_t st) {
    if (p.vol.nz == 1) return launch_brick_t<T, 32, 32, 1>(p, sino, vol, st);
    return launch_brick_t<T, 16, 16, 16>(p, sino, vol, st);
}

template <typename T>
static int launch_adj_batched_t(const PlanLaunch &L, int grid, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(L.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return (int)e;
    adjoint_brick_batched_kernel<T, 16, 16, 16><<<grid, 256, 0, st>>>(L);
    return (int)cudaGetLastError();
}

// bricks of the batched adjoint are 16^3 (3D volumes only)
int launch_adjoint_brick_batched(const PlanLaunch &L, int dtype, int grid, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_adj_batched_t<float>(L, grid, st);
        case PYRONN_BF16: return launch_adj_batched_t<__nv_bfloat16>(L, grid, st);
        case PYRONN_F16: return launch_adj_batched_t<__half>(L, grid, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

int adjoint_brick_batched_occupancy(int *blocks_per_sm) {
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,
                                                              adjoint_brick_batched_kernel<float, 16, 16, 16>, 256, 0);
}

int launch_adjoint_brick(const OpParams &p, const void *sino, void *vol, int dtype, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_brick_dims<float>(p, sino, vol, st);
        case PYRONN_BF16: return launch_brick_dims<__nv_bfloat16>(p, sino, vol, st);
        case PYRONN_F16: return launch_brick_dims<__half>(p, sino, vol, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace pyronn
