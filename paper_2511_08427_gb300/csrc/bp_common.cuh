// Per-(brick, view) set-up of the brick back-projectors (FP64 on the device) and their detector
// helpers, shared by the L1-path kernel (k_bp_brick.cu) and the TMA-staged one (k_bp_tma.cu).
#pragma once

#include "device_common.cuh"

namespace pyronn {

constexpr int BPB_X = 16, BPB_Y = 16, BPB_NT = BPB_X * BPB_Y, BPB_CHUNK = 32;

struct BpView {
    float Qa[3], Qb[3], Pw[3];   // per voxel-index step
    float w0;                    // depth ratio of the brick centre
    float fu, fv;                // fractional parts of u0, v0
    int U0, V0;                  // integer parts of u0, v0
    int flat;                    // 1: Qa_z == 0 and Pw_z == 0 (u, w constant along z)
    int valid;                   // 0: the brick centre is at or behind the source plane
    int eu, ev;                  // half-extent (pixels, rounded up) of the brick's shadow around (U0, V0):
                                 // every tap of the brick lies in [U0 - eu, U0 + eu] x [V0 - ev, V0 + ev];
                                 // -1: unbounded (the brick reaches the source plane)
};

// hz: half the brick's extent along z in voxels ((BZ - 1) / 2)
static __device__ void bp_view_setup(const OpParams &p, int view, const double Xb[3], double hz, BpView &o) {
    const double *x = p.views64 + (size_t)view * VIEW64_STRIDE;
    const double s[3] = {p.sx, p.sy, p.sz};
    double Pa[3], Pb[3], Pw[3], a0, b0, w0;
    if (p.perspective) {
        for (int i = 0; i < 3; ++i) {
            Pa[i] = x[i];
            Pb[i] = x[4 + i];
            Pw[i] = x[8 + i];
        }
        a0 = Pa[0] * Xb[0] + Pa[1] * Xb[1] + Pa[2] * Xb[2] + x[3];
        b0 = Pb[0] * Xb[0] + Pb[1] * Xb[1] + Pb[2] * Xb[2] + x[7];
        w0 = Pw[0] * Xb[0] + Pw[1] * Xb[1] + Pw[2] * Xb[2] + x[11];
    } else {
        const double *Dc = x, *eu = x + 3, *ev = x + 6;
        const double hu = 0.5 * (p.det.nu - 1), hv = 0.5 * (p.det.nv - 1);
        for (int i = 0; i < 3; ++i) {
            Pa[i] = eu[i] / p.du;
            Pb[i] = ev[i] / p.dv;
            Pw[i] = 0.0;
        }
        double Y[3] = {Xb[0] - Dc[0], Xb[1] - Dc[1], Xb[2] - Dc[2]};
        a0 = ((Y[0] * eu[0] + Y[1] * eu[1] + Y[2] * eu[2]) - p.ou) / p.du + hu;
        b0 = ((Y[0] * ev[0] + Y[1] * ev[1] + Y[2] * ev[2]) - p.ov) / p.dv + hv;
        w0 = 1.0;
    }
    o.valid = w0 > 0.0;
    if (!o.valid) w0 = 1.0;
    const double u0 = a0 / w0, v0 = b0 / w0;
    const double U = floor(u0), Vv = floor(v0);
    for (int i = 0; i < 3; ++i) {
        o.Qa[i] = (float)((Pa[i] - u0 * Pw[i]) * s[i]);
        o.Qb[i] = (float)((Pb[i] - v0 * Pw[i]) * s[i]);
        o.Pw[i] = (float)(Pw[i] * s[i]);
    }
    o.w0 = (float)w0;
    // clamp the integer parts far outside the detector (such views contribute nothing anyway)
    const double lim = 4.0e6;
    o.U0 = (int)fmin(fmax(U, -lim), lim);
    o.V0 = (int)fmin(fmax(Vv, -lim), lim);
    o.fu = (float)(u0 - U);
    o.fv = (float)(v0 - Vv);
    o.flat = (o.Qa[2] == 0.0f && o.Pw[2] == 0.0f);
    // shadow of the brick: voxel offsets d from its centre with |d_i| <= h_i (half the brick plus one
    // voxel of margin) project to |u - u0| <= sum |Qa_i| h_i / min w, min w = w0 - sum |Pw_i| h_i; the
    // taps of a voxel are floor(u) and floor(u) + 1, so one more pixel on each side
    const double h[3] = {0.5 * (BPB_X - 1) + 1.0, 0.5 * (BPB_Y - 1) + 1.0, hz + 1.0};
    double sa = 0.0, sb = 0.0, sw = 0.0;
    for (int i = 0; i < 3; ++i) {
        sa += fabs((Pa[i] - u0 * Pw[i]) * s[i]) * h[i];
        sb += fabs((Pb[i] - v0 * Pw[i]) * s[i]) * h[i];
        sw += fabs(Pw[i] * s[i]) * h[i];
    }
    const double wmin = w0 - sw;
    o.eu = o.ev = -1;
    if (o.valid && wmin > 0.0 && sa / wmin < 4096.0 && sb / wmin < 4096.0) {
        o.eu = (int)ceil(sa / wmin) + 2;
        o.ev = (int)ceil(sb / wmin) + 2;
    }
}

// floor and fraction; q is clamped to +-1e6 first (the magic addition needs |q| < 2^22; detector
// coordinates that far out contribute nothing)
static __device__ __forceinline__ void magic_floor(float q, int &i, float &f) {
    const float M = 12582912.0f;
    q = fminf(fmaxf(q, -1.0e6f), 1.0e6f);
    float t = __fadd_rd(q, M);
    i = __float_as_int(t) - 0x4B400000;
    f = q - (t - M);
}

template <typename T>
__device__ __forceinline__ float bilerp0(const T *__restrict__ q, int nu, int nv, int iu, int iv, float au, float av) {
    const bool u0 = (unsigned)iu < (unsigned)nu, u1 = (unsigned)(iu + 1) < (unsigned)nu;
    const bool v0 = (unsigned)iv < (unsigned)nv, v1 = (unsigned)(iv + 1) < (unsigned)nv;
    const int base = iv * nu + iu;   // one view holds fewer than 2^31 pixels
    const float q00 = (v0 && u0) ? ldg_f32(q + base) : 0.0f;
    const float q01 = (v0 && u1) ? ldg_f32(q + base + 1) : 0.0f;
    const float q10 = (v1 && u0) ? ldg_f32(q + base + nu) : 0.0f;
    const float q11 = (v1 && u1) ? ldg_f32(q + base + nu + 1) : 0.0f;
    const float r0 = fmaf(au, q01 - q00, q00);
    const float r1 = fmaf(au, q11 - q10, q10);
    return fmaf(av, r1 - r0, r0);
}

// One view of one brick's z-column through global memory (read-only L1 path): u, v are monotone along
// the column, so where every lane's end voxels read all four taps on the detector (a warp vote) the warp
// reads them without bounds tests; elsewhere each tap is tested. acc: the column's BZ sums.
template <typename T, int BZ, bool W2>
__device__ __forceinline__ void bp_view_global(const BpView &V, const T *__restrict__ q, int nu, int nv, float dx,
                                               float dy, float dz0, float (&acc)[BZ]) {
    float na = fmaf(V.Qa[0], dx, fmaf(V.Qa[1], dy, V.Qa[2] * dz0));
    float nb = fmaf(V.Qb[0], dx, fmaf(V.Qb[1], dy, V.Qb[2] * dz0));
    float w = fmaf(V.Pw[0], dx, fmaf(V.Pw[1], dy, fmaf(V.Pw[2], dz0, V.w0)));
    if (V.flat) {
        // Every lane of the warp is here (the view loop and the branches above are uniform): each
        // tests its own column, u fixed and v monotone in z (v_z = fma(z, Qb_z, nb) scaled by 1/w),
        // so the first and last voxel bound it; if all lanes' four taps lie on the detector, the
        // warp reads them without bounds tests
        const bool wpos = w > 0.0f;
        const float iw = wpos ? rcp_fast(w) : 0.0f;
        const float qu = fmaf(na, iw, V.fu);
        const float qv0 = fmaf(nb, iw, V.fv), qv1 = fmaf(fmaf((float)(BZ - 1), V.Qb[2], nb), iw, V.fv);
        const float lu = -(float)V.U0, hu = (float)(nu - 1 - V.U0);
        const float lv = -(float)V.V0, hv = (float)(nv - 1 - V.V0);
        const bool ok = wpos && qu >= lu && qu < hu && qv0 >= lv && qv0 < hv && qv1 >= lv && qv1 < hv;
        const float om = W2 ? iw * iw : 1.0f;
        if (__all_sync(0xffffffffu, ok)) {
            const float tu = __fadd_rd(qu, 12582912.0f);
            const float au = qu - (tu - 12582912.0f);
            const T *qc = q + (__float_as_int(tu) - 0x4B400000 + V.U0);
#pragma unroll
            for (int z = 0; z < BZ; ++z) {
                const float qv = fmaf(fmaf((float)z, V.Qb[2], nb), iw, V.fv);
                const float t = __fadd_rd(qv, 12582912.0f);
                const float av = qv - (t - 12582912.0f);
                const T *r = qc + (__float_as_int(t) - 0x4B400000 + V.V0) * nu;
                // the two lerps along u as one packed FP32x2 pair (each lane rounds as the scalar FMA)
                const f32x2 rr = lerp2(splat2(au), pack2(ldg_f32(r), ldg_f32(r + nu)),
                                       pack2(ldg_f32(r + 1), ldg_f32(r + nu + 1)));
                const float r0 = lo2(rr), r1 = hi2(rr);
                acc[z] = fmaf(om, fmaf(av, r1 - r0, r0), acc[z]);
            }
            return;
        }
        if (!wpos) return;
        int iu;
        float au;
        magic_floor(qu, iu, au);
        iu += V.U0;
        // the column iu and its bounds are shared by the brick's z voxels (32-bit detector
        // indices: one view holds fewer than 2^31 pixels)
        const bool u0 = (unsigned)iu < (unsigned)nu, u1 = (unsigned)(iu + 1) < (unsigned)nu;
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            int iv;
            float av;
            magic_floor(fmaf(fmaf((float)z, V.Qb[2], nb), iw, V.fv), iv, av);
            iv += V.V0;
            const bool v0 = (unsigned)iv < (unsigned)nv, v1 = (unsigned)(iv + 1) < (unsigned)nv;
            const T *r = q + (iv * nu + iu);
            const float q00 = (v0 && u0) ? ldg_f32(r) : 0.0f;
            const float q01 = (v0 && u1) ? ldg_f32(r + 1) : 0.0f;
            const float q10 = (v1 && u0) ? ldg_f32(r + nu) : 0.0f;
            const float q11 = (v1 && u1) ? ldg_f32(r + nu + 1) : 0.0f;
            const float r0 = fmaf(au, q01 - q00, q00);
            const float r1 = fmaf(au, q11 - q10, q10);
            acc[z] = fmaf(om, fmaf(av, r1 - r0, r0), acc[z]);
        }
    } else {
        // General views (u and w vary along z: tilted detectors, arbitrary trajectories). Along a
        // column, u(z) = (na + z Qa_z) / (w + z Pw_z) and v(z) are ratios of linear functions whose
        // denominator stays positive when it is positive at both ends, hence monotone: the end
        // voxels bound the column. Lanes whose columns lie on the detector with a margin of 1e-3
        // pixel (far above the rounding of these small quantities) read their taps without bounds
        // tests when the whole warp does; positions are formed per z from the column's start.
        {
            const float zl = (float)(BZ - 1);
            const float w1 = fmaf(zl, V.Pw[2], w);
            const bool wpos = w > 0.0f && w1 > 0.0f;
            const float iw0 = wpos ? rcp_fast(w) : 0.0f, iw1 = wpos ? rcp_fast(w1) : 0.0f;
            const float qu0 = fmaf(na, iw0, V.fu), qu1 = fmaf(fmaf(zl, V.Qa[2], na), iw1, V.fu);
            const float qv0 = fmaf(nb, iw0, V.fv), qv1 = fmaf(fmaf(zl, V.Qb[2], nb), iw1, V.fv);
            const float eps = 1e-3f;
            const float lu = -(float)V.U0 + eps, hu = (float)(nu - 1 - V.U0) - eps;
            const float lv = -(float)V.V0 + eps, hv = (float)(nv - 1 - V.V0) - eps;
            const bool ok = wpos && qu0 >= lu && qu0 < hu && qu1 >= lu && qu1 < hu && qv0 >= lv && qv0 < hv &&
                            qv1 >= lv && qv1 < hv;
            if (__all_sync(0xffffffffu, ok)) {
                // (u, v) positions and the two lerps along u as packed FP32x2 pairs (bit-identical lanes)
                const f32x2 M2 = splat2(12582912.0f);
                const f32x2 qab2 = pack2(V.Qa[2], V.Qb[2]), nab2 = pack2(na, nb), fuv2 = pack2(V.fu, V.fv);
#pragma unroll
                for (int z = 0; z < BZ; ++z) {
                    const float fz = (float)z;
                    const float iw = rcp_fast(fmaf(fz, V.Pw[2], w));
                    const f32x2 qq = fma2(fma2(splat2(fz), qab2, nab2), splat2(iw), fuv2);
                    const f32x2 t = add2_rd(qq, M2);
                    const f32x2 a = sub2(qq, sub2(t, M2));
                    const T *r = q + ((__float_as_int(hi2(t)) - 0x4B400000 + V.V0) * nu +
                                      (__float_as_int(lo2(t)) - 0x4B400000 + V.U0));
                    const f32x2 rr = lerp2(splat2(lo2(a)), pack2(ldg_f32(r), ldg_f32(r + nu)),
                                           pack2(ldg_f32(r + 1), ldg_f32(r + nu + 1)));
                    const float r0 = lo2(rr), r1 = hi2(rr);
                    const float om = W2 ? iw * iw : 1.0f;
                    acc[z] = fmaf(om, fmaf(hi2(a), r1 - r0, r0), acc[z]);
                }
                return;
            }
        }
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            if (w > 0.0f) {
                const float iw = rcp_fast(w);
                int iu, iv;
                float au, av;
                magic_floor(fmaf(na, iw, V.fu), iu, au);
                magic_floor(fmaf(nb, iw, V.fv), iv, av);
                const float om = W2 ? iw * iw : 1.0f;
                acc[z] = fmaf(om, bilerp0(q, nu, nv, iu + V.U0, iv + V.V0, au, av), acc[z]);
            }
            na += V.Qa[2];
            nb += V.Qb[2];
            w += V.Pw[2];
        }
    }
}

}  // namespace pyronn
