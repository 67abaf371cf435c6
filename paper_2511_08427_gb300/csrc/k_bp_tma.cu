// TMA-staged voxel-driven back-projector (same operator as bp_brick_kernel and bp_direct_kernel,
// Sec. 2.1: each voxel projected onto the detector, the bilinear, zero-padded detector values summed
// over the views).
//
// One CTA owns a 16 x 16 x BZ brick (each thread a z-column of BZ voxels, sums in registers over every
// view), like the L1-path brick kernel. The difference is where the detector taps come from: for every
// view, one thread copies the brick's shadow on the detector (a box of bu x bv pixels around the
// projection of the brick centre, sized on the host for the geometry) into shared memory with one 3D
// tensor copy, whose zero fill stands for the detector's zero padding. Views go in chunks (up to BT_CHUNK
// views, as many as let four CTAs share an SM) through two shared-memory stages: while the CTA
// back-projects one chunk, the next chunk's copies are in flight, so the taps are low-latency
// shared-memory loads instead of first-touch L1 misses, and need no bounds tests. One barrier per chunk
// orders the stages. The per-(brick, view) constants (FP64, a unit of low throughput on this GPU) are
// formed by a full warp for a group of about 32 views at a time, one lane per view. A warp takes the staged path for a view when every lane's column (whose u and v are
// monotone along z, so its end voxels bound it) falls inside the box with a margin; other warps, and
// views whose shadow exceeds the box (the box is sized from a sample of bricks), read through L1 as the
// brick kernel does. Every copy wait is bounded; a lost copy sets FLAG_TMA_TIMEOUT and the CTA leaves.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <type_traits>
#include <vector>

#include "bp_common.cuh"
#include "tma_common.cuh"

namespace pyronn {

constexpr int BT_CHUNK = 4;    // most views per stage (the configuration may use fewer, see cfg.chunk)
constexpr int BT_GROUP = 32;   // most views whose set-up one warp computes at once (one lane per view)

struct BpTmaCfg {
    int bu, bv;    // staged box per view (pixels); bu * element size is a multiple of 16 bytes
    int stride;    // elements between the views' boxes in shared memory: a tensor copy's destination must
                   // be 128-byte aligned, so bu * bv rounded up to a multiple of 128 bytes
    int chunk;     // views per stage (1 .. BT_CHUNK): as many as let four CTAs (three for 16-voxel
                   // columns) share an SM
    int valid;     // 0: the kernel does not apply (rows not a multiple of 16 bytes, box too large)
    int bz;        // voxels per thread along z (8 or 16)
};

// Set-up records of a group of consecutive views (chunk * floor(BT_GROUP / chunk) of them).
struct BtGroup {
    BpView v[BT_GROUP];
    int ub[BT_GROUP], vb[BT_GROUP];   // box origin on the detector (ub a multiple of 16 bytes / element)
    int staged[BT_GROUP];             // 1: the view's shadow fits the box and is copied
};

// Set-up of views n0 .. n0 + count - 1 (count <= 32) by the lanes of warp 0, one view per lane: the
// per-(brick, view) constants are formed in FP64, whose throughput is low, so a full warp forms them
// for a whole group at once rather than a few lanes per stage.
template <typename T, int BZ>
__device__ __forceinline__ void bt_group_setup(const OpParams &p, const BpTmaCfg &cfg, const double Xb[3], int n0,
                                               int count, BtGroup &G) {
    const int t = threadIdx.x;
    if (t >= count) return;
    const int n = n0 + t;
    G.staged[t] = 0;
    G.ub[t] = G.vb[t] = 0;
    BpView &V = G.v[t];
    if (n >= p.n_views) {
        V.valid = 0;
        return;
    }
    bp_view_setup(p, n, Xb, 0.5 * (BZ - 1), V);
    if (!V.valid || V.eu < 0) return;
    constexpr int align = 16 / (int)sizeof(T);
    const int u_lo = V.U0 - V.eu, u_hi = V.U0 + V.eu;
    const int ub = u_lo >= 0 ? (u_lo / align) * align : -(((-u_lo) + align - 1) / align) * align;
    const int vb = V.V0 - V.ev;
    // the box must hold the taps of every voxel; a box entirely off the detector is all zero and is
    // copied all the same (the copy fills it)
    if (u_hi - ub + 1 <= cfg.bu && 2 * V.ev + 1 <= cfg.bv) {
        G.ub[t] = ub;
        G.vb[t] = vb;
        G.staged[t] = 1;
    }
}

template <typename T, int BZ, bool W2>
__global__ void __launch_bounds__(BPB_NT, BZ > 8 ? 3 : 4) bp_tma_kernel(OpParams p, BpTmaCfg cfg, const __grid_constant__ CUtensorMap map,
                                                           const T *__restrict__ sino, T *__restrict__ vol) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ BtGroup grp[2];
    __shared__ unsigned long long bar[2];
    const unsigned raw = smem_u32(smem_raw);
    T *const stage0 = (T *)(smem_raw + (((raw + 127u) & ~127u) - raw));
    const int per_view = cfg.stride;                                  // slot of one view (128-byte multiple)
    const int chunk = cfg.chunk;
    const int K = BT_GROUP / chunk;                                   // chunks per group (>= 8)
    const int gsize = K * chunk;                                      // views per group
    const unsigned view_bytes = (unsigned)(sizeof(T) * cfg.bu * cfg.bv);   // bytes one copy delivers

    const int nbz = (p.vol.nz + BZ - 1) / BZ;
    const int bxi = blockIdx.x, byi = blockIdx.y, bzi = blockIdx.z % nbz, b = blockIdx.z / nbz;
    const int bx0 = bxi * BPB_X, by0 = byi * BPB_Y, bz0 = bzi * BZ;
    const int tid = threadIdx.x;
    const int lx = tid % BPB_X, ly = tid / BPB_X;
    const int i = bx0 + lx, j = by0 + ly;
    const T *sb = sino + (long long)b * p.sino_elems;
    const int nu = p.det.nu, nv = p.det.nv;
    double Xb[3];
    Xb[0] = (bx0 + 0.5 * (BPB_X - 1) - 0.5 * (p.vol.nx - 1)) * p.sx;
    Xb[1] = (by0 + 0.5 * (BPB_Y - 1) - 0.5 * (p.vol.ny - 1)) * p.sy;
    Xb[2] = (bz0 + 0.5 * (BZ - 1) - 0.5 * (p.vol.nz - 1)) * p.sz;
    const float dx = (float)lx - 0.5f * (BPB_X - 1), dy = (float)ly - 0.5f * (BPB_Y - 1);
    const float dz0 = -0.5f * (BZ - 1);

    float acc[BZ];
#pragma unroll
    for (int z = 0; z < BZ; ++z) acc[z] = 0.0f;

    const unsigned bars[2] = {smem_u32(&bar[0]), smem_u32(&bar[1])};
    if (tid == 0) {
        mbar_init(bars[0], 1);
        mbar_init(bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // Chunk ch holds views ch * chunk + c (c < chunk), whose records are entries (ch % K) * chunk + c of
    // grp[(ch / K) & 1], and goes through stage ch & 1. Thread 0 issues its copies once its group's
    // set-up is visible (after a barrier) and every thread is done with the chunk that last used the stage.
    auto issue = [&](int ch) {
        const BtGroup &G = grp[(ch / K) & 1];
        const int e0 = (ch % K) * chunk, s = ch & 1;
        unsigned bytes = 0;
        for (int c = 0; c < chunk; ++c) bytes += G.staged[e0 + c] ? view_bytes : 0u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the stage was last read by threads
        mbar_expect_tx(bars[s], bytes);
        for (int c = 0; c < chunk; ++c)
            if (G.staged[e0 + c])
                tma_load_3d(smem_u32(stage0 + (size_t)(s * chunk + c) * per_view), &map, bars[s], G.ub[e0 + c],
                            G.vb[e0 + c], b * p.n_views + ch * chunk + c);
    };

    const int nchunks = (p.n_views + chunk - 1) / chunk;
    if (tid < 32) bt_group_setup<T, BZ>(p, cfg, Xb, 0, gsize, grp[0]);
    __syncthreads();
    if (tid == 0) issue(0);
    int lost = -1;        // the first chunk whose copy did not arrive in time (for some thread)
    int mine_lost = 0;    // this thread's wait ran out
    for (int ch = 0; ch < nchunks; ++ch) {
        const int s = ch & 1;
        // records of the next group, before its first chunk's copies are issued: the group they replace
        // (two back) was finished by every thread at the barrier of an earlier chunk, as K >= 2
        if (tid < 32 && ch + 1 < nchunks && (ch + 1) % K == 0)
            bt_group_setup<T, BZ>(p, cfg, Xb, (ch + 1) * chunk, gsize, grp[((ch + 1) / K) & 1]);
        // the only barrier per chunk: every thread is done with chunk ch - 1 (stage s ^ 1 may be refilled),
        // the next group's records are visible, and a lost copy seen by any thread ends every thread's loop
        if (__syncthreads_or(mine_lost)) {
            lost = ch - 1;
            break;
        }
        if (tid == 0 && ch + 1 < nchunks) issue(ch + 1);
        // the lanes of a warp take one decision (the warp votes below need all 32 lanes)
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(bars[s], (unsigned)(ch >> 1) & 1u))) {
            mine_lost = 1;
            continue;
        }
        const BtGroup &G = grp[(ch / K) & 1];
        const int e0 = (ch % K) * chunk;
        for (int c = 0; c < chunk; ++c) {
            const int n = ch * chunk + c;
            if (n >= p.n_views) break;
            const BpView &V = G.v[e0 + c];
            if (!V.valid) continue;
            if (G.staged[e0 + c]) {
                const T *box = stage0 + (size_t)(s * chunk + c) * per_view;
                // tap (iu, iv) of the detector is box[(iv - vb) bu + (iu - ub)]; iu = floor(qu) + U0
                const int du0 = V.U0 - G.ub[e0 + c], dv0 = V.V0 - G.vb[e0 + c];
                const float eps = 1e-3f;
                const float lu = (float)(-du0) + eps, hu = (float)(cfg.bu - 1 - du0) - eps;
                const float lvv = (float)(-dv0) + eps, hvv = (float)(cfg.bv - 1 - dv0) - eps;
                const float na = fmaf(V.Qa[0], dx, fmaf(V.Qa[1], dy, V.Qa[2] * dz0));
                const float nb = fmaf(V.Qb[0], dx, fmaf(V.Qb[1], dy, V.Qb[2] * dz0));
                const float w = fmaf(V.Pw[0], dx, fmaf(V.Pw[1], dy, fmaf(V.Pw[2], dz0, V.w0)));
                const float zl = (float)(BZ - 1);
                const float w1 = fmaf(zl, V.Pw[2], w);
                const bool wpos = w > 0.0f && w1 > 0.0f;
                const float iw0 = wpos ? rcp_fast(w) : 0.0f, iw1 = wpos ? rcp_fast(w1) : 0.0f;
                const float qu0 = fmaf(na, iw0, V.fu), qu1 = fmaf(fmaf(zl, V.Qa[2], na), iw1, V.fu);
                const float qv0 = fmaf(nb, iw0, V.fv), qv1 = fmaf(fmaf(zl, V.Qb[2], nb), iw1, V.fv);
                const bool in = wpos && qu0 >= lu && qu0 < hu && qu1 >= lu && qu1 < hu && qv0 >= lvv && qv0 < hvv &&
                                qv1 >= lvv && qv1 < hvv;
                if (__all_sync(0xffffffffu, in)) {
                    // packed FP32x2 forms of the scalar arithmetic (each lane rounds as the scalar
                    // instruction does, so the result is the same bit for bit): the two lerps along u
                    // in one pair, and the (u, v) positions, or the v positions of two voxels, in another
                    const int bu = cfg.bu;
                    const f32x2 M2 = splat2(12582912.0f);
                    if (V.flat) {
                        // u and w constant along the column
                        const float tu = __fadd_rd(qu0, 12582912.0f);
                        const float au = qu0 - (tu - 12582912.0f);
                        const f32x2 au2 = splat2(au);
                        const T *bc = box + (__float_as_int(tu) - 0x4B400000 + du0);
                        const float om = W2 ? iw0 * iw0 : 1.0f;
                        const f32x2 qb2 = splat2(V.Qb[2]), nb2 = splat2(nb), iw2 = splat2(iw0), fv2 = splat2(V.fv);
#pragma unroll
                        for (int z = 0; z < BZ; z += 2) {
                            // voxels z and z + 1 (BZ is even)
                            const f32x2 qv = fma2(fma2(pack2((float)z, (float)(z + 1)), qb2, nb2), iw2, fv2);
                            const f32x2 t = add2_rd(qv, M2);
                            const f32x2 av = sub2(qv, sub2(t, M2));
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const T *r = bc + (__float_as_int(h ? hi2(t) : lo2(t)) - 0x4B400000 + dv0) * bu;
                                const f32x2 rr = lerp2(au2, pack2(to_f32(r[0]), to_f32(r[bu])),
                                                       pack2(to_f32(r[1]), to_f32(r[bu + 1])));
                                const float r0 = lo2(rr), r1 = hi2(rr);
                                acc[z + h] = fmaf(om, fmaf(h ? hi2(av) : lo2(av), r1 - r0, r0), acc[z + h]);
                            }
                        }
                    } else {
                        const f32x2 qab2 = pack2(V.Qa[2], V.Qb[2]), nab2 = pack2(na, nb), fuv2 = pack2(V.fu, V.fv);
#pragma unroll
                        for (int z = 0; z < BZ; ++z) {
                            const float fz = (float)z;
                            const float iw = rcp_fast(fmaf(fz, V.Pw[2], w));
                            const f32x2 q = fma2(fma2(splat2(fz), qab2, nab2), splat2(iw), fuv2);   // (u, v)
                            const f32x2 t = add2_rd(q, M2);
                            const f32x2 a = sub2(q, sub2(t, M2));
                            const T *r = box + ((__float_as_int(hi2(t)) - 0x4B400000 + dv0) * bu +
                                                (__float_as_int(lo2(t)) - 0x4B400000 + du0));
                            const f32x2 rr = lerp2(splat2(lo2(a)), pack2(to_f32(r[0]), to_f32(r[bu])),
                                                   pack2(to_f32(r[1]), to_f32(r[bu + 1])));
                            const float r0 = lo2(rr), r1 = hi2(rr);
                            const float om = W2 ? iw * iw : 1.0f;
                            acc[z] = fmaf(om, fmaf(hi2(a), r1 - r0, r0), acc[z]);
                        }
                    }
                    continue;
                }
            }
            bp_view_global<T, BZ, W2>(V, sb + (long long)n * nv * nu, nu, nv, dx, dy, dz0, acc);
        }
    }
    // a copy that ran out in the last chunk
    if (lost < 0 && __syncthreads_or(mine_lost)) lost = nchunks - 1;
    if (lost >= 0) {
        if (tid == 0) atomicAdd(p.flags + FLAG_TMA_TIMEOUT, 1);
        // wait (bounded) for the copies still in flight (this chunk's and the next one's) before the
        // shared memory goes away
        mbar_wait_bounded(bars[lost & 1], (unsigned)(lost >> 1) & 1u);
        if (lost + 1 < nchunks) mbar_wait_bounded(bars[(lost + 1) & 1], (unsigned)((lost + 1) >> 1) & 1u);
        return;
    }
    if (i < p.vol.nx && j < p.vol.ny) {
        T *vb = vol + (long long)b * p.vol_elems;
#pragma unroll
        for (int z = 0; z < BZ; ++z) {
            const int k = bz0 + z;
            if (k < p.vol.nz) vb[((long long)k * p.vol.ny + j) * p.vol.nx + i] = from_f32<T>(acc[z]);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------------------------

namespace {

// Shadow half-extents (pixels) of a 16 x 16 x BZ brick centred at Xb (world mm relative to the volume
// centre) in view record x, as the device set-up computes them; false where unbounded.
bool host_shadow(const pyronn_geom *g, const double *x, const double Xb[3], double hz, int &eu, int &ev) {
    const double s[3] = {g->sx, g->sy, g->sz};
    double Pa[3], Pb[3], Pw[3], a0, b0, w0;
    if (g->kind == 1) {
        for (int i = 0; i < 3; ++i) {
            Pa[i] = x[i];
            Pb[i] = x[4 + i];
            Pw[i] = x[8 + i];
        }
        a0 = Pa[0] * Xb[0] + Pa[1] * Xb[1] + Pa[2] * Xb[2] + x[3];
        b0 = Pb[0] * Xb[0] + Pb[1] * Xb[1] + Pb[2] * Xb[2] + x[7];
        w0 = Pw[0] * Xb[0] + Pw[1] * Xb[1] + Pw[2] * Xb[2] + x[11];
    } else {
        for (int i = 0; i < 3; ++i) {
            Pa[i] = x[3 + i] / g->du;
            Pb[i] = x[6 + i] / g->dv;
            Pw[i] = 0.0;
        }
        a0 = b0 = 0.0;
        w0 = 1.0;
    }
    if (!(w0 > 0.0)) return false;
    const double u0 = a0 / w0, v0 = b0 / w0;
    const double h[3] = {0.5 * (BPB_X - 1) + 1.0, 0.5 * (BPB_Y - 1) + 1.0, hz + 1.0};
    double sa = 0.0, sbb = 0.0, sw = 0.0;
    for (int i = 0; i < 3; ++i) {
        sa += std::fabs((Pa[i] - u0 * Pw[i]) * s[i]) * h[i];
        sbb += std::fabs((Pb[i] - v0 * Pw[i]) * s[i]) * h[i];
        sw += std::fabs(Pw[i] * s[i]) * h[i];
    }
    const double wmin = w0 - sw;
    if (!(wmin > 0.0) || !(sa / wmin < 4096.0) || !(sbb / wmin < 4096.0)) return false;
    eu = (int)std::ceil(sa / wmin) + 2;
    ev = (int)std::ceil(sbb / wmin) + 2;
    return true;
}

}  // namespace

// Box size for the staged back-projector: the largest shadow over a sample of bricks (every fourth
// brick along each axis, and the bricks at the volume's corners) and every view, plus the alignment of
// the box origin. Bricks whose shadow exceeds it take the L1 path. valid = 0 where the sinogram rows are
// not a multiple of 16 bytes, the volume is 2D, or the box would exceed 40 KB per stage.
static BpTmaCfg choose_bp_tma_cfg(const pyronn_geom *g, size_t elem, int bz) {
    BpTmaCfg c{};
    if (g->ndim != 3 || (g->nu * elem) % 16 != 0 || g->views_ext.empty()) return c;
    const int nbx = (g->nx + BPB_X - 1) / BPB_X, nby = (g->ny + BPB_Y - 1) / BPB_Y, nbz = (g->nz + bz - 1) / bz;
    std::vector<int> bxs, bys, bzs;
    for (int v = 0; v < nbx; v += 4) bxs.push_back(v);
    for (int v = 0; v < nby; v += 4) bys.push_back(v);
    for (int v = 0; v < nbz; v += 4) bzs.push_back(v);
    bxs.push_back(nbx - 1);
    bys.push_back(nby - 1);
    bzs.push_back(nbz - 1);
    const double hz = 0.5 * (bz - 1);
    std::vector<int> mu(g->n_views, 0), mv(g->n_views, 0);
    auto work = [&](int v0, int v1) {
        for (int n = v0; n < v1; ++n) {
            const double *x = g->views_ext.data() + (size_t)n * VIEW64_STRIDE;
            for (int a : bxs)
                for (int bb : bys)
                    for (int cc : bzs) {
                        const double Xb[3] = {(a * BPB_X + 0.5 * (BPB_X - 1) - 0.5 * (g->nx - 1)) * g->sx,
                                              (bb * BPB_Y + 0.5 * (BPB_Y - 1) - 0.5 * (g->ny - 1)) * g->sy,
                                              (cc * bz + 0.5 * (bz - 1) - 0.5 * (g->nz - 1)) * g->sz};
                        int eu = 0, ev = 0;
                        if (host_shadow(g, x, Xb, hz, eu, ev)) {
                            mu[n] = std::max(mu[n], eu);
                            mv[n] = std::max(mv[n], ev);
                        }
                    }
        }
    };
    const int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(work, (int)((long long)g->n_views * t / nt),
                                                  (int)((long long)g->n_views * (t + 1) / nt));
    work(0, (int)((long long)g->n_views / nt));
    for (auto &t : th) t.join();
    int eu = 0, ev = 0;
    for (int n = 0; n < g->n_views; ++n) {
        eu = std::max(eu, mu[n]);
        ev = std::max(ev, mv[n]);
    }
    const int align = 16 / (int)elem;
    const int ctas = bz > 8 ? 3 : 4;   // CTAs per SM the kernel is compiled for
    int bu = 2 * eu + 1 + (align - 1);
    bu = (bu + align - 1) / align * align;
    const int bv = 2 * ev + 1;
    if (eu <= 0 || bu > 256 || bv > 256) return c;
    // views per stage: as many (up to BT_CHUNK) as let the CTAs share an SM (228 KB, 1 KB reserved and
    // the static set-up records per CTA)
    const int stride = (int)((((size_t)bu * bv * elem + 127) / 128) * 128 / elem);
    const size_t view_bytes = (size_t)stride * elem;
    const size_t per_cta_fixed = 1024 + sizeof(BtGroup) * 2 + 16 + 128;
    int chunk = BT_CHUNK;
    while (chunk > 1 && ctas * (per_cta_fixed + 2 * chunk * view_bytes) > 228 * 1024) --chunk;
    if (2 * chunk * view_bytes > 100 * 1024) return c;
    c.bu = bu;
    c.bv = bv;
    c.stride = stride;
    c.chunk = chunk;
    c.valid = 1;
    c.bz = bz;
    return c;
}

template <typename T, int BZ, bool W2>
static int launch_bt(const OpParams &p, const BpTmaCfg &cfg, const void *sino, void *vol, cudaStream_t st) {
    auto enc = tma_encode_fn();
    if (!enc) return (int)cudaErrorNotSupported;
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (std::is_same<T, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                      : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    const size_t smem = (size_t)2 * cfg.chunk * cfg.stride * sizeof(T) + 128;
    auto kern = bp_tma_kernel<T, BZ, W2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    const int nbx = ceil_div(p.vol.nx, BPB_X), nby = ceil_div(p.vol.ny, BPB_Y), nbz = ceil_div(p.vol.nz, BZ);
    const int per_launch = 65535 / nbz > 0 ? 65535 / nbz : 1;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        const int nb = std::min(p.batch - b0, per_launch);
        const T *s0 = (const T *)sino + (size_t)b0 * p.sino_elems;
        // the sinograms of this launch as one 3D array: u, v, view (views of the batch items in order)
        cuuint64_t gdim[3] = {(cuuint64_t)p.det.nu, (cuuint64_t)p.det.nv, (cuuint64_t)p.n_views * nb};
        cuuint64_t gstride[2] = {(cuuint64_t)p.det.nu * sizeof(T), (cuuint64_t)p.det.nu * p.det.nv * sizeof(T)};
        cuuint32_t box[3] = {(cuuint32_t)cfg.bu, (cuuint32_t)cfg.bv, 1};
        cuuint32_t estride[3] = {1, 1, 1};
        CUtensorMap map;
        std::memset(&map, 0, sizeof(map));
        CUresult r = enc(&map, dt, 3, const_cast<T *>(s0), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return (int)cudaErrorInvalidValue;
        OpParams q = p;
        q.batch = nb;
        dim3 grid(nbx, nby, nbz * nb);
        kern<<<grid, BPB_NT, smem, st>>>(q, cfg, map, s0, (T *)vol + (size_t)b0 * p.vol_elems);
    }
    return (int)cudaGetLastError();
}

template <typename T>
static int launch_bt_t(const OpParams &p, const BpTmaCfg &cfg, const void *sino, void *vol, cudaStream_t st) {
    const bool w2 = p.perspective && p.weight == PYRONN_BP_INV_W2;
    if (cfg.bz == 16)
        return w2 ? launch_bt<T, 16, true>(p, cfg, sino, vol, st) : launch_bt<T, 16, false>(p, cfg, sino, vol, st);
    return w2 ? launch_bt<T, 8, true>(p, cfg, sino, vol, st) : launch_bt<T, 8, false>(p, cfg, sino, vol, st);
}

// The staged back-projector applies (3D, rows of 16-byte multiples, a box of bounded size)? Its columns
// are 16 voxels deep where the brick depth (bp_brick_depth) is 16, else 8.
bool bp_tma_usable(pyronn_geom *g, int dtype) {
    std::lock_guard<std::mutex> lk(g->mu);
    const int k = dtype;
    const int bz = bp_brick_depth(g->tuning.bp_brick_z, g->nz) == 16 ? 16 : 8;
    if (!g->bpt_ready[k] || g->bpt_cfg[k][5] != bz) {
        const BpTmaCfg c = choose_bp_tma_cfg(g, dtype_size(dtype), bz);
        g->bpt_cfg[k][0] = c.bu;
        g->bpt_cfg[k][1] = c.bv;
        g->bpt_cfg[k][2] = c.valid;
        g->bpt_cfg[k][3] = c.chunk;
        g->bpt_cfg[k][4] = c.stride;
        g->bpt_cfg[k][5] = bz;
        g->bpt_ready[k] = 1;
    }
    return g->bpt_cfg[k][2] != 0;
}

int launch_bp_tma(pyronn_geom *g, const OpParams &p, const void *sino, void *vol, int dtype, void *stream) {
    if (!bp_tma_usable(g, dtype)) return (int)cudaErrorInvalidValue;
    BpTmaCfg c{};
    c.bu = g->bpt_cfg[dtype][0];
    c.bv = g->bpt_cfg[dtype][1];
    c.chunk = g->bpt_cfg[dtype][3];
    c.stride = g->bpt_cfg[dtype][4];
    c.bz = g->bpt_cfg[dtype][5];
    c.valid = 1;
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_bt_t<float>(p, c, sino, vol, st);
        case PYRONN_BF16: return launch_bt_t<__nv_bfloat16>(p, c, sino, vol, st);
        case PYRONN_F16: return launch_bt_t<__half>(p, c, sino, vol, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace pyronn
