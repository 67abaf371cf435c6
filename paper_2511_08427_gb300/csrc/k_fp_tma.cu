// TMA-staged ray-driven forward projector (same operator as fp_direct_kernel, Sec. 2.1).
//
// Structure as in k_fp_slab.cu (one CTA per 16 x 16 detector tile of one view, slabs of D
// planes along the tile's dominant axis m, exact sample partition through integer slab
// boundaries), but the slab box is moved by the Tensor Memory Accelerator: one thread issues a
// cp.async.bulk.tensor load of a fixed-size box (chosen on the host as the largest footprint of
// any tile), the hardware zero-fills everything outside the volume, and two buffers (where they fit
// beside the other CTAs of an SM; the autotuner usually prefers one deeper buffer) let the load of
// slab s + 1 run under the sampling of slab s. The slabs' box origins are computed ahead by the lanes
// of warp 0, sixteen slabs at a time, so that a copy is issued right after the barrier that frees its
// buffer. Completion is tracked by mbarrier transaction counts; every wait is bounded, and a CTA whose
// copy does not arrive sets an error counter and leaves.
//
// Sample loop: positions relative to the box origin, floor / fraction by the round-down
// magic-number addition (no conversion-pipe instructions), eight shared-memory reads, seven
// lerps, one accumulate. By default the (x, y) positions, floors and fractions and the pairs of lerps
// along x and y run as packed FP32x2 instructions (two lanes per instruction, each rounding as the
// scalar instruction does, so the results are identical): the loop is issue-bound, and packing cuts
// about 8 % of its time.
//
// Box layout: the rays of a warp (16 x 2 pixels) spread across the tile's march axis. Where the
// tile marches along y or z they spread along x, the innermost axis of the volume, and read
// consecutive shared-memory words. Where it marches along x they would sit on different rows at
// nearly the same x, all on one word of each 16-byte bank group; there the slabs are staged from a
// y-fastest copy of the volume (made per call by a tiled transpose), so that y is the box's
// innermost axis. The sample loop works in the box's memory order (first, second, z) = (x, y, z)
// or (y, x, z).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>
#include <type_traits>

#include "device_common.cuh"
#include "host_rays.h"
#include "tma_common.cuh"

namespace pyronn {

constexpr int TMA_TU = FP_TILE_U, TMA_TV = FP_TILE_V, TMA_NT = TMA_TU * TMA_TV;
struct TmaMaps {
    CUtensorMap map[3];   // one box shape per march axis
};

struct SlabBox {
    int lo[3];      // box origin (x aligned for TMA)
    int fits;       // the tile's footprint in this slab fits the box
};

constexpr int FP_RING = 16;   // slab boxes computed ahead, one per lane of warp 0

template <bool RING>
struct FpTmaShared {
    unsigned long long bar[2];
    float corner[5][6];
    int srange[2];
    SlabBox box[2];                   // boxes of the slabs in the two copy slots (written by the issuing thread)
    SlabBox ring[RING ? FP_RING : 1]; // boxes of the next slabs of the tile (warp 0 only)
};

// One detector tile (tile_x, tile_y) of one view of volume b: returns false if a tensor copy was lost
// (the CTA must stop). bars / ph: the CTA's two slab mbarriers and the number of loads already
// consumed on each (the wait parity), carried across tiles by persistent launches. PK: the sample
// loop's arithmetic (FpTmaBox::packed) fixed at compile time, so that a kernel holds one sample loop
// (fewer live values, no spills in the loop), or -1 to read it from cfg (persistent launches, whose
// volumes may differ). RING: slab boxes computed ahead by warp 0 (below) or by thread 0 as it issues
// each copy (the persistent launches, whose small volumes' tiles have few slabs, run faster that way).
template <typename T, int PK, bool RING>
__device__ __forceinline__ bool fp_tma_tile(const OpParams &p, const FpTmaBox &cfg, const CUtensorMap *maps3,
                                            const T *__restrict__ vol, T *__restrict__ sino, int view, int b,
                                            int tile_x, int tile_y, T *const buf0, T *const buf1, FpTmaShared<RING> &sh,
                                            unsigned ph[2]) {
    const bool dbl = cfg.nbuf == 2;
    const int pk = PK >= 0 ? PK : cfg.packed;
    float (*s_corner)[6] = sh.corner;
    int *s_srange = sh.srange;
    const int tu0 = tile_x * TMA_TU, tv0 = tile_y * TMA_TV;
    const int tu1 = min(tu0 + TMA_TU, p.det.nu) - 1, tv1 = min(tv0 + TMA_TV, p.det.nv) - 1;
    const int tid = threadIdx.x;
    const int u = tu0 + tid % TMA_TU, v = tv0 + tid / TMA_TU;
    const bool active = (u <= tu1) && (v <= tv1);
    const FpRec &rec = p.fp[view];
    const T *vb = vol + (long long)b * p.vol_elems;

    __syncthreads();   // the previous tile's readers of the shared corner rays are done
    if (tid < 5) {
        float cu, cv;
        if (tid < 4) {
            cu = (float)((tid & 1) ? tu1 : tu0);
            cv = (float)((tid & 2) ? tv1 : tv0);
        } else {
            cu = 0.5f * (float)(tu0 + tu1);
            cv = 0.5f * (float)(tv0 + tv1);
        }
        RayIdx c = ray_setup(rec, p.vol, cu, cv);
        s_corner[tid][0] = c.cx; s_corner[tid][1] = c.cy; s_corner[tid][2] = c.cz;
        s_corner[tid][3] = c.dx; s_corner[tid][4] = c.dy; s_corner[tid][5] = c.dz;
    }
    if (tid == 0) {
        s_srange[0] = 1 << 30;
        s_srange[1] = -(1 << 30);
    }
    RayIdx r = ray_setup(rec, p.vol, (float)min(u, tu1), (float)min(v, tv1));
    int k0 = 0, k1 = -1;
    bool hit = active && ray_k_range(r, p.vol, p.dt, k0, k1);
    __syncthreads();

    int m;
    {
        float ax = fabsf(s_corner[4][3]), ay = fabsf(s_corner[4][4]), az = fabsf(s_corner[4][5]);
        m = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    }
    const int a1 = (m == 0) ? 1 : 0, a2 = (m == 2) ? 1 : 2;
    const int Nm = m == 0 ? p.vol.nx : (m == 1 ? p.vol.ny : p.vol.nz);
    const int N1 = a1 == 0 ? p.vol.nx : p.vol.ny, N2 = a2 == 1 ? p.vol.ny : p.vol.nz;
    const float cm = m == 0 ? r.cx : (m == 1 ? r.cy : r.cz);
    const float dm = m == 0 ? r.dx : (m == 1 ? r.dy : r.dz);
    const bool marchable = fabsf(dm) > 1e-3f * (fabsf(r.dx) + fabsf(r.dy) + fabsf(r.dz));
    const bool direct_ray = hit && !marchable;
    if (direct_ray) hit = false;
    const bool pos = dm > 0.0f;
    const float inv_step = marchable ? 1.0f / (p.dt * dm) : 0.0f;
    const int D = cfg.depth, G = cfg.guard;
    const int base0 = cfg.slab0;                        // slab s covers floor(q_m) in [base0 + s D, base0 + (s+1) D)
    const int nslab_all = (Nm + 1 - base0 + D - 1) / D; // enough slabs to reach plane Nm - 1
    const int BXb = m == 0 ? cfg.bx[0] : (m == 1 ? cfg.bx[1] : cfg.bx[2]);
    const int BYb = m == 0 ? cfg.by[0] : (m == 1 ? cfg.by[1] : cfg.by[2]);
    const int BZb = m == 0 ? cfg.bz[0] : (m == 1 ? cfg.bz[1] : cfg.bz[2]);
    const int box_elems = BXb * BYb * BZb;
    const unsigned box_bytes = (unsigned)(sizeof(T) * box_elems);
    const CUtensorMap *tmap = &maps3[m];
    // x-march tile staged from the y-fastest copy: the box's memory order is (y, x, z)
    const bool yt = m == 0 && cfg.xt;

    // slab range of this tile: union of the rays' in-box sample ranges
    if (hit) {
        float qa = fmaf(fmaf((float)k0, p.dt, 0.5f * p.dt), dm, cm);
        float qb = fmaf(fmaf((float)k1, p.dt, 0.5f * p.dt), dm, cm);
        float qlo = fmaxf(fminf(qa, qb), -1.0f), qhi = fminf(fmaxf(qa, qb), (float)Nm);
        int slo = ((int)floorf(qlo) - base0) / D, shi = ((int)floorf(qhi) - base0) / D;
        slo = max(min(slo, nslab_all - 1), 0);
        shi = max(min(shi, nslab_all - 1), 0);
        atomicMin(&s_srange[0], slo);
        atomicMax(&s_srange[1], shi);
    }
    __syncthreads();
    const int s_first = s_srange[0], s_last = s_srange[1];
    const int nsl = s_last >= s_first ? s_last - s_first + 1 : 0;
    const unsigned bars[2] = {smem_u32(&sh.bar[0]), smem_u32(&sh.bar[1])};
    const int align = 16 / (int)sizeof(T);

    // box of slab s (origin and whether the tile's footprint fits), from the corner rays' crossings of the
    // slab's end planes; the issuing thread shares it with the CTA through sh.box
    auto slab_box = [&](int s) {
        SlabBox sb;
        const int b_lo = base0 + s * D;
        const int b_hi = min(b_lo + D, Nm);
        float mn1 = 3e38f, mx1 = -3e38f, mn2 = 3e38f, mx2 = -3e38f;
        const float planes[2] = {(float)(b_lo - G), (float)(b_hi + G)};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float *cr = s_corner[c];
            float idm = 1.0f / cr[3 + m];
#pragma unroll
            for (int pl = 0; pl < 2; ++pl) {
                float t = (planes[pl] - cr[m]) * idm;
                float q1 = fmaf(t, cr[3 + a1], cr[a1]);
                float q2 = fmaf(t, cr[3 + a2], cr[a2]);
                mn1 = fminf(mn1, q1); mx1 = fmaxf(mx1, q1);
                mn2 = fminf(mn2, q2); mx2 = fmaxf(mx2, q2);
            }
        }
        const float gf = (float)(G + 2);
        mn1 = fmaxf(mn1, -gf); mx1 = fminf(mx1, (float)N1 + gf);
        mn2 = fmaxf(mn2, -gf); mx2 = fminf(mx2, (float)N2 + gf);
        const int lo1 = max((int)floorf(mn1) - 1, -1 - G), hi1 = min((int)floorf(mx1) + 2, N1 + G);
        const int lo2 = max((int)floorf(mn2) - 1, -1 - G), hi2 = min((int)floorf(mx2) + 2, N2 + G);
        const int lom = b_lo - G, him = b_hi + G;
        // (x, y, z) from (m, a1, a2): m = x -> (m, a1, a2); m = y -> (a1, m, a2); m = z -> (a1, a2, m)
        const int lx = m == 0 ? lom : lo1, hx = m == 0 ? him : hi1;
        const int ly = m == 0 ? lo1 : (m == 1 ? lom : lo2), hy = m == 0 ? hi1 : (m == 1 ? him : hi2);
        const int lz = m == 2 ? lom : lo2, hz = m == 2 ? him : hi2;
        // TMA: the innermost start coordinate (x, or y for the y-fastest copy) must be 16-byte aligned
        const int li = yt ? ly : lx;
        const int i0 = li >= 0 ? (li / align) * align : -(((-li) + align - 1) / align) * align;
        const int x0 = yt ? lx : i0, y0 = yt ? i0 : ly;
        sb.lo[0] = x0; sb.lo[1] = y0; sb.lo[2] = lz;
        sb.fits = (hx - x0 + 1 <= BXb) && (hy - y0 + 1 <= BYb) && (hz - lz + 1 <= BZb);
        return sb;
    };

    // The lanes of warp 0 compute the boxes of FP_RING slabs at a time (slab s_first + i0 + lane) into a
    // ring that only warp 0 touches; thread 0 reads a slab's box there when it issues the slab's copy, so
    // the corner-ray arithmetic is off the path between a slab's barrier and its copy. Called by all 32
    // lanes of warp 0.
    auto fill_ring = [&](int i0) {
        const int lane = tid & 31;
        __syncwarp();   // thread 0 has read the entries this call replaces
        if (lane < FP_RING && i0 + lane < nsl) sh.ring[lane] = slab_box(s_first + i0 + lane);
        __syncwarp();
    };

    auto box_for = [&](int i) { return RING ? sh.ring[i % FP_RING] : slab_box(s_first + i); };

    float acc = 0.0f;
    const float hdt = 0.5f * p.dt;
    if (nsl > 0) {
        if (RING && tid < 32) fill_ring(0);
        if (tid == 0) {
            const SlabBox sb0 = box_for(0);
            sh.box[0] = sb0;
            mbar_expect_tx(bars[0], box_bytes);
            tma_load_4d(smem_u32(buf0), tmap, bars[0], yt ? sb0.lo[1] : sb0.lo[0], yt ? sb0.lo[0] : sb0.lo[1],
                        sb0.lo[2], b);
        }
        for (int i = 0; i < nsl; ++i) {
            const int s = s_first + i;
            const int bi = dbl ? (i & 1) : 0;
            const unsigned parity = ph[bi] & 1u;
            // issued by thread 0; with the ring the whole of warp 0 takes the block (its lanes refill the
            // ring every FP_RING slabs), which measured faster than a separate refill branch
            if (dbl && tid < (RING ? 32 : 1) && i + 1 < nsl) {
                if (RING && (i + 1) % FP_RING == 0) fill_ring(i + 1);
                if (tid == 0) {
                    const SlabBox sbn = box_for(i + 1);
                    sh.box[(i + 1) & 1] = sbn;
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect_tx(bars[bi ^ 1], box_bytes);
                    tma_load_4d(smem_u32(bi ? buf0 : buf1), tmap, bars[bi ^ 1], yt ? sbn.lo[1] : sbn.lo[0],
                                yt ? sbn.lo[0] : sbn.lo[1], sbn.lo[2], b);
                }
            }
            // a copy lost anywhere aborts every CTA at its next slab, so the launch ends promptly (the
            // flag is read before the wait so that the two latencies overlap)
            int lost = 0;
            if (tid == 0) lost = *(volatile int *)(p.flags + FLAG_TMA_TIMEOUT);
            bool ok = mbar_wait_bounded(bars[bi], parity);
            if (lost != 0) ok = false;
            if (!__syncthreads_and(ok)) {
                if (tid == 0) atomicAdd(p.flags + FLAG_TMA_TIMEOUT, 1);
                // wait (bounded) for the copies still in flight before the shared memory goes away
                mbar_wait_bounded(bars[bi], parity);
                if (dbl && i + 1 < nsl) mbar_wait_bounded(bars[bi ^ 1], ph[bi ^ 1] & 1u);
                return false;
            }
            ++ph[bi];
            const SlabBox sb = sh.box[i & 1];
            const int b_lo = base0 + s * D;
            const int b_hi = min(b_lo + D, Nm);
            int ka = 0, kb = -1;
            if (hit) {
                if (pos) {
                    ka = (int)ceilf(fmaf((float)b_lo - cm, inv_step, -0.5f));
                    kb = (int)ceilf(fmaf((float)b_hi - cm, inv_step, -0.5f)) - 1;
                } else {
                    ka = (int)floorf(fmaf((float)b_hi - cm, inv_step, -0.5f)) + 1;
                    kb = (int)floorf(fmaf((float)b_lo - cm, inv_step, -0.5f));
                }
                ka = max(ka, k0);
                kb = min(kb, k1);
            }
            if (sb.fits) {
                const T *box = bi ? buf1 : buf0;
                // memory order of the box: (first, second, z) = (x, y, z), or (y, x, z) when yt; the
                // loop's "x" and "y" below are the first and second axes
                const int BF = yt ? BYb : BXb, BS = yt ? BXb : BYb;
                const int sy = BF, sz = BF * BS;
                // floor(q) + 2^23 + 2^22 is the bit pattern of q + 1.5 2^23 rounded down, so the box offset
                // sum floor(q_a) stride_a comes straight from the three bit patterns (unsigned wrap-around)
                const unsigned boff = 0x4B400000u * (unsigned)(sz + sy + 1);
                // position relative to the box origin: q = c0 + kf * step
                const float rcf = yt ? r.cy : r.cx, rdf = yt ? r.dy : r.dx;
                const float rcs = yt ? r.cx : r.cy, rds = yt ? r.dx : r.dy;
                const float c0x = fmaf(hdt, rdf, rcf - (float)(yt ? sb.lo[1] : sb.lo[0]));
                const float c0y = fmaf(hdt, rds, rcs - (float)(yt ? sb.lo[0] : sb.lo[1]));
                const float c0z = fmaf(hdt, r.dz, r.cz - (float)sb.lo[2]);
                const float stx = p.dt * rdf, sty = p.dt * rds, stz = p.dt * r.dz;
                float kf = (float)ka;
                // the eight corner values stay in registers while consecutive samples share a cell;
                // lanes that keep their cell issue no shared-memory reads
                int pbase = -1;
                float v000 = 0.0f, v001 = 0.0f, v010 = 0.0f, v011 = 0.0f;
                float v100 = 0.0f, v101 = 0.0f, v110 = 0.0f, v111 = 0.0f;
                const float M = 12582912.0f;
                const bool packed = pk != 0;   // 1: packed lerps; 2: packed lerps and positions
                auto sample = [&](int base, float ax, float ay, float az) {
                    if (base != pbase) {
                        const T *s0 = box + base;
                        v000 = to_f32(s0[0]); v001 = to_f32(s0[1]);
                        v010 = to_f32(s0[sy]); v011 = to_f32(s0[sy + 1]);
                        v100 = to_f32(s0[sz]); v101 = to_f32(s0[sz + 1]);
                        v110 = to_f32(s0[sz + sy]); v111 = to_f32(s0[sz + sy + 1]);
                        pbase = base;
                    }
                    if (packed) {
                        // the z = 0 and z = 1 lerps side by side in FP32x2 lanes: the same roundings as
                        // the scalar form, in 8 instead of 14 operations
                        const f32x2 c0010 = lerp2(splat2(ax), pack2(v000, v100), pack2(v001, v101));
                        const f32x2 c0111 = lerp2(splat2(ax), pack2(v010, v110), pack2(v011, v111));
                        const f32x2 c01 = lerp2(splat2(ay), c0010, c0111);
                        const float c0 = lo2(c01), c1 = hi2(c01);
                        acc += fmaf(az, c1 - c0, c0);
                    } else {
                        const float c00 = fmaf(ax, v001 - v000, v000);
                        const float c01 = fmaf(ax, v011 - v010, v010);
                        const float c10 = fmaf(ax, v101 - v100, v100);
                        const float c11 = fmaf(ax, v111 - v110, v110);
                        const float c0 = fmaf(ay, c01 - c00, c00);
                        const float c1 = fmaf(ay, c11 - c10, c10);
                        acc += fmaf(az, c1 - c0, c0);
                    }
                };
                // Positions are one correctly rounded FMA of the sample index, hence monotone in it along
                // each axis: when the first and the last sample's cells lie in the box (index in
                // [0, extent - 2] on every axis), all of them do and the loop needs no per-sample test.
                // The comparisons fail for NaN, which takes the checked loop.
                const float qax = fmaf(kf, stx, c0x), qbx = fmaf((float)kb, stx, c0x);
                const float qay = fmaf(kf, sty, c0y), qby = fmaf((float)kb, sty, c0y);
                const float qaz = fmaf(kf, stz, c0z), qbz = fmaf((float)kb, stz, c0z);
                const float ex = (float)(BF - 1), ey = (float)(BS - 1), ez = (float)(BZb - 1);
                if (qax >= 0.f && qbx >= 0.f && qax < ex && qbx < ex && qay >= 0.f && qby >= 0.f && qay < ey &&
                    qby < ey && qaz >= 0.f && qbz >= 0.f && qaz < ez && qbz < ez) {
                    if (pk == 2) {
                        // (x, y) positions, floors and fractions in FP32x2 lanes: the same roundings as
                        // the scalar loop below, in 5 instead of 9 operations per sample
                        const f32x2 st2 = pack2(stx, sty), c02 = pack2(c0x, c0y), M2 = splat2(M);
                        f32x2 kf2 = splat2(kf);
                        const f32x2 one2 = splat2(1.0f);
                        for (int k = ka; k <= kb; ++k) {
                            const f32x2 q2 = fma2(kf2, st2, c02);
                            const float qz = fmaf(lo2(kf2), stz, c0z);
                            const f32x2 t2 = add2_rd(q2, M2);
                            const float tz = __fadd_rd(qz, M);
                            const int base =
                                (int)((unsigned)__float_as_int(tz) * (unsigned)sz +
                                      ((unsigned)__float_as_int(hi2(t2)) * (unsigned)sy + ((unsigned)__float_as_int(lo2(t2)) - boff)));
                            const f32x2 a2 = sub2(q2, sub2(t2, M2));
                            sample(base, lo2(a2), hi2(a2), qz - (tz - M));
                            kf2 = add2(kf2, one2);
                        }
                    } else {
                        for (int k = ka; k <= kb; ++k, kf += 1.0f) {
                            const float qx = fmaf(kf, stx, c0x), qy = fmaf(kf, sty, c0y), qz = fmaf(kf, stz, c0z);
                            const float tx = __fadd_rd(qx, M), ty = __fadd_rd(qy, M), tz = __fadd_rd(qz, M);
                            const int base = (int)((unsigned)__float_as_int(tz) * (unsigned)sz +
                                                   ((unsigned)__float_as_int(ty) * (unsigned)sy + ((unsigned)__float_as_int(tx) - boff)));
                            sample(base, qx - (tx - M), qy - (ty - M), qz - (tz - M));
                        }
                    }
                } else {
                    for (int k = ka; k <= kb; ++k, kf += 1.0f) {
                        const float qx = fmaf(kf, stx, c0x), qy = fmaf(kf, sty, c0y), qz = fmaf(kf, stz, c0z);
                        const float tx = __fadd_rd(qx, M), ty = __fadd_rd(qy, M), tz = __fadd_rd(qz, M);
                        const int base = (int)((unsigned)__float_as_int(tz) * (unsigned)sz +
                                               ((unsigned)__float_as_int(ty) * (unsigned)sy + ((unsigned)__float_as_int(tx) - boff)));
                        // per-axis cell index in the box; a position outside (-2^22, 2^22), or NaN, gives an
                        // index far outside [0, extent - 1), so the test catches every sample off the box
                        const unsigned ix = (unsigned)(__float_as_int(tx) - 0x4B400000);
                        const unsigned iy = (unsigned)(__float_as_int(ty) - 0x4B400000);
                        const unsigned iz = (unsigned)(__float_as_int(tz) - 0x4B400000);
                        if (ix >= (unsigned)(BF - 1) || iy >= (unsigned)(BS - 1) || iz >= (unsigned)(BZb - 1)) {
                            atomicAdd(p.flags + FLAG_SLAB_OUT_OF_BOX, 1);
                            acc += trilerp_zero(vb, p.vol, (yt ? qy : qx) + (float)sb.lo[0],
                                                (yt ? qx : qy) + (float)sb.lo[1], qz + (float)sb.lo[2]);
                            pbase = -1;
                            continue;
                        }
                        sample(base, qx - (tx - M), qy - (ty - M), qz - (tz - M));
                    }
                }
            } else {
                if (tid == 0) atomicAdd(p.flags + FLAG_SLAB_OVERFLOW, 1);
                for (int k = ka; k <= kb; ++k) {
                    float t = fmaf((float)k, p.dt, hdt);
                    acc += trilerp_zero(vb, p.vol, fmaf(t, r.dx, r.cx), fmaf(t, r.dy, r.cy), fmaf(t, r.dz, r.cz));
                }
            }
            __syncthreads();   // everyone is done with this buffer before it is refilled
            // issued by thread 0, with warp 0 in the block where it refills the ring (as above)
            if (!dbl && tid < (RING ? 32 : 1) && i + 1 < nsl) {
                if (RING && (i + 1) % FP_RING == 0) fill_ring(i + 1);
                if (tid == 0) {
                    const SlabBox sbn = box_for(i + 1);
                    sh.box[(i + 1) & 1] = sbn;
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect_tx(bars[0], box_bytes);
                    tma_load_4d(smem_u32(buf0), tmap, bars[0], yt ? sbn.lo[1] : sbn.lo[0],
                                yt ? sbn.lo[0] : sbn.lo[1], sbn.lo[2], b);
                }
            }
        }
    }
    if (direct_ray) {
        atomicAdd(p.flags + FLAG_SLAB_DIRECT_RAY, 1);
        for (int k = k0; k <= k1; ++k) {
            float t = fmaf((float)k, p.dt, hdt);
            acc += trilerp_zero(vb, p.vol, fmaf(t, r.dx, r.cx), fmaf(t, r.dy, r.cy), fmaf(t, r.dz, r.cz));
        }
    }
    if (active)
        sino[(long long)b * p.sino_elems + ((long long)view * p.det.nv + v) * p.det.nu + u] = from_f32<T>(acc * p.dt);
    return true;
}

template <bool RING>
__device__ __forceinline__ void fp_tma_init_bars(FpTmaShared<RING> &sh) {
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&sh.bar[0]), 1);
        mbar_init(smem_u32(&sh.bar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

// 128-byte aligned slab buffers at the start of the dynamic shared memory
template <typename T>
__device__ __forceinline__ void fp_tma_buffers(unsigned char *smem_raw, int buf_elems, int nbuf, T *&buf0, T *&buf1) {
    const unsigned raw_u32 = smem_u32(smem_raw);
    const unsigned pad = ((raw_u32 + 127u) & ~127u) - raw_u32;
    buf0 = (T *)(smem_raw + pad);
    buf1 = nbuf == 2 ? (T *)(smem_raw + pad + sizeof(T) * (size_t)buf_elems) : buf0;
}

// MINB: CTAs per SM the register allocation must allow (4 where four slab buffers fit in shared memory)
template <typename T, int MINB, int PK>
__global__ void __launch_bounds__(TMA_NT, MINB) fp_tma_kernel(OpParams p, FpTmaBox cfg,
                                                           const __grid_constant__ TmaMaps maps,
                                                           const T *__restrict__ vol, T *__restrict__ sino) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ FpTmaShared<true> sh;
    T *buf0, *buf1;
    fp_tma_buffers<T>(smem_raw, cfg.buf_elems, cfg.nbuf, buf0, buf1);
    fp_tma_init_bars(sh);
    unsigned ph[2] = {0u, 0u};
    // grid (tile columns, views, tile rows x batch items): consecutive CTAs take the tiles of one tile row
    // in consecutive views, whose rays cross the same band of the volume, so the band stays in L2 while
    // the resident CTAs read it (see the launcher)
    const int ntv = (p.det.nv + TMA_TV - 1) / TMA_TV;
    fp_tma_tile<T, PK, true>(p, cfg, maps.map, vol, sino, blockIdx.y, blockIdx.z / ntv, blockIdx.x, blockIdx.z % ntv,
                       buf0, buf1, sh, ph);
}

// Persistent launch over the (view, tile) items of several volumes: each CTA takes the next item
// from a device counter until all are done. Volumes are ordered by decreasing cost per item.
struct PlanMaps {
    CUtensorMap map[PLAN_MAX][3];
};

template <typename T, int MINB, int PK>
__global__ void __launch_bounds__(TMA_NT, MINB) fp_tma_batched_kernel(const __grid_constant__ PlanLaunch L,
                                                                   const __grid_constant__ PlanMaps M) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ FpTmaShared<false> sh;
    __shared__ int s_item;
    fp_tma_init_bars(sh);
    unsigned ph[2] = {0u, 0u};
    const long long total = L.item_end[L.n - 1];
    for (;;) {
        __syncthreads();   // every thread has read the previous item number
        if (threadIdx.x == 0) s_item = atomicAdd(L.counter, 1);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        int i = 0;
        while (item >= L.item_end[i]) ++i;
        const PlanVolume &V = L.v[i];
        const long long local = item - (i ? L.item_end[i - 1] : 0);
        const int tiles = V.ntx * V.nty;
        const int view = (int)(local / tiles), t = (int)(local % tiles);
        T *buf0, *buf1;
        fp_tma_buffers<T>(smem_raw, V.cfg.buf_elems, V.cfg.nbuf, buf0, buf1);
        if (!fp_tma_tile<T, PK, false>(V.p, V.cfg, M.map[i], (const T *)V.in, (T *)V.out, view, 0, t % V.ntx, t / V.ntx,
                                buf0, buf1, sh, ph))
            return;
    }
}

// y-fastest copy of nvol volumes (x fastest): out[v][z][x][y] = in[v][z][y][x], through 32 x 32 tiles
// in shared memory so that both the reads and the writes are coalesced. blockIdx.z strides over the
// nz * nvol (z, volume) slices.
template <typename T>
__global__ void __launch_bounds__(256) transpose_xy_kernel(const T *__restrict__ in, T *__restrict__ out, int nx,
                                                           int ny, long long nslices) {
    __shared__ T tile[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    for (long long sl = blockIdx.z; sl < nslices; sl += gridDim.z) {
        const long long base = sl * nx * ny;
        __syncthreads();   // the previous slice's tile has been written out
        for (int j = threadIdx.y; j < 32; j += 8) {
            const int x = x0 + threadIdx.x, y = y0 + j;
            if (x < nx && y < ny) tile[j][threadIdx.x] = in[base + (long long)y * nx + x];
        }
        __syncthreads();
        for (int j = threadIdx.y; j < 32; j += 8) {
            const int y = y0 + threadIdx.x, x = x0 + j;
            if (x < nx && y < ny) out[base + (long long)x * ny + y] = tile[threadIdx.x][j];
        }
    }
}

// ---------------------------------------------------------------------------------------------
// host: box bound per march axis, tensor map, launch
// ---------------------------------------------------------------------------------------------
namespace {


// Per march axis, the largest cross-axis extents (in voxels) of any tile's staged box.
void tile_extents(const pyronn_geom *g, const FpRec &rec, int tu0, int tv0, int D, int G, int base0,
                  double ext[3][3]) {
    int tu1 = std::min(tu0 + TMA_TU, g->nu) - 1, tv1 = std::min(tv0 + TMA_TV, g->nv) - 1;
    RayD cr[4];
    for (int c = 0; c < 4; ++c) cr[c] = ray_setup_d(rec, g, (c & 1) ? tu1 : tu0, (c & 2) ? tv1 : tv0);
    RayD ctr = ray_setup_d(rec, g, 0.5 * (tu0 + tu1), 0.5 * (tv0 + tv1));
    const int dims[3] = {g->nx, g->ny, g->nz};
    double amax = std::max(std::fabs(ctr.d[0]), std::max(std::fabs(ctr.d[1]), std::fabs(ctr.d[2])));
    for (int m = 0; m < 3; ++m) {
        if (std::fabs(ctr.d[m]) < 0.999 * amax) continue;
        int a1 = (m == 0) ? 1 : 0, a2 = (m == 2) ? 1 : 2;
        int Nm = dims[m];
        int nslab = (Nm + 1 - base0 + D - 1) / D;
        for (int which = 0; which < 2; ++which) {
            int s = which ? nslab - 1 : 0;
            int b_lo = base0 + s * D, b_hi = std::min(b_lo + D, Nm);
            double planes[2] = {(double)(b_lo - G), (double)(b_hi + G)};
            double mn1 = 1e300, mx1 = -1e300, mn2 = 1e300, mx2 = -1e300;
            for (int c = 0; c < 4; ++c)
                for (int pl = 0; pl < 2; ++pl) {
                    double t = (planes[pl] - cr[c].c[m]) / cr[c].d[m];
                    double q1 = cr[c].c[a1] + t * cr[c].d[a1], q2 = cr[c].c[a2] + t * cr[c].d[a2];
                    mn1 = std::min(mn1, q1); mx1 = std::max(mx1, q1);
                    mn2 = std::min(mn2, q2); mx2 = std::max(mx2, q2);
                }
            // kernel: lo = floor(mn) - 1, hi = floor(mx) + 2 (clipped); extent <= ceil(mx - mn) + 4, +1 for FP32
            double e1 = std::min(std::ceil(mx1 - mn1) + 5.0, (double)(dims[a1] + 2 * G + 2));
            double e2 = std::min(std::ceil(mx2 - mn2) + 5.0, (double)(dims[a2] + 2 * G + 2));
            ext[m][a1] = std::max(ext[m][a1], e1);
            ext[m][a2] = std::max(ext[m][a2], e2);
        }
    }
}


}  // namespace

// The driver's tensor-map encoder, looked up once through the runtime (no link against libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// Box dimensions for the TMA kernel, or depth = 0 if it cannot be used (shared memory too small or
// the row pitch is not a multiple of 16 bytes). xt: x-march boxes may come from a y-fastest copy of
// the volume (taken where its rows, ny elements, are a multiple of 16 bytes too).
FpTmaBox choose_fp_tma_box(const pyronn_geom *g, size_t elem, int depth, int nbuf, int minb, int xt) {
    // automatic depth: the deeper slab where four CTAs still share an SM (fewer slab boundaries and copy
    // waits per ray), else 8 planes: 12 for FP32 (896 against 954 ms on the 512^3 workload; on the 256^3
    // one its box is too wide for four CTAs), 16 for 2-byte storage, whose boxes are half the bytes and
    // whose per-operand conversion the deeper slab repays (44.6 against 49.4 ms on the 256^3 workload, 963
    // against 1064 ms on the 512^3 one)
    if (depth == 0 && (elem == 2 || elem == 4)) {
        const FpTmaBox cd = choose_fp_tma_box(g, elem, elem == 2 ? 16 : 12, nbuf, minb, xt);
        if (cd.depth > 0 && cd.minb == 4) return cd;
    }
    FpTmaBox c{};
    const int align = 16 / (int)elem;
    if (((size_t)g->nx * elem) % 16 != 0) return c;
    const double smin = std::min(g->sx, std::min(g->sy, g->sz));
    if (!(g->dt / smin < 65535.0)) return c;   // steps of 2^16 voxels or more: another kernel
    c.xt = xt && ((size_t)g->ny * elem) % 16 == 0;
    // slab depth: a multiple of the x alignment so that x-march boxes start aligned
    c.depth = depth > 0 ? ((depth + align - 1) / align) * align : 8;
    c.nbuf = nbuf == 2 ? 2 : 1;   // default: one buffer (more CTAs per SM beat the copy overlap)
    c.guard = 1 + (int)std::floor(g->dt / smin);
    // slab planes start so that (first plane - guard) is a multiple of the x alignment
    c.slab0 = -1 - (((-1 - c.guard) % align) + align) % align;
    while (c.slab0 - c.guard > -1 - c.guard) c.slab0 -= align;   // keep the first slab at or below plane -1
    const int ntu = (g->nu + TMA_TU - 1) / TMA_TU, ntv = (g->nv + TMA_TV - 1) / TMA_TV;
    double ext[3][3] = {{0}};
    std::atomic<int> next(0);
    std::mutex mu;
    auto work = [&]() {
        double loc[3][3] = {{0}};
        for (int n = next.fetch_add(1); n < g->n_views; n = next.fetch_add(1))
            for (int j = 0; j < ntv; ++j)
                for (int i = 0; i < ntu; ++i)
                    tile_extents(g, g->fp_rec[n], i * TMA_TU, j * TMA_TV, c.depth, c.guard, c.slab0, loc);
        std::lock_guard<std::mutex> lk(mu);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) ext[a][b] = std::max(ext[a][b], loc[a][b]);
    };
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned i = 1; i < nt; ++i) th.emplace_back(work);
    work();
    for (auto &t : th) t.join();
    const int dims[3] = {g->nx, g->ny, g->nz};
    int maxel = 0;
    for (int m = 0; m < 3; ++m) {
        int e[3];
        for (int a = 0; a < 3; ++a) {
            // along m a slab's box spans planes b_lo - guard .. min(b_lo + depth, N) + guard, and the first
            // slab starts at slab0 (at or below plane -1)
            if (a == m) e[a] = std::min(c.depth + 2 * c.guard + 1, dims[a] - c.slab0 + 2 * c.guard + 1);
            else e[a] = (int)ext[m][a];
            if (a != m && e[a] == 0) e[a] = 1;   // axis never chosen: keep a valid box
        }
        if (m == 0 && c.xt) {
            // y-fastest copy: y is the innermost TMA dimension (room for the aligned start); the
            // rays of a warp read consecutive words of a row
            e[1] = ((e[1] + 2 * (align - 1)) / align) * align;
        } else {
            // x is the innermost TMA dimension: round up, plus room for the aligned start unless the
            // slab planes themselves start aligned (march along x)
            e[0] = m == 0 ? ((e[0] + align - 1) / align) * align : ((e[0] + 2 * (align - 1)) / align) * align;
            // march along x: all rays of a warp sit at nearly the same x, so a row pitch that is a
            // multiple of 32 bytes would fold their rows onto 4 or fewer bank groups; an odd multiple
            // of 16 bytes spreads consecutive rows over 8
            if (m == 0 && (e[0] * (int)elem) % 32 == 0) e[0] += align;
        }
        for (int a = 0; a < 3; ++a) e[a] = std::min(e[a], 256);
        c.bx[m] = e[0]; c.by[m] = e[1]; c.bz[m] = e[2];
        maxel = std::max(maxel, e[0] * e[1] * e[2]);
    }
    c.buf_elems = ((maxel * (int)elem + 127) / 128) * 128 / (int)elem;
    if ((size_t)c.nbuf * c.buf_elems * elem > 200 * 1024) c.depth = 0;   // does not fit: use another kernel
    // four CTAs per SM (registers capped at 64 per thread) where four copies of the slab buffers, the
    // static shared memory and the per-CTA reservation fit in the SM's 228 KB; else two
    const size_t per_cta = (size_t)c.nbuf * c.buf_elems * elem + 128 + 512 + 1024;
    const int auto_minb = 4 * per_cta <= 228 * 1024 ? 4 : 2;
    c.minb = (minb == 2 || minb == 4 || (minb == 3 && 3 * per_cta <= 228 * 1024)) ? minb : auto_minb;
    return c;
}

// Tensor maps of nb consecutive volumes (1 in plans) for the three march axes; with cfg.xt the x-march map
// covers the y-fastest copy vt.
template <typename T>
static int encode_maps(const OpParams &p, const FpTmaBox &cfg, const void *vol, const void *vt, int nb,
                       CUtensorMap maps[3]) {
    if (cfg.xt && !vt) return (int)cudaErrorInvalidValue;
    auto enc = tma_encode_fn();
    if (!enc) return (int)cudaErrorNotSupported;
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (std::is_same<T, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                      : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    const int nx = p.vol.nx, ny = p.vol.ny, nz = p.vol.nz;
    cuuint64_t gdim[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)nb};
    cuuint64_t gstride[3] = {(cuuint64_t)nx * sizeof(T), (cuuint64_t)nx * ny * sizeof(T),
                             (cuuint64_t)nx * ny * nz * sizeof(T)};
    cuuint32_t estride[4] = {1, 1, 1, 1};
    cuuint64_t gdim_t[4] = {(cuuint64_t)ny, (cuuint64_t)nx, (cuuint64_t)nz, (cuuint64_t)nb};
    cuuint64_t gstride_t[3] = {(cuuint64_t)ny * sizeof(T), (cuuint64_t)nx * ny * sizeof(T),
                               (cuuint64_t)nx * ny * nz * sizeof(T)};
    for (int m = 0; m < 3; ++m) {
        const bool t = m == 0 && cfg.xt;
        cuuint32_t box[4] = {(cuuint32_t)(t ? cfg.by[m] : cfg.bx[m]), (cuuint32_t)(t ? cfg.bx[m] : cfg.by[m]),
                             (cuuint32_t)cfg.bz[m], 1};
        CUresult r = enc(&maps[m], dt, 4, const_cast<void *>(t ? vt : vol), t ? gdim_t : gdim, t ? gstride_t : gstride,
                         box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return (int)cudaErrorInvalidValue;
    }
    return 0;
}

template <typename T>
static int launch_tma_t(const OpParams &p, const FpTmaBox &cfg, const void *vol, void *vol_t, void *sino,
                        cudaStream_t st, int make_copy) {
    if (cfg.xt && !vol_t) return (int)cudaErrorInvalidValue;
    const size_t smem = (size_t)cfg.nbuf * sizeof(T) * (size_t)cfg.buf_elems + 128;
    // one instantiation per (CTAs per SM, sample arithmetic)
    void (*kern)(OpParams, FpTmaBox, TmaMaps, const T *, T *);
    if (cfg.packed == 0)
        kern = cfg.minb == 4 ? fp_tma_kernel<T, 4, 0> : (cfg.minb == 3 ? fp_tma_kernel<T, 3, 0> : fp_tma_kernel<T, 2, 0>);
    else if (cfg.packed == 1)
        kern = cfg.minb == 4 ? fp_tma_kernel<T, 4, 1> : (cfg.minb == 3 ? fp_tma_kernel<T, 3, 1> : fp_tma_kernel<T, 2, 1>);
    else
        kern = cfg.minb == 4 ? fp_tma_kernel<T, 4, 2> : (cfg.minb == 3 ? fp_tma_kernel<T, 3, 2> : fp_tma_kernel<T, 2, 2>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    const int nx = p.vol.nx, ny = p.vol.ny, nz = p.vol.nz;
    // Grid order: tile columns fastest, then views, then tile rows and batch items. The CTAs resident at
    // one time are then the tiles of one tile row in about ten consecutive views; their rays cross one
    // band of the volume (the band of z that the row sees, widened by the cone angle), which stays in L2
    // while it is read. With views outermost the resident CTAs would sweep the whole volume once per view,
    // from DRAM once the volume exceeds L2. Views beyond the 65535 grid rows and batches beyond 65535
    // tile rows are split into several launches (tables and sinogram offset by the launch's first view).
    const int ntv = ceil_div(p.det.nv, TMA_TV);
    const int per_launch = 65535 / ntv > 0 ? 65535 / ntv : 1;
    const long long view_elems = (long long)p.det.nv * p.det.nu;
    for (int b0 = 0; b0 < p.batch; b0 += per_launch) {
        const int nb = p.batch - b0 < per_launch ? p.batch - b0 : per_launch;
        const T *vptr = (const T *)vol + b0 * p.vol_elems;
        T *tptr = cfg.xt ? (T *)vol_t + b0 * p.vol_elems : nullptr;
        if (cfg.xt && make_copy) {
            const long long nsl = (long long)nz * nb;
            dim3 tg(ceil_div(nx, 32), ceil_div(ny, 32), (unsigned)std::min<long long>(nsl, 65535));
            transpose_xy_kernel<T><<<tg, dim3(32, 8), 0, st>>>(vptr, tptr, nx, ny, nsl);
        }
        TmaMaps maps;
        std::memset(&maps, 0, sizeof(maps));
        const int rc = encode_maps<T>(p, cfg, vptr, tptr, nb, maps.map);
        if (rc) return rc;
        for (int v0 = 0; v0 < p.n_views; v0 += 65535) {
            const int nvw = p.n_views - v0 < 65535 ? p.n_views - v0 : 65535;
            OpParams q = p;
            q.fp = p.fp + v0;
            q.bp = p.bp ? p.bp + v0 : nullptr;
            q.views64 = p.views64 ? p.views64 + (size_t)v0 * VIEW64_STRIDE : nullptr;
            q.n_views = nvw;
            dim3 grid(ceil_div(p.det.nu, TMA_TU), nvw, ntv * nb);
            kern<<<grid, TMA_NT, smem, st>>>(q, cfg, maps, vptr, (T *)sino + b0 * p.sino_elems + v0 * view_elems);
        }
    }
    return (int)cudaGetLastError();
}

// the persistent kernel is compiled for four CTAs per SM (64 registers) where four CTAs' buffers fit
static bool batched_four(size_t smem) { return 4 * (smem + 512 + 1024) <= 228 * 1024; }

template <typename T>
static int launch_batched_t(const PlanLaunch &L, int grid, size_t smem, cudaStream_t st) {
    // the default sample arithmetic compiled in where every volume of the plan uses it (one sample loop
    // per kernel), else read per volume
    bool all2 = true;
    for (int i = 0; i < L.n; ++i) all2 = all2 && L.v[i].cfg.packed == 2;
    void (*kern)(PlanLaunch, PlanMaps);
    if (all2) kern = batched_four(smem) ? fp_tma_batched_kernel<T, 4, 2> : fp_tma_batched_kernel<T, 2, 2>;
    else kern = batched_four(smem) ? fp_tma_batched_kernel<T, 4, -1> : fp_tma_batched_kernel<T, 2, -1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    PlanMaps M;
    std::memset(&M, 0, sizeof(M));
    for (int i = 0; i < L.n; ++i) {
        const PlanVolume &V = L.v[i];
        if (V.cfg.xt) {
            if (!V.vt) return (int)cudaErrorInvalidValue;
            const int nx = V.p.vol.nx, ny = V.p.vol.ny;
            dim3 tg(ceil_div(nx, 32), ceil_div(ny, 32), (unsigned)std::min(V.p.vol.nz, 65535));
            transpose_xy_kernel<T><<<tg, dim3(32, 8), 0, st>>>((const T *)V.in, (T *)V.vt, nx, ny, V.p.vol.nz);
        }
        int rc = encode_maps<T>(V.p, V.cfg, V.in, V.vt, 1, M.map[i]);
        if (rc) return rc;
    }
    e = cudaMemsetAsync(L.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return (int)e;
    kern<<<grid, TMA_NT, smem, st>>>(L, M);
    return (int)cudaGetLastError();
}

int launch_fp_tma_batched(const PlanLaunch &L, int dtype, int grid, size_t smem, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_batched_t<float>(L, grid, smem, st);
        case PYRONN_BF16: return launch_batched_t<__nv_bfloat16>(L, grid, smem, st);
        case PYRONN_F16: return launch_batched_t<__half>(L, grid, smem, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

template <typename T>
static int batched_occupancy_t(size_t smem, int *blocks_per_sm) {
    auto kern = batched_four(smem) ? fp_tma_batched_kernel<T, 4, 2> : fp_tma_batched_kernel<T, 2, 2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, TMA_NT, smem);
    return (int)e;
}

int fp_tma_batched_occupancy(int dtype, size_t smem, int *blocks_per_sm) {
    switch (dtype) {
        case PYRONN_F32: return batched_occupancy_t<float>(smem, blocks_per_sm);
        case PYRONN_BF16: return batched_occupancy_t<__nv_bfloat16>(smem, blocks_per_sm);
        case PYRONN_F16: return batched_occupancy_t<__half>(smem, blocks_per_sm);
        default: return (int)cudaErrorInvalidValue;
    }
}

int launch_fp_tma(const OpParams &p, const FpTmaBox &cfg, const void *vol, void *vol_t, void *sino, int dtype,
                  void *stream, int make_copy) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (dtype) {
        case PYRONN_F32: return launch_tma_t<float>(p, cfg, vol, vol_t, sino, st, make_copy);
        case PYRONN_BF16: return launch_tma_t<__nv_bfloat16>(p, cfg, vol, vol_t, sino, st, make_copy);
        case PYRONN_F16: return launch_tma_t<__half>(p, cfg, vol, vol_t, sino, st, make_copy);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace pyronn
