// Internal declarations shared by the host geometry code, the C ABI and the CUDA kernels.
#pragma once

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pyronn.h"

namespace pyronn {

// ---------------------------------------------------------------------------------------------
// Device-side per-view records (FP32), built once per geometry on the host in FP64.
// ---------------------------------------------------------------------------------------------

// Ray family of one view, in world mm relative to the volume centre C:
//   reference point  Y(u, v) = R0 + u Ru + v Rv   (a point on the ray of pixel (u, v))
//   direction        D(u, v) = B0 + u Bu + v Bv   (unnormalised)
// Perspective views take Y on the plane through C parallel to the detector, so |Y| stays of the
// order of the volume size and the closest-point construction loses no FP32 precision.
struct FpRec {
    float R0[3], Ru[3], Rv[3];
    float B0[3], Bu[3], Bv[3];
};

// Filtered back-projection filter constants of one view (host FP64, stored FP32).
struct FbpRec {
    float scale;               // (pi / V) r^2 / tau: r = sid / sdd, tau = detector pitch at the volume centre
    float sdd;                 // source-detector distance, mm (0: parallel beam, no cosine weight)
    float b0[3], bu[3], bv[3]; // source -> pixel (u, v) = b0 + u bu + v bv, mm
};

// Projection of centred voxel indices (i - (Nx-1)/2, j - (Ny-1)/2, k - (Nz-1)/2, 1) to centred
// detector coordinates times depth: (u_c w, v_c w, w); u = u_c + (Nu-1)/2. Row-major 3 x 4.
struct BpRec {
    float P[12];
};

struct VolDims {
    int nx, ny, nz;
    float hx, hy, hz;      // (N - 1) / 2
    float isx, isy, isz;   // 1 / spacing (index units per mm)
};

struct DetDims {
    int nu, nv;
    float hu, hv;          // (N - 1) / 2
};

// Everything a kernel needs besides the data pointers.
struct OpParams {
    VolDims vol;
    DetDims det;
    int n_views;
    int batch;
    int perspective;       // 1: divide by w in BP; 0: affine (parallel) views
    int weight;            // BP weight mode (pyronn_bp_weight)
    float dt;              // sampling step, mm
    const FpRec *fp;       // device, n_views records
    const BpRec *bp;       // device, n_views records
    long long vol_elems;   // elements per volume
    long long sino_elems;  // elements per sinogram
    int *flags;            // device diagnostic counters (geometry-owned, see pyronn_geom_read_flags)
    // FP64 description (for per-brick constants computed on the device in double precision)
    const double *views64; // device, n_views x VIEW64_STRIDE extended FP64 records (see geometry.cpp)
    double sx, sy, sz;     // voxel spacing, mm
    double du, dv, ou, ov; // detector spacing / offset, mm
};

// Extended FP64 per-view record (all positions relative to the volume centre C, world mm):
//   perspective: [0..11] P with C folded in (maps X - C to (u w, v w, w)), [12..14] S - C,
//                [15..17] du eu, [18..20] dv ev, [21..23] D0 - S, [24..26] (du eu) x (dv ev),
//                [27] (D0 - S) . normal
//   parallel:    [0..2] Dc - C, [3..5] eu, [6..8] ev, [9..11] d (unit ray direction)
constexpr int VIEW64_STRIDE = 32;

// Diagnostic counters (device, per geometry).
enum {
    FLAG_SLAB_OUT_OF_BOX = 0,
    FLAG_SLAB_DIRECT_RAY = 1,
    FLAG_SLAB_OVERFLOW = 2,
    FLAG_TMA_TIMEOUT = 3,
    FLAG_ADJ_FIXED_SLABS = 4,
    FLAG_ADJ_FLOAT_SLABS = 5,
    N_FLAGS = 8
};

// Launch configuration of the slab-staged forward projector (chosen per geometry).
struct FpSlabCfg {
    int tu, tv;            // detector tile (rays per CTA = tu * tv)
    int depth;             // march slab depth in voxels
    int guard;             // extra staged planes on each side of a slab
    int smem_floats;       // staged box capacity
    int valid;             // 0: use the direct kernel
};

// Detector tile of one CTA of the TMA-staged forward projector (pixels along u, along v); the 32 lanes
// of a warp take 16 x 2 of its pixels
constexpr int FP_TILE_U = 16, FP_TILE_V = 16;

// Box shapes of the TMA-staged forward projector (chosen per geometry and element size).
struct FpTmaBox {
    int bx[3], by[3], bz[3];   // box extents (x, y, z) for march axis m = 0, 1, 2
    int depth, guard, slab0;   // slab depth (0: kernel unusable), guard planes, first slab plane
    int buf_elems;             // elements per buffer (max over axes)
    int nbuf;                  // 1 or 2 shared-memory buffers
    int minb;                  // CTAs per SM the single-volume kernel is compiled for (2 or 4)
    int xt;                    // x-march boxes come from a y-fastest copy of the volume (y innermost)
    int packed;                // sample loop: 0 scalar, 1 packed FP32x2 lerps, 2 packed lerps and (x, y) positions
};

// Slab-ordered adjoint configuration (chosen per geometry).
struct AdjSlabCfg {
    int depth, guard;          // slab depth, guard planes
    int box_cap;               // shared-memory box capacity (floats)
    int max_slabs;             // capacity of the per-tile slab table (dynamic shared memory, after the box)
    int valid;                 // 0: use the brick adjoint
    int allow_fixed;           // int32 fixed-point boxes where the per-slab bound allows
    int cell_fixed;            // fixed-point boxes: 1 cell-accumulated reductions, 0 one per sample
    int xpad;                  // x-march boxes get an odd row pitch (one word more than the x extent)
    int lanes;                 // lane-to-pixel mapping: 0 lanes along a tile row, 1 every other pixel of two rows
    int ypad;                  // y- and z-march boxes get a row pitch that is a multiple of 32 words where it fits
};

// Batched (persistent) launches: per-volume descriptions of one plan, in processing order.
constexpr int PLAN_MAX = 16;
struct PlanVolume {
    OpParams p;                // batch = 1
    FpTmaBox cfg;              // forward-projector boxes of this geometry and element type
    const void *in;            // input buffer (volume for FP, sinogram for adjoint / BP)
    void *out;                 // output buffer
    void *vt;                  // FP with cfg.xt: buffer for the y-fastest copy of the volume
    int ntx, nty;              // work tiles: detector tiles (FP) or volume bricks in x, y (adjoint, BP)
    int ntz;                   // bricks in z (adjoint, BP)
    int per_item;              // views per item group: FP items are (view, tile)
    AdjSlabCfg acfg;           // slab-ordered adjoint: slab configuration of this geometry
    float *acc;                // slab-ordered adjoint: FP32 accumulation volume (the output for FP32)
};
struct PlanLaunch {
    int n;
    long long item_end[PLAN_MAX];   // cumulative item counts
    PlanVolume v[PLAN_MAX];
    int *counter;              // device work counter (zeroed before the launch)
    int *flags;                // device flags (tensor-copy timeouts)
};

// Tuning knobs (pyronn_geom_set_tuning); 0 = automatic.
struct Tuning {
    int fp_depth = 0;          // slab depth of the TMA forward projector
    int fp_nbuf = 0;           // its number of buffers
    int fp_minb = 0;           // its CTAs per SM (2 or 4; 0 automatic)
    int adj_accum = 0;         // slab adjoint boxes: 0 automatic, 1 FP32 only, 2 fixed point with cells
    int fp_transpose = 0;      // TMA forward projector, x-march tiles: 0 y-fastest copy where usable, 1 never
    int adj_pitch = 0;         // slab adjoint, x-march boxes: 0 odd row pitch where it fits, 1 16-byte pitch
    int adj_depth = 0;         // slab adjoint: slab depth (0 automatic: the deepest that fits two CTAs per SM)
    int bp_brick_z = 0;        // brick back-projectors: voxels per thread along z (4, 8 or 16; 0 automatic, see
                               // bp_brick_depth)
    int adj_lanes = 0;         // slab adjoint lane-to-pixel mapping (0 automatic, 1 tile rows, 2 interleaved)
    int fp_packed = 0;         // TMA forward projector: 0 automatic (= 3), 1 scalar, 2 packed lerps, 3 packed lerps and positions
};

// Voxels per thread along z of the brick back-projectors for a volume of nz planes: the tuning value,
// or automatically 16 for volumes of at least 64 planes (the per-view set-up of a column is then spread
// over twice the voxels) and 8 below.
inline int bp_brick_depth(int tuning, int nz) { return tuning ? tuning : (nz >= 64 ? 16 : 8); }

}  // namespace pyronn

// ---------------------------------------------------------------------------------------------
// Geometry handle.
// ---------------------------------------------------------------------------------------------
struct pyronn_geom {
    int kind = 1;                  // 0 parallel, 1 perspective
    int ndim = 3;
    int nx = 0, ny = 0, nz = 0;
    double sx = 1, sy = 1, sz = 1;
    double ox = 0, oy = 0, oz = 0;
    int nu = 0, nv = 0;
    double du = 1, dv = 1, ou = 0, ov = 0;
    int n_views = 0;
    double dt = 0;
    std::vector<double> views;     // n_views x 12: P (perspective) or Dc, eu, ev, d (parallel)
    std::vector<pyronn::FpRec> fp_rec;
    std::vector<pyronn::BpRec> bp_rec;
    std::vector<double> views_ext;   // n_views x VIEW64_STRIDE (device copy: d_views64)

    // device state (one device per handle)
    std::mutex mu;
    int device = -1;
    pyronn::FpRec *d_fp = nullptr;
    pyronn::BpRec *d_bp = nullptr;
    int *d_flags = nullptr;
    double *d_views64 = nullptr;
    void *d_scratch = nullptr;     // FP32 accumulation buffer for reduced-precision adjoints
    size_t scratch_bytes = 0;
    pyronn::FbpRec *d_fbp = nullptr;   // FBP filter constants per view (uploaded on first use)
    void *tex_arr = nullptr;       // tiled gather texture of the texture projector (cudaArray_t)
    unsigned long long tex_obj = 0;    // its texture object
    void *d_tex_org = nullptr;     // tile origins (float2 per tile)
    int tex_batch = 0;             // volumes the array holds
    void *texf_arr = nullptr;      // 3D array of the hardware-filtered texture projector (cudaArray_t)
    unsigned long long texf_obj = 0;   // its texture object (linear filtering, border addressing)
    int texf_dtype = -1;           // element type the array holds
    int bpt_ready[3] = {0, 0, 0};  // staged back-projector: box chosen (per element type)
    int bpt_cfg[3][6] = {};        // its box (bu, bv), whether it applies, views per stage, slot stride, brick depth
    void *d_upd_sino = nullptr;    // work buffers of pyronn_adjoint_update on the unfused kernels
    void *d_upd_vol = nullptr;
    void *d_vol_t = nullptr;           // y-fastest copy of the volume for the TMA forward projector
    size_t vol_t_bytes = 0;
    void *copy_stream = nullptr;       // host-buffer entry points: stream of the overlapped downloads
    void *pipe_ev[9] = {};             // and the events that order it (one per view chunk, one final)
    size_t upd_sino_bytes = 0, upd_vol_bytes = 0;
    void *d_stage_in = nullptr;    // device buffers of the host-buffer entry points
    void *d_stage_out = nullptr;
    size_t stage_in_bytes = 0, stage_out_bytes = 0;

    int64_t sample_count = -1;     // cached pyronn_geom_count_samples
    pyronn::FpSlabCfg fp_cfg{};    // 0-initialised: chosen on first use
    int fp_cfg_ready = 0;
    pyronn::FpTmaBox tma_cfg[3] = {};   // per dtype
    pyronn::Tuning tuning;
    int tma_ready[3] = {0, 0, 0};
    int fp_variant = 0;            // 0 auto, 1 direct, 2 slab-staged (thread loads), 3 slab-staged (TMA), 4 texture
                                   // gather, 5 hardware-filtered texture (approximate weights, opt-in)
    int adj_variant = 0;           // 0 auto, 1 atomic scatter, 2 output-stationary bricks, 3 slab-ordered
    pyronn::AdjSlabCfg adj_cfg{};
    int adj_cfg_ready = 0;
    int bp_variant = 0;            // 0 auto, 1 one thread per voxel (absolute coordinates), 2 bricks (L1 path),
                                   // 3 bricks with TMA-staged detector shadows
};

namespace pyronn {

// error reporting (thread-local message)
int set_error(int code, const char *fmt, ...);
void clear_error();

// geometry helpers (geometry.cpp)
int finalize_geometry(pyronn_geom *g);          // build FP32 tables from views
int ensure_device(pyronn_geom *g);               // upload tables to the current device
OpParams make_params(const pyronn_geom *g, int batch);
FpSlabCfg choose_fp_slab_cfg(const pyronn_geom *g);
FpTmaBox choose_fp_tma_box(const pyronn_geom *g, size_t elem, int depth, int nbuf, int minb, int xt);
// vol_t: device buffer of batch x volume elements for the y-fastest copy (used when cfg.xt); make_copy 0:
// vol_t already holds the copy of vol (an earlier launch on the same stream made it)
int launch_fp_tma(const OpParams &p, const FpTmaBox &cfg, const void *vol, void *vol_t, void *sino, int dtype,
                  void *stream, int make_copy = 1);
int launch_fp_tma_batched(const PlanLaunch &L, int dtype, int grid, size_t smem, void *stream);
int launch_adjoint_brick_batched(const PlanLaunch &L, int dtype, int grid, void *stream);
int launch_residual(const void *a, const void *b, void *out, long long n, int dtype, void *stream);
int launch_fbp_filter(const OpParams &p, const FbpRec *rec, int filter, const void *in, void *out, int dtype,
                      void *stream);
int ensure_fbp(pyronn_geom *g);   // builds and uploads d_fbp (host FP64)
bool fp_tex_usable(const pyronn_geom *g, int batch, int dtype);
int launch_sim_jitter(const void *in, void *out, const int *shifts, int axis, int nu, int nv, long long n, int dtype,
                      void *stream);
int launch_sim_noise(const void *in, void *out, const float *noise, float mean, float sd, long long n, int dtype,
                     void *stream);
int launch_sim_ring(const void *in, void *out, const int *cols, const float *gains, int ncol, int nu, int nv, int n_views,
                    int v0, int v1, int batch, int dtype, void *stream);
int launch_sim_blur(const void *in, void *out, const float *angles, int length, int nu, int nv, int n_views, long long n,
                    int dtype, void *stream);
int launch_fp_tex(pyronn_geom *g, const OpParams &p, const void *vol, void *sino, void *stream);
bool fp_texf_usable(const pyronn_geom *g, int dtype);
bool bp_tma_usable(pyronn_geom *g, int dtype);
int launch_bp_tma(pyronn_geom *g, const OpParams &p, const void *sino, void *vol, int dtype, void *stream);
int launch_fp_texf(pyronn_geom *g, const OpParams &p, const void *vol, void *sino, int dtype, void *stream);
int launch_axpy(void *vol, const void *w, float alpha, long long n, int dtype, void *stream);
int launch_adjoint_slab_batched(const PlanLaunch &L, int dtype, int grid, size_t smem, void *stream);
int adjoint_slab_batched_occupancy(size_t smem, int *blocks_per_sm);
const AdjSlabCfg &geom_adj_cfg(pyronn_geom *g);   // cached per geometry (host computation)
int adjoint_brick_batched_occupancy(int *blocks_per_sm);
int launch_bp_brick_batched(const PlanLaunch &L, int dtype, int weight, int grid, void *stream);
int bp_brick_batched_occupancy(int *blocks_per_sm);
int fp_tma_batched_occupancy(int dtype, size_t smem, int *blocks_per_sm);

// kernel launchers (return a cudaError_t as int)
int launch_fp(const OpParams &p, const FpSlabCfg &cfg, const void *vol, void *sino, int dtype, void *stream);
int launch_fp_direct(const OpParams &p, const void *vol, void *sino, int dtype, void *stream);
int launch_adjoint(const OpParams &p, const void *sino, void *vol, float *acc32, int dtype, void *stream);
int launch_adjoint_brick(const OpParams &p, const void *sino, void *vol, int dtype, void *stream);
// dynamic shared memory of a slab-adjoint CTA: the box (box_cap floats, rounded to 16 bytes), then the
// slab table (max_slabs records)
size_t adjoint_slab_smem_bytes(int box_cap, int max_slabs);
AdjSlabCfg choose_adj_slab_cfg(const pyronn_geom *g);
int launch_adjoint_slab(const OpParams &p, const AdjSlabCfg &c, const void *sino, const void *sino_b, float y_scale,
                        bool accumulate, void *vol, float *acc32, int dtype, void *stream);
int launch_adjoint_scatter_acc(const OpParams &p, const void *sino, float *acc, void *vol, int dtype, void *stream);
int launch_bp(const OpParams &p, const void *sino, void *vol, int dtype, void *stream);
// bz: voxels per thread along z for 3D volumes (4, 8 or 16; 0 = 8)
int launch_bp_brick(const OpParams &p, int bz, const void *sino, void *vol, int dtype, void *stream);
int launch_bp_transpose(const OpParams &p, const void *vol, void *sino, float *acc32, int dtype, void *stream);

size_t dtype_size(int dtype);

// Grid size of a grid-stride element-wise kernel of 256 threads over n elements: enough CTAs for n, at
// most ctas_per_sm per SM of the current device (its SM count is queried once per device).
int stride_grid(long long n, int ctas_per_sm);

// Box extent (voxels) covering a span of index coordinates plus a margin, at most cap; -1 where the
// span is not finite (a corner ray parallel to the slab planes), which bounds nothing: the kernels
// test every tile's box against the buffer and send tiles that do not fit to global loads.
inline long long box_extent(double span, long long pad, long long cap) {
    if (!(span >= 0.0) || !std::isfinite(span)) return -1;
    if (!(span < (double)cap)) return cap;
    const long long e = (long long)std::ceil(span) + pad;
    return e < cap ? e : cap;
}

}  // namespace pyronn
