/*
 * pyronn.h — C ABI of the GB300 (sm_103a) CT projector library (libpyronn.so).
 *
 * Operators of "An update to PYRO-NN" (Schneider et al.):
 *   - the ray-driven forward projector A (Sec. 2.1: a ray per detector pixel, absorption
 *     accumulated along its path),
 *   - its exact transpose A^T (Sec. 2.2: "forward-projection operator A, with its adjoint"),
 *   - the voxel-driven back-projector (Sec. 2.1: each voxel projected onto the detector,
 *     detector values accumulated),
 * for 2D parallel, 2D fan and 3D cone-beam geometries (Sec. 2.1), with each view described by a
 * projection matrix so that calibrated matrices and arbitrary trajectories work (Sec. 2.1 last
 * sentence, Sec. 2.4 "Flexible Trajectory Modeling").
 *
 * Discretisation (the paper gives the operators in prose only; these are the library's
 * definitions, implemented identically by every kernel):
 *   voxel (i, j, k) of an (Nz, Ny, Nx) volume with spacing (sz, sy, sx) and centre offset
 *   (oz, oy, ox) sits at world ((i - (Nx-1)/2) sx + ox, (j - (Ny-1)/2) sy + oy, (k - (Nz-1)/2) sz + oz) mm;
 *   ray r is sampled at t_k = (k + 1/2) dt (k integer, dt in mm, default half the smallest voxel
 *   spacing) measured from its point closest to the volume centre; the volume is the
 *   trilinear (2D: bilinear) hat-function interpolant I, zero outside the grid;
 *     FP:      p_r = dt * sum_k I(c_r + t_k d_r)
 *     adjoint: (A^T y)_v = sum_r y_r dt sum_k prod_axes hat(q(r, k) - v)
 *     BP:      b_v = sum_views omega * (bilinear, zero-padded detector value at the projection of v),
 *              omega = 1 or 1 / w^2, w the depth ratio of v between source and detector plane.
 *
 * Memory layout (row-major, contiguous, owned by the caller, device memory unless stated):
 *   volume    [batch][Nz][Ny][Nx]   (2D: Nz = 1)
 *   sinogram  [batch][V][Nv][Nu]    (2D: Nv = 1)
 * Element type: PYRONN_F32, PYRONN_BF16 or PYRONN_F16 storage; all arithmetic is FP32.
 * Buffers must be 16-byte aligned.
 *
 * Errors: every call returns PYRONN_OK (0) or a negative pyronn_status; pyronn_last_error()
 * returns a message for the calling thread. Calls never abort and never trap on the device.
 * Operator calls are asynchronous on the given stream (a cudaStream_t passed as void*, NULL for
 * the legacy default stream) and never synchronise, except the *_host variants.
 * The first operator call of a geometry on a device uploads its per-view tables with a
 * synchronous copy; make that call before capturing a CUDA graph.
 *
 * Threads and streams: calls on different geometries are independent. Calls on one geometry may
 * come from several host threads (its lazily built tables, configurations and sample count are
 * set up under a lock), but on the device they must be ordered, on one stream or with events:
 * several operators use geometry-owned work buffers (the forward projector's y-fastest volume
 * copy, the FP32 accumulation of BF16 / FP16 adjoints, the update and host staging buffers). For
 * concurrent work use one geometry per stream, or a plan. The setters (pyronn_geom_set_step,
 * _set_variant, _set_tuning) and pyronn_geom_destroy must not run while another call uses the
 * same geometry.
 */
#ifndef PYRONN_H
#define PYRONN_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PYRONN_API __attribute__((visibility("default")))
#else
#define PYRONN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pyronn_geom *pyronn_geom_t;

typedef enum {
    PYRONN_OK = 0,
    PYRONN_INVALID_ARG = -1,
    PYRONN_UNSUPPORTED_DTYPE = -2,
    PYRONN_MISALIGNED = -3,
    PYRONN_CUDA_ERROR = -4,
    PYRONN_OOM = -5,
    PYRONN_SINGULAR = -6,
    PYRONN_DEVICE_CHECK_FAILED = -7
} pyronn_status;

typedef enum { PYRONN_F32 = 0, PYRONN_BF16 = 1, PYRONN_F16 = 2 } pyronn_dtype;

typedef enum { PYRONN_BP_PLAIN = 0, PYRONN_BP_INV_W2 = 1 } pyronn_bp_weight;

/* Volume description: the paper's volume_shape / volume_spacing (Listing 1), numpy (z, y, x)
 * order. ndim = 2 describes an image: shape[0] must be 1, spacing[0] and offset[0] are ignored.
 * The create calls return PYRONN_INVALID_ARG for a shape outside [1, 16384], an offset that is not
 * finite, a spacing (here or on the detector) that is not positive or whose value or reciprocal is
 * not finite in FP32, a geometry whose FP32 per-view tables would hold a non-finite entry, or a
 * default step (half the smallest spacing) that gives more than 2^22 samples across the volume. */
typedef struct {
    int ndim;
    int shape[3];        /* (Nz, Ny, Nx) */
    double spacing[3];   /* (sz, sy, sx) mm */
    double offset[3];    /* (oz, oy, ox) world position of the volume centre, mm */
} pyronn_vol_desc;

/* Detector description: the paper's detector_shape / detector_spacing (Listing 1), (rows, cols).
 * For 2D geometries shape[0] must be 1. offset shifts the detector centre along (ev, eu). */
typedef struct {
    int shape[2];        /* (Nv, Nu) */
    double spacing[2];   /* (dv, du) mm */
    double offset[2];    /* (ov, ou) mm */
} pyronn_det_desc;

/* ------------------------------------------------------------------------------------------
 * Geometry (host-side; FP64). The handle owns its host tables, its per-device view tables and
 * any scratch it needs; release it with pyronn_geom_destroy. Creation needs no GPU.
 * ---------------------------------------------------------------------------------------- */

/* 2D parallel beam (Sec. 2.1). View n at angle t = n * angular_range / n_views; rays run along
 * -(cos t, sin t); bin u lies at (u - (Nu-1)/2) du + ou along (-sin t, cos t). */
PYRONN_API int pyronn_geom_create_parallel2d(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                                  double angular_range, pyronn_geom_t *out);

/* 2D fan beam (Sec. 2.1): the z = 0 plane of the circular orbit below (sid = source-isocentre,
 * sdd = source-detector distance, Listing 1). */
PYRONN_API int pyronn_geom_create_fan2d(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                             double angular_range, double sid, double sdd, pyronn_geom_t *out);

/* 3D cone beam on a circular (helical_pitch_mm = 0) or helical orbit (Listing 1 parameters:
 * number_of_projections, angular_range, sdd, sid). View n at angle t = n * angular_range / n_views:
 * source sid (cos t, sin t, z_n), detector centre -(sdd - sid) (cos t, sin t, 0) + (0, 0, z_n),
 * eu = (-sin t, cos t, 0), ev = (0, 0, 1), z_n = pitch (n - (V-1)/2) (angular_range / V) / (2 pi).
 * The per-view matrices are built as in Sec. 2.4 (from source and detector positions). */
PYRONN_API int pyronn_geom_create_cone_circular(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                                     double angular_range, double sid, double sdd, double helical_pitch_mm,
                                     pyronn_geom_t *out);

/* 3D cone beam from source / detector positions and detector directions (Sec. 2.4, after
 * Graetz): src, det_centre, eu, ev are n_views x 3 world-mm arrays (eu, ev need not be unit:
 * they are normalised). P = M^-1 [I | -S] with M = [du eu | dv ev | D0 - S] and D0 the centre of
 * pixel (0, 0). Returns PYRONN_SINGULAR if a view's M is singular. */
PYRONN_API int pyronn_geom_create_from_positions(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                                      const double *src, const double *det_centre, const double *eu,
                                      const double *ev, pyronn_geom_t *out);

/* 3D cone beam from calibrated projection matrices (Sec. 2.1, Sec. 2.4): P is n_views x 3 x 4
 * row-major, mapping world (x, y, z, 1) mm to (u w, v w, w) with (u, v) pixel indices. Each
 * matrix is rescaled so that inv(P[:, :3]) has a first column of length du and w > 0 at the
 * volume centre. Returns PYRONN_SINGULAR if P[:, :3] is singular or w vanishes there. */
PYRONN_API int pyronn_geom_create_cone_matrices(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                                     const double *P, pyronn_geom_t *out);

/* 2D fan beam from 2 x 3 matrices (n_views x 2 x 3, world (x, y, 1) -> (u w, w)), or 2D parallel
 * beam when every matrix's last row is (0, 0, 1) (u = P[0] . (x, y, 1)). Normalised like the
 * 3D matrices (|inv(P[:, :2]) column 0| = du, w > 0 at the image centre). */
PYRONN_API int pyronn_geom_create_matrices2d(const pyronn_vol_desc *vol, const pyronn_det_desc *det, int n_views,
                                  const double *P, pyronn_geom_t *out);

/* Releases the handle with its host tables and every device buffer, stream and event it owns (on the
 * device they were created on). NULL is accepted and does nothing. The caller must make sure no
 * operation that uses g is still running on any stream (synchronise first); g is invalid afterwards. */
PYRONN_API int pyronn_geom_destroy(pyronn_geom_t g);

/* Sampling step along rays in mm (> 0). Default: half the smallest voxel spacing. PYRONN_INVALID_ARG
 * if the step or its reciprocal is not finite in FP32, or if the diagonal of the support box
 * ((-1, N) voxels on every axis) spans more than 2^22 steps. Steps of 2^16 voxels or more are accepted
 * and run on the direct projector and the brick adjoint (the slab-staged kernels need fewer). */
PYRONN_API int pyronn_geom_set_step(pyronn_geom_t g, double dt_mm);
/* The current step in mm, written to *dt_mm (PYRONN_INVALID_ARG for a NULL argument). */
PYRONN_API int pyronn_geom_get_step(pyronn_geom_t g, double *dt_mm);

/* Number of views, geometry kind (0 parallel, 1 perspective) and dimension (2 or 3); any output
 * pointer may be NULL. */
PYRONN_API int pyronn_geom_info(pyronn_geom_t g, int *n_views, int *kind, int *ndim);

/* Copy out the normalised per-view matrices: n_views x 12 doubles. Perspective views: P (3 x 4).
 * Parallel views: Dc[3], eu[3], ev[3], d[3] (detector centre, axes, ray direction). */
PYRONN_API int pyronn_geom_get_views(pyronn_geom_t g, double *out);

/* Exact number of (ray, sample) pairs whose sample lies inside the open support box (-1, N_a) on
 * every axis, summed over all views (FP64 host computation, multithreaded, cached). This is the
 * work unit of the forward projector's throughput. */
PYRONN_API int pyronn_geom_count_samples(pyronn_geom_t g, int64_t *total);

/* ------------------------------------------------------------------------------------------
 * Operators (device buffers, asynchronous on `stream`).
 * ---------------------------------------------------------------------------------------- */

/* Forward projection (Sec. 2.1 ray-driven; operator A of Sec. 2.2): sino = A vol, overwriting
 * sino. The TMA-staged projector may first copy the volume into a geometry-owned y-fastest buffer
 * (allocated on first use; see PYRONN_TUNE_FP_TRANSPOSE); since that buffer belongs to the
 * geometry, forward projections with one geometry on different streams must not overlap (use one
 * geometry per stream, or a plan, whose copies are per volume). */
PYRONN_API int pyronn_fp(pyronn_geom_t g, const void *vol, void *sino, int dtype, int batch, void *stream);

/* Matched adjoint (operator A^T of Sec. 2.2, the exact transpose of pyronn_fp):
 * vol = A^T sino, overwriting vol. For BF16/F16 storage the sum is formed in FP32 in a
 * geometry-owned scratch buffer (allocated on first use) and converted once at the end. */
PYRONN_API int pyronn_adjoint(pyronn_geom_t g, const void *sino, void *vol, int dtype, int batch, void *stream);

/* Fused gradient step (the data-term update of an iterative reconstruction, Sec. 2.2 "known operator"
 * networks; no dedicated passage in the paper): vol += alpha * A^T (sino - sino_b), accumulating into
 * vol in place. sino_b may be NULL (then vol += alpha A^T sino). With the slab-ordered adjoint the
 * residual is formed while the sinogram is read and the sum is added straight into vol (FP32), or into
 * an FP32 copy of vol that is converted back (BF16 / FP16); other adjoint kernels go through
 * geometry-owned work buffers (a residual sinogram and an adjoint volume, allocated on first use).
 * Same layouts, alignment and error behaviour as pyronn_adjoint; alpha must be finite. */
PYRONN_API int pyronn_adjoint_update(pyronn_geom_t g, const void *sino, const void *sino_b, double alpha, void *vol,
                                     int dtype, int batch, void *stream);

/* Filtered back-projection filter (Sec. 2.2: x = A^T F^T K F p with a ramp K, as in Listing 1's FDK
 * pipeline): out = per row, the cosine pre-weight of divergent beams (cos of each pixel's ray to the
 * detector normal), a direct convolution with the ramp's taps along u (filter 0 Ram-Lak: the ramp
 * band-limited to the detector's Nyquist frequency; 1 Shepp-Logan: times a sinc window) and the scale
 * (pi / V) r^2 / tau (r = sid / sdd at the volume centre, tau = detector pitch scaled to the volume
 * centre; parallel beams: r = 1, tau = du). pyronn_bp of out with weight PYRONN_BP_INV_W2 (divergent)
 * or PYRONN_BP_PLAIN (parallel) is the reconstruction of a [0, 2 pi) divergent or [0, pi) parallel
 * scan with V uniformly spaced views. sino and out are [batch][V][Nv][Nu] of one element type and may
 * be the same buffer; Nu <= 4096. Asynchronous on stream; status code as elsewhere. */
typedef enum { PYRONN_FILTER_RAM_LAK = 0, PYRONN_FILTER_SHEPP_LOGAN = 1 } pyronn_fbp_filter_kind;
PYRONN_API int pyronn_fbp_filter(pyronn_geom_t g, const void *sino, void *out, int filter, int dtype, int batch,
                                 void *stream);

/* ------------------------------------------------------------------------------------------
 * Acquisition-artifact simulation (Sec. 2.4). Sinograms [batch][V][Nv][Nu] of element type dtype
 * on the device; every random quantity is passed in (device arrays), so the calls are
 * deterministic. Asynchronous on stream; status code as elsewhere.
 * ---------------------------------------------------------------------------------------- */

/* Detector jitter: every detector row (axis 0: out[v][u] = sino[v][u - s], one int32 shift per
 * (item, view, row): [batch][V][Nv]) or column (axis 1: out[v][u] = sino[v - s][u], shifts
 * [batch][V][Nu]) moved by its shift in pixels, zero where the source lies outside. Not in place. */
PYRONN_API int pyronn_sim_detector_jitter(pyronn_geom_t g, const void *sino, void *out, const int32_t *shifts,
                                          int axis, int dtype, int batch, void *stream);

/* Gaussian noise: out = sino + mean + std * noise, noise an FP32 array of standard-normal samples
 * shaped like the sinogram. out may be sino. */
PYRONN_API int pyronn_sim_gaussian_noise(pyronn_geom_t g, const void *sino, void *out, const float *noise, double mean,
                                         double std, int dtype, int batch, void *stream);

/* Ring artifacts: out = sino, except detector columns columns[c] (int32, c < n_columns) of views
 * view_begin .. view_end - 1, which are multiplied by gains[c] (FP32; 0 = dead element). Columns
 * outside [0, Nu) are ignored. out may be sino. */
PYRONN_API int pyronn_sim_ring(pyronn_geom_t g, const void *sino, void *out, const int32_t *columns, const float *gains,
                               int n_columns, int view_begin, int view_end, int dtype, int batch, void *stream);

/* Gantry motion blur: each projection convolved with a line kernel of `length` samples (1 .. 1024),
 * unit total weight, rotated to its view's angle angles[view] (FP32 radians, [V]):
 * out(u, v) = (1 / L) sum_j bilinear(sino, u + t_j cos a, v + t_j sin a), t_j = j - (L - 1) / 2, zero
 * outside the detector. Not in place. */
PYRONN_API int pyronn_sim_motion_blur(pyronn_geom_t g, const void *sino, void *out, const float *angles, int length,
                                      int dtype, int batch, void *stream);

/* Voxel-driven back-projection (Sec. 2.1): vol = BP sino, overwriting vol; weight is a
 * pyronn_bp_weight. Not the transpose of pyronn_fp. */
PYRONN_API int pyronn_bp(pyronn_geom_t g, const void *sino, void *vol, int dtype, int batch, int weight, void *stream);

/* Exact transpose of pyronn_bp (the gradient of the voxel-driven back-projector with respect to
 * its sinogram, Sec. 2.1 "analytical gradients for all operators"): sino = BP^T vol, overwriting
 * sino. Each voxel spreads its value times omega over the four detector pixels around its
 * projection with the bilinear weights. BF16/F16 storage accumulates in FP32 scratch. */
PYRONN_API int pyronn_bp_transpose(pyronn_geom_t g, const void *vol, void *sino, int dtype, int batch, int weight,
                                   void *stream);

/* Matched adjoint that allocates no device memory (the paper has no counterpart: this is a
 * deployment variant of pyronn_adjoint's one-thread-per-ray atomic scatter). For callers that
 * cannot let a library call cudaMalloc, for example code running inside a memory pool that owns
 * the device or a pipeline that must not allocate after start-up. The per-view ray table and the
 * FP32 accumulator live in fixed device arrays of the library (at most 4096 views and 8M voxels
 * in total, volume x batch: 32 MiB), held by every GPU that loads the library until the process
 * exits; larger requests return PYRONN_INVALID_ARG. The first call on a device looks up the
 * arrays' device addresses (make it before any stream capture). Calls share the arrays: each call
 * clears the accumulator first, and calls that overlap on the GPU race, so serialise them.
 * Same arguments and result as pyronn_adjoint (vol is overwritten); asynchronous on stream. */
PYRONN_API int pyronn_adjoint_noalloc(pyronn_geom_t g, const void *sino, void *vol, int dtype, int batch,
                                      void *stream);

/* ------------------------------------------------------------------------------------------
 * Batched plans: many volumes, each with its own size and geometry, in one persistent launch per
 * operator (the paper's layers carry a batch dimension, Listing 1; here every batch member may
 * have its own geometry). Each CTA takes (view, detector tile) items (forward projection) or
 * volume-brick items (adjoint, back-projection) from a device work counter, largest items first.
 * Every call is one cudaMemsetAsync of the counter plus one kernel launch on `stream` (the forward
 * projection first adds one transpose launch per volume staged from a y-fastest copy) and allocates
 * nothing, so calls can be captured in a CUDA graph; the plan is created (and the geometries'
 * device tables uploaded) before capture.
 * ---------------------------------------------------------------------------------------- */
typedef struct pyronn_plan *pyronn_plan_t;

/* n (1..16) 3D geometries; dtype is the storage type of every buffer used with the plan. Volumes
 * whose rows (Nx elements) are not a multiple of 16 bytes cannot use tensor copies: their forward
 * projection runs as a separate per-geometry launch on the same stream. The plan allocates a
 * y-fastest copy buffer for every volume whose forward projection stages x-march boxes from one
 * (PYRONN_TUNE_FP_TRANSPOSE of its geometry at creation). The plan refers to the geometries (it
 * does not own them): keep them alive while the plan is used. */
PYRONN_API int pyronn_plan_create(int n, const pyronn_geom_t *geoms, int dtype, pyronn_plan_t *out);
PYRONN_API int pyronn_plan_destroy(pyronn_plan_t plan);

/* Item counts and persistent grid sizes: grids[3] = {forward, adjoint, back-projection}. */
PYRONN_API int pyronn_plan_info(pyronn_plan_t plan, int *n, int64_t *items_fp, int64_t *items_brick, int *grids);

/* vols / sinos: host arrays of n device pointers, in the order of the geometries given to
 * pyronn_plan_create. Same operators and overwrite semantics as pyronn_fp / pyronn_adjoint /
 * pyronn_bp with batch = 1 per geometry. */
PYRONN_API int pyronn_plan_fp(pyronn_plan_t plan, const void *const *vols, void *const *sinos, void *stream);
PYRONN_API int pyronn_plan_adjoint(pyronn_plan_t plan, const void *const *sinos, void *const *vols, void *stream);
PYRONN_API int pyronn_plan_bp(pyronn_plan_t plan, const void *const *sinos, void *const *vols, int weight,
                              void *stream);

/* Host-buffer variants: copy the input from host memory (pinned for best speed) into device
 * buffers owned by the geometry (allocated on first use), run the operator on `stream`, copy
 * the result back and synchronise the stream. With the TMA-staged projector the forward
 * projection runs the views in up to 8 chunks and downloads each chunk's sinogram rows on a
 * geometry-owned stream while the next chunk runs (the volume's upload precedes every view). */
PYRONN_API int pyronn_fp_host(pyronn_geom_t g, const void *vol_host, void *sino_host, int dtype, int batch, void *stream);
PYRONN_API int pyronn_adjoint_host(pyronn_geom_t g, const void *sino_host, void *vol_host, int dtype, int batch,
                        void *stream);

/* Kernel variant of an operator, for tests and tuning. op 0 = forward projection: variant 0
 * automatic (= 3 where usable, else 2), 1 one-thread-per-ray read-only-cache kernel, 2 slab-staged
 * shared-memory kernel filled by thread loads (falls back to 1 when the staged box cannot fit),
 * 3 slab-staged kernel filled by TMA tensor copies (needs a row pitch that is a multiple of 16
 * bytes; falls back to 2), 4 one thread per ray with texture gathers from a tiled 2D copy of the
 * volume (3D FP32 within the device's gather-texture limits, else as 0; the copy belongs to the
 * geometry, so forward projections with one geometry on different streams must not overlap), 5 one
 * thread per ray with the texture unit's trilinear filtering from a geometry-owned 3D texture copy of
 * the volume (the paper's "texture interpolation", Sec. 2.1: FP32 or FP16 storage of 3D volumes within
 * the device's 3D texture limits, else as 0; the hardware weighs the texels with 8-bit fractions, so
 * this variant is NOT the library's operator to FP32 accuracy but an approximation of it with a
 * relative error of the order of 1e-3; same stream restriction as variant 4).
 * op 1 = matched adjoint:
 * variant 0 automatic (= 3 where its box fits, else 2), 1 one-thread-per-ray FP32 global atomics,
 * 2 output-stationary bricks accumulated in shared memory, 3 slab-ordered: detector tiles march
 * the volume like the forward projector, scatter into shared-memory slab boxes and add each box to
 * the volume with vector reductions. op 2 = voxel-driven back-projection: variant 0 automatic
 * (= 3 where usable, else 2), 1 one thread per voxel in absolute detector
 * coordinates, 2 bricks with
 * detector coordinates relative to the brick centre's projection, taps read through L1, 3 the same
 * bricks with each view's shadow of the brick copied into shared memory by tensor copies, one chunk of
 * views ahead (3D volumes whose detector rows are a multiple of 16 bytes). All variants compute the same operator,
 * except forward-projection variant 5 (approximate interpolation weights). */
PYRONN_API int pyronn_geom_set_variant(pyronn_geom_t g, int op, int variant);

/* Tuning knobs of the kernels (used by the autotuner; 0 restores the automatic choice). All
 * settings compute the same operator. PYRONN_TUNE_FP_DEPTH: slab depth of the TMA-staged forward
 * projector in voxel planes (rounded up to the 16-byte x alignment); PYRONN_TUNE_FP_BUFFERS: 1 or
 * 2 shared-memory slab buffers (2 overlaps the next copy with sampling; 1 halves shared memory so
 * more CTAs fit on an SM); PYRONN_TUNE_ADJ_ACCUM: accumulation of the slab-ordered adjoint's
 * shared-memory boxes, 0 automatic (int32 fixed point with a power-of-two scale per tile and slab
 * wherever a bound on the box values allows it, with a quantum between 2^-22 and 2^-21 of the
 * tile's largest |y| dt, FP32 reductions elsewhere; fixed-point boxes take one reduction per sample
 * and corner), 1 FP32 reductions only, 2 as 0 but fixed-point boxes take one reduction per corner of
 * each cell a ray passes (weights summed in registers while the ray stays in the cell);
 * PYRONN_TUNE_FP_CTAS_PER_SM: CTAs per SM the TMA-staged forward projector is compiled for, 2, 3 or
 * 4 (4 caps registers at 64 per thread, 3 at 80; 3 needs three CTAs' slab buffers to fit in shared
 * memory; automatic: 4 where four CTAs' slab buffers fit); PYRONN_TUNE_FP_TRANSPOSE: 0 (automatic) lets the TMA-staged forward projector stage the
 * slabs of detector tiles that march along x from a y-fastest copy of the volume, made on the
 * call's stream into a geometry-owned buffer of the volume's size (allocated on first use), so that
 * the rays of a warp, which spread across y there, read consecutive shared-memory words; 1 stages
 * every slab from the volume itself; PYRONN_TUNE_ADJ_PITCH: 0 (automatic) gives the slab-ordered
 * adjoint's x-march boxes an odd row pitch (one word more than their x extent) wherever a slab depth
 * still fits two CTAs per SM with it, and its y- and z-march boxes a row pitch that is a multiple of 32
 * words wherever the padded box fits its capacity; 1 keeps rows of whole 16-byte groups everywhere; 2 as
 * 0 without the 32-word pitch; PYRONN_TUNE_ADJ_DEPTH: slab
 * depth of the slab-ordered adjoint in voxel planes, 2 .. 16 (0 automatic: the deepest of 8, 6, 5, 4 whose
 * box lets two CTAs share an SM; a depth whose box does not fit runs one CTA per SM, or the brick adjoint
 * if the box exceeds 160 KB); PYRONN_TUNE_BP_BRICK_Z: voxels per thread along z of the brick
 * back-projectors of 3D volumes, 4, 8 or 16 (0 automatic: 16 for volumes of at least 64 planes, else 8;
 * the staged back-projector, variant 3, takes 16 where the depth is 16 and 8 otherwise);
 * PYRONN_TUNE_ADJ_LANES: how the
 * slab-ordered adjoint's lanes take the pixels of a tile, 0 automatic (= 1), 1 the 32 lanes of a warp on
 * consecutive pixels of one tile row, 2 in each pass on every other pixel of two rows two pixels apart
 * (rays of adjacent pixels often share a cell, and their reductions then hit the same shared word);
 * PYRONN_TUNE_FP_PACKED: the TMA-staged projector's sample arithmetic, 0 automatic (= 3), 1 scalar FP32
 * instructions, 2 packed FP32x2 instructions for the pairs of lerps along x and y, 3 packed also for the
 * (x, y) positions, floors and fractions (identical results in every mode: each lane rounds as the
 * scalar instruction does). */
typedef enum {
    PYRONN_TUNE_FP_DEPTH = 0,
    PYRONN_TUNE_FP_BUFFERS = 1,
    PYRONN_TUNE_ADJ_ACCUM = 2,
    PYRONN_TUNE_FP_CTAS_PER_SM = 3,
    PYRONN_TUNE_FP_TRANSPOSE = 4,
    PYRONN_TUNE_ADJ_PITCH = 5,
    PYRONN_TUNE_ADJ_DEPTH = 6,
    PYRONN_TUNE_BP_BRICK_Z = 7,
    PYRONN_TUNE_ADJ_LANES = 8,
    PYRONN_TUNE_FP_PACKED = 9
} pyronn_tuning_param;
PYRONN_API int pyronn_geom_set_tuning(pyronn_geom_t g, int param, int value);

/* Autotuner (the batched pattern's tile and brick shapes chosen by measurement; the paper has no
 * dedicated passage): times every candidate configuration of one operator of g that runs on the kernel
 * it tunes, with CUDA events on `stream` after one warm-up launch each, and applies the fastest through
 * pyronn_geom_set_tuning (the choice stays with g). op 0: forward projection, in = volume, out =
 * sinogram; candidates (slab depth, buffers) of the TMA-staged projector. op 1: matched adjoint,
 * in = sinogram, out = volume; candidates (slab depth, pitch mode) of the slab-ordered adjoint. op 2:
 * voxel-driven back-projection (plain weights), in = sinogram, out = volume; candidates (brick depth,
 * variant): depths 4, 8, 16 of the L1-path bricks (variant 2) and the staged bricks (variant 3; 3D). Buffers hold one batch item of dtype (device memory, 16-byte aligned); out is
 * overwritten, in is only read; nothing is allocated beyond what the operators allocate on first use.
 * repeats: timed launches per candidate (1 .. 1000). result[4]: mean milliseconds per launch of the
 * chosen candidate, its two parameters and the number of candidates timed.
 * Synchronises the stream. PYRONN_INVALID_ARG if no candidate applies (the knobs are then left as
 * they were). */
PYRONN_API int pyronn_autotune(pyronn_geom_t g, int op, const void *in, void *out, int dtype, int repeats,
                               void *stream, double *result);

/* ------------------------------------------------------------------------------------------
 * Diagnostics.
 * ---------------------------------------------------------------------------------------- */

/* Read (and optionally reset) the geometry's device diagnostic counters, 8 ints: [0] samples of
 * the slab-staged projector that fell outside their staged box and were read from global memory
 * instead, [1] rays sampled outside the slab march (nearly parallel to the slabs), [2] slabs whose
 * box exceeded shared memory, [3] tensor copies that did not complete within the bounded wait (the
 * launch then stops early and its output is invalid); all zero is the expected state of [0..3].
 * [4], [5]: (tile, slab) boxes of the slab-ordered adjoint accumulated in int32 fixed point and in
 * FP32 (information, not errors). Synchronous (device-wide copy). */
PYRONN_API int pyronn_geom_read_flags(pyronn_geom_t g, int *out, int reset);

/* Forward-projector configuration that would be used for element type dtype (host computation,
 * no GPU needed), 20 ints: [0] kernel (1 direct, 2 slab thread-staged, 3 slab TMA-staged, 4 texture
 * gather, 5 hardware-filtered texture),
 * [1] slab depth, [2] guard planes, [3] first slab plane, [4..12] TMA box (x, y, z) for march
 * axes x, y, z, [13] elements per TMA buffer, [14] dynamic shared memory bytes per CTA,
 * [15] thread-staged box capacity (elements), [16] 1 if x-march boxes are staged from the y-fastest
 * copy of the volume (their innermost TMA axis is then y), [17..19] zero. */
PYRONN_API int pyronn_geom_fp_config(pyronn_geom_t g, int dtype, int *out);

/* Matched-adjoint configuration (host computation, no GPU needed), 8 ints: [0] kernel (1 atomic
 * scatter, 2 bricks, 3 slab-ordered), [1] slab depth, [2] guard planes, [3] shared-memory box
 * capacity in floats, [4] 1 if x-march boxes have an odd row pitch, [5] slab-table capacity,
 * [6] 1 if y- and z-march boxes get a 32-word row pitch where it fits, [7] zero. */
PYRONN_API int pyronn_geom_adjoint_config(pyronn_geom_t g, int *out);

/* Voxel-driven back-projector configuration for element type dtype (host computation, no GPU needed),
 * 8 ints: [0] kernel (1 one thread per voxel, 2 bricks through L1, 3 bricks with staged detector shadows),
 * [1], [2] the staged box per view in pixels (u, v; kernel 3), [3] voxels per thread along z, [4] views
 * per shared-memory stage (kernel 3), [5] elements between the views' boxes in shared memory (kernel 3;
 * a multiple of 128 bytes), [6..7] zero. */
PYRONN_API int pyronn_geom_bp_config(pyronn_geom_t g, int dtype, int *out);

/* Message describing the last error of the calling thread ("" if none). */
PYRONN_API const char *pyronn_last_error(void);

/* Library version, e.g. 100 for 0.1.0. */
PYRONN_API int pyronn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PYRONN_H */
