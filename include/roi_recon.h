/*
 * roi_recon.h -- C ABI of the GB300 local region-of-interest reconstruction library.
 *
 * Method: Pelt & Batenburg, "A method for locally approximating regularized
 * iterative tomographic reconstruction methods" (arXiv 1604.02292).
 *
 * The library reconstructs a square local part L (an "extended ROI box") of an
 * N x N image from a 2D parallel-beam sinogram.  It follows the
 * exterior-subtraction scheme the paper describes in Sec. 1: a global Ram-Lak
 * FBP (Eq. fbp), reprojection of that image outside L and subtraction from the
 * data (W = W_L + W_F, Eq. locouter), then a regularized iterative solve on L
 * only -- nonnegative SIRT (Eq. sirtit, Eq. sirtbox) or total variation
 * (Eq. priorsys with g = ||grad x||_1) by Chambolle-Pock.
 *
 * Conventions (every entry point):
 *   - Geometry (Sec. 2.1): pixel (i, j) = (row from the top, column) has centre
 *     (j - (N-1)/2, (N-1)/2 - i); bin d has centre t_d = d - (n_det-1)/2; a ray is
 *     x cos(theta) + y sin(theta) = t.  Sinograms are row-major [n_angles][n_det],
 *     images row-major [rows][columns], float32 unless stated.
 *   - Projector: Joseph's method, one ray per bin centre, sampled per row when
 *     |cos| >= |sin| (per column otherwise) with linear interpolation; the
 *     backprojector is its exact transpose.
 *   - Regions are given in pixel-index units: centre (cx = column, cy = row),
 *     radius r and margin m.  The extended box is the 2R x 2R pixels,
 *     R = ceil(r + m), whose centre indices are nearest to [c - R, c + R),
 *     clipped to the grid (Sec. 3.3 pads the local part and crops afterwards).
 *   - Streams: all device work of a handle is ordered on the CUDA stream given
 *     to roi_recon_create and is asynchronous with respect to the host, unless
 *     an entry point says it synchronizes.  Device pointers passed in must stay
 *     valid until that work completes.
 *   - Ownership: the handle owns its device copy of the sinogram, the cached
 *     FBP image and all scratch.  The caller owns every buffer it passes.
 *   - Errors: every entry point returns a roi_status and never throws or aborts.
 *     ROI_EINVAL for bad arguments, ROI_ESTATE for calls out of order,
 *     ROI_ENOMEM when a device allocation fails, ROI_ECUDA for other CUDA errors,
 *     ROI_ETIMEOUT when a bounded device-side wait gives up.  A message is kept
 *     per handle (roi_recon_last_error).
 *   - Threads: a handle may be used by one host thread at a time.
 */
#ifndef ROI_RECON_H
#define ROI_RECON_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct roi_recon* roi_recon_t;
typedef struct roi_batch_plan* roi_batch_plan_t;

typedef enum {
    ROI_OK = 0,
    ROI_EINVAL = 1,
    ROI_ENOMEM = 2,
    ROI_ESTATE = 3,
    ROI_ECUDA = 4,
    ROI_ETIMEOUT = 5,
    ROI_EBUSY = 6,
    ROI_ECANCELED = 7
} roi_status;

typedef enum { ROI_F32 = 0, ROI_BF16 = 1, ROI_F16 = 2 } roi_dtype;

typedef enum {
    ROI_SIRT_NONNEG = 0,   /* exterior subtraction, then nonnegative SIRT on the box (Sec. 1 scheme) */
    ROI_TV_CP = 1,         /* exterior subtraction, then TV by Chambolle-Pock on the box             */
    ROI_FILTER_SIRT = 2,   /* the paper's own method (Sec. 3): SIRT approximated by FBP with the
                              filters of Alg. filtcalc, the constraint x >= 0 applied on the box
                              by Alg. method; needs roi_recon_filter_prepare                     */
    ROI_FILTER_TV = 3,     /* the paper's method with FISTA for ||p - Wx||^2 + lambda TV(x), the
                              TV prox by inner_iters FGP iterations (Alg. methodfista); needs
                              roi_recon_filter_prepare                                           */
    ROI_FILTER_ISTA = 4    /* the paper's method with the ISTA prior of Eq. sirtista: soft
                              thresholding (at alpha lambda / 2) of the orthonormal 2D Haar
                              coefficients of the box, all levels; needs filter_prepare          */
} roi_regularizer;

/* Acquisition geometry (Sec. 2.1: N x N grid, N_d detectors, N_theta angles). */
typedef struct {
    int n_pix;             /* N >= 1                                                   */
    int n_angles;          /* N_theta >= 1                                             */
    int n_det;             /* N_d >= 1                                                 */
    const double* angles;  /* host array of n_angles radians, copied; NULL: a*pi/N_theta */
    roi_dtype storage;     /* storage of the resident sinogram: ROI_F32, ROI_BF16 or ROI_F16 */
    roi_dtype image_storage; /* storage of the cached FBP image and of the projector images
                              of batched / served solves: ROI_F32, ROI_BF16 or ROI_F16.
                              Arithmetic is float throughout.  A 16-bit sinogram with a
                              float32 image (image_storage = ROI_F32, the zero value) keeps
                              every image at full precision: the solve then differs from
                              the float32 path fed the same rounded data by float rounding
                              only.  A 16-bit image adds its own rounding to each solve.  */
} roi_geometry;

/* Region of interest in pixel-index units (see Conventions). */
typedef struct {
    double cx, cy;   /* centre: column, row            */
    double radius;   /* r > 0                           */
    double margin;   /* m >= 0, padding around the disk */
} roi_region;

typedef struct {
    roi_regularizer reg;   /* ROI_SIRT_NONNEG or ROI_TV_CP                                  */
    double lambda;         /* TV weight (CP); the data term is ||p' - W_L x||^2, no 1/2     */
    int iters;             /* iterations >= 0 (200 SIRT / 500 CP in the reference workloads) */
    int weighting;         /* SIRT: 0 = scalar alpha = 1/(N_theta N_d) (Sec. 3.1),
                              1 = row/column-sum weights x += C W_L^T R (p' - W_L x)          */
    int precond;           /* CP: 1 = diagonal steps (Pock & Chambolle 2011), 0 = 0.99/||K||  */
    int crop_disk;         /* 1: set output pixels outside the disk of radius r to 0          */
    int eval_objective;    /* 1: fill info->objective (the call then synchronizes)            */
    int inner_iters;       /* ROI_FILTER_TV: FGP iterations per outer iteration (0: 100)     */
} roi_solve_params;

/* Plan and result description of one local solve. */
typedef struct {
    int box_x0, box_y0, box_w, box_h;  /* extended box: columns [x0, x0+w), rows [y0, y0+h) */
    int window_max;                    /* max over angles of the number of bins reaching the box */
    int window_stride;                 /* row stride of window buffers (multiple of 4, >= max) */
    int iters_done;
    double step_L;                     /* CP with precond = 0: the ||K|| used; 0 otherwise      */
    double objective;                  /* eval_objective: ||W_L x - p'||^2 + lambda TV(x)        */
} roi_solve_info;

/* --------------------------------------------------------------------------
 * Handle life cycle and data
 * ------------------------------------------------------------------------ */

/* Create a handle for geometry *geom, ordering all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream) of the current device.
 * Allocates the sinogram, filter and FBP buffers (s N_theta N_d + 4 N_theta N_d + 2 i N^2
 * bytes, s and i = 4 for ROI_F32, 2 for ROI_BF16 / ROI_F16, of storage and image_storage;
 * a 16-bit image adds a float N^2 scratch at the first fbp).  With 16-bit storage every
 * stored value is rounded to nearest even; the ramp filter, projections and solves still
 * compute in float.  ROI_EINVAL for non-positive sizes or an unknown storage type,
 * ROI_ENOMEM if the device allocation fails.  *out is NULL on failure. */
roi_status roi_recon_create(const roi_geometry* geom, void* cuda_stream, roi_recon_t* out);

/* Release every resource of the handle (waits for its stream first).  NULL is ignored. */
void roi_recon_destroy(roi_recon_t h);

/* Message of the last failed call on this handle ("" if none).  Valid until the next call. */
const char* roi_recon_last_error(roi_recon_t h);

/* Copy the measured sinogram p (Sec. 2.1), [n_angles][n_det] of type dt (ROI_F32,
 * ROI_BF16 or ROI_F16), into the handle, converting it to the handle's storage type
 * (round to nearest even) on the device when the two differ.
 * on_device = 1: p is a device pointer (device-to-device copy, asynchronous);
 * on_device = 0: p is host memory, copied with cudaMemcpyAsync semantics: pageable
 * memory is consumed before the call returns, page-locked memory must stay unchanged
 * until the handle's stream has passed the copy.  Invalidates the cached FBP image. */
roi_status roi_recon_set_sinogram(roi_recon_t h, const void* p, roi_dtype dt, int on_device);

/* Truncated projection data (Sec. 5.6): p [n_angles][n_measured] holds only the central
 * n_measured bins of the handle's n_det-bin detector (bins [(n_det - n_measured)/2,
 * (n_det + n_measured)/2)); the bins outside are filled by constant padding with each
 * row's first / last measured value, as FBP-based methods do to reduce truncation
 * artifacts.  Everything downstream (fbp, exterior step, solves, filter_prepare) then
 * runs on the padded sinogram; results are meaningful inside the disk of diameter
 * n_measured around the rotation axis.  Other arguments as for roi_recon_set_sinogram.
 * ROI_EINVAL unless 1 <= n_measured <= n_det with n_det - n_measured even. */
roi_status roi_recon_set_sinogram_truncated(roi_recon_t h, const void* p, roi_dtype dt, int on_device,
                                           int n_measured);

/* Global filtered backprojection FBP(p, h) = W^T C_h p (Eq. fbp), Ram-Lak filter
 * scaled by pi/N_theta, on the whole N x N grid; the result is cached in the handle (in
 * its image storage type) for the exterior step, restricted to the field of view: pixels
 * whose centre lies farther than min(N, N_d)/2 from the rotation axis are set to 0 (the
 * detector misses them at some angles, so their FBP value is not determined by the data
 * and would make the reprojected exterior inconsistent).  out_or_null: optional device
 * [N][N] float32 copy of the cached image.  ROI_ESTATE before set_sinogram. */
roi_status roi_recon_fbp(roi_recon_t h, float* out_or_null);

/* Exterior subtraction (Sec. 1; Eq. locouter): p' = p - W M_F x_fbp on every ray that
 * reaches the extended box of *region (x_fbp: the cached image, inside its field of view).  window_out_or_null: optional device buffer
 * [n_angles][window_stride] float32 receiving p'; entry [a][k] belongs to bin
 * d0[a] + k, entries past the angle's width are 0.  d0_out_or_null: optional host
 * int[n_angles] receiving d0 (the call then synchronizes).  Sizes come from
 * roi_recon_plan.  ROI_ESTATE before fbp. */
roi_status roi_recon_reproject_exterior(roi_recon_t h, const roi_region* region,
                                        float* window_out_or_null, int* d0_out_or_null);

/* Local solve on the extended box of *region (Sec. 1 scheme; Eq. sirtit + Eq. sirtbox
 * with l = 0, or Eq. priorsys with TV by Chambolle-Pock), starting from x = 0.
 * Runs the exterior subtraction first.  out: [box_h][box_w] float32, a device
 * pointer when out_on_device = 1, host memory otherwise (the call then
 * synchronizes).  info (optional) receives the plan; its objective only when
 * params->eval_objective.  ROI_ESTATE before fbp, ROI_EINVAL for bad params or a
 * region whose box misses the grid. */
roi_status roi_recon_solve_local(roi_recon_t h, const roi_region* region, const roi_solve_params* params,
                                 float* out, int out_on_device, roi_solve_info* info);

/* Checkpoint / resume of roi_recon_solve_local (ROI_SIRT_NONNEG and ROI_TV_CP).  After a
 * solve_local without eval_objective the handle holds the iterate state of that solve:
 * SIRT x; CP x, xbar, the gradient dual (vx, vy) and the data dual on the window.
 * roi_recon_state_size gives its size in bytes: a 64-byte header (regularizer, weighting /
 * precond flag, lambda, box, window layout, iterations done) followed by those arrays,
 * float32, box-major [box_h][box_w] images and the window [n_angles][window_stride].
 * roi_recon_state_export copies it to dst (bytes >= the size; device memory when
 * on_device = 1, host memory otherwise); the call synchronizes.
 * A large box solved by the whole-region solver (see ROI_OPT_SINGLE_LAUNCH) leaves no
 * state: set ROI_OPT_SINGLE_LAUNCH = 0 for solves that are to be checkpointed.
 * roi_recon_solve_local_resume runs params->iters further iterations from such a state
 * (device or host memory) instead of from x = 0; everything else is as for solve_local,
 * and info->iters_done counts the state's iterations too.  The region must give the
 * state's box and window layout, and params->reg, weighting / precond and lambda must be
 * those of the solve that made it.  With the same sinogram and FBP, the result is
 * bit-identical to one uninterrupted solve of all the iterations (both run the same
 * operations in the same order).  ROI_ESTATE when the handle holds no state (no solve yet,
 * or forward_local, back_local, filter_prepare or another solve_local has used the solver
 * buffers since), ROI_EINVAL for a state that does not match the call. */
roi_status roi_recon_state_size(roi_recon_t h, size_t* bytes);
roi_status roi_recon_state_export(roi_recon_t h, void* dst, size_t bytes, int on_device);
roi_status roi_recon_solve_local_resume(roi_recon_t h, const roi_region* region, const roi_solve_params* params,
                                        const void* state, size_t bytes, int state_on_device, float* out,
                                        int out_on_device, roi_solve_info* info);

/* Many local solves in one call (Sec. 5.5: local reconstructions are independent and can
 * be computed in parallel; Sec. 1 scheme for each).  regions[n], params[n] (one per region;
 * SIRT and CP may be mixed; CP must use precond = 1; eval_objective is ignored), outs[n]:
 * [box_h][box_w] float32 each, device pointers when out_on_device = 1, host memory
 * otherwise (the call then synchronizes).  infos (optional) [n] receive each plan.
 * One persistent launch solves everything: its blocks each take whole regions, largest
 * first, exterior step included -- p' = (p - W x_fbp) + W_L x_fbp on the box, which is
 * p - W_F x_fbp by Eq. locouter, with the residual p - W x_fbp of every ray computed once
 * per FBP.  A region's result is bit-identical whatever else is in the batch and equals
 * the serving path's (roi_server_*); it agrees with roi_recon_solve_local to rounding (a
 * different split of the same sums).  Device memory: the residual (4 N_theta N_d bytes,
 * kept with the FBP image), the angle tables (about 90 N_theta bytes per region), and
 * scratch per SM for the largest region.  ROI_ESTATE before fbp, ROI_EINVAL naming the
 * offending region. */
roi_status roi_recon_solve_batch(roi_recon_t h, int n, const roi_region* regions, const roi_solve_params* params,
                                 float* const* outs, int out_on_device, roi_solve_info* infos);

/* A batch planned once and launched as one captured CUDA graph (Sec. 5.5; many local solves
 * in one persistent launch): create plans the batch exactly as roi_recon_solve_batch does
 * (same arguments; outs must be device pointers; SIRT and CP-TV regions only, ROI_EINVAL
 * otherwise), uploads the angle tables and region descriptors into device buffers of the
 * plan's own, and captures the launch -- the reset of the launch's queue or team barriers
 * and the persistent kernel -- into an instantiated CUDA graph (it synchronizes; options
 * such as the tile table, team table and wait limit are read then).  launch replays the
 * graph on the handle's stream after recomputing the residual p - W x_fbp if the sinogram
 * or FBP changed: a new sinogram of the same geometry (set_sinogram + fbp) is solved on the
 * same regions without host planning, and each result is bit-identical to solve_batch's on
 * that sinogram.  The outs and the handle must outlive the plan; destroy (or
 * roi_recon_destroy) waits for the handle's stream and frees the plan.  ROI_ESTATE for
 * launch before fbp; ROI_EINVAL for a plan of another handle. */
roi_status roi_recon_batch_plan_create(roi_recon_t h, int n, const roi_region* regions,
                                       const roi_solve_params* params, float* const* outs, roi_solve_info* infos,
                                       roi_batch_plan_t* out);
roi_status roi_recon_batch_plan_launch(roi_recon_t h, roi_batch_plan_t plan);
roi_status roi_recon_batch_plan_destroy(roi_recon_t h, roi_batch_plan_t plan);

/* Tiling (Sec. 5.5): the whole N x N image as non-overlapping tile x tile local
 * reconstructions placed next to each other.  Tile (ti, tj) covers rows [ti tile, (ti+1)
 * tile) and columns [tj tile, (tj+1) tile); it is solved as the region centred on the tile
 * with radius tile/2 and the given margin (its extended box, clipped to the grid), all
 * tiles in one roi_recon_solve_batch call, and the tile's square is copied from the box
 * result into out (device [N][N] float32).  params as for roi_recon_solve_batch, with
 * crop_disk = 0.  Synchronizes.  ROI_EINVAL unless tile is even and divides N. */
roi_status roi_recon_solve_tiled(roi_recon_t h, int tile, int margin, const roi_solve_params* params, float* out);

/* --------------------------------------------------------------------------
 * The paper's own local method (Sec. 3)
 * ------------------------------------------------------------------------ */

/* Prepares ROI_FILTER_SIRT solves of up to n_iters iterations on the resident sinogram:
 *  1. Alg. filtcalc on the whole N x N grid: with A = I - alpha W^T W (alpha =
 *     1/(N_theta N_d)) and c the unit impulse on the rotation axis (shared by the four
 *     central pixels when N is even), q_k = sum_{j<k} A^j c and the filters
 *     u_k = alpha W q_k, k = 1..n_iters, read at the integer detector offsets
 *     -(N_d-1)..N_d-1 from a detector with the acquisition's bin phase (even N_d: the
 *     mean of the bins at m -/+ 1/2).  Kept per handle (geometry-only) until a larger
 *     n_iters is asked for; n_iters pairs of full-grid projections.
 *  2. Disc subtraction (Sec. 3.3): p_d = p - g W D, D the disc of diameter N on the axis,
 *     g minimising the squared norm of the per-angle sums of p_d.
 *  3. The filtered sinograms C_{u_k} p_d for every k (4 n_iters N_theta N_d bytes), reused
 *     by every region of this sinogram; computed as in roi_recon_filter_conv (the filters
 *     packed for the tensor cores once per filter set: 32 n' N_theta 8 ceil((2 N_d - 1)/8)
 *     bytes, n' = n_iters rounded up to 16).  ROI_ETIMEOUT if a device wait gave up.
 * ROI_ESTATE before set_sinogram, ROI_EINVAL for n_iters < 1 or > 100000. */
roi_status roi_recon_filter_prepare(roi_recon_t h, int n_iters);

/* The filtered sinograms of Sec. 3.1 (Eq. sirtapp: iteration k of Alg. method filters the
 * sinogram with u_k) as one operator on caller data:
 *     out[k][a][d] = sum_{e < n_det} u[k][a][d - e + n_det - 1] p[a][e],  k < n,
 * u device [n][n_angles][2 n_det - 1], p device [n_angles][n_det], out device
 * [n][n_angles][n_det], float32, caller-owned (out must not overlap u or p).  Path as
 * ROI_OPT_FILTER_CONV says; the tensor-core path packs u into handle scratch first (see
 * filter_prepare for its size).  Synchronizes.  ROI_EINVAL for n < 1 or a NULL pointer,
 * ROI_ETIMEOUT if a device wait gave up. */
roi_status roi_recon_filter_conv(roi_recon_t h, int n, const float* u, const float* p, float* out);

/* After filter_prepare: the filters into device u_out [k][n_angles][2 n_det - 1] float32
 * (the first k = min(n_filters, prepared) of them; NULL to skip) and the disc grey value
 * into *disc_grey (host, optional).  ROI_ESTATE before filter_prepare. */
roi_status roi_recon_filter_get(roi_recon_t h, int n_filters, float* u_out, double* disc_grey);

/* --------------------------------------------------------------------------
 * Planning and single operators (for custom solvers and for verification)
 * ------------------------------------------------------------------------ */

/* Host-only ROI plan (no GPU needed): box and per-angle detector windows of the
 * rays that reach the box (rows of W_L that are not zero, Sec. 2.1).  info receives
 * box_* , window_max and window_stride; d0 and width (optional host int[n_angles])
 * receive each angle's first bin and bin count. */
roi_status roi_recon_plan(const roi_geometry* geom, const roi_region* region, roi_solve_info* info,
                          int* d0, int* width);

/* y = W_L x (Sec. 2.1): x device [box_h][box_w], y device [n_angles][window_stride]
 * (window layout as in roi_recon_reproject_exterior).  Needs only create. */
roi_status roi_recon_forward_local(roi_recon_t h, const roi_region* region, const float* x, float* y);

/* x = W_L^T y = M_L W^T y restricted to the box (Sec. 2.1), the exact transpose of
 * roi_recon_forward_local: y device window [n_angles][window_stride], x device
 * [box_h][box_w].  Needs only create. */
roi_status roi_recon_back_local(roi_recon_t h, const roi_region* region, const float* y, float* x);

/* q = C_h p: the resident sinogram filtered by the Ram-Lak filter scaled by pi/N_theta
 * (linear convolution, Eq. fbp), into device q [n_angles][n_det].  ROI_ESTATE before
 * set_sinogram. */
roi_status roi_recon_ramp_filter(roi_recon_t h, float* q);


/* --------------------------------------------------------------------------
 * Options and device-side status
 * ------------------------------------------------------------------------ */

typedef enum {
    /* 1 (default): run each SIRT / CP-TV solve_local as one cooperative launch.  When the
     * box's padded image fits in a block's shared memory (sides up to about 216 px): the
     * single-launch solver (all iterations in one kernel, grid barriers between phases).
     * Larger boxes: the whole-region solver of roi_recon_solve_batch, one team of every
     * co-resident block, exterior step p' = (p - W x_fbp) + W_L x_fbp (bit-identical to
     * solve_batch's result for the region; such a solve keeps no resumable state, and
     * eval_objective, CP with precond = 0 and resumed solves take the per-operator path).
     * 0: one launch per operator per iteration for every box. */
    ROI_OPT_SINGLE_LAUNCH = 0,
    /* time limit of one grid-barrier wait in a single-launch solve, microseconds
     * (default 1,000,000); a wait that runs out aborts the solve (see roi_recon_sync). */
    ROI_OPT_WAIT_LIMIT_US = 1,
    /* testing only: number of participants every grid or team barrier waits for beyond the
     * blocks launched (default 0).  Any value > 0 makes every cooperative solve time out:
     * single-launch solves, batched solves run by teams (few regions), large boxes of
     * solve_local, and (roi_server_set_option) requests solved by a team of a server.  For
     * a server, -1 keeps the team leaders away instead, so that the members' waits for
     * the leader's claim (the team mailbox) run out.  On a handle, > 0 also makes the
     * tensor-core filtered sinograms (filter_prepare, roi_recon_filter_conv) wait for
     * filter-bank bytes that never arrive: the call returns ROI_ETIMEOUT. */
    ROI_OPT_TEST_ABSENT_BLOCKS = 2,
    /* -1 (default): the phase B tile shape of each whole-region solve (solve_batch, large
     * boxes of solve_local, and requests served from this handle's sinogram) is taken from
     * the handle's tile table by box size (roi_recon_autotune); 0, 1, 2: that shape for
     * every region.  Shapes: 0 = 16 x 16 pixels per warp (runs of 8 pixels per lane),
     * 1 = 8 x 8 (runs of 2), 2 = 16 x 8 (runs of 4).  The shape changes how a pixel's
     * angles are grouped into partial sums, so results of different shapes agree to
     * rounding, not bit for bit; with one shape they are bit-identical wherever solved. */
    ROI_OPT_TILE_SHAPE = 3,
    /* path of the filtered sinograms (filter_prepare step 3, roi_recon_filter_conv):
     * 0 (default) the tensor cores (tcgen05 kind::tf32, each operand split into a tf32 head
     * and remainder, three products accumulated in fp32 in tensor memory) whenever a
     * detector row's expansion fits in shared memory (n_det up to about 2500 with 200
     * filters), else the FMA pipe; 1: the FMA pipe (fp32 direct sums).  The two agree to
     * float rounding. */
    ROI_OPT_FILTER_CONV = 4
} roi_option;

roi_status roi_recon_set_option(roi_recon_t h, roi_option opt, long long value);

/* Autotuner of the batching tier's tile shapes (Sec. 5.5: many independent local solves).
 * For each box-size class -- sides 48..96, 97..216 (image staged whole), 217..384 (image
 * streamed in bands), clipped to the grid -- it solves one batch of regions_per_class
 * seeded regions of that class (0: two per SM; SIRT and CP-TV alternating, iters
 * iterations, 0: 20) on this handle's sinogram with each tile shape (a warm-up, then the
 * best of two timed runs, CUDA events on the handle's stream), and keeps the fastest shape
 * per class in the handle's tile table; then, per class, the team size of few-region
 * batches (roi_recon_get_team_caps).  Both tables are also kept per geometry (grid,
 * angles, detector, image storage) for handles created later in the process.
 * shapes_out (optional, int[3]): the chosen shape per class; ms_out (optional,
 * double[3][3]): milliseconds per class and shape (0 for a class the grid cannot hold).
 * Synchronizes.  ROI_ESTATE before fbp. */
roi_status roi_recon_autotune(roi_recon_t h, int regions_per_class, int iters, int* shapes_out, double* ms_out);

/* The handle's tile table (int[3], one shape per box-size class, see ROI_OPT_TILE_SHAPE):
 * set it (ROI_EINVAL for an unknown shape) or read it.  A server reads the table of each
 * sinogram's handle when the sinogram is added. */
roi_status roi_recon_set_tile_shapes(roi_recon_t h, const int* shapes);
roi_status roi_recon_get_tile_shapes(roi_recon_t h, int* shapes);

/* The handle's team table (int[3], per box-size class as above): a batch of fewer regions
 * than half the blocks solves each region on a team of up to caps[c] blocks, c the class of
 * the batch's largest box (default 16; also bounded by the blocks per region).  A region's
 * result is the same bits for every team size.  roi_recon_autotune also times, per class,
 * a batch of 8 of its regions with caps 4, 8, 16 and 32 (with the class's chosen tile shape)
 * and keeps the fastest; it is cached with the tile table.  set: ROI_EINVAL for a cap
 * outside [1, 1024].  get: ms_out (optional, double[3][4]) receives the autotuner's
 * milliseconds per class and candidate (0 before it ran or for a class the grid cannot
 * hold). */
roi_status roi_recon_set_team_caps(roi_recon_t h, const int* caps);
roi_status roi_recon_get_team_caps(roi_recon_t h, int* caps, double* ms_out);

/* Wait for all work on the handle's stream, then report device-side failures: ROI_ETIMEOUT
 * if a single-launch solve gave up at a grid barrier since the last report (its output is
 * invalid; the context stays usable), ROI_ECUDA for a CUDA error.  solve_local calls this
 * itself whenever it synchronizes (host output). */
roi_status roi_recon_sync(roi_recon_t h);

/* Check build only (the library compiled with -DROI_CHECK; the Python binding loads that
 * variant when ROI_RECON_CHECK=1): the number of out-of-range indices the hot kernels'
 * checks have found since the last call -- image columns of ray samples and staged bins of
 * gathered pixels, each replaced by an in-range index when found -- with the first one's
 * site (1-2 single-launch solver, 3-5 whole-region solver, 6-7 one-launch-per-operator
 * projectors, 8 tensor-core filtered sinograms) and value in *site / *index (either may be NULL); the reports are cleared.
 * Waits for the device.  The product build has no checks and returns 0. */
int roi_recon_check_report(int* site, int* index);

/* --------------------------------------------------------------------------
 * Measurement
 * ------------------------------------------------------------------------ */

/* Kernel timing for profiling.  enable = 1 starts recording CUDA events around every
 * launch of the projector kernels and of the single-launch solver made by
 * roi_recon_solve_local, of the batched solver, and of the filtered-sinogram kernel (and
 * clears earlier records); enable = 0 stops.  Recording adds host work per launch, so
 * time whole steps with it off. */
roi_status roi_recon_set_timing(roi_recon_t h, int enable);

/* Launch count and summed device time (milliseconds, from the recorded events) of
 * kernel class `kernel` since timing was enabled: 0 = forward projector W_L
 * (ray-driven, fused dual/residual update), 1 = backprojector W_L^T (pixel gather,
 * fused primal update), 2 = single-launch solve (all iterations of one solve) or batched
 * solve (one launch), 3 = filtered sinograms (filter_prepare step 3, roi_recon_filter_conv;
 * the packing of the filter bank excluded).
 * Synchronizes the handle's stream. */
roi_status roi_recon_kernel_times(roi_recon_t h, int kernel, int* launches, double* total_ms);

/* Number of CUDA kernels this library has launched in this process (all handles). */
unsigned long long roi_recon_launch_count(void);

/* Testing only (process-wide, no GPU needed): the nth device or page-locked host allocation
 * the library makes from now on fails as if memory had run out, without allocating (the
 * call making it returns ROI_ENOMEM and leaves its handle or server usable); the later ones
 * succeed again.  nth = 0 turns it off.  ROI_EINVAL for nth < 0. */
roi_status roi_recon_test_fail_alloc(int nth);

/* --------------------------------------------------------------------------
 * Serving: continuous batching of ROI requests over resident sinograms
 * ------------------------------------------------------------------------ */

/* A server solves ROI requests (each the Sec. 1 scheme on one region of one resident
 * sinogram, Sec. 5.5: regions are independent) while more keep arriving.  One
 * cooperative kernel runs while there is work: its blocks form units -- single blocks
 * for small boxes, teams of team_blocks blocks for boxes of side >= large_side (and for
 * small ones while a team is idle, unless no_spill) -- that
 * take requests from rings in page-locked host memory mapped into the device, so a
 * request submitted while others are on the GPU starts as soon as a unit is free,
 * without a launch.  The host side (a progress engine, run by a background thread after
 * roi_server_start or by explicit roi_server_progress calls) admits requests in arrival
 * order while their state fits the device budget and their results fit the page-locked
 * result area, publishes them, polls completion words and recycles memory; the kernel
 * leaves after idle_us without work and is relaunched when work arrives.
 * A request's result is bit-identical whichever unit solves it and whatever runs beside
 * it, and equals roi_recon_solve_batch's for the same region (same exterior form).
 * Threads: submit / poll / take / stats may be called from any thread; the server
 * serialises them internally. */
typedef struct roi_server* roi_server_t;

typedef struct {
    size_t device_bytes;   /* HBM budget for the state of admitted requests (0: 4 GiB) */
    size_t host_bytes;     /* page-locked result area (0: 512 MiB) */
    int ring_slots;        /* request slots per unit pool (0: 1024) */
    int team_blocks;       /* blocks per team of the large-box pool (0: 16) */
    int teams;             /* teams (-1: every block but 24 in teams; 0: no team pool) */
    int large_side;        /* box side from which a request goes to the team pool (0: 256) */
    int idle_us;           /* the kernel leaves after this long without work (0: 2000) */
    int no_spill;          /* 0: a small-box request is admitted to an idle team when no
                              large one waits for it, and requests arriving at an idle server
                              run one at a time on one team of all blocks (a solo launch)
                              until a queue forms (lower latency at light load); 1: requests
                              go to their pool by size */
    int solo_queue_ms;     /* a solo launch leaves (and the pools take over) when the work
                              queued behind it exceeds this many milliseconds of estimated
                              whole-GPU solve time (0: 250) */
} roi_server_config;

typedef struct {
    long long id;          /* as returned by roi_server_submit */
    roi_status status;     /* ROI_OK; ROI_ETIMEOUT when a device wait gave up; ROI_ECANCELED
                              after roi_server_cancel */
    int sino;
    int box_x0, box_y0, box_w, box_h;
    int pool;              /* 0: one block, 1: a team */
    double t_submit_ms;    /* host monotonic clock (CLOCK_MONOTONIC), milliseconds */
    double t_publish_ms;   /* admitted and published to the device */
    double t_done_ms;      /* completion seen by the host */
} roi_server_completion;

typedef struct {
    long long submitted, completed, failed, pending, in_flight;
    long long kernel_launches;
    size_t device_in_use, device_peak, host_in_use, host_peak;
    int blocks, single_units, teams, team_blocks;
    long long cancelled;   /* requests removed from the queue by roi_server_cancel */
} roi_server_stats;

/* Creates a server on the current device (it owns a non-blocking stream).  cfg may be
 * NULL (defaults).  ROI_EINVAL for bad sizes, ROI_ENOMEM when the budgets cannot be
 * allocated.  Besides the two budgets, the first submit allocates the rings, a per-block
 * copy of a request's angle table, and up to 64 MB of per-band partial sums that solo
 * launches use for band-streamed boxes. */
roi_status roi_server_create(const roi_server_config* cfg, roi_server_t* out);

/* Registers the resident sinogram and FBP image of handle h (fbp done; ROI_ESTATE
 * otherwise) and computes its residual p - W x_fbp; *sino_id receives its index.  The
 * handle must outlive the server and its sinogram must not change while registered.
 * All sinograms must be added before the first submit. */
roi_status roi_server_add_sinogram(roi_server_t s, roi_recon_t h, int* sino_id);

/* Queues one request (params as for roi_recon_solve_batch: CP needs precond = 1).
 * Plans it on the host; *id receives its id.  ROI_EINVAL for a bad sinogram id,
 * region or params; ROI_ENOMEM when its state or result could never fit the budgets. */
roi_status roi_server_submit(roi_server_t s, int sino_id, const roi_region* region, const roi_solve_params* params,
                             long long* id);

/* Starts / stops the background progress thread. */
roi_status roi_server_start(roi_server_t s);
roi_status roi_server_stop(roi_server_t s);

/* One pass of the progress engine (admission, publication, completion, relaunch) for
 * callers that do not start the thread. */
roi_status roi_server_progress(roi_server_t s);

/* Moves up to max completion records into out; returns how many (0 if none, -1 on a
 * bad argument). */
int roi_server_poll(roi_server_t s, roi_server_completion* out, int max);

/* Copies the result of completed request id ([box_h][box_w] float32) into host memory
 * dst (may be NULL to discard) and releases it.  ROI_EBUSY if not complete yet,
 * ROI_EINVAL for an unknown id, the request's own status if it failed. */
roi_status roi_server_take(roi_server_t s, long long id, float* dst);

/* Removes request id from the queue if it is still waiting there (not yet admitted to the
 * device): it then completes at once with status ROI_ECANCELED (reported by poll; take
 * releases it and returns ROI_ECANCELED).  ROI_EBUSY if it is already on the device (it
 * runs to completion), ROI_EINVAL for an unknown or completed id. */
roi_status roi_server_cancel(roi_server_t s, long long id);

/* Server options, read at the next launch of the serving kernel: ROI_OPT_WAIT_LIMIT_US
 * (limit of the team barrier and mailbox waits, default 2 s) and ROI_OPT_TEST_ABSENT_BLOCKS
 * (testing only, see roi_option).  When a wait runs out the kernel leaves, the requests
 * it held complete with ROI_ETIMEOUT, and the server relaunches for the rest.  ROI_EINVAL
 * for ROI_OPT_SINGLE_LAUNCH or a value out of range. */
roi_status roi_server_set_option(roi_server_t s, roi_option opt, long long value);

/* Waits (running progress itself when the thread is not started) until every submitted
 * request has completed or timeout_ms has passed (ROI_EBUSY then). */
roi_status roi_server_drain(roi_server_t s, double timeout_ms);

roi_status roi_server_stats_get(roi_server_t s, roi_server_stats* out);
const char* roi_server_last_error(roi_server_t s);

/* Stops the thread, tells the kernel to leave once the requests it holds are done, waits
 * for it and frees everything; results not taken are dropped. */
void roi_server_destroy(roi_server_t s);

/* Host only (no GPU): the device-state and result bytes the server budgets for a request
 * on a sinogram of n_pix / n_angles / n_det whose handle has image storage type `storage`
 * (the projector images of a served solve are kept in it), and its box side. */
roi_status roi_server_footprint(int n_pix, int n_angles, int n_det, roi_dtype storage, const roi_region* region,
                                size_t* device_bytes, size_t* host_bytes, int* box_side);

/* --------------------------------------------------------------------------
 * Allocation-free variant
 * ------------------------------------------------------------------------ */

/* y = W_L x, the same operator as roi_recon_forward_local, without a handle and
 * without allocating device memory.  The paper has no counterpart: this entry point
 * serves callers that cannot allocate -- code whose device memory belongs to someone
 * else's fixed budget (a framework's caching allocator, a server that reserves HBM up
 * front) and loops that cannot take the implicit device synchronisation of
 * cudaMalloc / cudaFree.  It calls neither, nor anything that allocates.
 *   geom:    as for roi_recon_create; angles must be NULL (a*pi/N_theta), storage and
 *            image_storage ROI_F32.
 *   x:       device [box_h][box_w] float32; y: device [n_angles][window_stride] float32,
 *            sizes from roi_recon_plan; work is ordered on cuda_stream (NULL = legacy
 *            default stream) of the current device.
 *   err:     optional buffer of err_len bytes receiving a message on failure.
 * Scratch: a fixed 16 MiB device array inside the library holds the per-angle ray
 * table and two zero-padded copies of the box image (by rows and by columns, each row
 * padded to its length + 4 rounded up to a multiple of 4 floats).  Calls needing more
 * (about 90 bytes per angle plus 8 box_w box_h bytes for large boxes) fail with
 * ROI_EINVAL and say so in err.  The ray table is the plan roi_recon_plan returns for
 * the same geometry and region (the same host function makes it), so y has exactly the
 * window layout the caller sized it for; it reaches the device as kernel parameters.
 * Every GPU that loads the library keeps this array until the process exits.  With lazy
 * module loading (the CUDA default) the first call on each device loads the module that
 * holds the array, which allocates that module's memory and may synchronise; later calls
 * do neither, so make the first call before any stream capture.  Each call looks up the
 * array's address (cudaGetSymbolAddress, no allocation) with the caller's device current.
 * All calls share the array and it keeps the last call's contents; each call rewrites
 * what it reads, but calls that overlap on the GPU (other streams or host threads) race
 * on it, so serialise them. */
roi_status roi_recon_forward_local_noalloc(const roi_geometry* geom, const roi_region* region,
                                           const float* x, float* y, void* cuda_stream,
                                           char* err, int err_len);

#ifdef __cplusplus
}
#endif
#endif /* ROI_RECON_H */
