/*
 * quadbox.h -- C ABI of libquadbox, a GB300 (sm_103a) tile rasteriser for
 * 3D Gaussian Splatting with QuadBox binning and QPass traversal.
 *
 * Method: "QuadBox: Accelerating 3D Gaussian Splatting with Geometry-Aware
 * Boxes" (arXiv 2605.04844).  Section/equation references below are to that
 * paper.  Conventions the paper leaves open (near plane, Jacobian clamp, the
 * 0.3 low-pass dilation, the 0.99 opacity cap, the 1/255 skip, the 1e-4
 * transmittance stop, pixel centres at integer coordinates) follow the 3DGS
 * code base the paper builds on (Sec. 4.1).
 *
 * General rules for every entry point:
 *  - Pointers named d_* or documented as "device" are CUDA device pointers
 *    owned by the caller; the library never frees them.  Structs passed by
 *    pointer (qb_scene, qb_camera, qb_frame, ...) live in host memory.
 *  - All work is stream-ordered on the given stream (a cudaStream_t; NULL is
 *    the legacy default stream).  Nothing synchronises the host unless the
 *    function says so.
 *  - Every function returns a qb_status.  On failure qb_last_error() returns
 *    a message for the calling thread.  No C++ exception crosses the ABI.
 *  - Device-side failures (pair capacity exceeded, a bounded spin-wait that
 *    ran out) are recorded in a flag word inside the workspace and reported
 *    by the next function that synchronises (qb_frame_check, or
 *    qb_bin_emit with a non-NULL n_pairs_out).  A kernel never writes past a
 *    buffer because of them.
 *  - Tiles are 16 x 16 pixels; tile id = ty * tiles_x + tx.
 */
#ifndef QUADBOX_H
#define QUADBOX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *qb_stream_t; /* identical to cudaStream_t */

typedef enum {
    QB_OK = 0,
    QB_ERR_INVALID_ARG = 1, /* bad pointer, size, mode or alignment        */
    QB_ERR_CUDA = 2,        /* a CUDA runtime call failed                  */
    QB_ERR_CAPACITY = 3,    /* more Gaussian-tile pairs than pair_capacity */
    QB_ERR_TIMEOUT = 4,     /* a device spin-wait hit its iteration limit  */
    QB_ERR_STATE = 5        /* stages called out of order                  */
} qb_status;

/* Binning rule (how a Gaussian is mapped to tiles).
 *  AABB3S        vanilla 3DGS square box of side 6 sqrt(lambda_max) (Sec. 2).
 *  QUADBOX       four quadrant sub-boxes: the two along the major axis use
 *                the AdR extents (Eq. extents-closed), the other two are
 *                scaled by f (Eq. f-closed); tiles enumerated by QPass
 *                (Sec. 3.1.2, Sec. 3.2).
 *  ADR           the single opacity-aware AABB of AdR-Gaussian (Sec. 3.1.1).
 *  QUADBOX_NAIVE QUADBOX boxes enumerated by nested loops over each sub-box
 *                with overlap checks (the paper's QuadBox-dagger, Table 3).
 *  DUALBOX       only the two major-axis quadrants (Sec. 3.1.2); not
 *                conservative, images differ by design.
 * Sub-boxes are intersected with the 3-sigma rectangle unless
 * QB_BIN_NO_CLAMP is OR-ed into the mode; with the clamp, QUADBOX, ADR and
 * AABB3S produce identical images. */
typedef enum {
    QB_BIN_AABB3S = 0,
    QB_BIN_QUADBOX = 1,
    QB_BIN_ADR = 2,
    QB_BIN_QUADBOX_NAIVE = 3,
    QB_BIN_DUALBOX = 4
} qb_bin_mode;
#define QB_BIN_NO_CLAMP 0x100

/* How qb_bin_emit/qb_sort order the pairs by (tile, depth, index).  Both give
 * identical sorted values and ranges.
 *  DEPTH_FIRST  (default) sort the n Gaussians by (depth, index) once, emit
 *               each Gaussian's pairs in that order with 32-bit tile keys, then
 *               stable-sort the pairs on the tile bits only (with emit_fused
 *               the emit runs the first digit pass itself).
 *  FULL_KEY     emit in index order with 64-bit keys (tile << 31) | depth
 *               bits and stable-sort on all 31 + tile bits (SortPairs, Sec. 2). */
typedef enum { QB_SORT_DEPTH_FIRST = 0, QB_SORT_FULL_KEY = 1 } qb_sort_mode;

/* Pinhole camera.  viewmat: row-major 4x4 world->view, last row (0,0,0,1);
 * view space looks down +z.  Pixel (px, py) has its centre at
 * (px, py) = (fx x/z + cx, fy y/z + cy); normally cx = (width-1)/2.
 * tan_fov*: half-angle tangents (used by the Jacobian clamp).  campos: world
 * camera centre (for view-dependent colour).  znear: Gaussians with view
 * z <= znear are culled. */
typedef struct {
    float viewmat[16];
    float fx, fy, cx, cy;
    float tan_fovx, tan_fovy;
    float campos[3];
    int32_t width, height;
    float znear;
} qb_camera;

/* Scene in structure-of-arrays form, all device float32, row-major:
 * means [n,3]; scales [n,3] (log-scales if params_raw); quats [n,4] as
 * (w,x,y,z), any non-zero norm; opacities [n] (logits if params_raw);
 * sh [n,K,3] with K = (sh_degree+1)^2, sh_degree in 0..3, coefficient k
 * ordered l*l + l + m.  Colour = max(0, sum_k sh_k Y_k(dir) + 0.5) with dir
 * the unit vector from campos to the mean and Y_k the real spherical
 * harmonics carrying the Condon-Shortley phase (the 3DGS basis). */
typedef struct {
    const float *means;
    const float *scales;
    const float *quats;
    const float *opacities;
    const float *sh;
    int32_t n;
    int32_t sh_degree;
    int32_t params_raw;
} qb_scene;

/* Gradient outputs of qb_render_bwd, device float32, same shapes as the
 * qb_scene inputs.  The callee ACCUMULATES into them (+=); the caller zeroes
 * them first.  Gradients are w.r.t. the raw parameters when params_raw. */
typedef struct {
    float *means;
    float *scales;
    float *quats;
    float *opacities;
    float *sh;
} qb_scene_grads;

/* Per-frame state.  Create with qb_frame_init; the workspace is caller-
 * allocated device memory of at least qb_frame_workspace_bytes(...) bytes,
 * 256-byte aligned.  Fields are read-only for the caller. */
typedef struct {
    int32_t n, width, height, tiles_x, tiles_y;
    uint64_t pair_capacity;
    void *workspace;
    size_t workspace_bytes;
    /* written by the stages */
    int32_t bin_mode;       /* mode used by the last qb_preprocess        */
    int32_t sh_degree;
    int32_t key_bits;       /* significant key bits: 31 + tile bits       */
    int32_t stage;          /* 0 init, 1 preprocessed, 2 emitted, 3 sorted */
    uint64_t n_pairs;       /* host copy of P when known, else UINT64_MAX  */
    int32_t sort_digit_bits;  /* 8..11, radix digit width of qb_sort        */
    int32_t render_batch;     /* Gaussians staged per shared-memory batch   */
    int32_t sorted_in_alt;    /* internal: sorted pairs live in buffer 1    */
    int32_t sort_mode;        /* qb_sort_mode; set before qb_preprocess     */
    int32_t depth_in_alt;     /* internal: depth order lives in buffer 1    */
    int32_t emit_fused;       /* DEPTH_FIRST: 1 = the emit performs the tile
                                 sort's first digit pass (per-tile counts from
                                 the preprocess); 0 (default) = plain emit, the
                                 per-tile counts from a histogram of the
                                 emitted tile ids in qb_sort.  Frames of more
                                 than 24576 tiles (beyond the histogram's
                                 shared memory, e.g. 3840 x 2160) always take
                                 the fused emit; 1 selects it on any frame.
                                 Set before qb_preprocess                    */
    int32_t reserved[3];      /* internal */
} qb_frame;

/* Device arrays inside a frame workspace (for inspection and tests).  All
 * per-Gaussian arrays have n entries, indexed by Gaussian. */
typedef struct {
    float *xy;          /* [n][2]  mu^2D in pixels                          */
    float *conic_o;     /* [n][4]  (a, b, c, o): Lambda = [a b; b c], opacity */
    float *rgbd;        /* [n][4]  (r, g, b, depth)                         */
    float *box;         /* [n][4]  (x_max, y_max, f x_max, f y_max)         */
    float *r3;          /* [n]     3-sigma radius ceil(3 sqrt(lambda_max))  */
    int32_t *meta;      /* [n]     bit0 visible, bit1 orient (Sigma12 >= 0),
                                   bits2-4 colour channel clamped at 0      */
    uint32_t *counts;   /* [n]     tiles per Gaussian                       */
    uint32_t *offsets;  /* [n]     exclusive prefix of counts in emission order
                                   (index order, or depth order in DEPTH_FIRST) */
    uint64_t *keys;     /* [P]     FULL_KEY: (tile << 31) | depth bits, sorted after qb_sort */
    uint32_t *tile_keys;/* [P]     DEPTH_FIRST: scratch of the tile sort; the sorted
                                   tile ids are given by the ranges (qb_frame_tile_keys) */
    uint32_t *vals;     /* [P]     Gaussian index, in sorted order after qb_sort */
    uint32_t *depth_order; /* [n]  DEPTH_FIRST: Gaussians by (depth, index) */
    uint32_t *ranges;   /* [tiles][2] [start, end) into keys/vals           */
    float *t_final;     /* [H][W]  transmittance after the last contributor */
    int32_t *n_contrib; /* [H][W]  1 + position of the last contributor     */
    int32_t *n_eval;    /* [H][W]  list entries the pixel evaluated before it
                                   stopped (render statistics; written by
                                   qb_render_fwd_counted only)               */
    uint64_t *n_pairs;  /* [1]     P on the device                          */
    uint32_t *err_flags;/* [2]     [0]: bit0 capacity, bit1 timeout.  [1]:
                                   test-only, zero after qb_frame_init; a test
                                   may set it to k > 0 to exercise a bounded
                                   spin-wait: the second block of the last
                                   (values-only) tile-sort pass then finds its
                                   predecessor unpublished, gives up after k
                                   polls and raises TIMEOUT; the sorted values
                                   are then undefined (do not render them)  */
    uint32_t *order_counts; /* [2][64] tiles per work bucket, written by the
                                   forward render: [0] the render's order (by
                                   an estimate of each tile's work), [1] the
                                   backward's (by the tile's largest
                                   n_contrib); bucket j holds work in
                                   [16 (63 - j), 16 (64 - j)), bucket 0 all
                                   work from 1008 on                        */
    uint32_t *order_lists;  /* [2][64][tiles] the tile ids of each bucket,
                                   the first order_counts[o][j] of row j    */
} qb_frame_arrays;

/* Thread-local description of the last failure. */
const char *qb_last_error(void);

/* Library version string. */
const char *qb_version(void);

/* Number of CUDA kernels the library has launched in this process (all
 * threads, all devices), counted on the host at each launch. */
uint64_t qb_kernel_launches(void);

/* Instrumentation: when set, hook(kernel name, stream, user) is called on the
 * host immediately before each kernel launch of the library, on the thread
 * that launches it (e.g. to record a CUDA event on that stream, so kernel
 * durations can be measured in stream order).  NULL removes it.  The hook
 * must not call back into the library. */
typedef void (*qb_launch_hook)(const char *kernel, qb_stream_t stream, void *user);
void qb_set_launch_hook(qb_launch_hook hook, void *user);

/* Bytes of device workspace for a frame of n Gaussians, a width x height
 * image and room for pair_capacity Gaussian-tile pairs (pair_capacity
 * <= 2^30).  Returns 0 for invalid sizes. */
size_t qb_frame_workspace_bytes(int32_t n, int32_t width, int32_t height, uint64_t pair_capacity);

/* Binds a caller-owned workspace to *frame and resets the frame state.
 * Errors: INVALID_ARG for bad sizes, a NULL or misaligned workspace, or
 * workspace_bytes below qb_frame_workspace_bytes(...). */
qb_status qb_frame_init(qb_frame *frame, int32_t n, int32_t width, int32_t height,
                        uint64_t pair_capacity, void *d_workspace, size_t workspace_bytes,
                        qb_stream_t stream);

/* Device pointers of the frame's internal arrays. */
qb_status qb_frame_arrays_get(const qb_frame *frame, qb_frame_arrays *out);

/* Writes the sorted pairs' tile ids (tile t at every position of its range)
 * to d_out (device uint32 [n_out]) from the per-tile ranges, for inspection
 * in either sort mode; positions >= n_out are skipped.  Errors: STATE before
 * qb_sort, INVALID_ARG for a NULL d_out with n_out > 0. */
qb_status qb_frame_tile_keys(const qb_frame *frame, uint32_t *d_out, uint64_t n_out, qb_stream_t stream);

/* Synchronises the stream and reports device-side failures recorded in the
 * frame (CAPACITY, TIMEOUT); clears them. */
qb_status qb_frame_check(qb_frame *frame, qb_stream_t stream);

/* Stage 1 (Sec. 2 "Preprocess", Sec. 3.1): per Gaussian, EWA projection to
 * mu^2D and the conic Lambda = (Sigma^2D)^-1 (Eq. 4), depth, SH colour, the
 * opacity-aware threshold gamma = 2 ln(o / (1/255)) (Eq. 3, kept side),
 * the extents x_max, y_max (Eq. extents-closed), the stretching factor f
 * (Eq. f-closed), the 3-sigma radius, the mode's tile rectangles and the
 * QPass tile count.  scene->n must equal frame->n; mode is a qb_bin_mode,
 * optionally OR QB_BIN_NO_CLAMP. */
qb_status qb_preprocess(qb_frame *frame, const qb_scene *scene, const qb_camera *camera, int32_t mode,
                        qb_stream_t stream);

/* Stage 2 (Sec. 2 "DuplicateWithKeys", Sec. 3.2 QPass): exclusive scan of the
 * tile counts, then one (key, value) pair per Gaussian-tile overlap with
 * key = (tile << 31) | float bits of the depth (FULL_KEY) or the tile id
 * (DEPTH_FIRST, after sorting the Gaussians by depth), value = Gaussian
 * index, in emission order (each Gaussian's pairs at its scan offset).  In
 * DEPTH_FIRST with emit_fused the per-tile counts (from the preprocess) give
 * the ranges here, and in the QPass modes the emit also performs the first
 * digit pass of the tile sort, so the pairs leave it bucketed by their lowest
 * tile digit rather than in emission order; without emit_fused (the default)
 * qb_sort counts the emitted tile ids.
 * If n_pairs_out is non-NULL the host synchronises once to read P, stores it
 * in *n_pairs_out and frame->n_pairs, and returns CAPACITY (writing no pairs)
 * when P > pair_capacity.  With NULL nothing synchronises; an overflow is
 * then flagged on the device and reported by qb_frame_check. */
qb_status qb_bin_emit(qb_frame *frame, uint64_t *n_pairs_out, qb_stream_t stream);

/* Stage 3 (Sec. 2 "SortPairs"): stable LSD radix sort of the pairs with the
 * library's onesweep sort on the key bits [0, 31 + tile bits) (FULL_KEY),
 * then the per-tile [start, end) ranges; or (DEPTH_FIRST) a histogram of
 * the emitted tile ids giving the ranges and every pass's bucket offsets
 * (unless the fused emit already did), then the remaining digit passes on
 * the tile bits, whose last pass writes only the values (in vals,
 * sorted_in_alt = 0). */
qb_status qb_sort(qb_frame *frame, qb_stream_t stream);

/* Stage 4 (Sec. 2 "Render", Eq. 2): front-to-back compositing per pixel.
 * bg: host float[3] background colour (NULL = black).  d_img: device
 * float [3][height][width] (planar RGB), fully overwritten.  Also writes the
 * frame's t_final and n_contrib, which qb_render_bwd needs.  The tiles run
 * heaviest first: a first kernel files every tile by an estimate of its work
 * (order_counts[0] / order_lists[0] of qb_frame_arrays), and the render files
 * every tile again by its largest n_contrib for qb_render_bwd (the second
 * order); the image does not depend on the order. */
qb_status qb_render_fwd(qb_frame *frame, const float *bg, float *d_img, qb_stream_t stream);

/* Measurement only: qb_render_fwd (identical outputs) that also adds, over
 * all pixels, the (pixel, entry) evaluations of Eq. 2's loop up to each
 * pixel's stop to d_counts[0] and those whose exponent passed the power test
 * (not below the skip threshold, i.e. alpha was computed) to
 * d_counts[1].  d_counts: device uint64[2], accumulated (zero them first),
 * 8-byte aligned.  The counted kernel is slower than qb_render_fwd's; the
 * counts give the method's arithmetic work per frame for a roofline. */
qb_status qb_render_fwd_counted(qb_frame *frame, const float *bg, float *d_img, uint64_t *d_counts,
                                qb_stream_t stream);

/* Backward of stages 1 and 4 (differentiable rasteriser, Sec. 4.1): walks each
 * tile list in reverse from every pixel's last contributor, recomputing the
 * transmittance by division, and accumulates into grads the gradient of
 * sum(d_dL_dimg * image) w.r.t. the scene parameters.  scene, camera and bg
 * must be those of the forward pass.  d_dL_dimg: device float [3][H][W].
 * If d_grad_screen is non-NULL it receives the screen-space gradients,
 * double [n][9] = dL/d(mu_x, mu_y, Sigma11, Sigma12, Sigma22, o, r, g, b),
 * Sigma the 2D covariance with Sigma12 counted once (the conic gradient is
 * dL/dLambda = -Sigma dL/dSigma Sigma), and must be zeroed by the caller;
 * the sums over pixels are accumulated in float64.  Tiles run in the order
 * the last qb_render_fwd of this frame filed (heaviest first). */
qb_status qb_render_bwd(qb_frame *frame, const qb_scene *scene, const qb_camera *camera, const float *bg,
                        const float *d_dL_dimg, qb_scene_grads *grads, double *d_grad_screen,
                        qb_stream_t stream);

/* ------------------------------------------------------------------------ */
/* One optimisation step around the rasteriser (training integration).       */
/* ------------------------------------------------------------------------ */

/* L1 image loss: d_dL[i] = scale * sign(d_img[i] - d_target[i]) (0 where
 * equal), and, when d_loss is non-NULL, *d_loss += scale * sum |img - target|
 * (device double, accumulated; zero it first).  All device float [n].  With
 * scale = 1 / n this is the gradient of the mean absolute error. */
qb_status qb_l1_loss_grad(const float *d_img, const float *d_target, float *d_dL, uint64_t n, float scale,
                          double *d_loss, qb_stream_t stream);

/* Adam update (Kingma & Ba, bias-corrected) of n parameters in place, step
 * `step` >= 1: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).  d_m and d_v
 * are the caller's moment buffers (zero before the first step).  Apply it to
 * the raw scene arrays with the gradients qb_render_bwd accumulates. */
qb_status qb_adam_step(float *d_param, const float *d_grad, float *d_m, float *d_v, uint64_t n, float lr,
                       float beta1, float beta2, float eps, int32_t step, qb_stream_t stream);

/* Standalone pair sort (the sort used by qb_sort): sorts n (key, value)
 * pairs stably by key bits [0, end_bit) with the onesweep radix sort using
 * digit_bits-wide digits (8..11).  d_keys/d_vals hold the input; the result
 * ends in (d_keys, d_vals) if *result_in_alt is 0 on return, else in
 * (d_keys_alt, d_vals_alt).  d_scratch: device, at least
 * qb_sort_scratch_bytes(n, end_bit, digit_bits) bytes.  n <= 2^30. */
size_t qb_sort_scratch_bytes(uint64_t n, int32_t end_bit, int32_t digit_bits);
qb_status qb_sort_pairs(uint64_t *d_keys, uint32_t *d_vals, uint64_t *d_keys_alt, uint32_t *d_vals_alt,
                        uint64_t n, int32_t end_bit, int32_t digit_bits, void *d_scratch,
                        size_t scratch_bytes, int32_t *result_in_alt, qb_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Many cameras of one scene in one launch sequence (batched rendering).     */
/* ------------------------------------------------------------------------ */

#define QB_MAX_CAMERAS 256
#define QB_GROUP_MAX 16

/* Launch parameters of the batched path (picked by the autotuner).
 *  tiles_per_fetch  tiles a persistent render block takes from the global
 *                   tile-work queue at a time (1..8)
 *  render_batch     Gaussians staged per shared-memory batch (64, 128, 256)
 *  sort_digit_bits  radix digit width of each camera's tile sort (8..11)
 *  blocks_per_sm    persistent render blocks per SM (0: as many as fit) */
typedef struct {
    int32_t tiles_per_fetch;
    int32_t render_batch;
    int32_t sort_digit_bits;
    int32_t blocks_per_sm;
} qb_tune;

/* Batch state.  The preprocess runs once per group of `group` cameras
 * (<= QB_GROUP_MAX; one launch over every (camera, Gaussian) record of the
 * group, reading the scene once); every camera's pairs are then binned and
 * sorted like a frame into the camera's own slot; the render is one
 * persistent kernel fed by a global queue over the tiles of all n_cams
 * cameras, so cameras of uneven resolution balance across the GPU.  Images
 * are packed in one float buffer: camera k's planar [3][height][width] image
 * starts at float offset image_offset[k].  pair_capacity bounds the
 * Gaussian-tile pairs of one camera (<= 2^30).  A camera may have at most
 * 24576 tiles (render larger images as frames), and n_cams * n < 2^32.
 * Fields are read-only for the caller. */
typedef struct {
    int32_t n, n_cams, group, n_groups;
    uint64_t pair_capacity;
    void *workspace;
    size_t workspace_bytes;
    int32_t widths[QB_MAX_CAMERAS], heights[QB_MAX_CAMERAS];
    uint64_t image_offset[QB_MAX_CAMERAS];
    uint64_t total_floats;  /* size of the packed image buffer in floats */
    int32_t sh_degree, bin_mode, stage, sorted_tile_bits;
    int32_t reserved[8];
} qb_batch;

/* Bytes of device workspace for a batch (0 for invalid sizes). */
size_t qb_batch_workspace_bytes(int32_t n, int32_t n_cams, const int32_t *widths, const int32_t *heights,
                                int32_t group, uint64_t pair_capacity);

/* Binds a caller-owned, 256-byte aligned device workspace to *batch, writes
 * the render's per-camera table into it (synchronises the stream once) and
 * creates the batch's side streams: inside qb_render_batch the cameras of a
 * group are binned four at a time on side streams forked from the caller's
 * stream and joined back to it (captured into a CUDA graph with the rest).
 * Errors: INVALID_ARG for sizes outside the limits above. */
qb_status qb_batch_init(qb_batch *batch, int32_t n, int32_t n_cams, const int32_t *widths, const int32_t *heights,
                        int32_t group, uint64_t pair_capacity, void *d_workspace, size_t workspace_bytes,
                        qb_stream_t stream);

/* Destroys the side streams of a batch (after their work is done) and
 * unbinds its workspace; the caller still owns and frees the workspace. */
qb_status qb_batch_release(qb_batch *batch);

/* Forward of every camera of the batch (Sec. 2's pipeline with QuadBox
 * binning, Sec. 3, per camera): per group, one preprocess over all (camera,
 * Gaussian) records; per camera, the depth order of its records, scan, QPass
 * emit with camera-local tile ids, the tile histogram (ranges and bucket
 * offsets) and the stable tile sort into the camera's slot; then one
 * persistent render over the tiles of every camera.  cams: host array of
 * n_cams cameras whose sizes match qb_batch_init; tune: host, NULL for
 * defaults; d_images: device floats, total_floats of them.  No host
 * synchronisation and no allocation, so a call can be captured in a CUDA
 * graph (the cameras and tuning are then fixed in the graph); make one call
 * outside capture first.  Pair-capacity overflow is flagged on the device and
 * reported by qb_batch_check. */
qb_status qb_render_batch(qb_batch *batch, const qb_scene *scene, const qb_camera *cams, int32_t mode,
                          const qb_tune *tune, const float *bg, float *d_images, qb_stream_t stream);

/* Backward of the last qb_render_batch (same scene, cameras and bg):
 * accumulates into grads the gradient of sum(d_dL_dimages * images): one
 * persistent render backward over every camera's tiles, then the chain to
 * the scene parameters once per group.  d_dL_dimages is packed like the
 * images.  Capturable like the forward. */
qb_status qb_render_batch_bwd(qb_batch *batch, const qb_scene *scene, const qb_camera *cams, const float *bg,
                              const float *d_dL_dimages, qb_scene_grads *grads, qb_stream_t stream);

/* Synchronises and reports overflow or time-outs of the last batch calls;
 * if pairs_out (host, n_cams entries) is non-NULL it receives the pairs of
 * every camera. */
qb_status qb_batch_check(qb_batch *batch, uint64_t *pairs_out, qb_stream_t stream);

/* The same sort for callers that may not allocate device memory (no
 * counterpart in the paper).  Some callers cannot call cudaMalloc: a plug-in
 * whose host application owns all device memory, a render loop that must not
 * stall on an allocation, code that must keep a fixed device footprint.
 * Here the scratch lives in a fixed 16 MiB __device__ array inside the
 * library (qb_sort_pairs_noalloc_max_scratch() bytes), which every GPU that
 * loads the library holds until the process exits; no call allocates or
 * frees memory.  Sizes whose scratch (qb_sort_scratch_bytes(n, end_bit,
 * digit_bits) minus 256) exceeds that array are rejected with INVALID_ARG,
 * e.g. more than about 11M pairs at 44 key bits with 8-bit digits.
 * Arguments and result as for qb_sort_pairs.  Every call looks up the
 * array's device address on the current device (the first call on a device
 * may load the library's device code; make it before any stream capture).
 * All calls share the one array, and each call clears what must start at
 * zero, so calls whose work overlaps on the GPU (other streams, other host
 * threads) race with each other: serialise them.  Synchronises the stream
 * once, like qb_sort_pairs. */
size_t qb_sort_pairs_noalloc_max_scratch(void);
qb_status qb_sort_pairs_noalloc(uint64_t *d_keys, uint32_t *d_vals, uint64_t *d_keys_alt, uint32_t *d_vals_alt,
                                uint64_t n, int32_t end_bit, int32_t digit_bits, int32_t *result_in_alt,
                                qb_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* QUADBOX_H */
