/*
 * maskgs.h -- C ABI of libmaskgs, a GB300 (sm_103a) rasteriser for
 * MaskGaussian's masked rasterisation (Liu et al., "MaskGaussian: Adaptive 3D
 * Gaussian Representation from Probabilistic Masks", CVPR 2025,
 * arXiv 2412.20522).
 *
 * One training step of the method, as the paper describes it:
 *   1. mg_preprocess          sample each Gaussian's mask M_i (Sec. 3.3,
 *                             Gumbel-softmax over two existence scores) and
 *                             splat every Gaussian, unmasked, to a 2D
 *                             Gaussian with a view-dependent colour (Sec. 3.1)
 *   2. mg_depth_order, mg_bin order the splats by depth (Sec. 3.1: the blend
 *                             indexes Gaussians front to back) and duplicate each
 *                             visible splat once per 16x16 tile it intersects
 *                             (Sec. 3.1), keyed by (tile, depth)
 *   3. mg_sort                group the instances by tile, keeping the depth
 *                             order, and find each tile's range
 *   4. mg_render              masked alpha blending, Eq. 3-4
 *   5. mg_l1_loss_grad        an L1 render loss and dL/dC (Eq. 8's L_render)
 *   6. mg_render_backward     the mask gradient of Eq. 6 with the background
 *                             term of Appendix A, and the colour, opacity and
 *                             2D-geometry gradients of the same blend
 *   7. mg_preprocess_backward the chain rule back to the Gaussian parameters,
 *                             and through the straight-through Gumbel-softmax
 *                             to the existence scores
 * Fused forms of the same step: mg_render_l1 takes steps 4-5 in one kernel;
 * mg_render_l1_reset2d also resets the 2D-gradient accumulator that
 * mg_render_backward_accumulate then adds into (step 6 without its own
 * reset); mg_advance_iteration moves a device-side iteration on, so a step
 * captured in a CUDA graph samples a new mask on every replay.
 *
 * Conventions
 *   - Every array pointer is a caller-owned DEVICE pointer unless the comment
 *     says "host".  The library allocates nothing.
 *   - Every call only enqueues work on `stream` (a cudaStream_t); none
 *     synchronises, so the whole sequence can be captured in a CUDA graph.
 *   - Every call returns an mg_status.  Argument errors are detected on the
 *     host before anything is enqueued (MG_ERR_INVALID_ARG); a failed launch
 *     returns MG_ERR_CUDA.  Errors found on the device (instance capacity
 *     exceeded, a bounded wait that gave up) are written to the caller's
 *     device mg_status_word; read it after a synchronisation with
 *     mg_read_status.  No C++ exception crosses this interface.
 *   - Gaussians of all views live in one set of arrays.  A view sees the
 *     Gaussians [gaussian_offset, gaussian_offset + gaussian_count); several
 *     views of one scene share the range, a batch of scenes uses disjoint
 *     ranges.  Per-view outputs are concatenated in view order: view v's
 *     splat records start at record index R_v = sum_{u<v} gaussian_count_u,
 *     its tiles at T_v = sum_{u<v} tiles_x_u * tiles_y_u, its pixels at
 *     P_v = sum_{u<v} W_u * H_u.
 *   - Thread safety: concurrent calls on distinct buffers are independent.
 *     The library's only process-wide state is set once per device under a
 *     lock (the sort kernels' shared-memory limit; the address of the scratch
 *     array of mg_bin_noalloc, which itself must not be shared by overlapping
 *     calls); make the first call on a device outside stream capture.
 */
#ifndef MASKGS_H
#define MASKGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mg_stream_t;   /* same type as cudaStream_t */

typedef enum {
    MG_OK = 0,
    MG_ERR_INVALID_ARG = 1,
    MG_ERR_CUDA = 2,
    MG_ERR_CAPACITY = 3,     /* more (tile, Gaussian) instances than the buffers hold */
    MG_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    MG_ERR_UNSUPPORTED = 5,
    MG_ERR_BOUNDS = 6        /* an index or range outside its buffer (mg_validate_lists, or
                                a build with the bounds checks compiled in) */
} mg_status;

/* Mask modes (mg_raster_cfg.mask_mode):
 *   MG_MASK_GUMBEL    M_i sampled by Gumbel-max over the two scores, gradient
 *                     by the straight-through Gumbel-softmax (Sec. 3.3);
 *   MG_MASK_ALL_ONES  M_i = 1 (plain 3DGS, Eq. 1-2);
 *   MG_MASK_GIVEN     M_i read from given_mask;
 *   MG_MASK_STE       the deterministic ablation of Sec. 4.3 ("Effect of
 *                     Gumbel Softmax"): M_i = [l_0 - l_1 > ste_logit], i.e.
 *                     sigmoid(l_0 - l_1) above a threshold, with the
 *                     straight-through gradient of sigmoid(l_0 - l_1).
 * Mask application (mg_raster_cfg.mask_apply):
 *   MG_APPLY_RASTER   masked rasterisation, Eq. 3-4 (the method);
 *   MG_APPLY_OPACITY  the ablation of Sec. 4.3 ("Effect of Masked
 *                     Rasterization"): the splat's opacity is M_i o_i and it
 *                     blends as in Eq. 1-2, so a masked splat (alpha 0) is
 *                     filtered and receives no gradient; dL/dM_i = o_i dL/do'.
 * Mask loss (mg_raster_cfg.mask_loss), weighted by lambda_m (Eq. 8):
 *   MG_MASK_LOSS_L2   L_m = (sum_i M_i / N)^2 (Eq. 7);
 *   MG_MASK_LOSS_L1   L_m = sum_i M_i / N (the L1 form of Appendix C). */
enum { MG_MASK_GUMBEL = 0, MG_MASK_ALL_ONES = 1, MG_MASK_GIVEN = 2, MG_MASK_STE = 3 };
enum { MG_APPLY_RASTER = 0, MG_APPLY_OPACITY = 1 };
enum { MG_MASK_LOSS_L2 = 0, MG_MASK_LOSS_L1 = 1 };
/* Tile lists (mg_raster_cfg.bin_mode): MG_BIN_FILTERED drops the (Gaussian,
 * tile) pairs of the 3-sigma rectangle where the Gaussian stays under the
 * alpha floor at every pixel (no result changes; shorter lists); MG_BIN_RECT
 * keeps the whole rectangle, as the 3DGS rasteriser bins. */
enum { MG_BIN_FILTERED = 0, MG_BIN_RECT = 1 };
enum { MG_DTYPE_F32 = 0, MG_DTYPE_BF16 = 1, MG_DTYPE_F16 = 2 };
enum { MG_MAX_VIEWS = 64, MG_RECORD_FLOATS = 12, MG_GRAD2D_FLOATS = 12 };

/* Device status word.  Zero it before a step; kernels only ever raise it.
 * status: an mg_status; detail: which stage raised it (1 bin, 2 sort);
 * required: for MG_ERR_CAPACITY, the number of instances that was needed. */
typedef struct {
    int32_t status;
    int32_t detail;
    uint64_t required;
} mg_status_word;

/* Gaussian parameters (Sec. 3.1: centre p, opacity o, scales s, rotation q,
 * SH; Sec. 3.3: two mask scores).  Device arrays:
 *   means[n][3] FP32; log_scales[n][3] (s = exp(log_scales));
 *   quats[n][4] as (w, x, y, z), normalised inside;
 *   opacity_logit[n] (o = sigmoid(opacity_logit));
 *   sh[n][(sh_degree+1)^2][3], real SH with the Condon-Shortley phase,
 *     basis order l = 0..D, m = -l..l, colour = sum_k Y_k(dir) sh[k] + 0.5,
 *     clamped at 0; dir = normalise(p - cam_pos);
 *   mask_logits[n][2] FP32, index 0 = "present".
 * dtype is the storage of log_scales, quats, opacity_logit and sh: FP32, BF16
 * or FP16 (unpacked to FP32 on load; every computation is FP32).  Alignment:
 * sh 16 bytes, quats one row (16 or 8 bytes). */
typedef struct {
    int64_t n;
    int32_t sh_degree;       /* 0..3 */
    int32_t dtype;           /* MG_DTYPE_F32, MG_DTYPE_BF16 or MG_DTYPE_F16 */
    const void *means;
    const void *log_scales;
    const void *quats;
    const void *opacity_logit;
    const void *sh;
    const void *mask_logits;
} mg_gaussians;

/* Pinhole camera with OpenCV axes (x right, y down, z forward).
 * viewmat: row-major 3x4 world->camera, t = R p + t_cam.  Pixel (u, v) is
 * evaluated at its centre (u + 0.5, v + 0.5); p_bar = (fx tx/tz + cx,
 * fy ty/tz + cy).  Gaussians with tz <= near_plane are culled. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float viewmat[12];
    float cam_pos[3];
    float near_plane;
} mg_camera;

typedef struct {
    mg_camera cam;
    int64_t gaussian_offset;
    int64_t gaussian_count;
} mg_view;

/* tile_w x tile_h: 16x16 (the paper's grid, Sec. 3.1), 32x8 or 8x32 (256
 * pixels, both sides powers of two and at least 8; other shapes return
 * MG_ERR_INVALID_ARG).
 * Gumbel noise: u_k from Philox4x32-10 (Salmon et al., SC'11) with counter
 * (i, iteration_lo, iteration_hi, 0) and key (seed_lo, seed_hi), outputs 0 and
 * 1 mapped to (2 (x >> 9) + 1) 2^-24.  mask_mode MG_MASK_GIVEN reads
 * given_mask[n] (device, 0/1 bytes).  A view's scene is its Gaussian range:
 * views with equal ranges are views of one scene, and L_m is summed over the
 * distinct ranges, each over its own N = gaussian_count. */
typedef struct {
    int32_t tile_w, tile_h;
    float bg[3];
    float tau;               /* Gumbel-softmax temperature, > 0 */
    uint64_t seed;
    uint64_t iteration;
    int32_t mask_mode;       /* MG_MASK_* */
    int32_t mask_apply;      /* MG_APPLY_* */
    const uint8_t *given_mask;
    float lambda_m;          /* weight of L_m in L = L_render + lambda_m L_m (Eq. 8); 0 = off */
    int32_t mask_loss;       /* MG_MASK_LOSS_* */
    float ste_logit;         /* MG_MASK_STE threshold on l_0 - l_1 (FP32 comparison) */
    int32_t bin_mode;        /* MG_BIN_* */
    /* Splats staged in shared memory per batch by the render kernels (a
     * tuning choice; no result depends on it): render_batch 128 or 256 for
     * the forward, render_batch_bwd 64 or 128 for the backward, 0 = the
     * defaults (256, 128); other values return MG_ERR_INVALID_ARG. */
    int32_t render_batch;
    int32_t render_batch_bwd;
    /* Device word (nullable) added to `iteration` by the mask sample: a step
     * captured in a CUDA graph keeps every argument it was captured with, so
     * a training loop that replays it draws a new mask each step only if the
     * iteration lives in device memory and is advanced between replays
     * (mg_advance_iteration, captured with the step). */
    const uint64_t *iteration_dev;
} mg_raster_cfg;

/* Per-view preprocess outputs (R = sum_v gaussian_count_v records):
 *   record[R][12] FP32 render record: mean2d x, y; major axis ux, uy of the
 *     2D covariance; h1 = -log2(e)/(2 lambda_1), h2 = -log2(e)/(2 lambda_2)
 *     (so that o exp(-1/2 d^T Sigma^-1 d) = o exp2(h1 (d.u)^2 + h2 (d.u_perp)^2));
 *     o if M = 1, -o if M = 0 (opacity o > 0, the mask in the sign);
 *     e_min, a skip threshold just below log2(1/(255 o)) for the exponent
 *     (1 if o < 1/255: the splat never reaches the floor); r, g, b; depth tz.
 *   tiles_touched[R] u32, the record's candidate tiles for the binning: its
 *     whole 3-sigma rectangle (MG_BIN_RECT), or (MG_BIN_FILTERED) the tiles of
 *     that rectangle that meet the bounding box of the region where the tile
 *     filter can keep a tile -- a box computed by a fixed sequence of
 *     correctly rounded FP32 operations, with margins that make it hold every
 *     tile the filter keeps, so no list changes; 0 = no
 *     candidate (culled, or nothing of it can reach the floor in a tile);
 *   radius[R] i32 (pixels, 0 = culled),
 *   clamp[R] u8 (bit c: colour channel c was clamped at 0),
 *   bin_record[R][12] (48 bytes, 16-byte aligned) of a visible record, for
 *   the binning: FP32 px, py, a, b, c (the 2D covariance [[a, b], [b, c]]),
 *   11.1 det, b / a, b / c (decision-path values), then u32 x0 | y0 << 16
 *   (first tile column and row of the candidate rectangle), w (its width),
 *   the global id of its first tile, and the view's tiles per row gx; tile m
 *   of the rectangle (row-major) is first + (m / w) gx + m % w.
 *   With MG_APPLY_OPACITY the stored opacity is M o (+0 for a masked splat,
 *   e_min = 1).
 * Per-Gaussian (n):
 *   mask[n] u8 sampled M_i; mask_soft[n] f32 soft sample y_0 of the
 *   Gumbel-softmax (sigmoid(l_0 - l_1) for MG_MASK_STE, 1 for all-ones /
 *   given masks).
 * Per view (n_views), nullable: mask_count[v] u32 = sum of M_i over view v's
 *   Gaussian range (written by mg_preprocess; needed by mg_mask_loss and by
 *   mg_preprocess_backward when lambda_m != 0).
 * Nullable: depth_key[R] u32, the depth-order key of each record (the float
 *   bits of tz, 0xFFFFFFFF for a record that touches no tile); written by
 *   mg_preprocess when non-null, and then read by mg_depth_order instead of
 *   deriving the keys from record and tiles_touched. */
typedef struct {
    float *record;
    uint32_t *tiles_touched;
    int32_t *radius;
    uint8_t *clamp;
    float *bin_record;
    uint8_t *mask;
    float *mask_soft;
    uint32_t *mask_count;
    uint32_t *depth_key;
} mg_splats;

/* Gradients w.r.t. the per-view splats, grad2d[R][12] FP32:
 *   dL/dmean2d x, y; dL/dconic a, b, c (conic = Sigma^-1 = [[a, b], [b, c]],
 *   b the off-diagonal entry); dL/dopacity; dL/dr, g, b; dL/dM; 2 unused. */

/* Gradients w.r.t. the Gaussian parameters, same shapes as mg_gaussians,
 * FP32, OVERWRITTEN (summed over all views that see the Gaussian). */
typedef struct {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logit;
    float *sh;
    float *mask_logits;
} mg_param_grads;

/* ---- 1. preprocess (Sec. 3.1, Sec. 3.3) -------------------------------- */
/* Samples M_i once per Gaussian and splats every Gaussian of every view.
 * views: HOST array of n_views (1..MG_MAX_VIEWS) views.  The tile rectangle,
 * radius and depth key are computed by a fixed sequence of correctly rounded
 * FP32 operations (reproducible bit for bit).  Errors: MG_ERR_INVALID_ARG for
 * null pointers, n < 0, bad tile shape, sh_degree outside 0..3, a view range
 * outside [0, n), non-positive image size, tau <= 0. */
mg_status mg_preprocess(const mg_gaussians *g, const mg_view *views, int32_t n_views,
                        const mg_raster_cfg *cfg, const mg_splats *out,
                        mg_status_word *d_status, mg_stream_t stream);

/* ---- 2. depth order and bin (Sec. 3.1) ------------------------------------ */
/* Stable radix sort of the R splat records (all views) by the float bits of
 * their depth, records that touch no tile last: order[R] (u32 record indices).
 * Depth ties keep record order.  The keys are splats->depth_key when non-null
 * (as mg_preprocess wrote them), else derived from record and tiles_touched.
 * keys, keys_alt, order_alt: u32[R] scratch.  workspace:
 * mg_depth_order_workspace_bytes(R) bytes, any content. */
mg_status mg_depth_order(const mg_splats *splats, const mg_view *views, int32_t n_views,
                         const mg_raster_cfg *cfg, uint32_t *order, uint32_t *order_alt,
                         uint32_t *keys, uint32_t *keys_alt, void *workspace,
                         size_t workspace_bytes, mg_status_word *d_status, mg_stream_t stream);
size_t mg_depth_order_workspace_bytes(int64_t n_records);

/* Visits the R records in `order` (nullable: record order) and writes, for
 * position i, offsets[i] = sum_{j<i} tiles_touched[order[j]] (u32) and the
 * total K into *d_num_instances (device u64); then, for every record
 * r = order[i] and every tile of its candidate rectangle (row-major), the key
 * = global tile id (u32) and the value r at offsets[i] + k -- or, with
 * bin_mode MG_BIN_FILTERED, the key 0xFFFFFFFF when the record's Gaussian
 * stays under the alpha floor at every pixel of that tile (its quadratic form
 * above 2 ln 255 at every pixel centre, tested in correctly rounded FP32 from
 * bin_record): such a pair is a no-op, and mg_sort drops it.  Instances
 * beyond `capacity` are not written and raise MG_ERR_CAPACITY with
 * `required` = K.  workspace: device scratch of mg_bin_workspace_bytes(R)
 * bytes, any content. */
mg_status mg_bin(const mg_splats *splats, const mg_view *views, int32_t n_views,
                 const mg_raster_cfg *cfg, const uint32_t *order, uint32_t *offsets,
                 uint32_t *keys, uint32_t *vals, uint64_t capacity, uint64_t *d_num_instances,
                 void *workspace, size_t workspace_bytes, mg_status_word *d_status,
                 mg_stream_t stream);
size_t mg_bin_workspace_bytes(int64_t n_records);

/* The same as mg_bin, for callers that cannot allocate device memory (a
 * plugin whose host application owns every allocation, or code running where
 * cudaMalloc is not allowed): no workspace argument.  The paper has no
 * counterpart; this is a deployment convenience.
 * Its scratch is one file-scope device array inside the library, sized for at
 * most 2^24 records (sum of gaussian_count over the views); more records
 * return MG_ERR_INVALID_ARG.  The array (about 64 KB) is held on every GPU
 * that loads the library until the process exits.  The first call on each
 * device looks up the array's device address (with that device current) and
 * caches it; make that first call before any stream capture.  The cached
 * address does not survive cudaDeviceReset: do not call this function on a
 * device after resetting it in the same process.  Every call shares the one
 * array, so calls that overlap on the GPU (other streams, other threads) race:
 * serialise them.  Nothing is allocated: no cudaMalloc, no cudaFree. */
mg_status mg_bin_noalloc(const mg_splats *splats, const mg_view *views, int32_t n_views,
                         const mg_raster_cfg *cfg, const uint32_t *order, uint32_t *offsets,
                         uint32_t *keys, uint32_t *vals, uint64_t capacity,
                         uint64_t *d_num_instances, mg_status_word *d_status,
                         mg_stream_t stream);

/* ---- 3. sort + tile ranges (Sec. 3.1) -------------------------------------- */
/* Stable LSD radix sort (8-bit digits, single-pass "onesweep" passes with
 * decoupled look-back) of the first *d_num_instances (tile id, value) pairs by
 * the low key_bits bits of the tile id (mg_tile_bits); pairs whose key is
 * 0xFFFFFFFF (filtered by mg_bin) are dropped in the first pass, and the
 * number kept is written to *d_num_sorted (device u64, nullable).  Then
 * ranges[t] = [start, end) of the kept instances of global tile t
 * (n_tiles_total = sum of all views' tiles).  With the instances emitted in
 * depth order (mg_depth_order, then mg_bin), each tile's list comes out
 * ordered by (depth, record index) -- the order a full sort of 64-bit
 * (tile, depth) keys of record-ordered instances gives.  The sorted pairs end
 * in (keys, vals) when *result_in_alt (host int) is set to 0, else in
 * (keys_alt, vals_alt); it is known on the host from key_bits alone.  When
 * *d_num_instances exceeds capacity (mg_bin raised MG_ERR_CAPACITY) nothing is
 * sorted and every range is empty.  workspace: mg_sort_workspace_bytes(
 * capacity, key_bits) bytes, any content.  key_bits: 1..32 with
 * n_tiles_total <= 2^key_bits; capacity < 2^30.  The first call on a device
 * (of this or of mg_depth_order) sets the sort kernels' shared-memory limit:
 * make it outside stream capture. */
mg_status mg_sort(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                  const uint64_t *d_num_instances, uint64_t capacity, int32_t key_bits,
                  uint32_t *ranges, int64_t n_tiles_total, void *workspace,
                  size_t workspace_bytes, int32_t *result_in_alt, uint64_t *d_num_sorted,
                  mg_status_word *d_status, mg_stream_t stream);
size_t mg_sort_workspace_bytes(uint64_t capacity, int32_t key_bits);
/* The lists of mg_sort by another route, one pass over the whole tile id
 * (Sec. 3.1: each tile's Gaussians in depth order), that needs no depth order
 * of the records beforehand: the instances (keys = global tile ids, vals =
 * record indices, as mg_bin writes them, in any order -- mg_bin with a null
 * order emits them in record order) are grouped by tile by a counting pass
 * (per-tile counts, their scan, then a scatter of each tile's instances into
 * its range), and every tile's list is then ordered by (depth_key[record],
 * record) -- depth_key as mg_preprocess writes it (device u32[R], required).
 * Pairs keyed 0xFFFFFFFF are dropped.  Outputs: sorted_vals (u32[capacity]):
 * the records of tile t at [ranges[2t], ranges[2t+1]); *d_num_sorted
 * (nullable) = the number kept.  The lists equal mg_sort's on depth-ordered
 * instances bit for bit.  workspace: mg_sort_by_tile_workspace_bytes(
 * capacity, n_tiles_total) bytes, 16-byte aligned, any content.  When
 * *d_num_instances exceeds capacity nothing is sorted and every range is
 * empty.  Lists of up to 4096 records are ordered in shared memory, longer
 * ones in 4096-record chunks merged in the workspace.  The first call on a
 * device sets the kernels' shared-memory limit: make it outside stream
 * capture. */
mg_status mg_sort_by_tile(const uint32_t *keys, const uint32_t *vals, const uint32_t *depth_key,
                          const uint64_t *d_num_instances, uint64_t capacity,
                          int64_t n_tiles_total, uint32_t *sorted_vals, uint32_t *ranges,
                          void *workspace, size_t workspace_bytes, uint64_t *d_num_sorted,
                          mg_status_word *d_status, mg_stream_t stream);
size_t mg_sort_by_tile_workspace_bytes(uint64_t capacity, int64_t n_tiles_total);
/* Bits of a global tile id for a set of views: ceil(log2(n_tiles_total)), >= 1. */
int32_t mg_tile_bits(const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg);
int64_t mg_total_tiles(const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg);

/* ---- 4. render forward (Eq. 3-4) -------------------------------------------- */
/* Longest-first launch order of the tiles (all render calls take it):
 * tile_order[n_tiles_total] (u32) = the global tile ids, tiles with longer
 * lists first (by quarter-octave length classes; the order within a class is
 * unspecified).  One CTA renders one tile, so this only changes which tile
 * starts first (list scheduling, longest first), never a result.  ranges:
 * from mg_sort, 8-byte aligned. */
mg_status mg_tile_order(const uint32_t *ranges, int64_t n_tiles_total, uint32_t *tile_order,
                        mg_stream_t stream);

/* Per pixel, front to back over its tile's range: alpha = min(0.99,
 * o exp(power)); splats with alpha < 1/255 are skipped (masked or not);
 * test T' = T (1 - M alpha); if T' < 1e-4 blending stops before this splat;
 * else C += M alpha T c, T = T'.  Finally C += T bg.
 * Outputs: image[3][H][W] per view (at 3 P_v), final_T[H][W] and
 * n_contrib[H][W] per view (at P_v): n_contrib is the index in the tile's
 * list where blending stopped (the list length if it did not).
 * frag_count (nullable): device u64[4] of counters, accumulated (+=), taken
 * by a slower counting variant of the kernel: [0] (pixel, splat) pairs walked
 * (the sum of n_contrib, the pairs both render kernels evaluate), [1] of which
 * unmasked, [2] unmasked splats blended, [3] masked splats at or above the
 * alpha floor (the ones that receive dL/dM).
 * tile_order (nullable: tile-id order): from mg_tile_order. */
mg_status mg_render(const mg_splats *splats, const uint32_t *sorted_vals,
                    const uint32_t *ranges, const uint32_t *tile_order, const mg_view *views,
                    int32_t n_views, const mg_raster_cfg *cfg, float *image, float *final_T,
                    uint32_t *n_contrib, uint64_t *frag_count, mg_stream_t stream);

/* mg_render with the L1 render loss taken in the same kernel, from the
 * colours it has just composited (no second pass over the image): as
 * mg_render (without fragment counters), plus, for every view v and value i
 * of its image, dL_dimage[i] = sign(image[i] - target[i]) / (3 W_v H_v)
 * (sign(0) = 0) and *loss (device f32) += sum_v mean |image_v - target_v| --
 * the results of mg_l1_loss_grad, the loss summed in another order.  The
 * caller zeroes *loss.  target, dL_dimage: f32[sum_v 3 W_v H_v]. */
mg_status mg_render_l1(const mg_splats *splats, const uint32_t *sorted_vals,
                       const uint32_t *ranges, const uint32_t *tile_order,
                       const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg,
                       float *image, float *final_T, uint32_t *n_contrib, const float *target,
                       float *dL_dimage, float *loss, mg_stream_t stream);

/* mg_render_l1 that also zeroes grad2d[R][12] (16-byte aligned), the
 * accumulator of the render backward, for mg_render_backward_accumulate: the
 * render kernel's CTAs store the zeros while they render (its memory path is
 * nearly idle), so the training step needs no separate reset between the
 * render and its backward.  No paper counterpart: a scheduling choice. */
mg_status mg_render_l1_reset2d(const mg_splats *splats, const uint32_t *sorted_vals,
                               const uint32_t *ranges, const uint32_t *tile_order,
                               const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg,
                               float *image, float *final_T, uint32_t *n_contrib,
                               const float *target, float *dL_dimage, float *loss, float *grad2d,
                               mg_stream_t stream);

/* ---- 5. L1 render loss ------------------------------------------------------ */
/* For count = sum_v 3 W_v H_v values: dL_dimage[i] = sign(image[i] - target[i])
 * / (3 W_v H_v) of the view holding i (sign(0) = 0), and *loss (device f32)
 * += sum_v mean |image_v - target_v|.  The caller zeroes *loss.  image, target
 * and dL_dimage: 16-byte aligned. */
mg_status mg_l1_loss_grad(const float *image, const float *target, const mg_view *views,
                          int32_t n_views, float *dL_dimage, float *loss,
                          mg_stream_t stream);

/* ---- 6. render backward (Eq. 6, Appendix A) --------------------------------- */
/* Back-to-front replay of each pixel from n_contrib, recovering T_i =
 * T_{i+1} / (1 - M_i alpha_i) from final_T.  With b_{N+1} = bg and
 * b_i = M_i alpha_i c_i + (1 - M_i alpha_i) b_{i+1} (the colour behind and at
 * i, background folded in):
 *   dL/dM_i     = alpha_i T_i g.(c_i - b_{i+1})   (Eq. 6 + Appendix A)
 *   dL/dalpha_i = M_i T_i g.(c_i - b_{i+1})       (0 for a masked splat)
 *   dL/dc_i     = M_i alpha_i T_i g,   g = dL/dC,
 * then through the 0.99 clamp to opacity, conic and 2D mean.
 * grad2d[R][12] is ZEROED by this call and then accumulated.
 * counters (nullable): device u64[6] of profiling counters, accumulated, taken
 * by a slower counting variant: [0] (warp, splat) iterations after culling,
 * [1] of which masked, [2] unmasked with at least one contributing pixel,
 * [3] masked with one, [4] contributing pixels summed over [2], [5] batches.
 * tile_order (nullable): as for mg_render. */
mg_status mg_render_backward(const mg_splats *splats, const uint32_t *sorted_vals,
                             const uint32_t *ranges, const uint32_t *tile_order,
                             const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg,
                             const float *final_T, const uint32_t *n_contrib,
                             const float *dL_dimage, float *grad2d, uint64_t *counters,
                             mg_stream_t stream);

/* The same, adding into grad2d instead of zeroing it first: the caller provides
 * it zeroed (mg_render_l1_reset2d does so while it renders). */
mg_status mg_render_backward_accumulate(const mg_splats *splats, const uint32_t *sorted_vals,
                                        const uint32_t *ranges, const uint32_t *tile_order,
                                        const mg_view *views, int32_t n_views,
                                        const mg_raster_cfg *cfg, const float *final_T,
                                        const uint32_t *n_contrib, const float *dL_dimage,
                                        float *grad2d, uint64_t *counters, mg_stream_t stream);

/* ---- 7. preprocess backward ------------------------------------------------- */
/* Chain rule from grad2d through the 2D covariance (P = J W R S), the
 * quaternion normalisation, the scale exponential, the projection and the
 * SH colour (zero for clamped channels) to every parameter, summed over
 * views.  dL/dM_i is the sum over views of grad2d's dM (MG_APPLY_RASTER) or
 * o_i times the sum of dL/do' (MG_APPLY_OPACITY, where opacity_logit receives
 * M_i dL/do' sigma'), plus lambda_m dL_m/dM_i of the Gaussian's scene (first
 * view whose range holds i): 2 count / N^2 (L2) or 1 / N (L1), from
 * splats->mask_count.  mask_logits receive dL/dM y_0 (1 - y_0) / tau and its
 * negative (straight-through Gumbel-softmax, Sec. 3.3) for MG_MASK_GUMBEL,
 * dL/dM p (1 - p) and its negative with p = sigmoid(l_0 - l_1) for
 * MG_MASK_STE, zero otherwise.  Outputs are overwritten. */
mg_status mg_preprocess_backward(const mg_gaussians *g, const mg_view *views,
                                 int32_t n_views, const mg_raster_cfg *cfg,
                                 const mg_splats *splats, const float *grad2d,
                                 const mg_param_grads *out, mg_stream_t stream);

/* ---- 8. mask loss (Sec. 3.5, Eq. 7-8) ----------------------------------------- */
/* *iteration_dev += by on the stream (one thread), for the mask sample's
 * device-side iteration (mg_raster_cfg.iteration_dev, Sec. 3.3: a new
 * Gumbel sample every training step): enqueued after a step, it advances the
 * counter the next step reads, also inside a captured CUDA graph. */
mg_status mg_advance_iteration(uint64_t *iteration_dev, uint64_t by, mg_stream_t stream);

/* *loss (device f32) += lambda_m * sum over scenes of L_m, from
 * splats->mask_count (a scene = a distinct Gaussian range among the views,
 * N = its gaussian_count; empty ranges add nothing).  The gradient is added
 * by mg_preprocess_backward.  One tiny kernel; the caller zeroes *loss. */
mg_status mg_mask_loss(const mg_splats *splats, const mg_view *views, int32_t n_views,
                       const mg_raster_cfg *cfg, float *loss, mg_stream_t stream);

/* ---- 9. pruning (Sec. 3.5) ------------------------------------------------------- */
/* Draws n_draws (1..1024) independent masks per Gaussian and keeps the
 * Gaussians sampled present at least once: keep[i] = OR_d [l_0 + g_0 >=
 * l_1 + g_1] (u8 0/1), draw d with Philox counter (i, iteration_lo,
 * iteration_hi, d + 1) and key (seed_lo, seed_hi) -- disjoint from the
 * training draws (last counter word 0) -- and the same FP32 decision as
 * mg_preprocess.  The paper draws 10 times.  g->mask_logits is read (FP32). */
mg_status mg_prune_sample(const mg_gaussians *g, uint64_t seed, uint64_t iteration,
                          int32_t n_draws, uint8_t *keep, mg_stream_t stream);

/* Writable Gaussian arrays, laid out as in mg_gaussians with the same dtype. */
typedef struct {
    void *means;
    void *log_scales;
    void *quats;
    void *opacity_logit;
    void *sh;
    void *mask_logits;
} mg_gaussian_arrays;

/* Stream compaction of every attribute array of src to dst (rows with
 * keep[i] != 0, order kept; dst has room for src->n rows and must not
 * overlap src): *d_n_kept (device i64) = number kept, new_index[i] (device
 * i32, nullable) = row of i in dst or -1.  Single-pass scan with decoupled
 * look-back; a wait that gives up raises MG_ERR_TIMEOUT in d_status.
 * workspace: mg_compact_workspace_bytes(n) bytes, any content. */
mg_status mg_compact(const mg_gaussians *src, const uint8_t *keep, const mg_gaussian_arrays *dst,
                     int32_t *new_index, int64_t *d_n_kept, void *workspace,
                     size_t workspace_bytes, mg_status_word *d_status, mg_stream_t stream);
size_t mg_compact_workspace_bytes(int64_t n);

/* ---- 10. inference render (Sec. 4.2, rendering speed) ----------------------- */
/* Forward-only blend of splats made with MG_MASK_ALL_ONES (a pruned model
 * renders every Gaussian it keeps; masked records, if any, are skipped):
 * image[3][H][W] per view, as mg_render, without final_T and n_contrib.
 * tile_order (nullable): as for mg_render. */
mg_status mg_render_inference(const mg_splats *splats, const uint32_t *sorted_vals,
                              const uint32_t *ranges, const uint32_t *tile_order,
                              const mg_view *views, int32_t n_views, const mg_raster_cfg *cfg,
                              float *image, mg_stream_t stream);

/* ---- checks ------------------------------------------------------------------- */
/* Validates the tile lists the render calls consume (the paper has no
 * counterpart; a check in place of a memory sanitiser): for every tile t the
 * range [ranges[2t], ranges[2t+1]) is ordered and inside [0, *d_num_sorted),
 * the non-empty ranges of consecutive tiles do not overlap and their lengths
 * sum to *d_num_sorted, and every value sorted_vals[i] < n_records is a
 * record index.  A violation raises MG_ERR_BOUNDS in *d_status (detail 7:
 * a range, 8: a value, 9: the total; required = the offending tile, position
 * or total).  Only reads inside the given buffers: sorted_vals holds at least
 * *d_num_sorted values (nothing past capacity is read), ranges 2
 * n_tiles_total values.
 *
 * Builds with MG_DEBUG_BOUNDS defined (the library's debug build) also check,
 * inside the binning and sort kernels, every computed write position against
 * its buffer (a scatter slot against the instance count or capacity, a
 * duplication chunk's owner against the record count) and skip an
 * out-of-range write, raising MG_ERR_BOUNDS with the bad index. */
mg_status mg_validate_lists(const uint32_t *sorted_vals, const uint32_t *ranges,
                            int64_t n_tiles_total, const uint64_t *d_num_sorted,
                            uint64_t capacity, int64_t n_records, mg_status_word *d_status,
                            mg_stream_t stream);

/* ---- helpers ------------------------------------------------------------------ */
/* Synchronises `stream` and copies the device status word to *h_out (host). */
mg_status mg_read_status(const mg_status_word *d_status, mg_status_word *h_out,
                         mg_stream_t stream);
const char *mg_status_string(int32_t status);
const char *mg_version(void);

/* Self-test of the bounded device-side waits (the paper has no counterpart):
 * one thread runs the library's decoupled look-back on a flag that nothing
 * ever sets; after max_polls polls (0..2^24, each with a short sleep) it gives
 * up and raises MG_ERR_TIMEOUT with detail 4 in *d_status.  The context stays
 * usable; read the word with mg_read_status. */
mg_status mg_selftest_wait_timeout(int32_t max_polls, mg_status_word *d_status,
                                   mg_stream_t stream);

/* The same for the warp-wide look-back of the single-pass scans (the tile
 * count scan of mg_bin, the compaction of mg_compact): one warp waits for 32
 * predecessors that never publish; MG_ERR_TIMEOUT with detail 5. */
mg_status mg_selftest_warp_wait_timeout(int32_t max_polls, mg_status_word *d_status,
                                        mg_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MASKGS_H */
