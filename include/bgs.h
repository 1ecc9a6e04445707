/*
 * bgs.h -- C ABI of the balanced Gaussian-splat renderer (libbgs.so, sm_103a).
 *
 * The library implements the data-parallel hot path of Balanced 3DGS (Gui et al.,
 * arXiv 2412.17378): the tile-based front-to-back alpha-compositing render kernel of
 * 3D Gaussian Splatting ("renderCUDA"), its backward pass, and the projection and
 * binning steps that produce its inputs.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every array argument is a DEVICE pointer to caller-owned, contiguous memory
 *    (float32 / int32 / uint32 as typed), unless the comment says "host".  The library
 *    never frees caller memory and never keeps a caller pointer after the call returns.
 *  - `stream` is a cudaStream_t passed as void*; every call only enqueues work on it
 *    (except where a comment says the call synchronises).  NULL = legacy default stream.
 *  - Scratch memory (sort buffers, work lists, queue counters, gradient accumulators)
 *    belongs to the plan.  It is allocated with cudaMalloc on first need and grown on
 *    later calls; bgs_plan_reserve() sizes it up front.  Nothing is allocated while the
 *    stream is being captured into a CUDA graph: a call that would need to grow the
 *    workspace then fails with BGS_ERR_CAPACITY.
 *  - A plan may be used by one host thread and one stream at a time.
 *  - Return value: BGS_OK or a negative status.  bgs_last_error() gives a message
 *    (thread-local).  Outputs are unspecified after a failed call.
 *  - Image outputs are planar: color is [3, H, W], the others [H, W].
 *  - Pixel (x, y) is evaluated at coordinates (x, y) of the means2D frame.
 *
 * Per-pair rule (Eq. 3-4 and Algorithm 5, Appendix A of the paper; constants from
 * standard 3DGS since the paper omits them): for the depth-sorted Gaussians of the
 * pixel's tile, power = -1/2 (a dx^2 + c dy^2) - b dx dy with d = mean - pixel; skip if
 * power > 0; alpha = min(0.99, o exp(power)); skip if alpha < 1/255; T' = T (1 - alpha);
 * stop before accumulating if T' < 1e-4; else C += c alpha T, D += depth alpha T,
 * A += alpha T, T = T'.  Finally C += T bg.
 */
#ifndef BGS_H
#define BGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define BGS_OK 0
#define BGS_ERR_INVALID (-1)      /* bad argument (null pointer, size, tile shape, mode)   */
#define BGS_ERR_CAPACITY (-2)     /* caller buffer or plan workspace too small; see needed */
#define BGS_ERR_CUDA (-3)         /* a CUDA runtime call failed                             */
#define BGS_ERR_DEVICE_CHECK (-4) /* a device-side check tripped (reported by bgs_check)    */

/* Largest point-list length (num_entries, binning's K) any call accepts: list positions
   stay below 2^32 with room for the kernels' strides of up to 1024 entries. */
#define BGS_MAX_ENTRIES 4294963200LL /* 2^32 - 4096 */

/* ---- device-check bits (bgs_check / bgs_plan_stats) -------------------------------- */
#define BGS_CHECK_INDEX 1u        /* point_list held an index >= N                         */
#define BGS_CHECK_RANGE 2u        /* a tile range pointed past num_entries                 */
#define BGS_CHECK_OVERFLOW 4u     /* binning produced more entries than the capacity        */
#define BGS_CHECK_QUEUE 8u        /* a persistent pass did not run every queued item once   */

/* ---- render modes (Sec. 4 of the paper and its selector, Sec. 4.4) ------------------ */
#define BGS_MODE_AUTO 0     /* persistent queue; per-tile choice: Gaussian-wise for tiles whose
                               list is longer than plan.heavy_threshold, else pixel-wise        */
#define BGS_MODE_PIXEL 1    /* persistent queue (Sec. 4.1), every item pixel-wise               */
#define BGS_MODE_GAUSSIAN 2 /* persistent queue, every item Gaussian-wise (Sec. 4.2-4.3)        */
#define BGS_MODE_STATIC 3   /* plain pixel-wise static grid, one block per tile (Algorithm 4)  */
#define BGS_MODE_SELECT 4   /* self-adaptive selection (Sec. 4.4), single-view calls: render with
                               the balanced kernels (AUTO); every plan.select_period forward
                               calls, starting with the first, time the balanced forward against
                               the static pixel-wise forward on the call's frame (both run; the
                               outputs are the same); once the balanced forward is slower, use
                               the static kernels for every later call (irreversible, until
                               bgs_plan_selector_reset).  No measurement is taken while the
                               stream is being captured (timing needs a host synchronisation). */

/* ---- camera (Eq. 2: W = viewmat rotation, J = Jacobian of the pinhole map) ---------- */
typedef struct bgs_camera {
    int32_t width, height;   /* image size in pixels                                      */
    float fx, fy, cx, cy;    /* pinhole intrinsics: u = fx x/z + cx, v = fy y/z + cy       */
    float viewmat[16];       /* row-major 4x4 world->camera transform (camera looks at +z) */
    float near_plane;        /* Gaussians with camera z <= near_plane are culled (0.2)     */
    float lowpass;           /* added to the diagonal of the 2D covariance (0.3)           */
} bgs_camera;

/* ---- plan: tuning knobs + owned workspace ----------------------------------------- */
typedef struct bgs_plan_desc {
    int32_t heavy_threshold; /* AUTO mode: list length above which a tile is Gaussian-wise
                                (2147483647: no tile is)                                    */
    int32_t gw_pixels;       /* pixels one Gaussian-wise warp item covers: 1, 2, 4, 8 or 16 */
    int32_t queue_chunk;     /* work items a warp claims per atomicAdd on the queue (>= 1)  */
    int32_t blocks_per_sm;   /* persistent grid = SMs x blocks_per_sm; 0 = max resident     */
    int32_t lpt_order;       /* 1: work items ordered heaviest tile first (lengths in ~19 %
                                log buckets); 0: by kind only.  Gaussian-wise tiles come
                                first either way; tiles of one bucket come in no set order */
    int32_t device;          /* CUDA device ordinal; -1 = the current device at creation    */
    int32_t pixel_rows;      /* sub-tile of a pixel-wise item: 8 x (4 pixel_rows) pixels, one
                                warp, pixel_rows pixels per lane (1, 2 or 4)                 */
    int32_t select_period;   /* BGS_MODE_SELECT: forward calls between two timings (>= 1)   */
    int32_t bin_block;       /* binning: Gaussians per counting block, a multiple of 32, or 0
                                for automatic (>= 2048, about 4 blocks per SM, enough to
                                bound the tile histogram); changes speed only, not the lists */
    int32_t gw_segment;      /* Gaussian-wise tiles: list entries per segment (a multiple of
                                256, 256 .. 2^30; 2048).  A longer list is split into segments
                                walked by separate warps, and a merge pass composes each
                                pixel's segments (its stop taken by the sequential rule); the
                                split is skipped (one segment per tile) when it would need more
                                than 2^24 items or one per (segment, pixel group) over
                                num_entries / gw_segment segments                           */
} bgs_plan_desc;

typedef struct bgs_plan bgs_plan;

/* Counters accumulated by the render kernels since the last bgs_plan_reset_stats(). */
typedef struct bgs_stats {
    uint64_t eval_pairs;     /* (pixel, list entry) pairs the sequential rule visits       */
    uint64_t contrib_pairs;  /* pairs accumulated into a pixel                              */
    uint64_t items;          /* work items executed by the persistent kernels               */
    uint32_t check_bits;     /* BGS_CHECK_* bits raised by device checks                    */
    uint32_t last_num_items; /* work items in the last work list                            */
    uint64_t host_launches;  /* kernels of this library launched through the plan so far,
                                not counting the sort / scan kernels of the CUB library     */
} bgs_stats;

/* Fills *desc with defaults (threshold 512, 4 px per Gaussian-wise item, chunk 1,
   max resident blocks, LPT order on, current device, 2 pixel rows per lane, selector
   timing every 1000 forward calls, automatic binning blocks). */
void bgs_plan_desc_default(bgs_plan_desc *desc);
/* Creates a plan bound to desc->device.  Allocates a small device control block. */
int bgs_plan_create(const bgs_plan_desc *desc, bgs_plan **out);
int bgs_plan_destroy(bgs_plan *plan);
/* Replaces the tuning knobs (device unchanged). */
int bgs_plan_set(bgs_plan *plan, const bgs_plan_desc *desc);
int bgs_plan_get(const bgs_plan *plan, bgs_plan_desc *desc);
/* Grows the workspace for up to max_gaussians Gaussians, max_entries duplicated
   (Gaussian, tile) entries, max_tiles tiles and max_pixels pixels (all views together). */
int bgs_plan_reserve(bgs_plan *plan, int64_t max_gaussians, int64_t max_entries, int64_t max_tiles,
                     int64_t max_pixels);
/* Workspace bytes bgs_plan_reserve would hold for these sizes. */
size_t bgs_workspace_size(const bgs_plan *plan, int64_t max_gaussians, int64_t max_entries,
                          int64_t max_tiles, int64_t max_pixels);
/* Synchronises `stream`; returns BGS_ERR_DEVICE_CHECK (and clears the bits) if a device
   check tripped since the last call, else BGS_OK. */
int bgs_check(bgs_plan *plan, void *stream);
/* Synchronises `stream` and copies the counters (host pointer). */
int bgs_plan_stats(bgs_plan *plan, bgs_stats *out, void *stream);
int bgs_plan_reset_stats(bgs_plan *plan, void *stream);
/* Turns CUDA-event timing of the render kernels on (1) or off (0).  While on, every
   forward / backward render-kernel launch outside stream capture is bracketed by two
   events on the launching stream. */
int bgs_plan_timing(bgs_plan *plan, int enable);
/* Sums the recorded forward / backward kernel durations (ms) and their launch counts,
   then forgets them (waits for the recorded events). */
int bgs_plan_kernel_ms(bgs_plan *plan, double *fwd_ms, int32_t *fwd_n, double *bwd_ms, int32_t *bwd_n);
/* Number of SMs of the plan's device (host). */
int bgs_plan_num_sms(const bgs_plan *plan);
/* State of the BGS_MODE_SELECT selector (all outputs host, nullable): *switched = 1 once
   the static kernels were chosen; *calls = forward calls in SELECT mode; *measurements =
   timings taken; *last_balanced_ms / *last_static_ms = the last timing of each forward. */
int bgs_plan_selector(const bgs_plan *plan, int32_t *switched, int64_t *calls, int64_t *measurements,
                      double *last_balanced_ms, double *last_static_ms);
/* Restarts the selector: balanced kernels, no calls, no measurements. */
int bgs_plan_selector_reset(bgs_plan *plan);
/* Restores a selector state read with bgs_plan_selector (resuming a run from a checkpoint):
   switched 0 / 1, calls and measurements >= 0, the last timings >= 0. */
int bgs_plan_selector_restore(bgs_plan *plan, int32_t switched, int64_t calls, int64_t measurements,
                              double last_balanced_ms, double last_static_ms);
/* Fault injection for tests, on the host side (nothing faults on the device): which =
   BGS_CHECK_QUEUE marks every item of the next persistent pass's queue as already taken,
   so that pass renders nothing and its drain check raises BGS_CHECK_QUEUE, reported by the
   next bgs_check.  One-shot. */
int bgs_plan_inject_fault(bgs_plan *plan, uint32_t which);
const char *bgs_last_error(void);

/* ---- a1: projection (Eq. 1-3) ------------------------------------------------------
   Per Gaussian i: camera-space p = V [mean, 1]; culled if p.z <= near_plane.
   Sigma = R S S^T R^T with R from the normalised quaternion (w, x, y, z) and
   S = diag(exp(log_scale)); Sigma' = J W Sigma W^T J^T + lowpass I with J the
   Jacobian of the pinhole map at the tangent-clamped point (|x/z| <= 1.3 W/(2 fx)).
   Outputs: means2D [N,2] = (fx x/z + cx, fy y/z + cy); conic_opacity [N,4] =
   (a, b, c, o) with (a b; b c) = Sigma'^-1 and o = opacities[i]; depths [N] = p.z;
   radii [N] = ceil(3 sqrt(lambda_max)) with the eigenvalue discriminant floored at 0.1
   (0 when culled or when the Gaussian touches no tile); tiles_touched [N] = area of the
   tile rectangle (see bgs_bin_and_sort).  Inputs: means3D [N,3], log_scales [N,3],
   quats [N,4], opacities [N] (already in (0,1)).  cam is a host pointer. */
int bgs_preprocess(bgs_plan *plan, int64_t N, const float *means3D, const float *log_scales,
                   const float *quats, const float *opacities, const bgs_camera *cam, int32_t tile_w,
                   int32_t tile_h, float *means2D, float *conic_opacity, float *depths, int32_t *radii,
                   uint32_t *tiles_touched, void *stream);

/* ---- projection backward (the chain rule through Eq. 2-3; the paper prints none) ---
   Given dL/dmeans2D [N,2] (8-byte aligned), dL/dconic [N,3] (w.r.t. a, b, c as output by
   bgs_preprocess and consumed by the render; bgs_render_backward's dL_dconic) and
   dL/ddepths [N] (nullable), writes dL/dmeans3D [N,3], dL/dlog_scales [N,3] and
   dL/dquats [N,4] (w.r.t. the unnormalised input quaternion), overwriting them.  The
   projection is recomputed from the same inputs and camera as bgs_preprocess; Gaussians
   whose radii[i] is 0 (culled, or touching no tile) get zero.  The tangent clamp passes no
   gradient to the clamped coordinate.  The opacity and colour gradients of the render
   need no projection step (the render consumes opacities and colours as given). */
int bgs_preprocess_backward(bgs_plan *plan, int64_t N, const float *means3D, const float *log_scales,
                            const float *quats, const bgs_camera *cam, const int32_t *radii,
                            const float *dL_dmeans2D, const float *dL_dconic, const float *dL_ddepths,
                            float *dL_dmeans3D, float *dL_dlog_scales, float *dL_dquats, void *stream);

/* ---- a2: binning: per-tile depth-ordered lists (point_list of Algorithms 1-6) --------
   Gaussian i with radius r > 0 covers the tiles x in [floor((u-r)/tw),
   floor((u+(r+tw-1))/tw)), y likewise, clamped to the tile grid (float32, one rounding
   per operation).  Tile t's list holds the Gaussians covering t ordered by (float32
   depth bits, i) -- what a stable sort of (tile << 32 | depth bits, i) keys over all
   covered (tile, Gaussian) pairs gives; it is built by a depth sort of the N Gaussians
   and a counting sort over their tile rectangles (a stable radix sort on the tile id
   when the tile grid is too large for the counters).  point_list [capacity] receives
   the lists one after the other and ranges [T,2] (T = tiles_x * tiles_y) the half-open
   span of each tile (0,0 if empty).
   List truncation: when conic_opacity [N,4] (the render's conics and opacities, 16-byte
   aligned) is given, each tile's list is cut after the depth block of Gaussians at whose
   end every pixel of the tile is certified to have stopped (Algorithm 5 stops a pixel at
   the first pair that takes its transmittance below 1e-4; the entries behind that point
   are never read by the render, forward or backward).  The certificate is a product of
   factors 1 - a over the tile's Gaussians whose alpha is at least a at every pixel of the
   tile, at three opacity-relative levels a, below 1e-5; it never cuts an entry that the
   render's sequential rule visits, so every render output (images, n_contrib, n_eval,
   gradients) is the same as with the full lists.  Each kept list is a prefix of the full
   list.  Without conic_opacity (NULL), or on a tile grid whose counters do not fit in
   shared memory, the lists are complete.
   If the entry count K exceeds `capacity`, *needed (host, nullable) receives K,
   BGS_ERR_CAPACITY is returned and point_list / ranges are unspecified (nothing is
   written past capacity).  *num_rendered (host, nullable) receives K.  This call
   synchronises the stream once, at its end, to read K. */
int bgs_bin_and_sort(bgs_plan *plan, int64_t N, const float *means2D, const int32_t *radii,
                     const float *depths, const float *conic_opacity, int32_t W, int32_t H, int32_t tile_w,
                     int32_t tile_h, uint32_t *point_list, int64_t capacity, uint32_t *ranges,
                     int64_t *num_rendered, int64_t *needed, void *stream);

/* ---- a3-a5: render forward -------------------------------------------------------
   Inputs (the paper's XY, CO, F, D, PL): means2D [N,2], conic_opacity [N,4],
   colors [N,3], depths [N], point_list [num_entries] (values < N, num_entries <=
   BGS_MAX_ENTRIES), ranges [T,2].
   bg: host float[3].  Outputs (OC, OD, OA): out_color [3,H,W], out_depth [H,W],
   out_alpha [H,W] (= sum of weights = 1 - final_T), final_T [H,W], n_contrib [H,W]
   (list position + 1 of the last accumulated pair, 0 if none), n_eval [H,W] (nullable:
   pairs the sequential rule visits).  mode: BGS_MODE_*.  All modes give the same result
   up to float32 reassociation. */
int bgs_render_forward(bgs_plan *plan, int64_t N, const float *means2D, const float *conic_opacity,
                       const float *colors, const float *depths, const uint32_t *point_list,
                       int64_t num_entries, const uint32_t *ranges, int32_t W, int32_t H, int32_t tile_w,
                       int32_t tile_h, const float *bg, int32_t mode, float *out_color, float *out_depth,
                       float *out_alpha, float *final_T, int32_t *n_contrib, int32_t *n_eval, void *stream);

/* ---- a6: render backward ----------------------------------------------------------
   Gradient of L through the forward above, recomputing the blend back to front from
   final_T and n_contrib (no per-pair state is stored).  Inputs: the forward's inputs,
   its final_T / n_contrib, dL_dcolor [3,H,W], dL_ddepth [H,W] (nullable),
   dL_dalpha [H,W] (nullable).  Outputs (overwritten): dL_dmeans2D [N,2],
   dL_dconic [N,3] (w.r.t. a, b, c exactly as used in power), dL_dopacity [N],
   dL_dcolors [N,3], dL_ddepths [N] (nullable).  Where o exp(power) > 0.99 the alpha
   clamp is active and the pair passes no gradient to o or to the Gaussian's shape.
   The arrays must hold what the forward read (final_T and n_contrib only describe that
   blend).  When they are the same arrays (pointers and sizes) as the plan's last forward,
   its packed records are reused instead of being rebuilt; and when that forward split
   Gaussian-wise lists into segments (same render mode and knobs), the backward walks
   those tiles segment by segment from the boundary states it left in the plan.  The
   backward's own work list is ordered heaviest first by each tile's largest n_contrib
   (built once and reused by later backwards on the same list key). */
int bgs_render_backward(bgs_plan *plan, int64_t N, const float *means2D, const float *conic_opacity,
                        const float *colors, const float *depths, const uint32_t *point_list,
                        int64_t num_entries, const uint32_t *ranges, int32_t W, int32_t H, int32_t tile_w,
                        int32_t tile_h, const float *bg, int32_t mode, const float *final_T,
                        const int32_t *n_contrib, const float *dL_dcolor, const float *dL_ddepth,
                        const float *dL_dalpha, float *dL_dmeans2D, float *dL_dconic, float *dL_dopacity,
                        float *dL_dcolors, float *dL_ddepths, void *stream);

/* ---- a7: batched views (many cameras of one Gaussian set) and graph capture ----------
   A batched call renders V <= 32 views of N Gaussians in one persistent launch (the task
   pool of Sec. 4.1 spans all views).  Record v * N + g is Gaussian g seen from view v:
   per-record arrays (means2D, conic_opacity, depths, radii and their gradients) are
   [V * N, ...], view-major; colors [N, 3] are shared by the views.  The views' tiles form
   one global tile space, view v owning tile ids [sum_{u<v} T_u, sum_{u<=v} T_u) with
   T_u its tiles_x * tiles_y; ranges is [sum T_u, 2] and point_list holds record indices. */
typedef struct bgs_view {
    bgs_camera cam;                           /* host: camera and image size of the view     */
    float *out_color, *out_depth, *out_alpha; /* forward outputs [3,H,W], [H,W], [H,W]        */
    float *final_T;                           /* forward output [H,W], backward input         */
    int32_t *n_contrib;                       /* forward output [H,W], backward input         */
    int32_t *n_eval;                          /* forward output [H,W], nullable                */
    const float *dL_dcolor;                   /* backward input [3,H,W]                       */
    const float *dL_ddepth, *dL_dalpha;       /* backward inputs [H,W], nullable              */
} bgs_view;

#define BGS_BIN_NO_SYNC 1 /* bin_and_sort_batched: no host synchronisation (graph capture); an
                             entry count past capacity raises BGS_CHECK_OVERFLOW instead */

/* Projection (as bgs_preprocess) of N Gaussians into V views; views[] is a host array (only
   cam is read).  Outputs are [V * N, ...]. */
int bgs_preprocess_batched(bgs_plan *plan, int32_t V, const bgs_view *views, int64_t N, const float *means3D,
                           const float *log_scales, const float *quats, const float *opacities, int32_t tile_w,
                           int32_t tile_h, float *means2D, float *conic_opacity, float *depths, int32_t *radii,
                           uint32_t *tiles_touched, void *stream);
/* Projection backward of the batched projection: records v * N + g (radii, dL_dmeans2D,
   dL_dconic, dL_ddepths are [V * N, ...]); the gradients of Gaussian g [N, ...] are summed
   over the views. */
int bgs_preprocess_backward_batched(bgs_plan *plan, int32_t V, const bgs_view *views, int64_t N,
                                    const float *means3D, const float *log_scales, const float *quats,
                                    const int32_t *radii, const float *dL_dmeans2D, const float *dL_dconic,
                                    const float *dL_ddepths, float *dL_dmeans3D, float *dL_dlog_scales,
                                    float *dL_dquats, void *stream);
/* Binning (as bgs_bin_and_sort) of the V * N records into the global tile space: each
   view's lists are built in its own tile range, in view order, and point_list values are
   record indices.  Without BGS_BIN_NO_SYNC the call synchronises once at its end, returns
   BGS_ERR_CAPACITY if the entry count K exceeds capacity (*needed = K) and sets
   *num_rendered = K (both host, nullable).  With BGS_BIN_NO_SYNC it only enqueues work:
   lists are written up to capacity and an overflow raises BGS_CHECK_OVERFLOW.  Each view
   may have at most (opt-in shared memory per block / 4) tiles.  conic_opacity [V * N, 4]
   (nullable) truncates the lists as in bgs_bin_and_sort. */
int bgs_bin_and_sort_batched(bgs_plan *plan, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                             const int32_t *radii, const float *depths, const float *conic_opacity,
                             int32_t tile_w, int32_t tile_h, uint32_t *point_list, int64_t capacity,
                             uint32_t *ranges, int32_t flags, int64_t *num_rendered, int64_t *needed,
                             void *stream);
/* Forward (as bgs_render_forward) of all views in one persistent launch; outputs go to
   views[v].out_*.  mode: AUTO, PIXEL or GAUSSIAN. */
int bgs_render_forward_batched(bgs_plan *plan, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                               const float *conic_opacity, const float *colors, const float *depths,
                               const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges,
                               int32_t tile_w, int32_t tile_h, const float *bg, int32_t mode, void *stream);
/* Backward (as bgs_render_backward) of all views in one launch, reading views[v].final_T,
   n_contrib and dL_d*.  dL_dmeans2D, dL_dconic, dL_dopacity, dL_ddepths are per record
   ([V * N, ...]); dL_dcolors [N, 3] is summed over the views (colours are shared). */
int bgs_render_backward_batched(bgs_plan *plan, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                                const float *conic_opacity, const float *colors, const float *depths,
                                const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges,
                                int32_t tile_w, int32_t tile_h, const float *bg, int32_t mode, float *dL_dmeans2D,
                                float *dL_dconic, float *dL_dopacity, float *dL_dcolors, float *dL_ddepths,
                                void *stream);
/* As bgs_render_forward_batched / bgs_render_backward_batched with view-dependent colours:
   colors [V * N, 3] holds the colour of every record (view v's colours at rows v * N ..,
   e.g. from bgs_sh_to_rgb), and dL_dcolors [V * N, 3] receives the per-record colour
   gradients (no sum over the views). */
int bgs_render_forward_batched_vc(bgs_plan *plan, int32_t V, const bgs_view *views, int64_t N,
                                  const float *means2D, const float *conic_opacity, const float *colors,
                                  const float *depths, const uint32_t *point_list, int64_t num_entries,
                                  const uint32_t *ranges, int32_t tile_w, int32_t tile_h, const float *bg,
                                  int32_t mode, void *stream);
int bgs_render_backward_batched_vc(bgs_plan *plan, int32_t V, const bgs_view *views, int64_t N,
                                   const float *means2D, const float *conic_opacity, const float *colors,
                                   const float *depths, const uint32_t *point_list, int64_t num_entries,
                                   const uint32_t *ranges, int32_t tile_w, int32_t tile_h, const float *bg,
                                   int32_t mode, float *dL_dmeans2D, float *dL_dconic, float *dL_dopacity,
                                   float *dL_dcolors, float *dL_ddepths, void *stream);

/* ---- view-dependent colour from spherical harmonics (Sec. 2.1) ----------------------
   The paper represents a Gaussian's colour by spherical harmonics.  Basis: the real
   orthonormal spherical harmonics Y_k of degree <= `degree` (0..3) with the Condon-Shortley
   phase, ordered (l, m) = (0,0), (1,-1), (1,0), (1,1), (2,-2), ..., (3,3) (k = l^2 + l + m),
   evaluated at the unit direction d from view v's camera centre (solved from its viewmat)
   to means3D[i]:  rgb[v * N + i][c] = max(0, sum_{k < (degree+1)^2} Y_k(d) sh[i][k][c] + 1/2),
   clamped[v * N + i][c] = 1 where the sum + 1/2 was negative (0 otherwise).
   sh [N, stride, 3] f32 (stride >= (degree+1)^2 coefficient rows; rows past (degree+1)^2
   are not read), means3D [N, 3]; views: host array of V <= 32 (only cam.viewmat is read,
   which must be invertible); rgb [V * N, 3] (device) and clamped [V * N, 3] u8 (device,
   nullable).  A mean at a camera centre has no direction (NaN colour).  Errors:
   BGS_ERR_INVALID for a NULL plan / views / array, V or degree out of range, stride too
   small or a singular viewmat. */
int bgs_sh_to_rgb(bgs_plan *plan, int32_t V, const bgs_view *views, int64_t N, int32_t degree, int32_t stride,
                  const float *sh, const float *means3D, float *rgb, uint8_t *clamped, void *stream);
/* Gradients of bgs_sh_to_rgb: dL_drgb [V * N, 3] -> dL_dsh [N, stride, 3] (rows past
   (degree+1)^2 zeroed) and dL_dmeans3D [N, 3] (through the view direction), summed over the
   views and overwriting the outputs.  A clamped channel passes no gradient; the clamp
   decisions are recomputed with the forward's arithmetic. */
int bgs_sh_to_rgb_backward(bgs_plan *plan, int32_t V, const bgs_view *views, int64_t N, int32_t degree,
                           int32_t stride, const float *sh, const float *means3D, const float *dL_drgb,
                           float *dL_dsh, float *dL_dmeans3D, void *stream);
/* Autotuner: times forward (+ backward when `backward` is 1) passes of this frame under
   candidate plan knobs -- pixel_rows (sub-tile of pixel-wise items), heavy_threshold (the
   per-tile selector between pixel-wise and Gaussian-wise items), gw_pixels and
   queue_chunk -- and keeps the fastest in the plan (*best_ms, host, nullable, gets its
   time).  Arguments as bgs_render_forward_batched / bgs_render_backward_batched (the
   views' outputs and dL_dcolor buffers are used as scratch; dL_ddepths is not written).
   Synchronises the stream after every candidate; not for use inside a graph capture. */
int bgs_autotune_render(bgs_plan *plan, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                        const float *conic_opacity, const float *colors, const float *depths,
                        const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges, int32_t tile_w,
                        int32_t tile_h, const float *bg, int32_t backward, float *dL_dmeans2D, float *dL_dconic,
                        float *dL_dopacity, float *dL_dcolors, double *best_ms, void *stream);

/* Graph capture of a whole step: bgs_graph_begin starts capturing `stream` (thread-local
   mode), the caller enqueues its bgs_* calls (and its own work), bgs_graph_end ends the
   capture and instantiates the graph (kept by the plan, replacing an earlier one), and
   bgs_graph_launch replays it on `stream`.  Inside a capture the plan allocates nothing:
   run the step once before capturing (or call bgs_plan_reserve) so that its workspace is
   large enough, use BGS_BIN_NO_SYNC, and pass num_entries = the point_list capacity. */
int bgs_graph_begin(bgs_plan *plan, void *stream);
int bgs_graph_end(bgs_plan *plan, void *stream);
int bgs_graph_launch(bgs_plan *plan, void *stream);

/* ---- allocation-free forward ----------------------------------------------------------
   The paper has no counterpart to this entry point; it serves callers that cannot let
   the library allocate device memory -- a host application that owns all device memory
   under a fixed budget (a game engine, an inference server), a plugin loaded into such a
   process, or a runtime that forbids allocations after start-up.  It computes the same
   outputs as bgs_render_forward (persistent pixel-wise kernel, heaviest tiles first) from
   the same caller-owned inputs and outputs, needs no plan, and calls no cudaMalloc,
   cudaFree or other allocating routine.  Its scratch (work-queue counters and the tile
   order) lives in one fixed array of about 256 KiB in this library's device memory,
   present on every GPU that loads the library until the process exits; it holds at most
   65536 tiles, and larger tile grids are rejected with BGS_ERR_CAPACITY.  It runs on the
   caller's current device; the first call on a device looks up the array's device
   address (no allocation) and should come before any stream capture.  All calls share
   the array: each call resets what must start at zero, consecutive calls on one stream
   are independent, and calls that overlap on the GPU race.  Entries whose index is >= N
   or whose tile span passes num_entries are rendered transparent and raise
   BGS_CHECK_INDEX / BGS_CHECK_RANGE in the array.  check_bits (host, nullable): when
   given, the call waits for its own work on the stream, writes the bits this call raised
   and returns BGS_ERR_DEVICE_CHECK if any is set; when NULL it only enqueues work and the
   bits are not reported.  tile_w must be a multiple of 8 and tile_h of 4. */
int bgs_render_forward_noalloc(int64_t N, const float *means2D, const float *conic_opacity, const float *colors,
                               const float *depths, const uint32_t *point_list, int64_t num_entries,
                               const uint32_t *ranges, int32_t W, int32_t H, int32_t tile_w, int32_t tile_h,
                               const float *bg, float *out_color, float *out_depth, float *out_alpha, float *final_T,
                               int32_t *n_contrib, int32_t *n_eval, uint32_t *check_bits, void *stream);

/* ---- diagnostics -------------------------------------------------------------------
   Measures sustained per-SM issue rates of the FP32 pipe (FFMA) and of the MUFU ex2
   unit with dependent-chain-free loops on every SM; writes operations per SM per clock
   cycle (host) using the SM clock counter.  Synchronises. */
int bgs_probe_pipe_rates(bgs_plan *plan, double *fp32_per_sm_clk, double *ex2_per_sm_clk, void *stream);
/* y[i] = 2^x[i] with the exponential the render kernels use (ex2.approx.ftz). */
int bgs_debug_exp2(const float *x, float *y, int64_t n, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BGS_H */
