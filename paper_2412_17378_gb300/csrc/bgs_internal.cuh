// bgs_internal.cuh -- shared declarations of the CUDA library (device helpers, the
// plan's control block, per-pair blend rule, kernel launchers).  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bgs.h"

namespace bgs {

// ---- constants of the per-pair rule (Algorithm 5 with standard 3DGS constants) -------
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;  // log2(e): exp(x) = 2^(x log2 e)
constexpr float kLn2 = 0.6931471805599453f;    // ln(2)

constexpr int kMaxViews = 32;  // views of one batched call

// ---- device control block (one per plan) --------------------------------------------
struct DevCtrl {
    unsigned int queue_head;    // pixel-wise queue cursor (starts at num_gauss)
    unsigned int num_items;     // work items in the current list
    unsigned int check_bits;    // BGS_CHECK_* raised by device checks
    unsigned int num_gauss;     // items [0, num_gauss) are Gaussian-wise, the rest pixel-wise
    unsigned long long num_entries;  // K written by binning
    unsigned long long eval_pairs;
    unsigned long long contrib_pairs;
    unsigned long long items_done;
    unsigned int queue_head_g;  // Gaussian-wise queue cursor (starts at 0)
    unsigned int pass_items;    // items the current persistent pass completed
    unsigned long long bin_base;  // binning: entries of the call so far (= num_entries at its end)
    unsigned int warps_done;    // blocks of the current persistent pass that finished
    unsigned int pad1;
    // work-list build: items per sort key, each key's first item, blocks done (the counters
    // return to zero at the end of every build)
    unsigned int wl_cnt[256];
    unsigned int wl_off[256];
    unsigned int wl_done;
    unsigned int num_gauss0;    // Gaussian-wise items [0, num_gauss0) are first segments; the
                                // items [num_gauss0, num_gauss) later segments of long lists
    unsigned int gw_seg;        // entries per Gaussian-wise segment (0: lists are not split)
    unsigned int pad2;
    unsigned long long wl_extra;  // work-list build: later-segment items (returns to zero)
    // binning: each view's entry count and first point_list slot
    unsigned long long view_k[kMaxViews];
    unsigned long long view_base[kMaxViews];
};

// End of a persistent pass, per warp (lane 0), for a block of `warps_per_block` warps whose
// shared counters blk[0] (items) and blk[1] (finished warps) start at 0: the block's last
// warp adds the block's completed items to the pass total, and the pass's last block
// (`pass_blocks` in all) compares the total with the queued item count and raises
// BGS_CHECK_QUEUE unless every item ran exactly once.
__device__ __forceinline__ void finish_pass(DevCtrl *ctrl, unsigned long long items, unsigned int *blk,
                                            int warps_per_block, int pass_blocks) {
    atomicAdd(&blk[0], (unsigned int)items);
    __threadfence_block();
    if (atomicAdd(&blk[1], 1u) != (unsigned int)warps_per_block - 1u) return;
    atomicAdd(&ctrl->pass_items, atomicAdd(&blk[0], 0u));
    __threadfence();
    if (atomicAdd(&ctrl->warps_done, 1u) == (unsigned int)pass_blocks - 1u) {
        __threadfence();
        const unsigned int done = atomicAdd(&ctrl->pass_items, 0u);
        if (done != *((volatile unsigned int *)&ctrl->num_items)) atomicOr(&ctrl->check_bits, BGS_CHECK_QUEUE);
    }
}

// Pixel-wise items: Q = pixel rows per lane (the plan's sub-tile knob, 1, 2, 4 or 8).  For
// Q <= 4 an item covers 8 x 4Q pixels of a tile and lane l owns the pixels (l % 8, l / 8 +
// 4 q); for Q = 8 it covers 16 x 16 pixels and lane l owns (l % 16, l / 16 + 2 q), q < Q.
// Either way a lane's pixels share one column (and so their x-offset to a Gaussian).
__host__ __device__ constexpr int pix_item_w(int Q) { return Q == 8 ? 16 : 8; }
__host__ __device__ constexpr int pix_row_step(int Q) { return 32 / pix_item_w(Q); }
__host__ __device__ constexpr int pix_item_h(int Q) { return pix_row_step(Q) * Q; }

// ---- packed per-Gaussian record used by the render kernels (48 bytes) ---------------
//   a = (mx, my, qa, qb), b = (qc, o, hx, hy), c = (r, g, b, depth)
//   with (qa, qb, qc) = -log2(e) (a/2, b, c/2), so that the natural-log power of the
//   pair is ln2 * (qa dx^2 + qb dx dy + qc dy^2) and exp(power) = 2^(qa dx^2 + ...).
//   (hx, hy) are half-extents of a box around the mean outside which no pixel can reach
//   alpha >= 1/255 (negative: no pixel can); kernels use it to skip whole records for a
//   block of pixels.
struct __align__(16) Rec {
    float4 a, b, c;
};

// One work item of the persistent kernels.
//   x = tile id (global over views), y = kind << 31 | sub-item index inside the tile.
constexpr unsigned int kKindGauss = 1u << 31;

// ---- small device helpers ------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// hardware reciprocal approximation (a few ulp; used where the backward recovers T_i)
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void raise_check(DevCtrl *ctrl, unsigned int bit) {
    atomicOr(&ctrl->check_bits, bit);
}

// Half-extents of the region where alpha = min(0.99, o G) can reach 1/255: alpha >= 1/255
// needs o G >= 1/255, i.e. d^T Q d <= r^2 = 2 ln(255 o), whose bounding box has half-widths
// r sqrt((Q^-1)_xx) = r sqrt(c / det) and r sqrt(a / det) for Q = (a b; b c).  Widened by
// 0.1% and 0.01 px so that float32 evaluation of a pair never decides "valid" outside it.
__device__ __forceinline__ float2 alpha_box(float a, float b, float c, float o) {
    const float det = a * c - b * b;
    const float lo = 255.f * o;
    if (!(lo > 1.f)) return make_float2(-1.f, -1.f);  // alpha <= o < 1/255 everywhere
    if (!(det > 0.f)) return make_float2(3.0e38f, 3.0e38f);
    const float r2 = 2.f * logf(lo);
    return make_float2(sqrtf(r2 * c / det) * 1.001f + 0.01f, sqrtf(r2 * a / det) * 1.001f + 0.01f);
}

// Packs record g into a Rec (the conic is pre-scaled by -log2(e)/2); its colour is
// colour row cg (views of a batched call share the colours of their Gaussians).
__device__ __forceinline__ Rec make_rec(const float *__restrict__ means2D, const float *__restrict__ conic_opacity,
                                        const float *__restrict__ colors, const float *__restrict__ depths,
                                        unsigned int g, unsigned int cg) {
    Rec r;
    const float2 m = reinterpret_cast<const float2 *>(means2D)[g];
    const float4 co = reinterpret_cast<const float4 *>(conic_opacity)[g];
    const float2 box = alpha_box(co.x, co.y, co.z, co.w);
    r.a = make_float4(m.x, m.y, -0.5f * kLog2e * co.x, -kLog2e * co.y);
    r.b = make_float4(-0.5f * kLog2e * co.z, co.w, box.x, box.y);
    r.c = make_float4(colors[3 * cg], colors[3 * cg + 1], colors[3 * cg + 2], depths[g]);
    return r;
}

// true when the record cannot reach alpha >= 1/255 at any pixel whose centre lies within
// (hw, hh) of (cx, cy)
__device__ __forceinline__ bool box_misses(const float4 &a, const float4 &b, float cx, float cy, float hw, float hh) {
    return fabsf(a.x - cx) > b.z + hw || fabsf(a.y - cy) > b.w + hh;
}

__device__ __forceinline__ Rec make_rec(const float *__restrict__ means2D, const float *__restrict__ conic_opacity,
                                        const float *__restrict__ colors, const float *__restrict__ depths,
                                        unsigned int g) {
    return make_rec(means2D, conic_opacity, colors, depths, g, g);
}

// power2 = log2(e) * power of the pair (pixel px, py) = qa dx^2 + qb dx dy + qc dy^2,
// evaluated as hx + dy (bx + qc dy) with hx = qa dx^2 and bx = qb dx (shared by pixels of
// one column).  Written with explicit round-to-nearest intrinsics so that no kernel's
// compilation can contract or reorder it: every kernel, forward and backward, takes the
// same skip / stop decisions bit for bit.
struct PairX {
    float dx, hx, bx;
};

__device__ __forceinline__ PairX pair_x(float4 a, float px) {
    PairX r;
    r.dx = __fsub_rn(a.x, px);
    r.hx = __fmul_rn(__fmul_rn(a.z, r.dx), r.dx);
    r.bx = __fmul_rn(a.w, r.dx);
    return r;
}

__device__ __forceinline__ float pair_power2_y(const PairX &x, float ay, float qc, float py, float &dy) {
    dy = __fsub_rn(ay, py);
    return __fmaf_rn(dy, __fmaf_rn(qc, dy, x.bx), x.hx);
}

__device__ __forceinline__ float pair_power2(float4 a, float qc, float px, float py, float &dx, float &dy) {
    const PairX x = pair_x(a, px);
    dx = x.dx;
    return pair_power2_y(x, a.y, qc, py, dy);
}

// Transmittance after a pair, T (1 - alpha), as one fused multiply-add T - T alpha (one
// rounding); the pixel-wise kernels (static, persistent, allocation-free) and the
// backward's T recovery take their stop decision T' < 1e-4 on this value.  The
// Gaussian-wise kernels walk the entries of the stopping chunk with it too, but from a T in
// front of the chunk that is a product of chunk products (reassociated: about 2 ulp per
// 8-entry chunk and composition against this sequential chain), so a decision can only
// flip where T' lies within that rounding of 1e-4: inside the oracle's |T' - 1e-4| < 1e-9
// flag window at the list lengths of the tests.
__device__ __forceinline__ float next_T(float T, float al) { return __fmaf_rn(-T, al, T); }

// o G of a pair.  A pair is accumulated when power2 <= 0 and o G >= 1/255 (the same as
// alpha = min(0.99, o G) >= 1/255, since 1/255 < 0.99); alpha is formed only for those.
__device__ __forceinline__ float pair_oG(float power2, float o) { return __fmul_rn(o, ex2_approx(power2)); }

// ---- views ---------------------------------------------------------------------------
// A render call covers V views (1 for the single-view entry points).  Their tiles form
// one global tile space: view v owns tile ids [tile_base[v], tile_base[v+1]).  Record
// (and gradient) index v * n_per_view + g belongs to Gaussian g seen from view v.

struct ViewTable {
    int V;
    int W[kMaxViews], H[kMaxViews], tiles_x[kMaxViews], tiles_y[kMaxViews];
    int tile_base[kMaxViews + 1];
};

// view owning a global tile id (binary search over tile_base)
__device__ __forceinline__ int view_of(const ViewTable &vt, int tile) {
    int lo = 0, hi = vt.V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (vt.tile_base[mid] <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct ViewOut {  // forward outputs, per view
    float *out_color[kMaxViews], *out_depth[kMaxViews], *out_alpha[kMaxViews], *final_T[kMaxViews];
    int *n_contrib[kMaxViews], *n_eval[kMaxViews];
};

struct ViewGradIn {  // backward inputs, per view
    const float *final_T[kMaxViews];
    const int *n_contrib[kMaxViews];
    const float *dL_dcolor[kMaxViews], *dL_ddepth[kMaxViews], *dL_dalpha[kMaxViews];
};

// ---- launch parameter blocks -----------------------------------------------------------
struct FwdArgs {
    const Rec *recs;             // packed records [V * n_per_view]
    const float *means2D, *conic_opacity, *colors, *depths;  // ABI arrays (static kernel)
    const uint32_t *point_list;
    const uint2 *ranges;         // [total tiles]
    long long N;                 // number of records (V * n_per_view)
    long long num_entries;
    int tile_w, tile_h, num_tiles;
    float bg[3];
    ViewTable vt;
    ViewOut io;
    DevCtrl *ctrl;
    const uint2 *items;          // work list (persistent kernels)
    int pass_blocks;             // blocks of the persistent pass (both forward kernels when both run)
    int gw_pixels;
    const uint32_t *gw_exoff;    // per tile: its later-segment items' offset from num_gauss0
    float4 *gw_sum;              // per Gaussian-wise item, per pixel: the segment summary
    unsigned int *tile_cost;     // per tile (nullable, zeroed): the largest n_contrib of its pixels
    int pixel_rows;              // Q of the pixel-wise items
    int chunk;
};

// A pixel's record of one Gaussian-wise segment (2 x 16 bytes), per (segment item, pixel).
// Written by the segment item:
//   cd = colour and depth accumulated with the segment's own transmittance from 1;
//   t  = (transmittance after the segment, last contributor (index in the tile's list, bits;
//        -1: none), contributing pairs (bits), entries up to and including the stop (bits)
//        when the pixel stopped in the segment, else 0).
// Rewritten by the merge, for every segment the pixel reaches when its list has several:
//   cd = colour and depth accumulated behind the segment (with absolute weights, the
//        background's T_f bg included);  t.x = the transmittance behind the segment.
// That is the state a back-to-front walk holds when it enters the segment from behind.
struct GwSum {
    float4 cd;
    float4 t;
};

__device__ __forceinline__ bool tile_is_gauss(int mode, int heavy_threshold, uint32_t n) {
    return mode == BGS_MODE_GAUSSIAN || (mode == BGS_MODE_AUTO && n > (uint32_t)heavy_threshold);
}

struct BwdArgs {
    const Rec *recs;
    const float *means2D, *conic_opacity, *colors, *depths;
    const uint32_t *point_list;
    const uint2 *ranges;
    long long N;
    long long num_entries;
    int tile_w, tile_h, num_tiles;
    float bg[3];
    ViewTable vt;
    ViewGradIn gi;
    float *grad_acc;             // [N][12] accumulators (10 used)
    DevCtrl *ctrl;
    const uint2 *items;
    unsigned int *warp_items;  // per warp of the persistent pass: items it completed
    int pixel_rows;
    int chunk;
    // segmented walk of the tiles the last forward split (bseg_mode: its render mode, -1:
    // none): the forward's per-tile segment item positions and boundary states
    int bseg_mode, heavy_threshold, gw_pixels;
    const uint2 *gw_tile;
    const GwSum *gw_sum;
};

// Records a message for bgs_last_error() and returns code.
int set_error(int code, const char *msg);

// ---- launchers (each returns cudaGetLastError() of its launch) ------------------------
// N Gaussians seen from V cameras: record v * N + g (V = 1 for a single view)
cudaError_t launch_preprocess(long long N, int V, const float *means3D, const float *log_scales, const float *quats,
                              const float *opacities, const bgs_camera *cams, int tile_w, int tile_h,
                              float *means2D, float *conic_opacity, float *depths, int *radii,
                              uint32_t *tiles_touched, cudaStream_t s);
// projection backward: dL/d(means2D, conic a b c, depth) of the records [V N] ->
// dL/d(means3D, log_scales, quats) [N] summed over the views (radius-0 records skipped)
cudaError_t launch_preprocess_backward(long long N, int V, const float *means3D, const float *log_scales,
                                       const float *quats, const bgs_camera *cams, const int *radii,
                                       const float *dL_dmeans2D, const float *dL_dconic, const float *dL_ddepths,
                                       float *dL_dmeans3D, float *dL_dlog_scales, float *dL_dquats, cudaStream_t s);
// idx[i] = i for i in [lo, hi)
cudaError_t launch_iota(long long lo, long long hi, uint32_t *idx, cudaStream_t s);

cudaError_t launch_touched(long long N, const float *means2D, const int *radii, const float *depths, int W, int H,
                           int tile_w, int tile_h, uint32_t *touched, uint32_t *dkey, uint32_t *idx, cudaStream_t s);
cudaError_t launch_gather_u32(long long N, const uint32_t *src, const uint32_t *order, uint32_t *dst, cudaStream_t s);
template <typename KeyT>
cudaError_t launch_duplicate(long long N, const uint32_t *order, const float *means2D, const int *radii,
                             const unsigned long long *offsets, int W, int H, int tile_w, int tile_h, KeyT *keys,
                             uint32_t *vals, long long capacity, cudaStream_t s);
cudaError_t launch_count_total(long long N, const uint32_t *touched, const unsigned long long *offsets,
                               DevCtrl *ctrl, cudaStream_t s);
template <typename KeyT>
cudaError_t launch_ranges(const KeyT *keys, long long K, uint2 *ranges, cudaStream_t s);

// counting-sort binning (binning.cu)
// shared memory of the count kernel (tile counters + one 512-bit mask slice per tile group)
size_t bin_count_smem(int tx, int ty);
int bin_mask_groups(int tx, int ty);
cudaError_t setup_bin_kernels(int tx, int ty);
// also writes each sorted position's record rect[s] = (x0 | w << 16, y0 | h << 16, Gaussian
// index, 0) (both rectangle words 0 when empty) and the (block, tile group) masks, W32
// words each (a multiple of 16)
// blocks [b_lo, b_hi) of the counting pass; skipP (nullable): the exclusive 2D prefix of the
// tiles known to have stopped before b_lo (k_bin_stopped), whose Gaussians are left out
cudaError_t launch_bin_count(long long N, int G, int b_lo, int b_hi, const uint32_t *order, const float *means2D,
                             const int *radii, int W, int H, int tw, int th, uint32_t *Hm, uint4 *rect, uint32_t *masks,
                             int W32, const int *skipP, cudaStream_t s);
// the tiles whose credits over blocks [0, B1) certify that every pixel stopped, as the
// exclusive 2D prefix P [(ty + 1) x (tx + 1)] of their indicator; P's buffer holds tx ty more
// words behind the prefix (the per-tile sums)
cudaError_t launch_bin_stopped(int B1, int tx, int ty, const uint16_t *D, int *P, cudaStream_t s);
// per tile column: exclusive prefix of H over the blocks and the total; with the credits D
// (nullable) the column is cut after the block b_sat[t] at which they certify that every
// pixel of the tile has stopped (b_sat written when bsat is not null)
cudaError_t launch_bin_colscan(int B, int T, uint32_t *Hm, const uint16_t *D, uint32_t *total, uint32_t *bsat,
                               cudaStream_t s);
// per block and tile: fixed-point credits toward that certificate (k_bin_credit)
size_t bin_credit_smem(int tx, int ty);
cudaError_t launch_bin_credit(long long N, int G, int b_lo, int b_hi, const uint4 *rect, const float *means2D,
                              const float *conic_opacity, int W, int H, int tw, int th, uint16_t *D, cudaStream_t s);
// ranges of view v's tiles, offset by the view's first point_list slot (the sum of the entry
// counts of views 0..v-1, stored in ctrl->view_base[v] for the scatter)
cudaError_t launch_bin_ranges(int T, const uint32_t *start, const uint32_t *total, uint2 *ranges, int v,
                              DevCtrl *ctrl, cudaStream_t s);
cudaError_t launch_bin_scatter(long long N, int G, int B, int W32, const uint4 *rect, int W, int H, int tw, int th,
                               const uint32_t *Hm, const uint32_t *start, const uint32_t *masks, uint32_t *point_list,
                               long long capacity, const uint32_t *bsat, uint32_t *item_start, int num_sms, int v,
                               const DevCtrl *ctrl, cudaStream_t s);
// ctrl->view_k[v] = view v's entry count (64-bit sum of its tile totals)
cudaError_t launch_bin_view_total(int T, const uint32_t *total, int v, DevCtrl *ctrl, cudaStream_t s);
// num_entries = bin_base = the sum of the V views' counts; raises BGS_CHECK_OVERFLOW past
// capacity or BGS_MAX_ENTRIES
cudaError_t launch_bin_finish(int V, long long capacity, DevCtrl *ctrl, cudaStream_t s);

// view-dependent colour from spherical harmonics (sh.cu); backward: dL_drgb -> dL_dsh,
// dL_dmeans3D (summed over the V <= kMaxViews camera centres campos [V,3], host)
cudaError_t launch_sh(bool backward, long long N, int degree, int stride, const float *sh, const float *means3D,
                      int V, const float *campos, float *rgb, uint8_t *clamped, const float *dL_drgb, float *dL_dsh,
                      float *dL_dmeans3D, cudaStream_t s);

// recs[i] from means2D[i], conic_opacity[i], depths[i] and colors[i % n_colors]
cudaError_t launch_pack(long long N, const float *means2D, const float *conic_opacity, const float *colors,
                        long long n_colors, const float *depths, Rec *recs, cudaStream_t s);

// Work list of the persistent kernels, by bucket counting over the tiles' sort keys:
// k_wl_count gives every tile its place in its key's bucket and (last block) the buckets'
// first items and the ctrl counts; k_wl_emit writes the items (positions past `capacity`
// items raise BGS_CHECK_OVERFLOW and are skipped).  The order of tiles within one key is
// unspecified.
// gw_segment: entries per Gaussian-wise segment (0: lists are not split); exoff [num_tiles]
// (nullable when gw_segment is 0) receives each tile's later-segment offset; extra_cap: the
// most later-segment items the list may hold (beyond it the lists are not split).
// bseg_mode >= 0 (a pixel-wise list for the backward): the tiles that the last forward, in
// that render mode, split into segments get their pixel-wise items once per segment
// (ctrl->gw_seg, the forward's segment length, is kept).  gw_tile [num_tiles] (nullable):
// per Gaussian-wise tile of a forward list, (first first-segment item, first later-segment
// item).  cost [num_tiles] (nullable): the per-tile load that orders the list heaviest first
// (default: the list length).
cudaError_t launch_worklist_buckets(const uint2 *ranges, int num_tiles, const ViewTable &vt, int tile_w, int tile_h,
                                    int mode, int heavy_threshold, int lpt, int gw_pixels, int pixel_rows,
                                    int gw_segment, long long extra_cap, uint32_t *slot, uint32_t *exoff,
                                    uint2 *items, long long capacity, int bseg_mode, uint2 *gw_tile,
                                    const uint32_t *cost, DevCtrl *ctrl, cudaStream_t s);

// queue of the current list: rewind for another pass / mark exhausted (fault injection)
cudaError_t launch_rewind_queue(DevCtrl *ctrl, cudaStream_t s);
cudaError_t launch_exhaust_queue(DevCtrl *ctrl, cudaStream_t s);

cudaError_t launch_forward_static(const FwdArgs &a, cudaStream_t s);
cudaError_t launch_forward_gauss(const FwdArgs &a, int grid, cudaStream_t s);
cudaError_t launch_forward_pixel(const FwdArgs &a, int grid, bool after_gauss, cudaStream_t s);
// composes the Gaussian-wise segment summaries per pixel; after both forward kernels
cudaError_t launch_forward_gw_merge(const FwdArgs &a, int grid, cudaStream_t s);
int forward_balanced_block_threads();
const void *forward_gauss_kernel(int gw_pixels);
const void *forward_gw_merge_kernel(int gw_pixels);
const void *forward_pixel_kernel(int pixel_rows);

cudaError_t launch_backward_static(const BwdArgs &a, cudaStream_t s);
cudaError_t launch_backward_balanced(const BwdArgs &a, int grid, cudaStream_t s);
int backward_balanced_block_threads();
const void *backward_balanced_kernel(const BwdArgs &a);  // the instantiation a would launch
// gradients of N records; colours have n_colors rows (n_colors < N: summed over views)
cudaError_t launch_grad_finalize(long long N, long long n_colors, const float4 *acc, const float *conic_opacity,
                                 float *dL_dmeans2D, float *dL_dconic, float *dL_dopacity, float *dL_dcolors,
                                 float *dL_ddepths, const unsigned int *warp_items, int n_warps, DevCtrl *ctrl,
                                 cudaStream_t s);

}  // namespace bgs
