// worklist.cu -- a3: per-tile load statistics and the work list of the persistent kernels.
//
// The paper's task pool (Sec. 4.1) holds whole tiles; its fine-grained variant
// (Sec. 4.3) splits each tile into 4-pixel tasks, and its selector (Sec. 4.4) chooses
// between the Gaussian-wise and the pixel-wise kernel.  Here the choice is made per
// tile from its list length n (the paper names "the Gaussians of a tile" as the key
// load-balance metric, Sec. 4.4):
//   n >  heavy_threshold -> Gaussian-wise items of P pixels (one warp each), and, for a list
//                           longer than gw_segment entries, one item per further segment
//                           of gw_segment entries and P pixels (the cross-warp split),
//   n <= heavy_threshold -> pixel-wise items of 8 x 4Q pixels (one warp, Q pixels per lane).
// The work list holds the Gaussian-wise first-segment items, then the later-segment items,
// then the pixel-wise items.
// Tiles of all views of a batched call share one global tile space.
// Items of heavier tiles are queued first (longest-processing-time order) so the long
// items start early and the light ones fill the tail.
#include <cub/block/block_scan.cuh>

#include "bgs_internal.cuh"

namespace bgs {

// Items of tile t: Gaussian-wise (first segments), P pixels each; else pixel-wise sub-blocks of
// its visible part.
__device__ __forceinline__ uint32_t tile_items(int t, bool gauss, const ViewTable &vt, int tile_w, int tile_h,
                                               int gw_pixels, int pixel_rows) {
    const int v = view_of(vt, t);
    const int lt = t - vt.tile_base[v];
    const int tx = lt % vt.tiles_x[v], ty = lt / vt.tiles_x[v];
    const int vw = min(tile_w, vt.W[v] - tx * tile_w), vh = min(tile_h, vt.H[v] - ty * tile_h);
    if (gauss) return (uint32_t)((vw * vh + gw_pixels - 1) / gw_pixels);
    const int iw = pix_item_w(pixel_rows), ih = pix_item_h(pixel_rows);
    return (uint32_t)(((vw + iw - 1) / iw) * ((vh + ih - 1) / ih));
}

// Items of a pixel-wise list's tile that the forward rendered Gaussian-wise with its list
// split into segments of L entries (bseg_mode: the forward's render mode, -1 for a list
// without segments): the tile's c pixel-wise items once per segment (sub-item = segment *
// c + item), so that the backward walks each segment on its own.
__device__ __forceinline__ uint32_t bwd_segments(int bseg_mode, int heavy_threshold, unsigned L, uint32_t n) {
    if (bseg_mode < 0 || L == 0u || n <= L || !tile_is_gauss(bseg_mode, heavy_threshold, n)) return 1u;
    return (n - 1u) / L + 1u;
}

// Later-segment items of a Gaussian-wise tile with first-segment items `groups` and list
// length n: one per (segment after the first, pixel group).
__device__ __forceinline__ unsigned long long tile_extra(bool gauss, uint32_t groups, uint32_t n, int gw_segment) {
    if (!gauss || gw_segment <= 0 || n <= (uint32_t)gw_segment) return 0ull;
    return (unsigned long long)groups * (unsigned long long)((n - 1u) / (uint32_t)gw_segment);
}

// The list is ordered by a descending 8-bit key per tile: its kind in the top bit (Gaussian-
// wise tiles first) and, when lpt is on, a log-scale bucket of its list length below it
// (heaviest first; lengths within ~19% share a bucket): bucket = 4 floor(log2 n) + the two
// bits after the leading one, + 1 (0 for an empty tile).
__device__ __forceinline__ uint32_t length_bucket(uint32_t n) {
    if (n == 0u) return 0u;
    const int e = 31 - __clz(n);
    const uint32_t m = e >= 2 ? (n >> (e - 2)) & 3u : (n << (2 - e)) & 3u;
    return min(127u, 4u * (uint32_t)e + m + 1u);
}

// ---- bucket-counting build (any grid, two launches) ----------------------------------------
// The key takes at most 256 values, so no sort is needed: a tile's items go to its key's
// bucket, the buckets in descending key order.  Within a bucket the order of the tiles
// follows the atomics (it changes only when items start, never what they compute).  At the
// grids of a frame (thousands to ~10^5 tiles) this is two short launches, where a block
// radix sort in one block or a device-wide sort chain is bound by latency.
constexpr int kWlcThreads = 256;  // one thread per key in the offset pass

__device__ __forceinline__ uint32_t wl_sort_key(uint32_t n, bool gauss, int lpt) {
    const uint32_t kind = gauss ? 1u : 0u;
    return lpt ? (kind << 7) | length_bucket(n) : kind;
}

// Per block: items per key in shared memory (a tile's slot within its block's share is the
// atomic's old value), then one global atomic per key gives the block's share its place in
// the key's bucket; a block scan of the tiles' later-segment items and one global atomic
// give each tile its later-segment offset.  The last block to finish reads the totals
// (clearing them for the next build), scans them in descending key order into the buckets'
// first items and publishes the list's item counts and queue cursors.  When the
// later-segment items exceed extra_cap, no list is split (segment size 0).
__global__ void __launch_bounds__(kWlcThreads) k_wl_count(const uint2 *__restrict__ ranges, int T, const ViewTable vt,
                                                           int tile_w, int tile_h, int mode, int heavy_threshold,
                                                           int lpt, int gw_pixels, int pixel_rows, int gw_segment,
                                                           long long extra_cap, uint32_t *__restrict__ slot,
                                                           uint32_t *__restrict__ exoff, int bseg_mode,
                                                           const uint32_t *__restrict__ cost, DevCtrl *ctrl) {
    using Scan = cub::BlockScan<uint32_t, kWlcThreads>;
    using Scan64 = cub::BlockScan<unsigned long long, kWlcThreads>;
    __shared__ union {
        typename Scan::TempStorage s32;
        typename Scan64::TempStorage s64;
    } scan_tmp;
    __shared__ uint32_t s_cnt[256], s_base[256];
    __shared__ unsigned long long s_xbase;
    __shared__ bool s_last;
    s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    const int t = blockIdx.x * kWlcThreads + threadIdx.x;
    // a backward list segmented like the last forward: that forward's segment length
    const unsigned Lb = bseg_mode >= 0 ? *((volatile unsigned int *)&ctrl->gw_seg) : 0u;
    uint32_t key = 0u, local = 0u;
    unsigned long long extra = 0ull;
    if (t < T) {
        const uint2 rg = ranges[t];
        const uint32_t n = rg.y >= rg.x ? rg.y - rg.x : 0u;
        const bool gauss = tile_is_gauss(mode, heavy_threshold, n);
        key = wl_sort_key(cost ? cost[t] : n, gauss, lpt);
        const uint32_t c = tile_items(t, gauss, vt, tile_w, tile_h, gw_pixels, pixel_rows) *
                           (gauss ? 1u : bwd_segments(bseg_mode, heavy_threshold, Lb, n));
        local = atomicAdd(&s_cnt[key], c);
        extra = tile_extra(gauss, c, n, gw_segment);
    }
    if (gw_segment > 0) {  // grid-uniform
        unsigned long long xoff, xtotal;
        Scan64(scan_tmp.s64).ExclusiveSum(extra, xoff, xtotal);
        if (threadIdx.x == 0) s_xbase = xtotal ? atomicAdd(&ctrl->wl_extra, xtotal) : 0ull;
        __syncthreads();
        if (t < T) exoff[t] = (uint32_t)(s_xbase + xoff);  // used only when the total fits extra_cap
    }
    __syncthreads();
    {
        const uint32_t c = s_cnt[threadIdx.x];
        if (c) s_base[threadIdx.x] = atomicAdd(&ctrl->wl_cnt[threadIdx.x], c);
    }
    __syncthreads();
    if (t < T) slot[t] = s_base[key] + local;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctrl->wl_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        const unsigned long long E = gw_segment > 0 ? atomicExch(&ctrl->wl_extra, 0ull) : 0ull;
        const bool split = gw_segment > 0 && E <= (unsigned long long)extra_cap;
        s_xbase = split ? E : 0ull;
        // a segmented backward list keeps the forward's segment length (its kernel reads it)
        if (bseg_mode < 0) ctrl->gw_seg = split ? (unsigned int)gw_segment : 0u;
    }
    __syncthreads();
    const uint32_t E = (uint32_t)s_xbase;
    // thread i takes key 255 - i, so the scan runs in descending key order
    const int k = kWlcThreads - 1 - (int)threadIdx.x;
    const uint32_t c = atomicExch(&ctrl->wl_cnt[k], 0u);
    uint32_t off, total;
    Scan(scan_tmp.s32).ExclusiveSum(c, off, total);
    // Gaussian-wise keys (kind bit set) are the largest; the pixel-wise buckets follow the
    // later-segment items, and the first pixel-wise key's offset is the number of
    // first-segment items
    const int pix_top = lpt ? 127 : 0;
    ctrl->wl_off[k] = k <= pix_top ? off + E : off;
    if (k == pix_top) {
        ctrl->num_gauss0 = off;
        ctrl->num_gauss = off + E;
        ctrl->queue_head = off + E;
    }
    if (threadIdx.x == 0) {
        ctrl->num_items = total + E;
        ctrl->queue_head_g = 0u;
        ctrl->pass_items = 0u;
        ctrl->warps_done = 0u;
        ctrl->wl_done = 0u;
    }
}

// A thread per tile writes the tile's items at its bucket's first item + its slot, and its
// later-segment items (sub-item index = segment * groups + group, segment >= 1) at
// num_gauss0 + its offset.
__global__ void __launch_bounds__(256) k_wl_emit(const uint2 *__restrict__ ranges, int T, const ViewTable vt,
                                                 int tile_w, int tile_h, int mode, int heavy_threshold, int lpt,
                                                 int gw_pixels, int pixel_rows, const uint32_t *__restrict__ slot,
                                                 const uint32_t *__restrict__ exoff, uint2 *__restrict__ items,
                                                 long long capacity, int bseg_mode, uint2 *__restrict__ gw_tile,
                                                 const uint32_t *__restrict__ cost, DevCtrl *ctrl) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const uint2 rg = ranges[t];
    const uint32_t n = rg.y >= rg.x ? rg.y - rg.x : 0u;
    const bool gauss = tile_is_gauss(mode, heavy_threshold, n);
    const unsigned Lb = bseg_mode >= 0 ? ctrl->gw_seg : 0u;
    const uint32_t c = tile_items(t, gauss, vt, tile_w, tile_h, gw_pixels, pixel_rows) *
                       (gauss ? 1u : bwd_segments(bseg_mode, heavy_threshold, Lb, n));
    const long long pos = (long long)ctrl->wl_off[wl_sort_key(cost ? cost[t] : n, gauss, lpt)] + slot[t];
    if (pos + (long long)c > capacity) {
        raise_check(ctrl, BGS_CHECK_OVERFLOW);
        return;
    }
    const uint32_t kindbit = gauss ? kKindGauss : 0u;
    for (uint32_t q = 0; q < c; ++q) items[pos + q] = make_uint2((uint32_t)t, kindbit | q);
    const int seg = (int)ctrl->gw_seg;
    const unsigned long long x = tile_extra(gauss, c, n, seg);
    // where a Gaussian-wise tile's segment items sit (for a backward that reads their summaries)
    if (gw_tile && gauss) gw_tile[t] = make_uint2((uint32_t)pos, x ? ctrl->num_gauss0 + exoff[t] : 0u);
    if (x == 0ull) return;
    const long long xpos = (long long)ctrl->num_gauss0 + exoff[t];
    if (xpos + (long long)x > capacity) {
        raise_check(ctrl, BGS_CHECK_OVERFLOW);
        return;
    }
    for (uint32_t q = 0; q < (uint32_t)x; ++q) items[xpos + q] = make_uint2((uint32_t)t, kKindGauss | (c + q));
}

cudaError_t launch_worklist_buckets(const uint2 *ranges, int num_tiles, const ViewTable &vt, int tile_w, int tile_h,
                                    int mode, int heavy_threshold, int lpt, int gw_pixels, int pixel_rows,
                                    int gw_segment, long long extra_cap, uint32_t *slot, uint32_t *exoff,
                                    uint2 *items, long long capacity, int bseg_mode, uint2 *gw_tile,
                                    const uint32_t *cost, DevCtrl *ctrl, cudaStream_t s) {
    if (num_tiles < 0 || (gw_segment > 0 && !exoff)) return cudaErrorInvalidValue;
    const int blocks = num_tiles > 0 ? (num_tiles + kWlcThreads - 1) / kWlcThreads : 1;
    k_wl_count<<<blocks, kWlcThreads, 0, s>>>(ranges, num_tiles, vt, tile_w, tile_h, mode, heavy_threshold, lpt,
                                              gw_pixels, pixel_rows, gw_segment, extra_cap, slot, exoff, bseg_mode,
                                              cost, ctrl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || num_tiles == 0) return e;
    k_wl_emit<<<(num_tiles + 255) / 256, 256, 0, s>>>(ranges, num_tiles, vt, tile_w, tile_h, mode, heavy_threshold,
                                                      lpt, gw_pixels, pixel_rows, slot, exoff, items, capacity,
                                                      bseg_mode, gw_tile, cost, ctrl);
    return cudaGetLastError();
}

// Rewinds the queue of the current (pixel-wise) list for another persistent pass.
__global__ void k_rewind_queue(DevCtrl *ctrl) {
    ctrl->queue_head = ctrl->num_gauss;
    ctrl->queue_head_g = 0u;
    ctrl->pass_items = 0u;
    ctrl->warps_done = 0u;
}

// Host-requested fault: marks every queued item as taken, so the next pass runs none of
// them (its drain check must then raise BGS_CHECK_QUEUE).
__global__ void k_exhaust_queue(DevCtrl *ctrl) {
    ctrl->queue_head = ctrl->num_items;
    ctrl->queue_head_g = ctrl->num_gauss;
}

cudaError_t launch_rewind_queue(DevCtrl *ctrl, cudaStream_t s) {
    k_rewind_queue<<<1, 1, 0, s>>>(ctrl);
    return cudaGetLastError();
}

cudaError_t launch_exhaust_queue(DevCtrl *ctrl, cudaStream_t s) {
    k_exhaust_queue<<<1, 1, 0, s>>>(ctrl);
    return cudaGetLastError();
}

}  // namespace bgs
