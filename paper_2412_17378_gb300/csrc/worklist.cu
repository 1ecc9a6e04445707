// worklist.cu -- a3: per-tile load statistics and the work list of the persistent kernels.
//
// The paper's task pool (Sec. 4.1) holds whole tiles; its fine-grained variant
// (Sec. 4.3) splits each tile into 4-pixel tasks, and its selector (Sec. 4.4) chooses
// between the Gaussian-wise and the pixel-wise kernel.  Here the choice is made per
// tile from its list length n (the paper names "the Gaussians of a tile" as the key
// load-balance metric, Sec. 4.4):
//   n >  heavy_threshold -> Gaussian-wise items of P pixels (one warp each),
//   n <= heavy_threshold -> pixel-wise items of 8 x 4Q pixels (one warp, Q pixels per lane).
// Tiles of all views of a batched call share one global tile space.
// Items of heavier tiles are queued first (longest-processing-time order) so the long
// items start early and the light ones fill the tail.
#include <cub/block/block_radix_sort.cuh>
#include <cub/block/block_scan.cuh>

#include "bgs_internal.cuh"

namespace bgs {

__device__ __forceinline__ bool tile_is_gauss(int mode, int heavy_threshold, uint32_t n) {
    return mode == BGS_MODE_GAUSSIAN || (mode == BGS_MODE_AUTO && n > (uint32_t)heavy_threshold);
}

// Items of tile t: Gaussian-wise, P pixels each; else pixel-wise sub-blocks of its visible part.
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

__device__ __forceinline__ uint32_t tile_item_count(int t, uint32_t n, const ViewTable &vt, int tile_w, int tile_h,
                                                    int mode, int heavy_threshold, int gw_pixels, int pixel_rows) {
    return tile_items(t, tile_is_gauss(mode, heavy_threshold, n), vt, tile_w, tile_h, gw_pixels, pixel_rows);
}

// Sort key of each tile for the descending stable sort: its kind in the top bit (Gaussian-
// wise tiles first) and, when lpt is on, a log-scale bucket of its list length below it
// (heaviest first; lengths within ~19% share a bucket): bucket = 4 floor(log2 n) + the two
// bits after the leading one, + 1 (0 for an empty tile).  One 8-bit radix pass sorts it.
__device__ __forceinline__ uint32_t length_bucket(uint32_t n) {
    if (n == 0u) return 0u;
    const int e = 31 - __clz(n);
    const uint32_t m = e >= 2 ? (n >> (e - 2)) & 3u : (n << (2 - e)) & 3u;
    return min(127u, 4u * (uint32_t)e + m + 1u);
}

__global__ void k_tile_counts(const uint2 *__restrict__ ranges, int num_tiles, int mode, int heavy_threshold, int lpt,
                              uint32_t *__restrict__ tile_key, uint32_t *__restrict__ tile_idx) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= num_tiles) return;
    const uint2 rg = ranges[t];
    const uint32_t n = rg.y >= rg.x ? rg.y - rg.x : 0u;
    const uint32_t kind = tile_is_gauss(mode, heavy_threshold, n) ? 1u : 0u;
    tile_key[t] = lpt ? (kind << 7) | length_bucket(n) : kind;
    tile_idx[t] = (uint32_t)t;
}

cudaError_t launch_tile_counts(const uint2 *ranges, int num_tiles, int mode, int heavy_threshold, int lpt,
                               uint32_t *tile_key, uint32_t *tile_idx, cudaStream_t s) {
    if (num_tiles == 0) return cudaSuccess;
    k_tile_counts<<<(num_tiles + 255) / 256, 256, 0, s>>>(ranges, num_tiles, mode, heavy_threshold, lpt, tile_key,
                                                         tile_idx);
    return cudaGetLastError();
}

__global__ void k_gather_counts(const uint32_t *__restrict__ order, int num_tiles, const uint2 *__restrict__ ranges,
                                const ViewTable vt, int tile_w, int tile_h, int mode, int heavy_threshold,
                                int gw_pixels, int pixel_rows, uint32_t *__restrict__ counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= num_tiles) return;
    const int t = (int)order[i];
    const uint2 rg = ranges[t];
    const uint32_t n = rg.y >= rg.x ? rg.y - rg.x : 0u;
    counts[i] = tile_item_count(t, n, vt, tile_w, tile_h, mode, heavy_threshold, gw_pixels, pixel_rows);
}

cudaError_t launch_gather_counts(const uint32_t *order, int num_tiles, const uint2 *ranges, const ViewTable &vt,
                                 int tile_w, int tile_h, int mode, int heavy_threshold, int gw_pixels,
                                 int pixel_rows, uint32_t *counts, cudaStream_t s) {
    if (num_tiles == 0) return cudaSuccess;
    k_gather_counts<<<(num_tiles + 255) / 256, 256, 0, s>>>(order, num_tiles, ranges, vt, tile_w, tile_h, mode,
                                                            heavy_threshold, gw_pixels, pixel_rows, counts);
    return cudaGetLastError();
}

// One warp per tile writes the tile's items at its offset; the last tile also publishes
// the total and resets the queue cursor.
__global__ void k_emit_items(const uint32_t *__restrict__ order, const uint32_t *__restrict__ counts,
                             const uint32_t *__restrict__ offsets, int num_tiles, const uint2 *__restrict__ ranges,
                             int mode, int heavy_threshold, uint2 *__restrict__ items, DevCtrl *ctrl) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= num_tiles) return;
    const uint32_t t = order[i];
    const uint2 rg = ranges[t];
    const uint32_t n = rg.y >= rg.x ? rg.y - rg.x : 0u;
    const uint32_t kind = tile_is_gauss(mode, heavy_threshold, n) ? kKindGauss : 0u;
    const uint32_t c = counts[i], off = offsets[i];
    for (uint32_t q = lane; q < c; q += 32) items[off + q] = make_uint2(t, kind | q);
    if (lane == 0) {
        // Gaussian-wise tiles come first: the boundary between the kinds sets num_gauss
        bool next_gauss = false;
        if (i + 1 < num_tiles) {
            const uint2 rn = ranges[order[i + 1]];
            next_gauss = tile_is_gauss(mode, heavy_threshold, rn.y >= rn.x ? rn.y - rn.x : 0u);
        }
        uint32_t ng = 0xffffffffu;
        if (i == 0 && !kind) ng = 0u;
        if (kind && !next_gauss) ng = off + c;
        if (ng != 0xffffffffu) {
            ctrl->num_gauss = ng;
            ctrl->queue_head = ng;
            ctrl->queue_head_g = 0u;
            ctrl->pass_items = 0u;
            ctrl->warps_done = 0u;
        }
        if (i == num_tiles - 1) ctrl->num_items = off + c;
    }
}

cudaError_t launch_emit_items(const uint32_t *order, const uint32_t *counts, const uint32_t *offsets, int num_tiles,
                              const uint2 *ranges, int mode, int heavy_threshold, uint2 *items, DevCtrl *ctrl,
                              cudaStream_t s) {
    if (num_tiles == 0) return cudaSuccess;
    const long long threads = (long long)num_tiles * 32;
    k_emit_items<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(order, counts, offsets, num_tiles, ranges, mode,
                                                                   heavy_threshold, items, ctrl);
    return cudaGetLastError();
}

// ---- one-block build for grids of up to kWlMaxTiles tiles ---------------------------------
// The same list as k_tile_counts + the stable descending key sort + k_gather_counts + the
// exclusive scan + k_emit_items, in one launch: each of 1024 threads loads 8 tiles' ranges,
// a block radix sort orders the keys (descending, stable: equal keys keep the tile order;
// padding entries carry key 0 and indices past T, so they sort after every tile), a block
// scan of the sorted tiles' item counts gives every tile its first item, and each thread
// writes its tiles' items.  At a few thousand tiles the multi-kernel chain is dominated by
// launch latency.
constexpr int kWlThreads = 1024, kWlPerThread = 8;
constexpr int kWlMaxTiles = kWlThreads * kWlPerThread;

__global__ void __launch_bounds__(kWlThreads) k_build_worklist(const uint2 *__restrict__ ranges, int T,
                                                                const ViewTable vt, int tile_w, int tile_h, int mode,
                                                                int heavy_threshold, int lpt, int gw_pixels,
                                                                int pixel_rows, uint2 *__restrict__ items,
                                                                DevCtrl *ctrl) {
    using Sort = cub::BlockRadixSort<uint32_t, kWlThreads, kWlPerThread, uint32_t>;
    using Scan = cub::BlockScan<uint32_t, kWlThreads>;
    __shared__ union {
        typename Sort::TempStorage sort;
        typename Scan::TempStorage scan;
    } tmp;
    __shared__ uint32_t n_gauss;
    if (threadIdx.x == 0) n_gauss = 0u;
    uint32_t key[kWlPerThread], tile[kWlPerThread];
#pragma unroll
    for (int j = 0; j < kWlPerThread; ++j) {
        const int t = threadIdx.x * kWlPerThread + j;
        key[j] = 0u;
        tile[j] = (uint32_t)t;
        if (t < T) {
            const uint2 rg = ranges[t];
            const uint32_t n = rg.y >= rg.x ? rg.y - rg.x : 0u;
            const uint32_t kind = tile_is_gauss(mode, heavy_threshold, n) ? 1u : 0u;
            key[j] = lpt ? (kind << 7) | length_bucket(n) : kind;
        }
    }
    Sort(tmp.sort).SortDescending(key, tile, 0, lpt ? 8 : 1);
    __syncthreads();  // tmp is reused by the scan
    // this thread now holds sorted positions threadIdx.x * kWlPerThread + j
    uint32_t cnt[kWlPerThread], sum = 0u, gsum = 0u;
#pragma unroll
    for (int j = 0; j < kWlPerThread; ++j) {
        const int r = threadIdx.x * kWlPerThread + j;
        const bool gauss = (lpt ? key[j] >> 7 : key[j]) != 0u;
        cnt[j] = r < T ? tile_items((int)tile[j], gauss, vt, tile_w, tile_h, gw_pixels, pixel_rows) : 0u;
        sum += cnt[j];
        if (gauss && r < T) gsum += cnt[j];
    }
    uint32_t off, total;
    Scan(tmp.scan).ExclusiveSum(sum, off, total);
    if (gsum) atomicAdd(&n_gauss, gsum);
#pragma unroll
    for (int j = 0; j < kWlPerThread; ++j) {
        const uint32_t kindbit = (lpt ? key[j] >> 7 : key[j]) != 0u ? kKindGauss : 0u;
        for (uint32_t q = 0; q < cnt[j]; ++q) items[off + q] = make_uint2(tile[j], kindbit | q);
        off += cnt[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // Gaussian-wise tiles sort first (the kind is the key's top bit): items [0, num_gauss)
        const uint32_t ng = n_gauss;
        ctrl->num_gauss = ng;
        ctrl->queue_head = ng;
        ctrl->queue_head_g = 0u;
        ctrl->pass_items = 0u;
        ctrl->warps_done = 0u;
        ctrl->num_items = total;
    }
}

int worklist_one_block_max_tiles() { return kWlMaxTiles; }

cudaError_t launch_build_worklist(const uint2 *ranges, int num_tiles, const ViewTable &vt, int tile_w, int tile_h,
                                  int mode, int heavy_threshold, int lpt, int gw_pixels, int pixel_rows,
                                  uint2 *items, DevCtrl *ctrl, cudaStream_t s) {
    if (num_tiles < 0 || num_tiles > kWlMaxTiles) return cudaErrorInvalidValue;
    k_build_worklist<<<1, kWlThreads, 0, s>>>(ranges, num_tiles, vt, tile_w, tile_h, mode, heavy_threshold, lpt,
                                              gw_pixels, pixel_rows, items, ctrl);
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
