// binning.cu -- a2: per-tile depth-ordered lists in one pass over the duplicated entries.
//
// After the Gaussians are sorted by depth (ties by index), every per-tile list is the
// subsequence of that order whose rectangles cover the tile.  Conceptually every Gaussian
// emits one (tile, index) entry per covered tile in depth order (entry e of the stream
// belongs to the Gaussian whose exclusive entry offset is the last one <= e) and the
// entries are stably partitioned by tile.  The stream is cut into chunks of kChunk
// consecutive entries, regenerated from the Gaussians' rectangles whenever needed:
//   1. k_chunk_first - first Gaussian of every chunk.
//   2. k_bin_count   - chunk b counts its entries per tile in shared memory: H[b][t].
//   3. k_bin_colscan - exclusive scan of every column of H over b (in place) and the tile
//                      totals n[t]; (CUB) exclusive scan of n -> tile starts; ranges.
//   4. k_bin_sort_scatter - chunk b regenerates its entries, sorts them by tile in shared
//                      memory with a stable block radix sort, ranks each entry inside its
//                      tile's run and writes its Gaussian index to
//                      start[t] + H[b][t] + rank, the runs coalesced.
// The result is the stable (depth, index) order per tile; the K entries are written once
// and never sorted in global memory.
#include <cub/block/block_exchange.cuh>
#include <cub/block/block_radix_sort.cuh>
#include <cub/block/block_scan.cuh>

#include "bgs_internal.cuh"

namespace bgs {

__device__ __forceinline__ void rect_of(const float2 *__restrict__ means2D, const int *__restrict__ radii, uint32_t g,
                                        int tw, int th, int tx, int ty, int &x0, int &y0, int &w, int &cnt) {
    x0 = y0 = 0;
    w = 1;
    cnt = 0;
    const int r = radii[g];
    if (r <= 0) return;
    const float2 m = means2D[g];
    // same float32 operations as the preprocess and oracle rectangles
    int x1, y1;
    x0 = (int)floorf(__fdiv_rn(__fsub_rn(m.x, (float)r), (float)tw));
    x1 = (int)floorf(__fdiv_rn(__fadd_rn(m.x, (float)(r + tw - 1)), (float)tw));
    y0 = (int)floorf(__fdiv_rn(__fsub_rn(m.y, (float)r), (float)th));
    y1 = (int)floorf(__fdiv_rn(__fadd_rn(m.y, (float)(r + th - 1)), (float)th));
    x0 = min(max(x0, 0), tx);
    x1 = min(max(x1, 0), tx);
    y0 = min(max(y0, 0), ty);
    y1 = min(max(y1, 0), ty);
    if (x1 > x0 && y1 > y0) {
        w = x1 - x0;
        cnt = w * (y1 - y0);
    }
}

// first Gaussian (depth position) of every chunk of kChunk entries
__global__ void __launch_bounds__(256) k_chunk_first(long long N, const unsigned long long *__restrict__ offsets,
                                                     const uint32_t *__restrict__ counts, long long chunk,
                                                     long long num_chunks, uint32_t *__restrict__ first) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const unsigned long long c = counts[s];
    if (c == 0) return;
    const unsigned long long off = offsets[s];
    for (unsigned long long b = (off + chunk - 1) / chunk; b * chunk < off + c && (long long)b < num_chunks; ++b)
        first[b] = (uint32_t)s;
}

// Visits the entries [e0, e1) of the depth-ordered entry stream: fn(local position, tile, Gaussian index).
// Warps take 32 consecutive Gaussians at a time (strided over the block) starting at
// s_first; each one's entries are spread over the warp's lanes.
template <typename Fn>
__device__ __forceinline__ void for_chunk_entries(long long N, const uint32_t *__restrict__ order,
                                                  const unsigned long long *__restrict__ offsets,
                                                  const float2 *__restrict__ means2D, const int *__restrict__ radii,
                                                  int tw, int th, int tx, int ty, long long s_first,
                                                  unsigned long long e0, unsigned long long e1, Fn fn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (long long base = s_first + 32ll * warp;; base += 32ll * nwarps) {
        const long long s = base + lane;
        int x0 = 0, y0 = 0, w = 1, c = 0;
        uint32_t g = 0;
        unsigned long long off = e1;
        if (s < N) {
            off = offsets[s];
            if (off < e1) {
                g = order[s];
                rect_of(means2D, radii, g, tw, th, tx, ty, x0, y0, w, c);
            }
        }
        // the warp's first Gaussian starts past the chunk: every later one does too
        if (__shfl_sync(0xffffffffu, off, 0) >= e1 || base >= N) break;
        unsigned pending = __ballot_sync(0xffffffffu, c > 0 && off < e1 && off + (unsigned long long)c > e0);
        while (pending) {
            const int q = __ffs(pending) - 1;
            pending &= pending - 1;
            const int cq = __shfl_sync(0xffffffffu, c, q), wq = __shfl_sync(0xffffffffu, w, q);
            const int xq = __shfl_sync(0xffffffffu, x0, q), yq = __shfl_sync(0xffffffffu, y0, q);
            const uint32_t gq = __shfl_sync(0xffffffffu, g, q);
            const unsigned long long oq = __shfl_sync(0xffffffffu, off, q);
            const int k0 = oq < e0 ? (int)(e0 - oq) : 0;
            const int k1 = (int)min((unsigned long long)cq, e1 - oq);
            for (int k = k0 + lane; k < k1; k += 32) {
                const int dy = k / wq;
                fn((int)(oq + k - e0), (yq + dy) * tx + xq + (k - dy * wq), gq);
            }
        }
    }
}

__global__ void __launch_bounds__(512) k_bin_count(long long N, const uint32_t *__restrict__ order,
                                                   const unsigned long long *__restrict__ offsets,
                                                   const uint32_t *__restrict__ first,
                                                   const unsigned long long *view_entries,
                                                   const float2 *__restrict__ means2D, const int *__restrict__ radii,
                                                   int tw, int th, int tx, int ty, uint32_t *__restrict__ H) {
    extern __shared__ uint32_t cnt_s[];
    const int T = tx * ty;
    const int b = blockIdx.x;
    for (int t = threadIdx.x; t < T; t += blockDim.x) cnt_s[t] = 0u;
    __syncthreads();
    const unsigned long long K = *view_entries;
    const unsigned long long e0 = (unsigned long long)b * kChunk, e1 = min(K, e0 + kChunk);
    if (e0 < e1)
        for_chunk_entries(N, order, offsets, means2D, radii, tw, th, tx, ty, first[b], e0, e1,
                          [&](int, int t, uint32_t) { atomicAdd(&cnt_s[t], 1u); });
    __syncthreads();
    uint32_t *row = H + (size_t)b * T;
    for (int t = threadIdx.x; t < T; t += blockDim.x) row[t] = cnt_s[t];
}

// Block (32 tiles) x (32 row groups): per column t, exclusive prefix over b in place, and
// the column total n[t].
__global__ void __launch_bounds__(1024) k_bin_colscan(int B, int T, uint32_t *__restrict__ H,
                                                      uint32_t *__restrict__ total) {
    __shared__ uint32_t part[32][33];
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int t = blockIdx.x * 32 + lx;
    const int rows = (B + 31) / 32;
    const int b0 = ly * rows, b1 = min(B, b0 + rows);
    uint32_t sum = 0;
    if (t < T)
        for (int b = b0; b < b1; ++b) sum += H[(size_t)b * T + t];
    part[ly][lx] = sum;
    __syncthreads();
    if (ly == 0) {
        uint32_t run = 0;
        for (int gq = 0; gq < 32; ++gq) {
            const uint32_t v = part[gq][lx];
            part[gq][lx] = run;
            run += v;
        }
        if (t < T) total[t] = run;
    }
    __syncthreads();
    if (t < T) {
        uint32_t off = part[ly][lx];
        for (int b = b0; b < b1; ++b) {
            const uint32_t h = H[(size_t)b * T + t];
            H[(size_t)b * T + t] = off;
            off += h;
        }
    }
}

// ranges[t] = bin_base + [start[t], start[t] + n[t]) for the tiles of one view ((0,0) for
// an empty tile).
__global__ void k_bin_ranges(int T, const uint32_t *__restrict__ start, const uint32_t *__restrict__ total,
                             uint2 *__restrict__ ranges, const DevCtrl *ctrl) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const uint32_t base = (uint32_t)ctrl->bin_base;
    const uint32_t a = base + start[t], n = total[t];
    ranges[t] = n ? make_uint2(a, a + n) : make_uint2(0u, 0u);
}

// Adds the view's entry count (computed in 64 bits from the per-tile totals) to bin_base;
// flags an overflow past the point_list capacity or past the view's chunk capacity.
__global__ void k_bin_advance(int T, const uint32_t *__restrict__ total, long long capacity, int view,
                              long long chunk_capacity, DevCtrl *ctrl) {
    __shared__ unsigned long long part[32];
    unsigned long long n = 0;
    for (int t = threadIdx.x; t < T; t += blockDim.x) n += total[t];
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long k = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) k += part[w];
        const unsigned long long next = ctrl->bin_base + k;
        ctrl->bin_base = next;
        ctrl->num_entries = next;
        if ((long long)next > capacity || next >= 0xffffffffull ||
            (long long)ctrl->view_entries[view] > chunk_capacity)
            atomicOr(&ctrl->check_bits, (unsigned)BGS_CHECK_OVERFLOW);
    }
}

// Chunk b: regenerate its entries, stable block radix sort by tile, rank inside each
// tile's run, write index g to bin_base + start[t] + H[b][t] + rank.
constexpr int kSortThreads = 512;
constexpr int kSortItems = kChunk / kSortThreads;
using SortKey = uint16_t;  // tile ids of a view are < 65536
using BlockSortT = cub::BlockRadixSort<SortKey, kSortThreads, kSortItems, uint32_t>;
using BlockScanT = cub::BlockScan<int, kSortThreads>;
using BlockExchangeT = cub::BlockExchange<uint32_t, kSortThreads, kSortItems>;

struct SortSmem {
    union {
        struct {
            SortKey key[kChunk];
            uint32_t val[kChunk];
        } stage;
        typename BlockSortT::TempStorage sort;
        SortKey sorted_key[kChunk];
        typename BlockExchangeT::TempStorage exchange;
    } u;
    typename BlockScanT::TempStorage scan;
};

size_t bin_sort_smem() { return sizeof(SortSmem); }

__global__ void __launch_bounds__(kSortThreads) k_bin_sort_scatter(
    long long N, const uint32_t *__restrict__ order, const unsigned long long *__restrict__ offsets,
    const uint32_t *__restrict__ first, const unsigned long long *view_entries, const DevCtrl *ctrl,
    const float2 *__restrict__ means2D, const int *__restrict__ radii, int tw, int th, int tx, int ty,
    const uint32_t *__restrict__ H, const uint32_t *__restrict__ start, uint32_t *__restrict__ point_list,
    long long capacity, int end_bit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &sm = *reinterpret_cast<SortSmem *>(smem_raw);
    const int T = tx * ty;
    const int b = blockIdx.x;
    const unsigned long long K = *view_entries;
    const unsigned long long e0 = (unsigned long long)b * kChunk, e1 = min(K, e0 + kChunk);
    if (e0 >= e1) return;  // uniform over the block
    const int n = (int)(e1 - e0);
    // 1. the chunk's entries in stream order (padding sorts last and is never written)
    for (int i = threadIdx.x; i < kChunk; i += kSortThreads) {
        if (i >= n) {
            sm.u.stage.key[i] = (SortKey)0xffffu;
            sm.u.stage.val[i] = 0xffffffffu;
        }
    }
    for_chunk_entries(N, order, offsets, means2D, radii, tw, th, tx, ty, first[b], e0, e1,
                      [&](int i, int t, uint32_t g) {
                          sm.u.stage.key[i] = (SortKey)t;
                          sm.u.stage.val[i] = g;
                      });
    __syncthreads();
    SortKey keys[kSortItems];
    uint32_t vals[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        keys[j] = sm.u.stage.key[threadIdx.x * kSortItems + j];
        vals[j] = sm.u.stage.val[threadIdx.x * kSortItems + j];
    }
    __syncthreads();
    // 2. stable sort by tile (blocked arrangement in, blocked out)
    BlockSortT(sm.u.sort).Sort(keys, vals, 0, end_bit);
    __syncthreads();
    // 3. rank inside the tile's run: position minus the run's first position (max-scan of heads)
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) sm.u.sorted_key[threadIdx.x * kSortItems + j] = keys[j];
    __syncthreads();
    int heads[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int p = threadIdx.x * kSortItems + j;
        heads[j] = (p == 0 || sm.u.sorted_key[p - 1] != keys[j]) ? p : 0;
    }
    __syncthreads();
    BlockScanT(sm.scan).InclusiveScan(heads, heads, [](int a, int b) { return a > b ? a : b; });
    // 4. global slots, then write in striped order (consecutive threads, consecutive slots)
    const uint32_t base = (uint32_t)ctrl->bin_base;
    const uint32_t *row = H + (size_t)b * T;
    uint32_t pos[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int p = threadIdx.x * kSortItems + j;
        const int t = (int)keys[j];
        pos[j] = (p < n && t < T) ? base + start[t] + row[t] + (uint32_t)(p - heads[j]) : 0xffffffffu;
    }
    BlockExchangeT(sm.u.exchange).BlockedToStriped(pos);
    __syncthreads();
    BlockExchangeT(sm.u.exchange).BlockedToStriped(vals);
#pragma unroll
    for (int j = 0; j < kSortItems; ++j)
        if (pos[j] != 0xffffffffu && (long long)pos[j] < capacity) point_list[pos[j]] = vals[j];
}

size_t bin_count_smem(int T) { return sizeof(uint32_t) * (size_t)T; }

cudaError_t setup_bin_kernels(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bin_sort_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bin_sort_smem());
    return e;
}

cudaError_t launch_chunk_first(long long N, const unsigned long long *offsets, const uint32_t *counts, long long B,
                               uint32_t *first, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    k_chunk_first<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, offsets, counts, kChunk, B, first);
    return cudaGetLastError();
}

cudaError_t launch_bin_count(long long N, int B, const uint32_t *order, const unsigned long long *offsets,
                             const uint32_t *first, const unsigned long long *view_entries, const float *means2D,
                             const int *radii, int W, int H, int tw, int th, uint32_t *Hm, cudaStream_t s) {
    const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    k_bin_count<<<B, 512, bin_count_smem(tx * ty), s>>>(N, order, offsets, first, view_entries,
                                                         reinterpret_cast<const float2 *>(means2D), radii, tw, th, tx,
                                                         ty, Hm);
    return cudaGetLastError();
}

cudaError_t launch_bin_colscan(int B, int T, uint32_t *Hm, uint32_t *total, cudaStream_t s) {
    k_bin_colscan<<<(T + 31) / 32, dim3(32, 32), 0, s>>>(B, T, Hm, total);
    return cudaGetLastError();
}

cudaError_t launch_bin_ranges(int T, const uint32_t *start, const uint32_t *total, uint2 *ranges, DevCtrl *ctrl,
                              cudaStream_t s) {
    k_bin_ranges<<<(T + 255) / 256, 256, 0, s>>>(T, start, total, ranges, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_bin_advance(int T, const uint32_t *total, long long capacity, int view, long long chunk_capacity,
                               DevCtrl *ctrl, cudaStream_t s) {
    k_bin_advance<<<1, 1024, 0, s>>>(T, total, capacity, view, chunk_capacity, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_bin_sort_scatter(long long N, int B, const uint32_t *order, const unsigned long long *offsets,
                                    const uint32_t *first, const unsigned long long *view_entries, const DevCtrl *ctrl,
                                    const float *means2D, const int *radii, int W, int H, int tw, int th,
                                    const uint32_t *Hm, const uint32_t *start, uint32_t *point_list, long long capacity,
                                    int end_bit, cudaStream_t s) {
    const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    k_bin_sort_scatter<<<B, kSortThreads, bin_sort_smem(), s>>>(N, order, offsets, first, view_entries, ctrl,
                                                                 reinterpret_cast<const float2 *>(means2D), radii, tw,
                                                                 th, tx, ty, Hm, start, point_list, capacity, end_bit);
    return cudaGetLastError();
}

}  // namespace bgs
