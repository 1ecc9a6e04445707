// binning.cu -- a2: per-tile depth-ordered lists by a counting sort over tile rectangles.
//
// After the Gaussians are sorted by depth (ties by index), every per-tile list is the
// subsequence of that order whose rectangles cover the tile.  The lists are built without
// materialising and sorting the K duplicated entries:
//   1. k_bin_count   - the depth order is cut into B blocks of G consecutive Gaussians;
//                      block b counts, in shared memory, how many of its Gaussians cover
//                      each tile: H[b][t].
//   2. k_bin_colscan - exclusive scan of every column of H over b (in place) and the tile
//                      totals n[t].
//   3. (CUB) exclusive scan of n -> tile start; k_bin_ranges writes ranges and K.
//   4. k_bin_scatter - one warp per block walks its Gaussians in depth order and writes
//                      each one's index at start[t] + H[b][t] + (running count of the tile
//                      inside the block), for every tile t of its rectangle.
// The result is the stable (depth, index) order per tile.  Traffic is O(B T + K) words
// instead of the ~26 bytes per entry of a two-pass radix sort of (tile, index) pairs.
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

__global__ void __launch_bounds__(256) k_bin_count(long long N, int G, const uint32_t *__restrict__ order,
                                                   const float2 *__restrict__ means2D, const int *__restrict__ radii,
                                                   int tw, int th, int tx, int ty, uint32_t *__restrict__ H) {
    extern __shared__ uint32_t cnt_s[];
    const int T = tx * ty;
    const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = threadIdx.x; t < T; t += blockDim.x) cnt_s[t] = 0u;
    __syncthreads();
    const long long s0 = (long long)b * G, s1 = min(N, s0 + G);
    for (long long base = s0 + 32ll * warp; base < s1; base += 32ll * nwarps) {
        const long long s = base + lane;
        int x0 = 0, y0 = 0, w = 1, c = 0;
        if (s < s1) rect_of(means2D, radii, order[s], tw, th, tx, ty, x0, y0, w, c);
        unsigned pending = __ballot_sync(0xffffffffu, c > 0);
        while (pending) {
            const int q = __ffs(pending) - 1;
            pending &= pending - 1;
            const int cq = __shfl_sync(0xffffffffu, c, q), wq = __shfl_sync(0xffffffffu, w, q);
            const int xq = __shfl_sync(0xffffffffu, x0, q), yq = __shfl_sync(0xffffffffu, y0, q);
            for (int k = lane; k < cq; k += 32) {
                const int dy = k / wq;
                atomicAdd(&cnt_s[(yq + dy) * tx + xq + (k - dy * wq)], 1u);
            }
        }
    }
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

// Adds the view's entry count (computed in 64 bits from the per-tile totals) to bin_base.
__global__ void k_bin_advance(int T, const uint32_t *__restrict__ total, long long capacity, DevCtrl *ctrl) {
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
        if ((long long)next > capacity || next >= 0xffffffffull) atomicOr(&ctrl->check_bits, (unsigned)BGS_CHECK_OVERFLOW);
    }
}

// One warp per block of the depth order: walks its Gaussians in order and writes each
// Gaussian index into the lists of the tiles its rectangle covers.
__global__ void __launch_bounds__(32) k_bin_scatter(long long N, int G, const uint32_t *__restrict__ order,
                                                    const float2 *__restrict__ means2D, const int *__restrict__ radii,
                                                    int tw, int th, int tx, int ty, const uint32_t *__restrict__ H,
                                                    const uint32_t *__restrict__ start, uint32_t *__restrict__ point_list,
                                                    long long capacity, const DevCtrl *ctrl) {
    extern __shared__ uint32_t pos_s[];
    const int T = tx * ty;
    const int b = blockIdx.x, lane = threadIdx.x;
    const uint32_t *row = H + (size_t)b * T;
    const uint32_t base = (uint32_t)ctrl->bin_base;
    for (int t = lane; t < T; t += 32) pos_s[t] = base + start[t] + row[t];
    __syncwarp();
    const long long s0 = (long long)b * G, s1 = min(N, s0 + G);
    for (long long base = s0; base < s1; base += 32) {
        const long long s = base + lane;
        uint32_t g = 0;
        int x0 = 0, y0 = 0, w = 1, c = 0;
        if (s < s1) {
            g = order[s];
            rect_of(means2D, radii, g, tw, th, tx, ty, x0, y0, w, c);
        }
        unsigned pending = __ballot_sync(0xffffffffu, c > 0);
        while (pending) {  // in depth order: lowest lane first
            const int q = __ffs(pending) - 1;
            pending &= pending - 1;
            const int cq = __shfl_sync(0xffffffffu, c, q), wq = __shfl_sync(0xffffffffu, w, q);
            const int xq = __shfl_sync(0xffffffffu, x0, q), yq = __shfl_sync(0xffffffffu, y0, q);
            const uint32_t gq = __shfl_sync(0xffffffffu, g, q);
            for (int k = lane; k < cq; k += 32) {  // distinct tiles: no two lanes share a counter
                const int dy = k / wq;
                const int t = (yq + dy) * tx + xq + (k - dy * wq);
                const uint32_t p = pos_s[t];
                pos_s[t] = p + 1u;
                if ((long long)p < capacity) point_list[p] = gq;
            }
            __syncwarp();
        }
    }
}

size_t bin_count_smem(int T) { return sizeof(uint32_t) * (size_t)T; }

cudaError_t setup_bin_kernels(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

cudaError_t launch_bin_count(long long N, int G, int B, const uint32_t *order, const float *means2D, const int *radii,
                             int W, int H, int tw, int th, uint32_t *Hm, cudaStream_t s) {
    const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    k_bin_count<<<B, 256, bin_count_smem(tx * ty), s>>>(N, G, order, reinterpret_cast<const float2 *>(means2D), radii,
                                                         tw, th, tx, ty, Hm);
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

cudaError_t launch_bin_advance(int T, const uint32_t *start, const uint32_t *total, long long capacity, DevCtrl *ctrl,
                               cudaStream_t s) {
    (void)start;
    k_bin_advance<<<1, 1024, 0, s>>>(T, total, capacity, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_bin_scatter(long long N, int G, int B, const uint32_t *order, const float *means2D, const int *radii,
                               int W, int H, int tw, int th, const uint32_t *Hm, const uint32_t *start,
                               uint32_t *point_list, long long capacity, const DevCtrl *ctrl, cudaStream_t s) {
    const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    k_bin_scatter<<<B, 32, bin_count_smem(tx * ty), s>>>(N, G, order, reinterpret_cast<const float2 *>(means2D), radii,
                                                          tw, th, tx, ty, Hm, start, point_list, capacity, ctrl);
    return cudaGetLastError();
}

}  // namespace bgs
