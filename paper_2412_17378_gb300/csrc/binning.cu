// binning.cu -- a2: per-tile depth-ordered lists by a counting sort over tile rectangles.
//
// After the Gaussians are sorted by depth (ties by index), every per-tile list is the
// subsequence of that order whose rectangles cover the tile.  The lists are built without
// materialising and sorting the K duplicated entries:
//   1. k_bin_count   - the depth order is cut into B blocks of G consecutive Gaussians;
//                      block b counts how many of its Gaussians cover each tile, H[b][t],
//                      as a 2D difference array in shared memory (4 updates per
//                      rectangle) followed by a prefix sum along x then y.  It also stores
//                      every sorted position's packed rectangle for step 4.
//   2. k_bin_colscan - exclusive scan of every column of H over b (in place) and the tile
//                      totals n[t].
//   3. (CUB) exclusive scan of n -> tile start; k_bin_ranges writes ranges and K.
//   4. k_bin_scatter - block (b, tile row), one warp, the row's write positions
//                      start[t] + H[b][t] in shared memory.  The warp visits the block's
//                      Gaussians that cover its row in depth order; lane l appends the
//                      Gaussian's index to the l-th tile of its x-range.  Blocks run row
//                      after row in launch order, so the slice of the point list being
//                      written (a few tile rows) stays resident in L2 while its sectors fill
//                      up from many blocks.
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
                                                   int tw, int th, int tx, int ty, uint32_t *__restrict__ H,
                                                   uint32_t *__restrict__ rect_x, uint32_t *__restrict__ rect_y) {
    extern __shared__ uint32_t d_s[];
    const int T = tx * ty;
    const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = threadIdx.x; t < T; t += blockDim.x) d_s[t] = 0u;
    __syncthreads();
    // 2D difference array: +1 at (x0, y0) and (x1, y1), -1 at (x1, y0) and (x0, y1)
    // (modulo 2^32; the prefix sums below give the exact non-negative counts)
    const long long s0 = (long long)b * G, s1 = min(N, s0 + G);
    for (long long s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        int x0, y0, w, c;
        rect_of(means2D, radii, order[s], tw, th, tx, ty, x0, y0, w, c);
        uint32_t px = 0u, py = 0u;  // packed (x0 | w << 16, y0 | h << 16); h = 0 if empty
        if (c > 0) {
            const int h = c / w, x1 = x0 + w, y1 = y0 + h;
            px = (uint32_t)x0 | ((uint32_t)w << 16);
            py = (uint32_t)y0 | ((uint32_t)h << 16);
            atomicAdd(&d_s[y0 * tx + x0], 1u);
            if (x1 < tx) atomicAdd(&d_s[y0 * tx + x1], 0xffffffffu);
            if (y1 < ty) {
                atomicAdd(&d_s[y1 * tx + x0], 0xffffffffu);
                if (x1 < tx) atomicAdd(&d_s[y1 * tx + x1], 1u);
            }
        }
        rect_x[s] = px;
        rect_y[s] = py;
    }
    __syncthreads();
    // prefix along x: one warp per tile row, 32 columns per step
    for (int y = warp; y < ty; y += nwarps) {
        uint32_t carry = 0u;
        for (int xb = 0; xb < tx; xb += 32) {
            const int x = xb + lane;
            uint32_t v = x < tx ? d_s[y * tx + x] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (x < tx) d_s[y * tx + x] = v + carry;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    // prefix along y: one thread per tile column, written straight to H[b]
    uint32_t *row = H + (size_t)b * T;
    for (int x = threadIdx.x; x < tx; x += blockDim.x) {
        uint32_t run = 0u;
        for (int y = 0; y < ty; ++y) {
            run += d_s[y * tx + x];
            row[y * tx + x] = run;
        }
    }
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

// Block (b, row): one warp; the row's write positions start[t] + H[b][t] live in shared
// memory.  The block's Gaussians that cover the row are compacted (depth order kept) 32 at
// a time into a shared list and visited in order; for each, lane l appends the Gaussian's
// index to the l-th tile of its x-range.
__global__ void __launch_bounds__(32) k_bin_scatter(uint32_t N, uint32_t G, const uint32_t *__restrict__ order,
                                                    const uint32_t *__restrict__ rect_x,
                                                    const uint32_t *__restrict__ rect_y, int tx, int ty,
                                                    const uint32_t *__restrict__ H, const uint32_t *__restrict__ start,
                                                    uint32_t *__restrict__ point_list, uint32_t capacity,
                                                    const DevCtrl *ctrl) {
    extern __shared__ uint32_t pos_s[];
    __shared__ uint2 hit_s[32];  // (x0 | w << 16, index) of the group's Gaussians on the row
    const int b = blockIdx.x, r = blockIdx.y, lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    const size_t t0 = (size_t)r * tx;
    const uint32_t *hrow = H + (size_t)b * tx * ty + t0;
    const uint32_t base = (uint32_t)ctrl->bin_base;
    for (int x = lane; x < tx; x += 32) pos_s[x] = base + start[t0 + x] + hrow[x];
    __syncwarp();
    const uint32_t s0 = (uint32_t)b * G, s1 = min(N, s0 + G);
    // 512 Gaussians per pass: all rectangle / index loads of the pass are issued before any
    // is used (two dependent rounds instead of one per 32 Gaussians)
    constexpr int kPre = 16;
    for (uint32_t cb = s0; cb < s1; cb += 32 * kPre) {
        uint32_t py[kPre], span[kPre], g[kPre];
#pragma unroll
        for (int i = 0; i < kPre; ++i) {
            const uint32_t s = cb + 32 * i + lane;
            py[i] = s < s1 ? rect_y[s] : 0u;
        }
#pragma unroll
        for (int i = 0; i < kPre; ++i) {
            const uint32_t s = cb + 32 * i + lane;
            const bool on_row = (uint32_t)(r - (int)(py[i] & 0xffffu)) < (py[i] >> 16);  // y0 <= r < y0 + h
            span[i] = on_row ? rect_x[s] : 0u;  // x0 | w << 16 (w = 0: not on this row)
            g[i] = on_row ? order[s] : 0u;
        }
        for (int i = 0; i < kPre; ++i) {
            const bool hit = (span[i] >> 16) != 0u;
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (m == 0u) continue;
            if (hit) hit_s[__popc(m & lt)] = make_uint2(span[i], g[i]);
            __syncwarp();
            const int nh = __popc(m);
#pragma unroll 1
            for (int c = 0; c < nh; ++c) {  // depth order
                const uint2 e = hit_s[c];
                const int x0 = (int)(e.x & 0xffffu), w = (int)(e.x >> 16);
                // distinct tiles: no two lanes share a counter
                if (lane < w) {
                    const uint32_t pp = pos_s[x0 + lane];
                    pos_s[x0 + lane] = pp + 1u;
                    if (pp < capacity) point_list[pp] = e.y;
                }
                if (w > 32) {  // rare: ranges wider than the warp
#pragma unroll 1
                    for (int k = lane + 32; k < w; k += 32) {
                        const uint32_t pp = pos_s[x0 + k];
                        pos_s[x0 + k] = pp + 1u;
                        if (pp < capacity) point_list[pp] = e.y;
                    }
                }
                __syncwarp();
            }
        }
    }
}

size_t bin_count_smem(int T) { return sizeof(uint32_t) * (size_t)T; }

cudaError_t setup_bin_kernels(int tx, int ty) {
    const size_t sc = bin_count_smem(tx * ty), ss = sizeof(uint32_t) * (size_t)tx;
    cudaError_t e = cudaSuccess;
    if (sc > 48 * 1024) e = cudaFuncSetAttribute(k_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
    if (e == cudaSuccess && ss > 48 * 1024)
        e = cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    return e;
}

cudaError_t launch_bin_count(long long N, int G, int B, const uint32_t *order, const float *means2D, const int *radii,
                             int W, int H, int tw, int th, uint32_t *Hm, uint32_t *rect_x, uint32_t *rect_y,
                             cudaStream_t s) {
    const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    k_bin_count<<<B, 256, bin_count_smem(tx * ty), s>>>(N, G, order, reinterpret_cast<const float2 *>(means2D), radii,
                                                         tw, th, tx, ty, Hm, rect_x, rect_y);
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

cudaError_t launch_bin_scatter(long long N, int G, int B, const uint32_t *order, const uint32_t *rect_x,
                               const uint32_t *rect_y, int W, int H, int tw, int th, const uint32_t *Hm,
                               const uint32_t *start, uint32_t *point_list, long long capacity, const DevCtrl *ctrl,
                               cudaStream_t s) {
    const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    // indices, sorted positions and list slots are < 2^32 (checked by the callers)
    const uint32_t cap = capacity >= 0xffffffffll ? 0xffffffffu : (uint32_t)capacity;
    k_bin_scatter<<<dim3(B, ty), 32, sizeof(uint32_t) * tx, s>>>((uint32_t)N, (uint32_t)G, order, rect_x, rect_y, tx,
                                                                 ty, Hm, start, point_list, cap, ctrl);
    return cudaGetLastError();
}

}  // namespace bgs
