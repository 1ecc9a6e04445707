// binning.cu -- a2: per-tile depth-ordered lists by a counting sort over tile rectangles.
//
// After the Gaussians are sorted by depth (ties by index), every per-tile list is the
// subsequence of that order whose rectangles cover the tile.  The lists are built without
// materialising and sorting the K duplicated entries:
//   1. k_bin_count   - the depth order is cut into B blocks of G consecutive Gaussians;
//                      block b counts how many of its Gaussians cover each tile, H[b][t],
//                      as a 2D difference array in shared memory (4 updates per
//                      rectangle) followed by a prefix sum along x then y.  It also stores
//                      every sorted position's packed rectangle and Gaussian index (one
//                      16-byte record) and, per group of 8 x 4 tiles C, a bit mask of the
//                      block's Gaussians whose rectangle meets C.
//   2. k_bin_colscan - exclusive scan of every column of H over b (in place) and the tile
//                      totals n[t].
//   3. (CUB) exclusive scan of n -> tile start; k_bin_ranges writes ranges and K.
//   4. k_bin_scatter - block (b, C), one warp, lane l owns tile l of C and keeps its write
//                      position start[t] + H[b][t] in a register.  The warp visits the
//                      Gaussians flagged in the (b, C) mask in depth order; every lane whose
//                      tile the rectangle covers appends the Gaussian's index.  A lane stages
//                      its appends in a 16-word ring in shared memory and writes each
//                      completed 32-byte sector of its run with two 16-byte stores, so the
//                      point list is written in whole sectors (not one word per request).
// The result is the stable (depth, index) order per tile.  Traffic is O(B T + K) words
// instead of the ~26 bytes per entry of a two-pass radix sort of (tile, index) pairs.
#include "bgs_internal.cuh"

namespace bgs {

constexpr int kCbW = 8, kCbH = 4;  // tile group of one scatter warp (a tile per lane)

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
                                                   uint4 *__restrict__ rect, uint32_t *__restrict__ masks, int W32) {
    extern __shared__ uint32_t d_s[];  // [T] tile counters, then [nC][16] mask words
    const int T = tx * ty;
    const int ncx = (tx + kCbW - 1) / kCbW, nC = ncx * ((ty + kCbH - 1) / kCbH);
    uint32_t *m_s = d_s + T;
    const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = threadIdx.x; t < T + 16 * nC; t += blockDim.x) d_s[t] = 0u;
    __syncthreads();
    const long long s0 = (long long)b * G, s1 = min(N, s0 + G);
    // 512 Gaussians (16 mask words per C) at a time
    for (int sub = 0; sub < W32 / 16; ++sub) {
        const long long c0 = s0 + 512ll * sub, c1 = min(s1, c0 + 512);
        for (long long s = c0 + threadIdx.x; s < c1; s += blockDim.x) {
            int x0, y0, w, c;
            const uint32_t g = order[s];
            rect_of(means2D, radii, g, tw, th, tx, ty, x0, y0, w, c);
            uint32_t px = 0u, py = 0u;  // packed (x0 | w << 16, y0 | h << 16); h = 0 if empty
            if (c > 0) {
                const int h = c / w, x1 = x0 + w, y1 = y0 + h;
                px = (uint32_t)x0 | ((uint32_t)w << 16);
                py = (uint32_t)y0 | ((uint32_t)h << 16);
                // 2D difference array: +1 at (x0, y0) and (x1, y1), -1 at (x1, y0) and
                // (x0, y1) (modulo 2^32; the prefix sums below give the exact counts)
                atomicAdd(&d_s[y0 * tx + x0], 1u);
                if (x1 < tx) atomicAdd(&d_s[y0 * tx + x1], 0xffffffffu);
                if (y1 < ty) {
                    atomicAdd(&d_s[y1 * tx + x0], 0xffffffffu);
                    if (x1 < tx) atomicAdd(&d_s[y1 * tx + x1], 1u);
                }
                const int li = (int)(s - c0);
                const uint32_t bit = 1u << (li & 31);
                for (int cy = y0 / kCbH; cy <= (y1 - 1) / kCbH; ++cy)
                    for (int cx = x0 / kCbW; cx <= (x1 - 1) / kCbW; ++cx)
                        atomicOr(&m_s[(cy * ncx + cx) * 16 + (li >> 5)], bit);
            }
            rect[s] = make_uint4(px, py, g, 0u);
        }
        __syncthreads();
        // the sub-block's mask words: (b, C) words [16 sub, 16 sub + 16)
        for (int k = threadIdx.x; k < 16 * nC; k += blockDim.x) {
            masks[((size_t)b * nC + (k >> 4)) * W32 + 16 * sub + (k & 15)] = m_s[k];
            m_s[k] = 0u;
        }
        __syncthreads();
    }
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

// Writes the completed sector [done, done + 8) of a lane's run from its ring (words below
// run0 belong to the previous block's run of the tile and are left alone).  The ring is
// slot-major, ring_s[slot * 32 + lane]: appends and these reads are bank-conflict free.
__device__ __forceinline__ void flush_sector(const uint32_t *ring_s, int lane, uint32_t done, uint32_t run0,
                                             uint32_t *__restrict__ point_list, uint32_t capacity, bool vec_ok) {
    const uint32_t *src = ring_s + ((done & 15u) << 5) + lane;
    uint32_t v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = src[32 * j];
    if (vec_ok && done >= run0 && done + 8u <= capacity) {
        uint4 *dst = reinterpret_cast<uint4 *>(point_list + done);  // 32-byte aligned
        dst[0] = make_uint4(v[0], v[1], v[2], v[3]);
        dst[1] = make_uint4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (done + j >= run0 && done + j < capacity) point_list[done + j] = v[j];
    }
}

// Block (b, cx, cy): one warp, lane l owns tile (8 cx + l % 8, 4 cy + l / 8) of the group.
// Single-warp blocks: a block's shared memory is released as soon as its warp is done
// (blocks of several warps hold it until the slowest one finishes, and reached fewer
// resident warps).
__global__ void __launch_bounds__(32) k_bin_scatter(uint32_t G, int W32, const uint4 *__restrict__ rect, int tx, int ty,
                                                    const uint32_t *__restrict__ H, const uint32_t *__restrict__ start,
                                                    const uint32_t *__restrict__ masks,
                                                    uint32_t *__restrict__ point_list, uint32_t capacity, int vec_ok,
                                                    const DevCtrl *ctrl) {
    // per flagged Gaussian of the pass: (lanes whose tile its rectangle covers, Gaussian
    // index), .y holding its sorted position until the hit is known; and the lanes' 16-word
    // output rings, slot-major.  7 KB of shared memory a block in all, so that 32 blocks
    // (the per-SM block limit) fit an SM.
    __shared__ uint2 hit_s[512];
    __shared__ uint32_t ring_s[16 * 32];
    const int b = blockIdx.x, cx = blockIdx.y, cy = blockIdx.z, lane = threadIdx.x;
    const int nC = ((tx + kCbW - 1) / kCbW) * ((ty + kCbH - 1) / kCbH);
    const int C = cy * ((tx + kCbW - 1) / kCbW) + cx;
    const int gx0 = cx * kCbW, gy0 = cy * kCbH;
    const int ltx = gx0 + (lane % kCbW), lty = gy0 + (lane / kCbW);
    const bool own = ltx < tx && lty < ty;
    const unsigned own_mask = __ballot_sync(0xffffffffu, own);
    const size_t t = (size_t)lty * tx + ltx;
    const uint32_t base = (uint32_t)ctrl->bin_base;
    uint32_t pos = own ? base + start[t] + H[(size_t)b * tx * ty + t] : 0u;
    const uint32_t run0 = pos;
    uint32_t done = pos & ~7u;  // positions below done are written (or precede the run)
    uint32_t *ring = ring_s + lane;
    const uint32_t *mk = masks + ((size_t)b * nC + C) * W32;
    const uint32_t s0 = (uint32_t)b * G;
    for (int wb = 0; wb < W32; wb += 16) {  // 512 Gaussians per pass
        uint32_t word = lane < 16 ? mk[wb + lane] : 0u;
        const uint32_t cnt = (uint32_t)__popc(word);
        uint32_t incl = cnt;
        for (int o = 1; o < 16; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const int total = (int)__shfl_sync(0xffffffffu, incl, 15);
        if (total == 0) continue;
        // compact the flagged positions in depth order (word by word, bit by bit)
        uint32_t off = incl - cnt;
        while (word) {
            const int bit = __ffs(word) - 1;
            word &= word - 1u;
            hit_s[off++].y = s0 + 32u * (uint32_t)(wb + lane) + (uint32_t)bit;
        }
        __syncwarp();
        // per flagged Gaussian: the lanes whose tile its rectangle covers (a nonempty
        // rectangle meeting the group: the masks flag no other)
        for (int k = lane; k < total; k += 32) {
            const uint4 rc = rect[hit_s[k].y];
            const int x0 = (int)(rc.x & 0xffffu) - gx0, x1 = x0 + (int)(rc.x >> 16);
            const int y0 = (int)(rc.y & 0xffffu) - gy0, y1 = y0 + (int)(rc.y >> 16);
            const uint32_t lx0 = (uint32_t)max(x0, 0), lx1 = (uint32_t)min(x1, kCbW);
            const uint32_t ly0 = (uint32_t)max(y0, 0), ly1 = (uint32_t)min(y1, kCbH);
            const uint32_t cols = ((1u << lx1) - 1u) ^ ((1u << lx0) - 1u);
            const uint32_t rows = (ly1 >= 4u ? 0xffffffffu : (1u << (8u * ly1)) - 1u) ^ ((1u << (8u * ly0)) - 1u);
            hit_s[k] = make_uint2(rows & (cols * 0x01010101u) & own_mask, rc.z);
        }
        __syncwarp();
        // depth order, 8 visits at a time, then the remaining total % 8 one by one; at most 8
        // appends between two checks: at most one newly completed sector, and no ring slot
        // overwritten before it is written out
        const int full = total & ~7;
        for (int k0 = 0; k0 < full; k0 += 8) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                // branch-free: the slot of position pos is free (pos - done < 16), so every
                // lane writes it and only the lanes whose tile is covered advance past it
                const uint2 e = hit_s[k0 + j];
                ring[(pos & 15u) << 5] = e.y;
                pos += (e.x >> lane) & 1u;
            }
            if (done + 8u <= pos) {
                flush_sector(ring_s, lane, done, run0, point_list, capacity, vec_ok != 0);
                done += 8u;
            }
        }
        if (full < total) {
            for (int k = full; k < total; ++k) {
                const uint2 e = hit_s[k];
                ring[(pos & 15u) << 5] = e.y;
                pos += (e.x >> lane) & 1u;
            }
            if (done + 8u <= pos) {
                flush_sector(ring_s, lane, done, run0, point_list, capacity, vec_ok != 0);
                done += 8u;
            }
        }
        __syncwarp();
    }
    // the last, partial sector
    for (uint32_t p = done; p < pos; ++p)
        if (p >= run0 && p < capacity) point_list[p] = ring[(p & 15u) << 5];
}

size_t bin_count_smem(int tx, int ty) {
    const size_t nC = (size_t)((tx + kCbW - 1) / kCbW) * ((ty + kCbH - 1) / kCbH);
    return sizeof(uint32_t) * ((size_t)tx * ty + 16 * nC);
}

int bin_mask_groups(int tx, int ty) { return ((tx + kCbW - 1) / kCbW) * ((ty + kCbH - 1) / kCbH); }

cudaError_t setup_bin_kernels(int tx, int ty) {
    const size_t sc = bin_count_smem(tx, ty);
    if (sc <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
}

cudaError_t launch_bin_count(long long N, int G, int B, const uint32_t *order, const float *means2D, const int *radii,
                             int W, int H, int tw, int th, uint32_t *Hm, uint4 *rect, uint32_t *masks, int W32,
                             cudaStream_t s) {
    const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    k_bin_count<<<B, 256, bin_count_smem(tx, ty), s>>>(N, G, order, reinterpret_cast<const float2 *>(means2D), radii,
                                                        tw, th, tx, ty, Hm, rect, masks, W32);
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

cudaError_t launch_bin_scatter(long long N, int G, int B, int W32, const uint4 *rect, int W, int H, int tw, int th,
                               const uint32_t *Hm, const uint32_t *start, const uint32_t *masks, uint32_t *point_list,
                               long long capacity, const DevCtrl *ctrl, cudaStream_t s) {
    (void)N;
    const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    // indices, sorted positions and list slots are < 2^32 (checked by the callers)
    const uint32_t cap = capacity >= 0xffffffffll ? 0xffffffffu : (uint32_t)capacity;
    const int vec_ok = (reinterpret_cast<uintptr_t>(point_list) & 31u) == 0u;
    const dim3 grid(B, (tx + kCbW - 1) / kCbW, (ty + kCbH - 1) / kCbH);
    k_bin_scatter<<<grid, 32, 0, s>>>((uint32_t)G, W32, rect, tx, ty, Hm, start, masks, point_list, cap, vec_ok, ctrl);
    return cudaGetLastError();
}

}  // namespace bgs
