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
//   1'. k_bin_credit - (optional, when the conics are given) per block and tile, credits
//                      that certify where every pixel of a tile has stopped (see below).
//   2. k_bin_colscan - exclusive scan of every column of H over b (in place) and the tile
//                      totals n[t]; with credits, each tile's list is cut after the block
//                      at which its pixels are certified to have stopped.
//   3. (CUB) exclusive scan of n -> tile start; k_bin_view_total sums the view's count;
//      k_bin_ranges writes the ranges, offset by the view's first point_list slot (the
//      counts of the views before it: the views of a batched call run concurrently up to
//      here, and each view's scatter waits only for the counts of the views before it).
//   4. k_bin_scatter - item (b, C), one warp, lane l owns tile l of C and keeps its write
//                      position start[t] + H[b][t] in a register.  The warp visits the
//                      Gaussians flagged in the (b, C) mask in depth order; every lane whose
//                      tile the rectangle covers (and whose list was not cut before b)
//                      appends the index.  A lane stages
//                      its appends in a 16-word ring in shared memory and writes each
//                      completed 32-byte sector of its run with two 16-byte stores, so the
//                      point list is written in whole sectors (not one word per request).
// The result is the stable (depth, index) order per tile.  Traffic is O(B T + K) words
// instead of the ~26 bytes per entry of a two-pass radix sort of (tile, index) pairs.
#include <algorithm>
#include <mutex>

#include "bgs_internal.cuh"

namespace bgs {

constexpr int kCbW = 8, kCbH = 4;  // tile group of one scatter warp (a tile per lane)

// The tile rectangle of a record with mean m and radius r (r <= 0: empty).
__device__ __forceinline__ void rect_of(float2 m, int r, int tw, int th, int tx, int ty, int &x0, int &y0, int &w,
                                        int &cnt) {
    x0 = y0 = 0;
    w = 1;
    cnt = 0;
    if (r <= 0) return;
    // same float32 operations as the preprocess and oracle rectangles: a quotient rounded once
    // (for a power-of-two tile side, the product by its exact reciprocal is that quotient)
    int x1, y1;
    const bool px2 = (tw & (tw - 1)) == 0, py2 = (th & (th - 1)) == 0;
    const float itw = 1.f / (float)tw, ith = 1.f / (float)th;
    const float ax = __fsub_rn(m.x, (float)r), bx = __fadd_rn(m.x, (float)(r + tw - 1));
    const float ay = __fsub_rn(m.y, (float)r), by = __fadd_rn(m.y, (float)(r + th - 1));
    x0 = (int)floorf(px2 ? __fmul_rn(ax, itw) : __fdiv_rn(ax, (float)tw));
    x1 = (int)floorf(px2 ? __fmul_rn(bx, itw) : __fdiv_rn(bx, (float)tw));
    y0 = (int)floorf(py2 ? __fmul_rn(ay, ith) : __fdiv_rn(ay, (float)th));
    y1 = (int)floorf(py2 ? __fmul_rn(by, ith) : __fdiv_rn(by, (float)th));
    x0 = min(max(x0, 0), tx);
    x1 = min(max(x1, 0), tx);
    y0 = min(max(y0, 0), ty);
    y1 = min(max(y1, 0), ty);
    if (x1 > x0 && y1 > y0) {
        w = x1 - x0;
        cnt = w * (y1 - y0);
    }
}

constexpr int kCountThreads = 512;  // one thread per Gaussian of a 512-Gaussian sub-block
constexpr int kLaneGroups = 8;      // tile groups a lane flags by itself (more: the whole warp)

__global__ void __launch_bounds__(kCountThreads) k_bin_count(long long N, int G, const uint32_t *__restrict__ order,
                                                   const float2 *__restrict__ means2D, const int *__restrict__ radii,
                                                   int tw, int th, int tx, int ty, uint32_t *__restrict__ H,
                                                   uint4 *__restrict__ rect, uint32_t *__restrict__ masks, int W32,
                                                   int b_off, const int *__restrict__ skipP) {
    // [T] tile counters, then (16-byte aligned) [nC][16] mask words, then [nC / 32] bits of
    // the groups whose tiles all stopped before this pass
    extern __shared__ __align__(16) uint32_t d_s[];
    const int T = tx * ty;
    const int ncx = (tx + kCbW - 1) / kCbW, ncy = (ty + kCbH - 1) / kCbH, nC = ncx * ncy;
    const int T4 = (T + 3) & ~3;
    uint32_t *m_s = d_s + T4, *closed_s = m_s + 16 * nC;
    const int b = blockIdx.x + b_off, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = threadIdx.x; t < T4 + 16 * nC; t += blockDim.x) d_s[t] = 0u;
    if (skipP) {
        // a group whose tiles all stopped before this pass: no list reaches this block there,
        // and the scatter opens no (block, group) item of it, so its mask words are not written
        const int w1 = tx + 1;
        for (int c0 = warp * 32; c0 < nC; c0 += nwarps * 32) {
            const int C = c0 + lane;
            bool closed = false;
            if (C < nC) {
                const int gx0 = (C % ncx) * kCbW, gy0 = (C / ncx) * kCbH;
                const int gx1 = min(gx0 + kCbW, tx), gy1 = min(gy0 + kCbH, ty);
                const int n = skipP[gy1 * w1 + gx1] - skipP[gy0 * w1 + gx1] - skipP[gy1 * w1 + gx0] + skipP[gy0 * w1 + gx0];
                closed = n == (gx1 - gx0) * (gy1 - gy0);
            }
            const unsigned m = __ballot_sync(0xffffffffu, closed);
            if (lane == 0) closed_s[c0 >> 5] = m;
        }
    }
    __syncthreads();
    const long long s0 = (long long)b * G, s1 = min(N, s0 + G);
    // 512 Gaussians (16 mask words per C) at a time, a thread per Gaussian.  The loads are
    // pipelined across the sub-blocks: a thread holds the depth order two sub-blocks ahead
    // and the mean and radius one ahead, so the two dependent gathers of a sub-block overlap
    // the atomics, barriers and mask stores of the one before it.
    const int nb = (int)(s1 - s0);  // Gaussians of this block (<= G)
    const uint32_t *ord = order + s0;
    uint4 *rec = rect + s0;
    int i = threadIdx.x;  // position in the block
    uint32_t g = 0u, g_next = 0u;
    float2 m = make_float2(0.f, 0.f);
    int r = 0;
    if (i < nb) g = ord[i];
    if (i + kCountThreads < nb) g_next = ord[i + kCountThreads];
    if (i < nb) {
        r = radii[g];
        m = means2D[g];
    }
    for (int sub = 0; sub < W32 / 16; ++sub, i += kCountThreads) {
        float2 m_next = make_float2(0.f, 0.f);
        int r_next = 0;
        uint32_t g_after = 0u;
        if (i + kCountThreads < nb) {
            r_next = radii[g_next];
            m_next = means2D[g_next];
        }
        if (i + 2 * kCountThreads < nb) g_after = ord[i + 2 * kCountThreads];
        // a rectangle meeting more than kLaneGroups tile groups is flagged by the whole warp
        // below (one group per lane), not by its own lane's loop: the warp would otherwise
        // wait on its largest Gaussian's loop with one lane active
        int gx0 = 0, gy0 = 0, ngx = 1, ng = 0;
        if (i < nb) {
            int x0, y0, w, c;
            rect_of(m, r, tw, th, tx, ty, x0, y0, w, c);
            if (c > 0 && skipP) {
                // every tile the rectangle covers stopped in the blocks before this pass: the
                // Gaussian is past the end of all its lists (treated as covering nothing)
                const int x1 = x0 + w, y1 = y0 + c / w, w1 = tx + 1;
                if (skipP[y1 * w1 + x1] - skipP[y0 * w1 + x1] - skipP[y1 * w1 + x0] + skipP[y0 * w1 + x0] == c) c = 0;
            }
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
                // the Gaussian's bit (lane) in word `warp` of every group its rectangle meets
                gx0 = x0 / kCbW;
                gy0 = y0 / kCbH;
                ngx = (x1 - 1) / kCbW - gx0 + 1;
                ng = ngx * ((y1 - 1) / kCbH - gy0 + 1);
                if (ng <= kLaneGroups) {
                    for (int cy = gy0; cy <= (y1 - 1) / kCbH; ++cy)
                        for (int cx = gx0; cx < gx0 + ngx; ++cx)
                            atomicOr(&m_s[(cy * ncx + cx) * 16 + warp], 1u << lane);
                }
            }
            rec[i] = make_uint4(px, py, g, 0u);
        }
        for (unsigned big = __ballot_sync(0xffffffffu, ng > kLaneGroups); big; big &= big - 1u) {
            const int src = __ffs(big) - 1;
            const int bgx0 = __shfl_sync(0xffffffffu, gx0, src), bgy0 = __shfl_sync(0xffffffffu, gy0, src);
            const int bngx = __shfl_sync(0xffffffffu, ngx, src), bng = __shfl_sync(0xffffffffu, ng, src);
            for (int k = lane; k < bng; k += 32) {
                const int cy = bgy0 + k / bngx, cx = bgx0 + k % bngx;
                atomicOr(&m_s[(cy * ncx + cx) * 16 + warp], 1u << src);
            }
        }
        g = g_next;
        m = m_next;
        r = r_next;
        g_next = g_after;
        __syncthreads();
        // the sub-block's mask words: (b, C) words [16 sub, 16 sub + 16), 16 bytes a store (the
        // word arrays are 16-word aligned: W32 is a multiple of 16)
        for (int k = threadIdx.x; k < 4 * nC; k += blockDim.x) {
            uint4 *src = reinterpret_cast<uint4 *>(m_s) + k;
            const int C = k >> 2;
            if (!skipP || !((closed_s[C >> 5] >> (C & 31)) & 1u))
                reinterpret_cast<uint4 *>(masks + ((size_t)b * nC + C) * W32 + 16 * sub)[k & 3] = *src;
            *src = make_uint4(0u, 0u, 0u, 0u);
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

// ---- list truncation credits -----------------------------------------------------------
// A pixel stops (Algorithm 5) at the first pair that would take its transmittance below
// 1e-4, so the entries of a tile's list past the point where every pixel of the tile has
// stopped are never read, by the forward or the backward.  A Gaussian whose alpha is at
// least a at every pixel of a tile lowers the transmittance of each of its pixels by a
// factor <= 1 - a; once the product of such factors over a prefix of the tile's list is
// below 1e-5 (ten times under the stop threshold, which absorbs float32 rounding of the
// blend), every pixel of the tile has stopped within that prefix.
//
// k_bin_credit computes, per block b of G depth-ordered Gaussians and per tile, the block's
// sum of floor(256 ln(1 / (1 - a))) (fixed point, 1/256 nat) over its Gaussians and three
// levels a = max(f o, 1.01 / 255), f = 0.15, 0.45, 0.8: a Gaussian credits a tile with the
// highest level whose ellipse {d^T Q d <= 2 ln(o / a')} (a' = a (1 + 2^-9)) holds the
// tile's whole pixel rectangle (widened by half a pixel).  Alpha is log-concave, so that
// rectangle lies inside the level set iff its corners do, and per tile row the tiles
// inside form an interval: the intersection of the ellipse's chords at the row's two edges,
// shrunk by float32 error margins.  Only tiles of the Gaussian's own tile rectangle (where
// it has list entries) are credited.  Each row interval is one +/- pair of a per-row
// difference array in shared memory, so a Gaussian costs O(its tile rows), not O(its
// tiles).  Near-singular conics (det < 1e-5 a c), whose pairs may round to a positive power
// and be skipped, earn no credit.
constexpr uint32_t kCreditThr = 2948;  // ceil(256 ln(1e5))

// Work units: one per (Gaussian, tile row inside its lowest level set's vertical extent);
// a unit credits the row for every level whose set spans it (the levels share the row's
// chord centres).  Each warp takes 32 Gaussians at a time and spreads their units evenly
// over its lanes (a few large Gaussians would otherwise hold the warp for tens of rows); the
// warps of a block share only the credit counters, so they run without block barriers
// until the final prefix pass.
template <int kCrWarps>
__global__ void __launch_bounds__(kCrWarps * 32) k_bin_credit(long long N, int G, const uint4 *__restrict__ rect,
                                                              const float2 *__restrict__ means2D,
                                                              const float4 *__restrict__ conic_opacity, int tw,
                                                              int th, int tx, int ty, uint16_t *__restrict__ D,
                                                              int b_off) {
    extern __shared__ uint32_t w_s[];  // [T] per-row difference arrays of the credits
    // per warp, per lane's Gaussian: mx, my, 1 / qa, qb / qa, det, qa r^2 of the 3 levels;
    // the credit steps, first and end rows of the levels; the rectangle's columns, levels
    __shared__ float s_g[kCrWarps][32][8];
    __shared__ uint32_t s_dw[kCrWarps][32][3];
    __shared__ int s_j[kCrWarps][32][6];
    __shared__ int s_rx[kCrWarps][32][2];
    __shared__ int s_scan[kCrWarps][32];
    const int T = tx * ty;
    const int b = blockIdx.x + b_off, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < T; i += kCrWarps * 32) w_s[i] = 0u;
    __syncthreads();
    const long long s0 = (long long)b * G, s1 = min(N, s0 + G);
    const float fr[3] = {0.15f, 0.45f, 0.8f};
    const float itw = 1.f / (float)tw, ith = 1.f / (float)th;
    // level set {o G >= a'} of a level a = f o, a' = a (1 + 2^-9): r^2 = 2 ln(o / a') is a
    // constant of f (0.999 shrinks it against float32 rounding); a level clamped at
    // 1.01 / 255 computes its logarithm.  ln(1 / (f (1 + 2^-9))) for f = 0.15, 0.45, 0.8,
    // rounded down:
    const float r2c[3] = {2.f * 1.8951687f * 0.999f, 2.f * 0.7965564f * 0.999f, 2.f * 0.2211923f * 0.999f};
    // the next round's rectangle is loaded a round ahead (the conic gather behind it then
    // waits for one memory round trip, not two)
    uint4 rc_next = s0 + 32ll * warp + lane < s1 ? rect[s0 + 32ll * warp + lane] : make_uint4(0u, 0u, 0u, 0u);
    for (long long c0 = s0 + 32ll * warp; c0 < s1; c0 += 32ll * kCrWarps) {
        // (1) per Gaussian: its levels, their credits and the rows their level sets span
        const long long s = c0 + lane;
        const uint4 rc = rc_next;
        if (s + 32ll * kCrWarps < s1) rc_next = rect[s + 32ll * kCrWarps];
        int units = 0;
        if (s < s1) {
            const int rw = (int)(rc.x >> 16), rh = (int)(rc.y >> 16);
            if (rw > 0 && rh > 0) {
                const int rx0 = (int)(rc.x & 0xffffu), ry0 = (int)(rc.y & 0xffffu);
                const float4 co = conic_opacity[rc.z];
                const float qa = co.x, qb = co.y, qc = co.z, o = co.w;
                const float det = qa * qc - qb * qb;
                // r^2 < 2 ln(255 / 1.01) < 11.1 at every level: a Gaussian whose widest level
                // set cannot hold half a tile in x or y earns nothing
                if (qa > 0.f && det >= 1e-5f * qa * qc && 11.1f * qc >= det * (0.25f * tw * tw) &&
                    11.1f * qa >= det * (0.25f * th * th)) {
                    const float2 m = means2D[rc.z];
                    const float iqa = 1.f / qa, idet = 1.f / det;
                    float *gp = s_g[warp][lane];
                    gp[0] = m.x;
                    gp[1] = m.y;
                    gp[2] = iqa;
                    gp[3] = qb * iqa;
                    gp[4] = det;
                    s_rx[warp][lane][0] = rx0;
                    s_rx[warp][lane][1] = rx0 + rw;
                    uint32_t wprev = 0u;
                    int jlo = 0, jhi = 0;  // rows of the lowest credited level
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        s_dw[warp][lane][k] = 0u;
                        s_j[warp][lane][2 * k] = s_j[warp][lane][2 * k + 1] = 0;
                    }
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float fo = fr[k] * o;
                        const bool clamped = fo < 1.01f / 255.f;
                        const float lv = clamped ? 1.01f / 255.f : fo;
                        const float lv2 = lv * (1.f + 1.f / 512.f);
                        if (!(o > lv2)) break;
                        const float r2 = clamped ? 2.f * logf(o / lv2) * 0.999f : r2c[k];
                        // the level set's half-extents: no tile fits when below half a tile
                        if (r2 * qc < det * (0.25f * tw * tw) || r2 * qa < det * (0.25f * th * th)) break;
                        // floor(256 ln(1 / (1 - a))), shrunk by 0.1% (covers __logf's error)
                        const uint32_t wk = (uint32_t)floorf(-256.f * __logf(1.f - fminf(lv, 0.99f)) * 0.999f);
                        if (wk <= wprev) continue;
                        // tile rows whose band [j th - 0.5, (j + 1) th - 0.5] lies within the level
                        // set's vertical extent my -+ ey, inside the rectangle (a row taken in
                        // by rounding gets empty chords below and no credit)
                        const float ey = fminf(__fsqrt_rn(r2 * qa * idet), 1e8f);
                        const int j0 = max(ry0, (int)ceilf((fmaxf(m.y - ey, -1e8f) + 0.5f) * ith));
                        const int j1 = min(ry0 + rh, (int)floorf((fminf(m.y + ey, 1e8f) + 0.5f) * ith));
                        if (j1 <= j0) break;  // the higher levels' sets lie inside this one
                        if (wprev == 0u) {
                            jlo = j0;
                            jhi = j1;
                        }
                        gp[5 + k] = qa * r2;
                        s_dw[warp][lane][k] = wk - wprev;
                        s_j[warp][lane][2 * k] = j0;
                        s_j[warp][lane][2 * k + 1] = j1;
                        wprev = wk;
                    }
                    units = jhi - jlo;
                }
            }
        }
        // (2) inclusive scan of the lanes' unit counts
        int v = units;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += u;
        }
        s_scan[warp][lane] = v;
        const int total = __shfl_sync(0xffffffffu, v, 31);
        __syncwarp();
        // (3) the units: per level spanning the row, the level-set ellipse's chords at the
        // row's two edges, their intersection, and one +/- pair of the row's difference array
        for (int u = lane; u < total; u += 32) {
            int lo = 0, hi = 31;  // owner: first lane g with scan[g] > u
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_scan[warp][mid] > u) hi = mid;
                else lo = mid + 1;
            }
            const int g = lo;
            const float *gp = s_g[warp][g];
            const float mx = gp[0], my = gp[1], iqa = gp[2], bqa = gp[3], det = gp[4];
            // the first credited level's rows start the owner's unit range
            int k0 = 0;
            while (s_dw[warp][g][k0] == 0u) ++k0;
            const int j = s_j[warp][g][2 * k0] + (u - (g > 0 ? s_scan[warp][g - 1] : 0));
            float ctr[2], d2[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {  // the row's edges: chord centres, det dy^2
                const float dy = (float)((j + e) * th) - 0.5f - my;
                ctr[e] = mx - bqa * dy;
                d2[e] = det * dy * dy;
            }
            const int rx0 = s_rx[warp][g][0], rx1 = s_rx[warp][g][1];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const uint32_t dw = s_dw[warp][g][k];
                if (dw == 0u || j < s_j[warp][g][2 * k] || j >= s_j[warp][g][2 * k + 1]) continue;
                const float ar2 = gp[5 + k];
                float lo_x = -1e8f, hi_x = 1e8f;
#pragma unroll
                for (int e = 0; e < 2; ++e) {  // x in ctr -+ half (empty: half < 0)
                    const float disc = ar2 - d2[e] - 1e-6f * ar2;
                    // approximate square root and reciprocals: their few-ulp errors are far
                    // inside the 0.1% + 0.02 px the half-width is shrunk by
                    const float half = disc > 0.f ? disc * rsqrtf(disc) * iqa * 0.999f - 0.02f : -1e30f;
                    lo_x = fmaxf(lo_x, ctr[e] - half);
                    hi_x = fminf(hi_x, ctr[e] + half);
                }
                lo_x = fmaxf(lo_x, -1e8f);
                hi_x = fminf(hi_x, 1e8f);
                if (!(hi_x - lo_x >= (float)tw)) continue;
                // tiles i with [i tw - 0.5, i tw + tw - 0.5] inside [lo, hi], within the
                // rectangle (the product by 1 / tw rounds by far less than the 0.02 px the
                // chords were shrunk by)
                const int i0 = max(rx0, (int)ceilf((lo_x + 0.5f) * itw));
                const int i1 = min(rx1, (int)floorf((hi_x + 0.5f) * itw));
                if (i1 <= i0) continue;
                atomicAdd(&w_s[j * tx + i0], dw);
                if (i1 < tx) atomicAdd(&w_s[j * tx + i1], 0u - dw);
            }
        }
        __syncwarp();
    }
    __syncthreads();
    // prefix along each tile row (warp per row), saturated to 16 bits on the way out
    for (int y = warp; y < ty; y += kCrWarps) {
        uint32_t carry = 0u;
        for (int xb = 0; xb < tx; xb += 32) {
            const int x = xb + lane;
            uint32_t v = x < tx ? w_s[y * tx + x] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (x < tx) D[(size_t)b * T + y * tx + x] = (uint16_t)min(v + carry, 65535u);
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
}

// Block (32 tiles) x (32 row groups): per column t, exclusive prefix over b in place, and
// the column total n[t].  With the credits D (nullable): the column is cut after the first
// block b_sat[t] at whose end the credits summed over blocks 0..b reach thr (every pixel of
// the tile has stopped there); n[t] then counts blocks 0..b_sat only, and blocks past b_sat
// keep stale values that the scatter never reads.  b_sat = B - 1 when the credits never
// reach thr (or without D).
__global__ void __launch_bounds__(1024) k_bin_colscan(int B, int T, uint32_t *__restrict__ H,
                                                      const uint16_t *__restrict__ D, uint32_t thr,
                                                      uint32_t *__restrict__ total, uint32_t *__restrict__ bsat) {
    __shared__ uint32_t part[32][33], partD[32][33];
    __shared__ uint32_t s_gsat[32], s_runD[32], s_bsat[32], s_partH[32];
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int t = blockIdx.x * 32 + lx;
    const int rows = (B + 31) / 32;
    const int b0 = ly * rows, b1 = min(B, b0 + rows);
    uint32_t sum = 0, sumD = 0;
    if (t < T)
        for (int b = b0; b < b1; ++b) {
            sum += H[(size_t)b * T + t];
            if (D) sumD = min(sumD + (uint32_t)D[(size_t)b * T + t], 0x7fffffffu);
        }
    part[ly][lx] = sum;
    partD[ly][lx] = sumD;
    __syncthreads();
    if (ly == 0) {  // the row group in which the credits reach thr (32: none)
        uint32_t run = 0;
        int gsat = 32;
        if (D)
            for (int gq = 0; gq < 32; ++gq) {
                if (run + partD[gq][lx] >= thr) {
                    gsat = gq;
                    break;
                }
                run += partD[gq][lx];
            }
        s_gsat[lx] = (uint32_t)gsat;
        s_runD[lx] = run;
        s_bsat[lx] = (uint32_t)(B - 1);
        s_partH[lx] = 0u;
    }
    __syncthreads();
    const int gsat = (int)s_gsat[lx];
    if (ly == gsat && t < T) {  // the block inside that group, and the counts up to it
        uint32_t run = s_runD[lx], ph = 0;
        int bs = b1 - 1;
        for (int b = b0; b < b1; ++b) {
            ph += H[(size_t)b * T + t];
            run += D[(size_t)b * T + t];
            if (run >= thr) {
                bs = b;
                break;
            }
        }
        s_bsat[lx] = (uint32_t)bs;
        s_partH[lx] = ph;
    }
    __syncthreads();
    if (ly == 0) {
        uint32_t run = 0;
        for (int gq = 0; gq < 32 && gq <= gsat; ++gq) {
            const uint32_t v = part[gq][lx];
            part[gq][lx] = run;
            run += (gq == gsat) ? s_partH[lx] : v;
        }
        if (t < T) {
            total[t] = run;
            if (bsat) bsat[t] = s_bsat[lx];
        }
    }
    __syncthreads();
    if (t < T && ly <= gsat) {
        const int bend = min(b1, (int)s_bsat[lx] + 1);
        uint32_t off = part[ly][lx];
        for (int b = b0; b < bend; ++b) {
            const uint32_t h = H[(size_t)b * T + t];
            H[(size_t)b * T + t] = off;
            off += h;
        }
    }
}

// ranges[t] = base + [start[t], start[t] + n[t]) for the tiles of view v ((0,0) for an empty
// tile), base = the entries of views 0..v-1; block 0 stores base for the scatter.
__global__ void k_bin_ranges(int T, const uint32_t *__restrict__ start, const uint32_t *__restrict__ total,
                             uint2 *__restrict__ ranges, int v, DevCtrl *ctrl) {
    unsigned long long b64 = 0;
    for (int u = 0; u < v; ++u) b64 += ctrl->view_k[u];
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->view_base[v] = b64;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const uint32_t base = (uint32_t)b64;  // past 2^32 the call raises BGS_CHECK_OVERFLOW
    const uint32_t a = base + start[t], n = total[t];
    ranges[t] = n ? make_uint2(a, a + n) : make_uint2(0u, 0u);
}

// view_k[v] = the view's entry count, summed in 64 bits from the per-tile totals.
__global__ void k_bin_view_total(int T, const uint32_t *__restrict__ total, int v, DevCtrl *ctrl) {
    __shared__ unsigned long long part[32];
    unsigned long long n = 0;
    for (int t = threadIdx.x; t < T; t += blockDim.x) n += total[t];
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long k = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) k += part[w];
        ctrl->view_k[v] = k;
    }
}

// The call's entry count over its V views; overflow check.
__global__ void k_bin_finish(int V, long long capacity, DevCtrl *ctrl) {
    unsigned long long k = 0;
    for (int u = 0; u < V; ++u) k += ctrl->view_k[u];
    ctrl->bin_base = k;
    ctrl->num_entries = k;
    if ((long long)k > capacity || (long long)k > BGS_MAX_ENTRIES) atomicOr(&ctrl->check_bits, (unsigned)BGS_CHECK_OVERFLOW);
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
// Work items of the scatter: the (depth block b, tile group C) pairs with b at most the last
// block any tile of C keeps (every pair without truncation), numbered C-major.  One block:
// item_start[C] = exclusive prefix of min(B, max over C's tiles of b_sat + 1), and
// item_start[nC] = the item count.
__global__ void __launch_bounds__(1024) k_bin_items(int nC, int tx, int ty, int B, const uint32_t *__restrict__ bsat,
                                                    uint32_t *__restrict__ item_start) {
    __shared__ uint32_t part[1024];
    const int tid = threadIdx.x;
    const int per = (nC + 1023) / 1024;
    const int c0 = min(nC, tid * per), c1 = min(nC, c0 + per);
    const int ncx = (tx + kCbW - 1) / kCbW;
    uint32_t local = 0;
    for (int C = c0; C < c1; ++C) {
        uint32_t n = (uint32_t)B;
        if (bsat) {
            uint32_t gmax = 0;
            const int gx0 = (C % ncx) * kCbW, gy0 = (C / ncx) * kCbH;
            for (int y = gy0; y < min(ty, gy0 + kCbH); ++y)
                for (int x = gx0; x < min(tx, gx0 + kCbW); ++x) gmax = max(gmax, bsat[(size_t)y * tx + x]);
            n = min((uint32_t)B, gmax + 1u);
        }
        item_start[C] = n;  // the count, turned into the offset below
        local += n;
    }
    part[tid] = local;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan of the threads' sums
        const uint32_t v = tid >= off ? part[tid - off] : 0u;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    uint32_t run = part[tid] - local;
    for (int C = c0; C < c1; ++C) {
        const uint32_t n = item_start[C];
        item_start[C] = run;
        run += n;
    }
    if (tid == 1023) item_start[nC] = part[1023];
}

// With truncated lists (bsat given) the blocks stride over the work items of k_bin_items,
// item -> (C, b); with complete lists every (b, C) is an item and block i takes item i
// (C = i / B, b = i % B) once.  Item (b, C): one warp, lane l owns tile l of C; lanes whose
// list ends before b append nothing.
__global__ void __launch_bounds__(32) k_bin_scatter(uint32_t G, int W32, const uint4 *__restrict__ rect, int tx, int ty,
                                                    const uint32_t *__restrict__ H, const uint32_t *__restrict__ start,
                                                    const uint32_t *__restrict__ masks,
                                                    uint32_t *__restrict__ point_list, uint32_t capacity, int vec_ok,
                                                    const uint32_t *__restrict__ bsat,
                                                    const uint32_t *__restrict__ item_start, int nC, int B,
                                                    int v, const DevCtrl *ctrl) {
    // per flagged Gaussian of the pass: (lanes whose tile its rectangle covers, Gaussian
    // index), .y holding its sorted position until the hit is known; and the lanes' 16-word
    // output rings, slot-major.  7 KB of shared memory a block in all, so that 32 blocks
    // (the per-SM block limit) fit an SM.
    __shared__ uint2 hit_s[512];
    __shared__ uint32_t ring_s[16 * 32];
    const int lane = threadIdx.x;
    const int ncx = (tx + kCbW - 1) / kCbW;
    const bool listed = bsat != nullptr;
    const uint32_t n_items = listed ? item_start[nC] : (uint32_t)B * (uint32_t)nC;
    const uint32_t base = (uint32_t)ctrl->view_base[v];
    uint32_t *ring = ring_s + lane;
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        int C, b;
        if (listed) {
            int lo = 0, hi = nC - 1;  // C: the last group with item_start[C] <= it
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (item_start[mid] <= it) lo = mid;
                else hi = mid - 1;
            }
            C = lo;
            b = (int)(it - item_start[C]);
        } else {
            C = (int)(it / (uint32_t)B);
            b = (int)(it % (uint32_t)B);
        }
        const int gx0 = (C % ncx) * kCbW, gy0 = (C / ncx) * kCbH;
        const int ltx = gx0 + (lane % kCbW), lty = gy0 + (lane / kCbW);
        const size_t t = (size_t)lty * tx + ltx;
        // a lane whose tile's list was cut before block b appends nothing
        const bool own = ltx < tx && lty < ty && (bsat == nullptr || (uint32_t)b <= bsat[t]);
        const unsigned own_mask = __ballot_sync(0xffffffffu, own);
        if (own_mask == 0u) continue;
        uint32_t pos = own ? base + start[t] + H[(size_t)b * tx * ty + t] : 0u;
        const uint32_t run0 = pos;
        uint32_t done = pos & ~7u;  // positions below done are written (or precede the run)
        const uint32_t *mk = masks + ((size_t)b * nC + C) * W32;
        const uint32_t s0 = (uint32_t)b * G;
        // The flagged positions of the item's mask words, 16 words (512 Gaussians) a pass,
        // gathered in depth order into hit_s across passes and visited in batches of up to 512
        // hits: one round of rectangle gathers serves all passes of a sparse item.
        auto visit = [&](int total) {
            // per flagged Gaussian: the lanes whose tile its rectangle covers (a nonempty
            // rectangle meeting the group: the masks flag no other), among the lanes whose
            // list is still open; hits that reach no such lane are dropped (in place: a hit
            // moves to a slot at or before its own, after the warp has read the round)
            int kept = 0;
            for (int k0 = 0; k0 < total; k0 += 32) {
                const int k = k0 + lane;
                uint32_t cover = 0u, idx = 0u;
                if (k < total) {
                    const uint4 rc = rect[hit_s[k].y];
                    const int x0 = (int)(rc.x & 0xffffu) - gx0, x1 = x0 + (int)(rc.x >> 16);
                    const int y0 = (int)(rc.y & 0xffffu) - gy0, y1 = y0 + (int)(rc.y >> 16);
                    const uint32_t lx0 = (uint32_t)max(x0, 0), lx1 = (uint32_t)min(x1, kCbW);
                    const uint32_t ly0 = (uint32_t)max(y0, 0), ly1 = (uint32_t)min(y1, kCbH);
                    const uint32_t cols = ((1u << lx1) - 1u) ^ ((1u << lx0) - 1u);
                    const uint32_t rows =
                        (ly1 >= 4u ? 0xffffffffu : (1u << (8u * ly1)) - 1u) ^ ((1u << (8u * ly0)) - 1u);
                    cover = rows & (cols * 0x01010101u) & own_mask;
                    idx = rc.z;
                }
                const unsigned keep = __ballot_sync(0xffffffffu, cover != 0u);
                if (cover != 0u) hit_s[kept + __popc(keep & ((1u << lane) - 1u))] = make_uint2(cover, idx);
                kept += __popc(keep);
            }
            __syncwarp();
            // depth order, 8 visits at a time, then the remaining kept % 8 one by one; at most 8
            // appends between two checks: at most one newly completed sector, and no ring slot
            // overwritten before it is written out
            const int full = kept & ~7;
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
            if (full < kept) {
                for (int k = full; k < kept; ++k) {
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
        };
        int acc = 0;  // hits gathered in hit_s[0, acc)
        uint32_t next = lane < 16 ? mk[lane] : 0u;
        for (int wb = 0; wb < W32; wb += 16) {
            uint32_t word = next;
            next = (lane < 16 && wb + 16 < W32) ? mk[wb + 16 + lane] : 0u;  // the next pass's words, early
            const uint32_t cnt = (uint32_t)__popc(word);
            uint32_t incl = cnt;
            for (int o = 1; o < 16; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            const int total = (int)__shfl_sync(0xffffffffu, incl, 15);
            if (total == 0) continue;
            if (acc + total > 512) {
                visit(acc);
                acc = 0;
            }
            // compact the flagged positions in depth order (word by word, bit by bit)
            uint32_t off = (uint32_t)acc + incl - cnt;
            while (word) {
                const int bit = __ffs(word) - 1;
                word &= word - 1u;
                hit_s[off++].y = s0 + 32u * (uint32_t)(wb + lane) + (uint32_t)bit;
            }
            __syncwarp();
            acc += total;
        }
        if (acc) visit(acc);
        // the last, partial sector
        for (uint32_t p = done; p < pos; ++p)
            if (p >= run0 && p < capacity) point_list[p] = ring[(p & 15u) << 5];
        __syncwarp();
    }
}

size_t bin_count_smem(int tx, int ty) {
    const size_t nC = (size_t)((tx + kCbW - 1) / kCbW) * ((ty + kCbH - 1) / kCbH);
    return sizeof(uint32_t) * ((((size_t)tx * ty + 3) & ~(size_t)3) + 16 * nC + (nC + 31) / 32);
}

int bin_mask_groups(int tx, int ty) { return ((tx + kCbW - 1) / kCbW) * ((ty + kCbH - 1) / kCbH); }

// Raises a kernel's dynamic shared-memory limit on the current device to at least `bytes`,
// never lowering it: launches captured in a CUDA graph keep their own (possibly larger)
// size, and a replay of them needs the limit the capture saw.  slot: one per kernel.
static cudaError_t raise_dyn_smem(const void *kernel, int slot, size_t bytes) {
    constexpr int kSlots = 4, kDevices = 64;
    static std::mutex mu;
    static int limit[kSlots][kDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDevices || slot < 0 || slot >= kSlots) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)bytes <= limit[slot][dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) limit[slot][dev] = (int)bytes;
    return e;
}

cudaError_t setup_bin_kernels(int tx, int ty) {
    const size_t sc = bin_count_smem(tx, ty);
    if (sc <= 48 * 1024) return cudaSuccess;
    return raise_dyn_smem((const void *)k_bin_count, 0, sc);
}

cudaError_t launch_bin_count(long long N, int G, int b_lo, int b_hi, const uint32_t *order, const float *means2D,
                             const int *radii, int W, int H, int tw, int th, uint32_t *Hm, uint4 *rect, uint32_t *masks,
                             int W32, const int *skipP, cudaStream_t s) {
    const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    if (b_hi <= b_lo) return cudaSuccess;
    k_bin_count<<<b_hi - b_lo, kCountThreads, bin_count_smem(tx, ty), s>>>(
        N, G, order, reinterpret_cast<const float2 *>(means2D), radii, tw, th, tx, ty, Hm, rect, masks, W32, b_lo, skipP);
    return cudaGetLastError();
}

// Per tile, the credits of blocks [0, B1): a thread per (tile, chunk of `chunk` blocks) adds
// its chunk's sum, capped at thr (only whether the total reaches thr matters; the cap keeps
// the total far below 2^32), to S[t].
__global__ void k_bin_stopped(int B1, int T, int chunk, const uint16_t *__restrict__ D, uint32_t thr,
                              uint32_t *__restrict__ S) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int b0 = (int)blockIdx.y * chunk, b1 = min(B1, b0 + chunk);
    uint32_t sum = 0;
    for (int b = b0; b < b1; ++b) sum += (uint32_t)D[(size_t)b * T + t];
    if (sum) atomicAdd(&S[t], min(sum, thr));
}

// P [(ty + 1) x (tx + 1)]: the exclusive 2D prefix of the stopped tiles' indicator (S[t] >=
// thr), P[y][x] = #stopped tiles (x' < x, y' < y), built in shared memory by one block.
__global__ void __launch_bounds__(1024) k_bin_prefix2d(int tx, int ty, const uint32_t *__restrict__ S, uint32_t thr,
                                                       int *__restrict__ P) {
    extern __shared__ int p_s[];
    const int w1 = tx + 1, n = (tx + 1) * (ty + 1), lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int y = i / w1, x = i - y * w1;
        p_s[i] = (x > 0 && y > 0 && S[(y - 1) * tx + (x - 1)] >= thr) ? 1 : 0;
    }
    __syncthreads();
    for (int y = 1 + warp; y <= ty; y += nwarps) {  // along x, a warp per row
        int carry = 0;
        for (int xb = 1; xb <= tx; xb += 32) {
            const int x = xb + lane;
            int v = x <= tx ? p_s[y * w1 + x] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (x <= tx) p_s[y * w1 + x] = v + carry;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    for (int x = 1 + (int)threadIdx.x; x <= tx; x += blockDim.x) {  // along y, a thread per column
        int run = 0;
        for (int y = 1; y <= ty; ++y) {
            run += p_s[y * w1 + x];
            p_s[y * w1 + x] = run;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) P[i] = p_s[i];
}

size_t bin_stopped_smem(int tx, int ty) { return sizeof(int) * (size_t)(tx + 1) * (ty + 1); }

cudaError_t launch_bin_stopped(int B1, int tx, int ty, const uint16_t *D, int *P, cudaStream_t s) {
    const int T = tx * ty;
    // the per-tile sums live behind the prefix in P's buffer
    uint32_t *S = reinterpret_cast<uint32_t *>(P + (size_t)(tx + 1) * (ty + 1));
    cudaError_t e = cudaMemsetAsync(S, 0, sizeof(uint32_t) * (size_t)T, s);
    if (e != cudaSuccess) return e;
    if (B1 > 0) {
        const int chunk = std::max(32, (B1 + 65534) / 65535);
        const dim3 grid((unsigned)std::max(1, (T + 255) / 256), (unsigned)((B1 + chunk - 1) / chunk));
        k_bin_stopped<<<grid, 256, 0, s>>>(B1, T, chunk, D, kCreditThr, S);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const size_t smem = bin_stopped_smem(tx, ty);
    if (smem > 48 * 1024 && (e = raise_dyn_smem((const void *)k_bin_prefix2d, 3, smem)) != cudaSuccess) return e;
    k_bin_prefix2d<<<1, 1024, smem, s>>>(tx, ty, S, kCreditThr, P);
    return cudaGetLastError();
}

cudaError_t launch_bin_colscan(int B, int T, uint32_t *Hm, const uint16_t *D, uint32_t *total, uint32_t *bsat,
                               cudaStream_t s) {
    k_bin_colscan<<<(T + 31) / 32, dim3(32, 32), 0, s>>>(B, T, Hm, D, kCreditThr, total, bsat);
    return cudaGetLastError();
}

// dynamic shared memory of k_bin_credit (one credit counter per tile)
static size_t bin_credit_dyn_smem(int tx, int ty) { return sizeof(uint32_t) * (size_t)tx * ty; }
// static shared memory of k_bin_credit per warp (its unit tables)
constexpr size_t kCrWarpSmem = 2560;
// all of k_bin_credit's shared memory at its smallest block (16 warps): the counters and the
// per-warp unit tables (+ slack)
size_t bin_credit_smem(int tx, int ty) { return bin_credit_dyn_smem(tx, ty) + 16 * kCrWarpSmem + 4096; }

cudaError_t launch_bin_credit(long long N, int G, int b_lo, int b_hi, const uint4 *rect, const float *means2D,
                              const float *conic_opacity, int W, int H, int tw, int th, uint16_t *D, cudaStream_t s) {
    const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    if (b_hi <= b_lo) return cudaSuccess;
    const size_t smem = bin_credit_dyn_smem(tx, ty);
    // 32 warps a block where their tables fit next to the counters (a large grid leaves room
    // for one block per SM only), else 16; the static tables plus the counters pass the 48 KB
    // default already on small grids: opt in to the dynamic size (the limit only ever grows)
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const float2 *m2 = reinterpret_cast<const float2 *>(means2D);
    const float4 *co = reinterpret_cast<const float4 *>(conic_opacity);
    if (smem + 32 * kCrWarpSmem + 4096 <= (size_t)optin) {
        if ((e = raise_dyn_smem((const void *)k_bin_credit<32>, 2, smem)) != cudaSuccess) return e;
        k_bin_credit<32><<<b_hi - b_lo, 32 * 32, smem, s>>>(N, G, rect, m2, co, tw, th, tx, ty, D, b_lo);
    } else {
        if ((e = raise_dyn_smem((const void *)k_bin_credit<16>, 1, smem)) != cudaSuccess) return e;
        k_bin_credit<16><<<b_hi - b_lo, 16 * 32, smem, s>>>(N, G, rect, m2, co, tw, th, tx, ty, D, b_lo);
    }
    return cudaGetLastError();
}

cudaError_t launch_bin_ranges(int T, const uint32_t *start, const uint32_t *total, uint2 *ranges, int v,
                              DevCtrl *ctrl, cudaStream_t s) {
    k_bin_ranges<<<std::max(1, (T + 255) / 256), 256, 0, s>>>(T, start, total, ranges, v, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_bin_view_total(int T, const uint32_t *total, int v, DevCtrl *ctrl, cudaStream_t s) {
    k_bin_view_total<<<1, 1024, 0, s>>>(T, total, v, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_bin_finish(int V, long long capacity, DevCtrl *ctrl, cudaStream_t s) {
    k_bin_finish<<<1, 1, 0, s>>>(V, capacity, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_bin_scatter(long long N, int G, int B, int W32, const uint4 *rect, int W, int H, int tw, int th,
                               const uint32_t *Hm, const uint32_t *start, const uint32_t *masks, uint32_t *point_list,
                               long long capacity, const uint32_t *bsat, uint32_t *item_start, int num_sms, int v,
                               const DevCtrl *ctrl, cudaStream_t s) {
    (void)N;
    const int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    const int nC = bin_mask_groups(tx, ty);
    // indices, sorted positions and list slots are < 2^32 (checked by the callers)
    const uint32_t cap = capacity > BGS_MAX_ENTRIES ? (uint32_t)BGS_MAX_ENTRIES : (uint32_t)capacity;
    const int vec_ok = (reinterpret_cast<uintptr_t>(point_list) & 31u) == 0u;
    // truncated lists: a persistent grid (32 single-warp blocks per SM, the per-SM block limit)
    // over the open items; complete lists: one block per (b, C), scheduled by the hardware
    long long grid = (long long)B * nC;
    if (bsat) {
        k_bin_items<<<1, 1024, 0, s>>>(nC, tx, ty, B, bsat, item_start);
        grid = std::min<long long>((long long)num_sms * 32, grid);
    }
    k_bin_scatter<<<(unsigned)std::max<long long>(1, grid), 32, 0, s>>>((uint32_t)G, W32, rect, tx, ty, Hm, start,
                                                                         masks, point_list, cap, vec_ok, bsat,
                                                                         item_start, nC, B, v, ctrl);
    return cudaGetLastError();
}

}  // namespace bgs
