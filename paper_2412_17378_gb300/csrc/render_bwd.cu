// render_bwd.cu -- a6: backward render kernels.
//
// The paper describes only the forward kernel; its backward (Sec. 3 cites the L2
// atomic bottleneck of 3DGS gradients) is derived here from Eq. 4.  With
// T_i = prod_{j<i}(1 - alpha_j), R_i the colour accumulated behind entry i normalised by
// T_{i+1} (R starts at the background), and T_f the final transmittance:
//   dL/dc_i      = alpha_i T_i dL/dC
//   dL/dalpha_i  = T_i [ (c_i - R_i) . dL/dC + (d_i - Rd_i) dL/dD ] + T_f/(1-alpha_i) dL/dA
//   R_{i-1}      = alpha_i c_i + (1 - alpha_i) R_i       (same for depth, Rd starts at 0)
// and alpha = min(0.99, o G), G = exp(power): dL/do = G dL/dalpha and dL/dpower =
// o G dL/dalpha where the clamp is inactive (both 0 where o G > 0.99).
// Each pixel walks its tile's list from its last contributor back to the front,
// recovering T_i = T_{i+1} / (1 - alpha_i) from the stored final T (no per-pair state is
// kept by the forward).  All lanes of a warp visit the same list entry at the same step,
// so the per-Gaussian contributions of the warp's pixels are summed with shuffles and added
// to a packed accumulator [N][12] with two red.add instructions (warp-aggregated atomics).
// With gp = dL/dpower2 of a pair, the mean and conic gradients of a Gaussian are sums of
// gp times (dx, dy, dx^2, dx dy, dy^2) combined with the Gaussian's (constant) conic, so a
// lane only sums gp, gp dy and gp dy^2 over its pixels (which share dx), forms the five
// moments once, and the conic is applied after the warp sum.  Two identities shorten the
// per-pair work: R_i enters dL/dalpha only through R_i . dL/dC, so a pixel carries that
// scalar (updated by the same recurrence) instead of R_i; and dL/do = sum G dL/dalpha =
// (sum gp) / o, so the opacity gradient is the gp sum, divided by o once per Gaussian in the
// final pass, which scales and scatters the accumulator into the ABI's gradient arrays.
#include <algorithm>

#include "bgs_internal.cuh"

namespace bgs {

constexpr unsigned kFullB = 0xffffffffu;
constexpr int kBwdWarps = 8;

struct PixState {
    float T, Tf, g0, g1, g2, gD, gA;
    float Rg, Rd;  // R . dL/dC (colour behind the entry, dotted with the pixel's colour gradient), depth behind
    int nc;
};

__device__ __forceinline__ PixState load_pixel(const BwdArgs &a, int v, int px, int py, bool inside) {
    PixState s;
    if (inside) {
        const int W = a.vt.W[v];
        const long long HW = (long long)W * a.vt.H[v];
        const long long pid = (long long)py * W + px;
        s.T = a.gi.final_T[v][pid];
        s.nc = a.gi.n_contrib[v][pid];
        const float *gc = a.gi.dL_dcolor[v];
        s.g0 = gc[pid];
        s.g1 = gc[HW + pid];
        s.g2 = gc[2 * HW + pid];
        s.gD = a.gi.dL_ddepth[v] ? a.gi.dL_ddepth[v][pid] : 0.f;
        s.gA = a.gi.dL_dalpha[v] ? a.gi.dL_dalpha[v][pid] : 0.f;
    } else {
        s.T = 1.f;
        s.nc = 0;
        s.g0 = s.g1 = s.g2 = s.gD = s.gA = 0.f;
    }
    s.Tf = s.T;
    s.Rg = a.bg[0] * s.g0 + a.bg[1] * s.g1 + a.bg[2] * s.g2;
    s.Rd = 0.f;
    return s;
}

// Per-lane sums of one record's pair contributions over the lane's pixels.
struct PairSums {
    float g, gy, gyy;  // sum of gp, gp dy, gp dy^2 (gp = dL/dpower2, power2 the log2 exponent)
    float c0, c1, c2;  // sum of alpha T dL/dC           (-> dL/dcolour)
    float d;           // sum of alpha T dL/dD           (-> dL/ddepth)
};

__device__ __forceinline__ PairSums zero_sums() {
    PairSums a;
    a.g = a.gy = a.gyy = a.c0 = a.c1 = a.c2 = a.d = 0.f;
    return a;
}

// One (pixel, entry) step of the backward walk: adds the pair's contributions to a
// (nothing when the pair is skipped).  dL/dalpha_i = T_i [(c_i - R_i) . dL/dC + (d_i - Rd_i)
// dL/dD] + T_f / (1 - alpha_i) dL/dA; then R_{i-1} = R_i + alpha_i (c_i - R_i), carried as
// Rg = R . dL/dC.  Extra = false: no depth / alpha output gradients (dL/dD = dL/dA = 0), their
// terms are compiled out.
template <bool Extra>
__device__ __forceinline__ bool pair_backward(const Rec &r, const PairX &x, float pyf, bool active, PixState &s,
                                              PairSums &a) {
    float dy;
    const float p2 = pair_power2_y(x, r.a.y, r.b.x, pyf, dy);
    const float oG = pair_oG(p2, r.b.y);
    const bool valid = active && p2 <= 0.f && oG >= kAlphaMin;
    if (valid) {
        const float al = fminf(kAlphaMax, oG);
        const float om = 1.f - al;
        const float io = rcp_approx(om);  // om in [0.01, 1]
        s.T = s.T * io;                   // T_i
        const float w = al * s.T;
        a.c0 += w * s.g0;
        a.c1 += w * s.g1;
        a.c2 += w * s.g2;
        const float diff = (r.c.x * s.g0 + r.c.y * s.g1 + r.c.z * s.g2) - s.Rg;  // (c_i - R_i) . dL/dC
        float dLda = s.T * diff;
        if (Extra) {
            a.d += w * s.gD;
            const float dd = r.c.w - s.Rd;
            dLda += s.T * dd * s.gD + s.Tf * io * s.gA;
            s.Rd += al * dd;
        }
        s.Rg += al * diff;
        // alpha = min(0.99, o G): no gradient through the clamp (branch-free)
        const float gp = oG <= kAlphaMax ? oG * dLda : 0.f;  // dL/dpower2 = o G dL/dalpha
        const float gpy = gp * dy;
        a.g += gp;
        a.gy += gpy;
        a.gyy += gpy * dy;
    }
    return valid;
}

// Adds the lane sums of one record, over the warp's 32 lanes, to the record's accumulator
// row acc[0..9]:
//   acc0..4 = sum gp (dx, dy, dx^2, dx dy, dy^2), acc5 = sum gp (= o sum G dL/dalpha),
//   acc6..8 = colour sums, acc9 = depth sum
// (dx = mean_x - px is shared by the lane's pixels; the final pass applies the Gaussian's
// conic to the first two moments, once per Gaussian).  The eight values (the five moments,
// sum gp, two colour channels) are reduced by recursive halving over lane bits 4, 3, 2
// (4 + 2 + 1 shuffles), leaving in lane l the sum of element (l >> 2) & 7 over the 8 lanes
// that share l's bits 1, 0; the third colour channel (and the depth sum, halved against it
// over bit 4) takes three butterflies.  The four partial sums of every value are then added
// by the atomics themselves: one red.add instruction from all 32 lanes for the eight
// values, one from lanes 0-3 (and 16-19) for colour channel 2 (and depth).  Stopping the
// trees two levels early shortens the per-record dependency chain by two shuffles; L2
// absorbs the extra atomic operations.
template <bool Extra>
__device__ __forceinline__ void warp_reduce_red(const PairSums &s, float dx, float *acc, int lane) {
    const float sdx = dx * s.g;
    float v[8] = {sdx, s.gy, dx * sdx, dx * s.gy, s.gyy, s.g, s.c0, s.c1};
    float h4[4], h2[2];
    {
        const bool hi = (lane & 16) != 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float send = hi ? v[j] : v[j + 4];
            h4[j] = (hi ? v[j + 4] : v[j]) + __shfl_xor_sync(kFullB, send, 16);
        }
    }
    {
        const bool hi = (lane & 8) != 0;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float send = hi ? h4[j] : h4[j + 2];
            h2[j] = (hi ? h4[j + 2] : h4[j]) + __shfl_xor_sync(kFullB, send, 8);
        }
    }
    float t;
    {
        const bool hi = (lane & 4) != 0;
        t = (hi ? h2[1] : h2[0]) + __shfl_xor_sync(kFullB, hi ? h2[0] : h2[1], 4);
    }
    float u;  // colour channel 2 (lanes with bit 4 clear) / depth (bit 4 set) when Extra
    if (Extra) {
        const bool hi = (lane & 16) != 0;
        u = (hi ? s.d : s.c2) + __shfl_xor_sync(kFullB, hi ? s.c2 : s.d, 16);
    } else {
        u = s.c2 + __shfl_xor_sync(kFullB, s.c2, 16);
    }
    u += __shfl_xor_sync(kFullB, u, 8);
    u += __shfl_xor_sync(kFullB, u, 4);
    if (t != 0.f) atomicAdd(acc + ((lane >> 2) & 7), t);
    const bool ul = Extra ? (lane & 12) == 0 : lane < 4;  // lanes 0-3 (and 16-19)
    if (ul && u != 0.f) atomicAdd(acc + ((Extra && (lane & 16)) ? 9 : 8), u);
}

// Record of list entry j and its index g; an index >= N raises BGS_CHECK_INDEX and yields a
// transparent record (its box misses every pixel) with index 0.
__device__ __forceinline__ Rec load_rec_bwd(const BwdArgs &a, uint32_t j, uint32_t &g) {
    g = a.point_list[j];
    Rec r;
    if ((long long)g >= a.N) {
        raise_check(a.ctrl, BGS_CHECK_INDEX);
        g = 0;
        r.a = make_float4(0.f, 0.f, 0.f, 0.f);
        r.b = make_float4(0.f, 0.f, -1.f, -1.f);
        r.c = make_float4(0.f, 0.f, 0.f, 0.f);
        return r;
    }
    return a.recs[g];
}

__device__ __forceinline__ uint2 load_range_bwd(const BwdArgs &a, int tile) {
    uint2 rg = a.ranges[tile];
    if (rg.y < rg.x || (long long)rg.y > a.num_entries) {
        raise_check(a.ctrl, BGS_CHECK_RANGE);
        rg = make_uint2(0, 0);
    }
    return rg;
}

// =====================================================================================
// plain pixel-wise static backward: one block per tile, block-wide staging
// =====================================================================================
__global__ void __launch_bounds__(1024) k_backward_static(BwdArgs a) {
    extern __shared__ Rec srec[];  // [nthreads] records, then [nthreads] indices
    __shared__ int s_max;
    const int nthreads = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    const int tile = blockIdx.x;  // single view
    const int tx = tile % a.vt.tiles_x[0], ty = tile / a.vt.tiles_x[0];
    const int px = tx * a.tile_w + tid % a.tile_w, py = ty * a.tile_h + tid / a.tile_w;
    const bool inside = px < a.vt.W[0] && py < a.vt.H[0];
    uint2 rg = a.ranges[tile];
    if (rg.y < rg.x || (long long)rg.y > a.num_entries) {
        if (tid == 0) raise_check(a.ctrl, BGS_CHECK_RANGE);
        rg = make_uint2(0, 0);
    }
    PixState s = load_pixel(a, 0, px, py, inside);
    if (s.nc > (int)(rg.y - rg.x)) s.nc = (int)(rg.y - rg.x);
    if (tid == 0) s_max = 0;
    __syncthreads();
    atomicMax(&s_max, s.nc);
    __syncthreads();
    const uint32_t hi = rg.x + (uint32_t)s_max;
    const float pxf = (float)px, pyf = (float)py;
    uint32_t *sidx = reinterpret_cast<uint32_t *>(srec + nthreads);
    for (uint32_t top = hi; top > rg.x; top -= min((uint32_t)nthreads, top - rg.x)) {
        const uint32_t lo = top - min((uint32_t)nthreads, top - rg.x);
        const int cnt = (int)(top - lo);
        __syncthreads();
        if (tid < cnt) {
            const uint32_t j = top - 1 - tid;
            const uint32_t g = a.point_list[j];
            Rec r;
            if ((long long)g < a.N) {
                r = make_rec(a.means2D, a.conic_opacity, a.colors, a.depths, g);
            } else {
                raise_check(a.ctrl, BGS_CHECK_INDEX);
                r.a = make_float4(0.f, 0.f, 0.f, 0.f);
                r.b = r.a;
                r.c = r.a;
            }
            srec[tid] = r;
            sidx[tid] = (long long)g < a.N ? g : 0u;
        }
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const Rec r = srec[k];
            const int pos = (int)(top - 1 - k - rg.x);
            const PairX x = pair_x(r.a, pxf);
            PairSums sums = zero_sums();
            const bool valid = pair_backward<true>(r, x, pyf, pos < s.nc, s, sums);
            if (__any_sync(kFullB, valid)) warp_reduce_red<true>(sums, x.dx, a.grad_acc + 12ull * sidx[k], lane);
        }
    }
}

cudaError_t launch_backward_static(const BwdArgs &a, cudaStream_t s) {
    const int threads = a.tile_w * a.tile_h;
    const int tiles = a.vt.tiles_x[0] * a.vt.tiles_y[0];
    if (tiles == 0) return cudaSuccess;
    k_backward_static<<<tiles, threads, (sizeof(Rec) + sizeof(uint32_t)) * threads, s>>>(a);
    return cudaGetLastError();
}

// =====================================================================================
// balanced persistent backward: warps pull pixel-wise items (8x4 sub-blocks)
// =====================================================================================
// Pixel-wise item: an 8 x 4Q sub-block; lane l owns the pixels (l % 8, l / 8 + 4 q).  The
// lane adds its pixels' contributions before the warp-wide reduction, so one reduction
// serves 32 Q pixels.  In a tile that the last forward split into segments of L entries
// (Gaussian-wise, reading the forward's boundary states), the item walks one segment
// [e0, e1) of the list: a pixel whose last contributor lies behind the segment enters it
// with the state the merge stored for it (T behind the segment, colour and depth behind it
// over that T); one whose last contributor lies inside starts there as usual; the others
// have nothing in it.
template <int Q, bool Extra>
__device__ __forceinline__ void bwd_pixel_item(const BwdArgs &a, int tile, int sub, unsigned L, Rec *buf,
                                               uint32_t *gbuf, int lane) {
    constexpr int kItemW = pix_item_w(Q), kItemH = pix_item_h(Q), kRowStep = pix_row_step(Q);
    const int v = view_of(a.vt, tile);
    const int lt = tile - a.vt.tile_base[v];
    const int tx = lt % a.vt.tiles_x[v], ty = lt / a.vt.tiles_x[v];
    const int x0 = tx * a.tile_w, y0 = ty * a.tile_h;
    const int vw = min(a.tile_w, a.vt.W[v] - x0), vh = min(a.tile_h, a.vt.H[v] - y0);
    const int cxs = (vw + kItemW - 1) / kItemW;
    const uint2 rg = load_range_bwd(a, tile);
    const int n = (int)(rg.y - rg.x);
    // the segment of a split tile (seg < 0: the whole list)
    int seg = -1;
    uint32_t e0 = rg.x, e1 = rg.y;
    if (L != 0u && (uint32_t)n > L && tile_is_gauss(a.bseg_mode, a.heavy_threshold, (uint32_t)n)) {
        const int per_tile = cxs * ((vh + kItemH - 1) / kItemH);
        seg = sub / per_tile;
        sub -= seg * per_tile;
        e0 = rg.x + (uint32_t)seg * L;
        e1 = (uint32_t)min((unsigned long long)rg.y, (unsigned long long)e0 + L);
    }
    const int sx = sub % cxs, sy = sub / cxs;
    const int px = x0 + sx * kItemW + (lane % kItemW);
    const int py0 = y0 + sy * kItemH + (lane / kItemW);
    PixState s[Q];
    float pyf[Q];
    int maxnc = 0;
    const int P = a.gw_pixels, groups = (vw * vh + P - 1) / P;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int py = py0 + kRowStep * q;
        const bool inside = px < x0 + vw && py < y0 + vh;
        s[q] = load_pixel(a, v, px, py, inside);
        if (s[q].nc > n) s[q].nc = n;
        if (seg >= 0) {
            const uint32_t end = rg.x + (uint32_t)s[q].nc;  // one past the last contributor
            if (end <= e0) {
                s[q].nc = 0;  // nothing of this pixel in the segment
            } else if (end >= e1 && inside) {
                // enter from behind: the merge's state at the segment's end
                const int qp = (py - y0) * vw + (px - x0), group = qp / P;
                const uint2 gt = a.gw_tile[tile];
                const size_t si = seg == 0 ? (size_t)gt.x + group : (size_t)gt.y + (size_t)(seg - 1) * groups + group;
                const GwSum st = a.gw_sum[si * P + qp % P];
                const float iT = 1.f / st.t.x;
                s[q].T = st.t.x;
                s[q].Rg = (st.cd.x * s[q].g0 + st.cd.y * s[q].g1 + st.cd.z * s[q].g2) * iT;
                s[q].Rd = st.cd.w * iT;
                s[q].nc = (int)(e1 - rg.x);
            }
        }
        maxnc = max(maxnc, s[q].nc);
        pyf[q] = (float)py;
    }
    maxnc = __reduce_max_sync(kFullB, maxnc);
    const uint32_t hi = rg.x + (uint32_t)maxnc;
    const float pxf = (float)px;
    const float bcx = (float)(x0 + sx * kItemW) + 0.5f * (kItemW - 1);
    const float bcy = (float)(y0 + sy * kItemH) + 0.5f * (kItemH - 1);
    for (uint32_t top = hi; top > e0;) {
        const uint32_t lo = top - min(32u, top - e0);
        const int cnt = (int)(top - lo);
        bool hit = false;
        __syncwarp();
        if (lane < cnt) {
            uint32_t g;
            const Rec r = load_rec_bwd(a, top - 1 - lane, g);
            buf[lane] = r;
            gbuf[lane] = g;
            hit = !box_misses(r.a, r.b, bcx, bcy, 0.5f * (kItemW - 1), 0.5f * (kItemH - 1));
        }
        // back to front over the records whose alpha box reaches the pixel block
        unsigned live = __ballot_sync(kFullB, hit);
        __syncwarp();
        while (live) {
            const int k = __ffs(live) - 1;
            live &= live - 1;
            const Rec r = buf[k];
            const int pos = (int)(top - 1 - k - rg.x);
            const PairX px2 = pair_x(r.a, pxf);  // shared by the lane's pixels (same column)
            PairSums sums = zero_sums();
            bool any = false;
#pragma unroll
            for (int q = 0; q < Q; ++q) any |= pair_backward<Extra>(r, px2, pyf[q], pos < s[q].nc, s[q], sums);
            if (__any_sync(kFullB, any)) warp_reduce_red<Extra>(sums, px2.dx, a.grad_acc + 12ull * gbuf[k], lane);
        }
        top = lo;
    }
}

// The walk is latency-bound (dependent FP32 chains, shuffle trees): with colour-only output
// gradients and up to 4 rows per lane the kernel fits 64 registers, so 4 blocks (32 warps)
// stay resident per SM instead of 3.  The other variants would spill there: 3 blocks for
// the depth / alpha gradients at up to 4 rows, no bound at 8 rows.
template <int Q, bool Extra>
__global__ void __launch_bounds__(kBwdWarps * 32, (Q <= 4 && !Extra) ? 4 : (Q <= 4 ? 3 : 1))
    k_backward_balanced(BwdArgs a) {
    __shared__ Rec sbuf[kBwdWarps][32];
    __shared__ uint32_t sidx[kBwdWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Rec *buf = sbuf[warp];
    uint32_t *gbuf = sidx[warp];
    const unsigned num_items = a.ctrl->num_items;
    const unsigned chunk = (unsigned)a.chunk;
    // segment length of the tiles the last forward split (0: no segmented walk)
    const unsigned L = a.bseg_mode >= 0 ? a.ctrl->gw_seg : 0u;
    unsigned long long st_items = 0;
    while (true) {
        unsigned first = 0;
        if (lane == 0) first = atomicAdd(&a.ctrl->queue_head, chunk);
        first = __shfl_sync(kFullB, first, 0);
        if (first >= num_items) break;
        const unsigned end = min(first + chunk, num_items);
        for (unsigned it = first; it < end; ++it) {
            const uint2 item = a.items[it];
            bwd_pixel_item<Q, Extra>(a, (int)item.x, (int)(item.y & ~kKindGauss), L, buf, gbuf, lane);
            ++st_items;
        }
    }
    // the warp's completed items; k_grad_finalize checks their sum (the queue's drain)
    if (lane == 0) a.warp_items[blockIdx.x * kBwdWarps + warp] = (unsigned int)st_items;
}

int backward_balanced_block_threads() { return kBwdWarps * 32; }
static bool has_extra(const BwdArgs &a) {
    for (int v = 0; v < a.vt.V; ++v)
        if (a.gi.dL_ddepth[v] || a.gi.dL_dalpha[v]) return true;
    return false;
}

const void *backward_balanced_kernel(const BwdArgs &a) {
    const bool e = has_extra(a);
    switch (a.pixel_rows) {
        case 1: return e ? (const void *)k_backward_balanced<1, true> : (const void *)k_backward_balanced<1, false>;
        case 2: return e ? (const void *)k_backward_balanced<2, true> : (const void *)k_backward_balanced<2, false>;
        case 4: return e ? (const void *)k_backward_balanced<4, true> : (const void *)k_backward_balanced<4, false>;
        case 8: return e ? (const void *)k_backward_balanced<8, true> : (const void *)k_backward_balanced<8, false>;
        default: return nullptr;
    }
}

cudaError_t launch_backward_balanced(const BwdArgs &a, int grid, cudaStream_t s) {
    const void *k = backward_balanced_kernel(a);
    if (!k) return cudaErrorInvalidValue;
    BwdArgs arg = a;
    void *params[] = {&arg};
    return cudaLaunchKernel(k, dim3(grid), dim3(kBwdWarps * 32), params, 0, s);
}

// ---- accumulator -> ABI gradient arrays ----------------------------------------------
// Record i's accumulator row -> its gradients.  Colours are shared by the views of a
// batched call when n_colors < N (records g, g + n_colors, ... are Gaussian g seen from
// each view): then a thread takes Gaussian g, finalizes its records one view after another
// and writes its colour gradient summed over them, reading each accumulator row once.
__device__ __forceinline__ void finalize_record(long long i, const float4 *__restrict__ acc,
                                                const float4 *__restrict__ conic_opacity,
                                                float *__restrict__ dL_dmeans2D, float *__restrict__ dL_dconic,
                                                float *__restrict__ dL_dopacity, float *__restrict__ dL_ddepths,
                                                float &cr, float &cg, float &cb) {
    const float4 a0 = acc[3 * i], a1 = acc[3 * i + 1], a2 = acc[3 * i + 2];
    const float4 co = conic_opacity[i];
    // power = ln2 * power2 with power2 = qa dx^2 + qb dx dy + qc dy^2 and (qa, qb, qc) the
    // record's pre-scaled conic; d power / d mean = ln2 (2 qa dx + qb dy, 2 qc dy + qb dx),
    // summed over the pairs from the moments sum gp dx (a0.x) and sum gp dy (a0.y);
    // d power / d(a, b, c) = (-dx^2 / 2, -dx dy, -dy^2 / 2)
    const float qa = -0.5f * kLog2e * co.x, qb = -kLog2e * co.y, qc = -0.5f * kLog2e * co.z;
    dL_dmeans2D[2 * i] = kLn2 * (2.f * qa * a0.x + qb * a0.y);
    dL_dmeans2D[2 * i + 1] = kLn2 * (2.f * qc * a0.y + qb * a0.x);
    dL_dconic[3 * i] = -0.5f * a0.z;
    dL_dconic[3 * i + 1] = -a0.w;
    dL_dconic[3 * i + 2] = -0.5f * a1.x;
    // sum gp / o = sum G dL/dalpha (a record with o = 0 has alpha = 0 everywhere: no pair)
    dL_dopacity[i] = co.w > 0.f ? a1.y / co.w : 0.f;
    if (dL_ddepths) dL_ddepths[i] = a2.y;
    cr += a1.z;
    cg += a1.w;
    cb += a2.x;
}

__global__ void __launch_bounds__(256) k_grad_finalize(long long N, long long n_colors, const float4 *__restrict__ acc,
                                                       const float4 *__restrict__ conic_opacity,
                                                       float *__restrict__ dL_dmeans2D, float *__restrict__ dL_dconic,
                                                       float *__restrict__ dL_dopacity, float *__restrict__ dL_dcolors,
                                                       float *__restrict__ dL_ddepths,
                                                       const unsigned int *__restrict__ warp_items, int n_warps,
                                                       DevCtrl *ctrl) {
    if (blockIdx.x == 0 && n_warps > 0) {
        // drain check of the persistent backward pass: every queued item ran exactly once
        __shared__ unsigned int part[8];
        unsigned int sum = 0;
        for (int w = threadIdx.x; w < n_warps; w += blockDim.x) sum += warp_items[w];
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int total = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += part[w];
            if (total != ctrl->num_items) atomicOr(&ctrl->check_bits, BGS_CHECK_QUEUE);
        }
    }
    // a thread per record (colours per record), or per Gaussian over its views (shared colours)
    const bool shared = n_colors > 0 && n_colors < N;
    const long long stride = shared ? n_colors : N;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= stride) return;
    float cr = 0.f, cg = 0.f, cb = 0.f;
    for (long long i = g; i < N; i += stride)
        finalize_record(i, acc, conic_opacity, dL_dmeans2D, dL_dconic, dL_dopacity, dL_ddepths, cr, cg, cb);
    if (n_colors > 0) {
        dL_dcolors[3 * g] = cr;
        dL_dcolors[3 * g + 1] = cg;
        dL_dcolors[3 * g + 2] = cb;
    }
}

cudaError_t launch_grad_finalize(long long N, long long n_colors, const float4 *acc, const float *conic_opacity,
                                 float *dL_dmeans2D, float *dL_dconic, float *dL_dopacity, float *dL_dcolors,
                                 float *dL_ddepths, const unsigned int *warp_items, int n_warps, DevCtrl *ctrl,
                                 cudaStream_t s) {
    if (N == 0 && n_warps == 0) return cudaSuccess;
    const long long threads = (n_colors > 0 && n_colors < N) ? n_colors : N;
    k_grad_finalize<<<(unsigned)std::max<long long>(1, (threads + 255) / 256), 256, 0, s>>>(
        N, n_colors, acc, reinterpret_cast<const float4 *>(conic_opacity), dL_dmeans2D, dL_dconic, dL_dopacity,
        dL_dcolors, dL_ddepths, warp_items, n_warps, ctrl);
    return cudaGetLastError();
}

}  // namespace bgs
