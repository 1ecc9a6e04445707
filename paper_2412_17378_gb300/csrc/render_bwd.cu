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
// to a packed accumulator [N][12] with one red.add instruction (warp-aggregated atomics).
// A final pass scales and scatters the accumulator into the ABI's gradient arrays.
#include "bgs_internal.cuh"

namespace bgs {

constexpr unsigned kFullB = 0xffffffffu;
constexpr int kBwdWarps = 8;

struct PixState {
    float T, Tf, g0, g1, g2, gD, gA, R0, R1, R2, Rd;
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
    s.R0 = a.bg[0];
    s.R1 = a.bg[1];
    s.R2 = a.bg[2];
    s.Rd = 0.f;
    return s;
}

// One (pixel, entry) step of the backward walk.  Adds the pair's 10 gradient
// contributions (nothing when the pair is skipped) to v[]:
//   v0 = dL/dpower (2 qa dx + qb dy), v1 = dL/dpower (2 qc dy + qb dx),
//   v2 = dL/dpower dx^2, v3 = dL/dpower dx dy, v4 = dL/dpower dy^2,
//   v5 = dL/do, v6..8 = dL/dc, v9 = dL/d(depth)
// (power is the natural-log exponent; the final pass applies the ln2 and -1/2 factors).
// Extra = false: no depth / alpha output gradients (dL/dD = dL/dA = 0), their terms are
// compiled out.
template <bool Extra>
__device__ __forceinline__ bool pair_backward(const Rec &r, const PairX &x, float pyf, bool active, PixState &s,
                                              float v[10]) {
    float dy, G;
    const float dx = x.dx;
    const float p2 = pair_power2_y(x, r.a.y, r.b.x, pyf, dy);
    const float al = pair_alpha(p2, r.b.y, G);
    const bool valid = active && p2 <= 0.f && al >= kAlphaMin;
    if (valid) {
        const float om = 1.f - al;
        const float io = rcp_approx(om);  // om in [0.01, 1]
        s.T = s.T * io;  // T_i
        const float w = al * s.T;
        v[6] += w * s.g0;
        v[7] += w * s.g1;
        v[8] += w * s.g2;
        float dLda = s.T * ((r.c.x - s.R0) * s.g0 + (r.c.y - s.R1) * s.g1 + (r.c.z - s.R2) * s.g2);
        if (Extra) {
            v[9] += w * s.gD;
            dLda += s.T * (r.c.w - s.Rd) * s.gD + s.Tf * io * s.gA;
            s.Rd = al * r.c.w + om * s.Rd;
        }
        s.R0 = al * r.c.x + om * s.R0;
        s.R1 = al * r.c.y + om * s.R1;
        s.R2 = al * r.c.z + om * s.R2;
        const float o = r.b.y;
        if (o * G <= kAlphaMax) {
            const float gp = o * G * dLda;  // dL/dpower
            v[0] += gp * (2.f * r.a.z * dx + r.a.w * dy);
            v[1] += gp * (2.f * r.b.x * dy + r.a.w * dx);
            v[2] += gp * dx * dx;
            v[3] += gp * dx * dy;
            v[4] += gp * dy * dy;
            v[5] += G * dLda;
        }
    }
    return valid;
}

// Sums v[0..9] over the warp's 32 lanes and adds the 10 totals to acc[0..9].  Recursive
// halving (reduce-scatter): at each of 4 stages a lane keeps one half of its remaining
// values and adds the partner's copy of that half (16 -> 8 -> 4 -> 2 -> 1 values, the
// vector padded to 16), then one butterfly step completes the sum.  Lane l ends with
// element (l >> 1) & 15; the even lanes holding elements 0..9 issue one red.add each, all
// in the same instruction.
__device__ __forceinline__ void warp_reduce_red10(const float v[10], float *acc, int lane) {
    float a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = j < 10 ? v[j] : 0.f;
#pragma unroll
    for (int stage = 0; stage < 4; ++stage) {
        const int off = 16 >> stage;  // 16, 8, 4, 2
        const int half = 8 >> stage;  // 8, 4, 2, 1
        const bool hi = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const float send = hi ? a[j] : a[j + half];
            const float keep = hi ? a[j + half] : a[j];
            a[j] = keep + __shfl_xor_sync(kFullB, send, off);
        }
    }
    const float tot = a[0] + __shfl_xor_sync(kFullB, a[0], 1);
    const int idx = (lane >> 1) & 15;
    if ((lane & 1) == 0 && idx < 10 && tot != 0.f) atomicAdd(acc + idx, tot);
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
            float v[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const bool valid = pair_backward<true>(r, pair_x(r.a, pxf), pyf, pos < s.nc, s, v);
            if (__any_sync(kFullB, valid)) warp_reduce_red10(v, a.grad_acc + 12ull * sidx[k], lane);
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
// serves 32 Q pixels.
template <int Q, bool Extra>
__device__ __forceinline__ void bwd_pixel_item(const BwdArgs &a, int tile, int sub, Rec *buf, uint32_t *gbuf,
                                               int lane) {
    constexpr int kItemH = 4 * Q;
    const int v = view_of(a.vt, tile);
    const int lt = tile - a.vt.tile_base[v];
    const int tx = lt % a.vt.tiles_x[v], ty = lt / a.vt.tiles_x[v];
    const int x0 = tx * a.tile_w, y0 = ty * a.tile_h;
    const int vw = min(a.tile_w, a.vt.W[v] - x0), vh = min(a.tile_h, a.vt.H[v] - y0);
    const int cxs = (vw + kPixItemW - 1) / kPixItemW;
    const int sx = sub % cxs, sy = sub / cxs;
    const int px = x0 + sx * kPixItemW + (lane & 7);
    const int py0 = y0 + sy * kItemH + (lane >> 3);
    const uint2 rg = load_range_bwd(a, tile);
    const int n = (int)(rg.y - rg.x);
    PixState s[Q];
    float pyf[Q];
    int maxnc = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int py = py0 + 4 * q;
        s[q] = load_pixel(a, v, px, py, px < x0 + vw && py < y0 + vh);
        if (s[q].nc > n) s[q].nc = n;
        maxnc = max(maxnc, s[q].nc);
        pyf[q] = (float)py;
    }
    maxnc = __reduce_max_sync(kFullB, maxnc);
    const uint32_t hi = rg.x + (uint32_t)maxnc;
    const float pxf = (float)px;
    const float bcx = (float)(x0 + sx * kPixItemW) + 3.5f;
    const float bcy = (float)(y0 + sy * kItemH) + 0.5f * (kItemH - 1);
    for (uint32_t top = hi; top > rg.x;) {
        const uint32_t lo = top - min(32u, top - rg.x);
        const int cnt = (int)(top - lo);
        bool hit = false;
        __syncwarp();
        if (lane < cnt) {
            uint32_t g;
            const Rec r = load_rec_bwd(a, top - 1 - lane, g);
            buf[lane] = r;
            gbuf[lane] = g;
            hit = !box_misses(r.a, r.b, bcx, bcy, 3.5f, 0.5f * (kItemH - 1));
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
            float v[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool any = false;
#pragma unroll
            for (int q = 0; q < Q; ++q) any |= pair_backward<Extra>(r, px2, pyf[q], pos < s[q].nc, s[q], v);
            if (__any_sync(kFullB, any)) warp_reduce_red10(v, a.grad_acc + 12ull * gbuf[k], lane);
        }
        top = lo;
    }
}

template <int Q, bool Extra>
__global__ void __launch_bounds__(kBwdWarps * 32) k_backward_balanced(BwdArgs a) {
    __shared__ Rec sbuf[kBwdWarps][32];
    __shared__ uint32_t sidx[kBwdWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Rec *buf = sbuf[warp];
    uint32_t *gbuf = sidx[warp];
    const unsigned num_items = a.ctrl->num_items;
    const unsigned chunk = (unsigned)a.chunk;
    while (true) {
        unsigned first = 0;
        if (lane == 0) first = atomicAdd(&a.ctrl->queue_head, chunk);
        first = __shfl_sync(kFullB, first, 0);
        if (first >= num_items) break;
        const unsigned end = min(first + chunk, num_items);
        for (unsigned it = first; it < end; ++it) {
            const uint2 item = a.items[it];
            bwd_pixel_item<Q, Extra>(a, (int)item.x, (int)(item.y & ~kKindGauss), buf, gbuf, lane);
        }
    }
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
// batched call: when n_colors < N, the colour gradient of Gaussian g sums the rows
// g, g + n_colors, ... (one per view) in k_grad_colors instead.
__global__ void __launch_bounds__(256) k_grad_finalize(long long N, long long n_colors, const float4 *__restrict__ acc,
                                                       float *__restrict__ dL_dmeans2D, float *__restrict__ dL_dconic,
                                                       float *__restrict__ dL_dopacity, float *__restrict__ dL_dcolors,
                                                       float *__restrict__ dL_ddepths) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 a0 = acc[3 * i], a1 = acc[3 * i + 1], a2 = acc[3 * i + 2];
    // power = ln2 * power2; d power / d mean = ln2 (2 qa dx + qb dy, 2 qc dy + qb dx);
    // d power / d(a, b, c) = (-dx^2 / 2, -dx dy, -dy^2 / 2)
    dL_dmeans2D[2 * i] = kLn2 * a0.x;
    dL_dmeans2D[2 * i + 1] = kLn2 * a0.y;
    dL_dconic[3 * i] = -0.5f * a0.z;
    dL_dconic[3 * i + 1] = -a0.w;
    dL_dconic[3 * i + 2] = -0.5f * a1.x;
    dL_dopacity[i] = a1.y;
    if (n_colors == N) {
        dL_dcolors[3 * i] = a1.z;
        dL_dcolors[3 * i + 1] = a1.w;
        dL_dcolors[3 * i + 2] = a2.x;
    }
    if (dL_ddepths) dL_ddepths[i] = a2.y;
}

__global__ void __launch_bounds__(256) k_grad_colors(long long N, long long n_colors, const float4 *__restrict__ acc,
                                                     float *__restrict__ dL_dcolors) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_colors) return;
    float r = 0.f, gg = 0.f, b = 0.f;
    for (long long i = g; i < N; i += n_colors) {
        const float4 a1 = acc[3 * i + 1], a2 = acc[3 * i + 2];
        r += a1.z;
        gg += a1.w;
        b += a2.x;
    }
    dL_dcolors[3 * g] = r;
    dL_dcolors[3 * g + 1] = gg;
    dL_dcolors[3 * g + 2] = b;
}

cudaError_t launch_grad_finalize(long long N, long long n_colors, const float4 *acc, float *dL_dmeans2D,
                                 float *dL_dconic, float *dL_dopacity, float *dL_dcolors, float *dL_ddepths,
                                 cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    k_grad_finalize<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, n_colors, acc, dL_dmeans2D, dL_dconic, dL_dopacity,
                                                                 dL_dcolors, dL_ddepths);
    if (n_colors != N && n_colors > 0)
        k_grad_colors<<<(unsigned)((n_colors + 255) / 256), 256, 0, s>>>(N, n_colors, acc, dL_dcolors);
    return cudaGetLastError();
}

}  // namespace bgs
