// render_fwd.cu -- a4/a5: forward render kernels.
//
//  k_forward_static    plain pixel-wise kernel on a static grid (one block per tile, one
//                      thread per pixel, block-wide staging of the tile's records in
//                      shared memory) -- the paper's "naive renderCUDA" (Algorithm 4)
//                      with the shared-memory staging of features and depths of
//                      Sec. 5.2.2.  It is the baseline the balanced kernel is timed against.
//  k_forward_gauss / k_forward_pixel
//                      persistent kernels (Sec. 4.1's inter-block dynamic distribution,
//                      taken down to warp granularity): every warp pulls work items from
//                      a device atomic queue.  The work list holds the Gaussian-wise items
//                      first, then the pixel-wise ones; each kind has its own kernel (and
//                      register budget) and its own queue cursor:
//                        - Gaussian-wise (Sec. 4.2, Algorithm 6, fine-grained per
//                          Sec. 4.3): P pixels of a tile, the lanes splitting a segment of
//                          the list into contiguous chunks and composing them with a
//                          shuffle prefix product; segments of one tile run on separate
//                          warps and k_forward_gw_merge composes them per pixel;
//                        - pixel-wise: an 8x8 sub-block of a tile, two pixels per lane,
//                          walking the tile's list through a warp-private shared memory
//                          window of 32 records.
//
// All evaluate each (pixel, entry) pair with the same code (pair_power2 / pair_oG), so
// their skip decisions agree bit for bit, and the pixel-wise kernels' stop decisions too;
// the Gaussian-wise kernel's transmittance product is reassociated (see next_T).
// Results of all kernels equal the sequential rule of Algorithm 5 up to float32
// reassociation of the transmittance product (Sec. 4: "without any precision loss").
#include "bgs_internal.cuh"

namespace bgs {

constexpr unsigned kFull = 0xffffffffu;

// The accumulated alpha sum_i alpha_i T_i telescopes to 1 - T (T_i - T_{i+1} summed), so it is
// written from the final T instead of being summed per pair.
__device__ __forceinline__ void write_pixel(const FwdArgs &a, int v, int px, int py, float T, float c0, float c1,
                                            float c2, float D, int last, int neval) {
    const int W = a.vt.W[v];
    const long long HW = (long long)W * a.vt.H[v];
    const long long pid = (long long)py * W + px;
    float *oc = a.io.out_color[v];
    oc[pid] = c0 + T * a.bg[0];
    oc[HW + pid] = c1 + T * a.bg[1];
    oc[2 * HW + pid] = c2 + T * a.bg[2];
    a.io.out_depth[v][pid] = D;
    a.io.out_alpha[v][pid] = 1.f - T;
    a.io.final_T[v][pid] = T;
    a.io.n_contrib[v][pid] = last;
    if (a.io.n_eval[v]) a.io.n_eval[v][pid] = neval;
}

// Validated tile range: an out-of-bounds span raises BGS_CHECK_RANGE and renders empty.
__device__ __forceinline__ uint2 load_range(const FwdArgs &a, int tile) {
    uint2 rg = a.ranges[tile];
    if (rg.y < rg.x || (long long)rg.y > a.num_entries) {
        raise_check(a.ctrl, BGS_CHECK_RANGE);
        rg = make_uint2(0, 0);
    }
    return rg;
}

// Record of list entry j; an index >= N raises BGS_CHECK_INDEX and yields a transparent record.
__device__ __forceinline__ Rec load_rec(const FwdArgs &a, uint32_t j) {
    const uint32_t g = a.point_list[j];
    if ((long long)g >= a.N) {
        raise_check(a.ctrl, BGS_CHECK_INDEX);
        Rec r;
        r.a = make_float4(0.f, 0.f, 0.f, 0.f);
        r.b = make_float4(0.f, 0.f, 0.f, 0.f);
        r.c = r.b;
        return r;
    }
    return a.recs[g];
}

// =====================================================================================
// plain pixel-wise static kernel
// =====================================================================================
__global__ void __launch_bounds__(1024) k_forward_static(FwdArgs a) {
    extern __shared__ Rec srec[];
    const int nthreads = blockDim.x;
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;  // single view: global tile id = tile of view 0
    const int tx = tile % a.vt.tiles_x[0], ty = tile / a.vt.tiles_x[0];
    const int px = tx * a.tile_w + tid % a.tile_w, py = ty * a.tile_h + tid / a.tile_w;
    const bool inside = px < a.vt.W[0] && py < a.vt.H[0];
    uint2 rg = a.ranges[tile];
    if (rg.y < rg.x || (long long)rg.y > a.num_entries) {
        if (tid == 0) raise_check(a.ctrl, BGS_CHECK_RANGE);
        rg = make_uint2(0, 0);
    }
    const float pxf = (float)px, pyf = (float)py;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, D = 0.f;
    int last = 0, neval = (int)(rg.y - rg.x), nacc = 0;
    bool done = !inside;
    for (uint32_t base = rg.x; base < rg.y; base += nthreads) {
        if (__syncthreads_count(done) == nthreads) break;
        const uint32_t j = base + tid;
        if (j < rg.y) {
            const uint32_t g = a.point_list[j];
            if ((long long)g < a.N) {
                srec[tid] = make_rec(a.means2D, a.conic_opacity, a.colors, a.depths, g);
            } else {
                raise_check(a.ctrl, BGS_CHECK_INDEX);
                srec[tid].b = make_float4(0.f, 0.f, 0.f, 0.f);
                srec[tid].a = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        const int cnt = min(nthreads, (int)(rg.y - base));
        for (int k = 0; !done && k < cnt; ++k) {
            const float4 ra = srec[k].a;
            const float4 rb = srec[k].b;
            float dx, dy;
            const float p2 = pair_power2(ra, rb.x, pxf, pyf, dx, dy);
            const float oG = pair_oG(p2, rb.y);
            if (!(p2 <= 0.f && oG >= kAlphaMin)) continue;
            const float al = fminf(kAlphaMax, oG);
            const float tt = next_T(T, al);
            if (tt < kTMin) {
                done = true;
                neval = (int)(base + k + 1 - rg.x);
                break;
            }
            const float4 rc = srec[k].c;
            const float w = al * T;
            c0 += w * rc.x;
            c1 += w * rc.y;
            c2 += w * rc.z;
            D += w * rc.w;
            T = tt;
            last = (int)(base + k + 1 - rg.x);
            ++nacc;
        }
    }
    if (inside) write_pixel(a, 0, px, py, T, c0, c1, c2, D, last, neval);
    // evaluated / contributing pair counters
    unsigned long long e = inside ? (unsigned long long)neval : 0ull, c = inside ? (unsigned long long)nacc : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(kFull, e, o);
        c += __shfl_xor_sync(kFull, c, o);
    }
    if ((tid & 31) == 0) {
        atomicAdd(&a.ctrl->eval_pairs, e);
        atomicAdd(&a.ctrl->contrib_pairs, c);
    }
}

cudaError_t launch_forward_static(const FwdArgs &a, cudaStream_t s) {
    const int threads = a.tile_w * a.tile_h;
    const int tiles = a.vt.tiles_x[0] * a.vt.tiles_y[0];
    if (tiles == 0) return cudaSuccess;
    const size_t smem = sizeof(Rec) * threads;
    k_forward_static<<<tiles, threads, smem, s>>>(a);
    return cudaGetLastError();
}

// =====================================================================================
// balanced persistent kernel
// =====================================================================================
constexpr int kWarpsPerBlock = 8;

struct TileGeom {
    int v;               // view
    int x0, y0, vw, vh;  // tile origin and the part of it inside the view's image
};

__device__ __forceinline__ TileGeom tile_geom(const FwdArgs &a, int tile) {
    TileGeom t;
    t.v = view_of(a.vt, tile);
    const int lt = tile - a.vt.tile_base[t.v];
    const int tx = lt % a.vt.tiles_x[t.v], ty = lt / a.vt.tiles_x[t.v];
    t.x0 = tx * a.tile_w;
    t.y0 = ty * a.tile_h;
    t.vw = min(a.tile_w, a.vt.W[t.v] - t.x0);
    t.vh = min(a.tile_h, a.vt.H[t.v] - t.y0);
    return t;
}

// Pixel-wise item: an 8 x 4Q sub-block of a tile; lane l owns the pixels (l % 8, l / 8 + 4 q).
// The warp walks the tile's list through a warp-private window of 32 records in shared
// memory; each record is read once per lane (broadcast) and applied to the lane's Q
// pixels, which share dx.
template <int Q>
__device__ __forceinline__ void pixel_item(const FwdArgs &a, int tile, int sub, Rec *buf, int lane,
                                           unsigned long long &st_eval, unsigned long long &st_acc) {
    constexpr int kItemW = pix_item_w(Q), kItemH = pix_item_h(Q), kRowStep = pix_row_step(Q);
    const TileGeom tg = tile_geom(a, tile);
    const int cxs = (tg.vw + kItemW - 1) / kItemW;
    const int sx = sub % cxs, sy = sub / cxs;
    const int px = tg.x0 + sx * kItemW + (lane % kItemW);
    const int py0 = tg.y0 + sy * kItemH + (lane / kItemW);
    const uint2 rg = load_range(a, tile);
    const float pxf = (float)px;
    // centre and half-extent of the item's pixel block (for skipping records that miss it)
    const float bcx = (float)(tg.x0 + sx * kItemW) + 0.5f * (kItemW - 1);
    const float bcy = (float)(tg.y0 + sy * kItemH) + 0.5f * (kItemH - 1);
    float pyf[Q], T[Q], c0[Q], c1[Q], c2[Q], D[Q];
    int last[Q], neval[Q], nacc[Q];
    bool done[Q], inside[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int py = py0 + kRowStep * q;
        inside[q] = px < tg.x0 + tg.vw && py < tg.y0 + tg.vh;
        pyf[q] = (float)py;
        T[q] = 1.f;
        c0[q] = c1[q] = c2[q] = D[q] = 0.f;
        last[q] = 0;
        neval[q] = (int)(rg.y - rg.x);
        nacc[q] = 0;
        done[q] = !inside[q];
    }
    for (uint32_t base = rg.x; base < rg.y; base += 32) {
        bool lane_done = true;
#pragma unroll
        for (int q = 0; q < Q; ++q) lane_done = lane_done && done[q];
        if (__all_sync(kFull, lane_done)) break;
        const uint32_t j = base + lane;
        bool hit = false;
        __syncwarp();
        if (j < rg.y) {
            const Rec r = load_rec(a, j);
            buf[lane] = r;
            hit = !box_misses(r.a, r.b, bcx, bcy, 0.5f * (kItemW - 1), 0.5f * (kItemH - 1));
        }
        // records whose alpha box reaches the item's pixel block; the others are skipped
        unsigned live = __ballot_sync(kFull, hit);
        __syncwarp();
        const int pos0 = (int)(base - rg.x);
        while (live) {
            const int k = __ffs(live) - 1;
            live &= live - 1;
            const float4 ra = buf[k].a;
            const float4 rb = buf[k].b;
            const PairX px2 = pair_x(ra, pxf);  // shared by the lane's pixels (same column)
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                float dy;
                const float p2 = pair_power2_y(px2, ra.y, rb.x, pyf[q], dy);
                const float oG = pair_oG(p2, rb.y);
                if (!done[q] && p2 <= 0.f && oG >= kAlphaMin) {
                    const float al = fminf(kAlphaMax, oG);
                    const float tt = next_T(T[q], al);
                    if (tt < kTMin) {
                        done[q] = true;
                        neval[q] = pos0 + k + 1;
                    } else {
                        const float4 rc = buf[k].c;
                        const float w = al * T[q];
                        c0[q] += w * rc.x;
                        c1[q] += w * rc.y;
                        c2[q] += w * rc.z;
                        D[q] += w * rc.w;
                        T[q] = tt;
                        last[q] = pos0 + k + 1;
                        ++nacc[q];
                    }
                }
            }
        }
    }
    int mlast = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (inside[q]) {
            write_pixel(a, tg.v, px, py0 + kRowStep * q, T[q], c0[q], c1[q], c2[q], D[q], last[q], neval[q]);
            st_eval += (unsigned long long)neval[q];
            st_acc += (unsigned long long)nacc[q];
            mlast = max(mlast, last[q]);
        }
    }
    // the tile's largest n_contrib: the backward's per-tile cost (its work list's order)
    if (a.tile_cost) {
        mlast = __reduce_max_sync(kFull, mlast);
        if (lane == 0 && mlast > 0) atomicMax(a.tile_cost + tile, (unsigned int)mlast);
    }
}

// ---- Gaussian-wise items (Sec. 4.2-4.3, Algorithm 6) ------------------------------------
// The lanes of a warp split a tile's depth-sorted list and combine transmittance with a
// prefix product over lanes, as in Algorithm 6, but at chunk granularity: each lane blends a
// contiguous chunk of kGwChunk entries serially (its own transmittance starts at 1), then a
// prefix product composes the chunks with the over-operator
// (C1, T1) o (C2, T2) = (C1 + T1 C2, T1 T2), once per round instead of once per entry.
// An item covers P pixels: the warp's lanes are PXL pixel-lanes x NCH = 32 / PXL chunk-lanes,
// each lane holding PPL of the item's pixels, so that the PXL lanes of one chunk read the same
// records (one gather serves PXL x PPL pixels) and a round covers NCH chunks.  The list is
// further cut into segments of gw_segment entries handled by separate warps (cross-warp
// splitting of one pixel's list): a segment item walks its segment for its P pixels from
// transmittance 1 and writes each pixel's segment summary (C, D, T, last contributor,
// contributing pairs).  k_forward_gw_merge then composes a pixel's segments in list order
// and, in the segment where the composed transmittance falls below 1e-4, walks the entries
// again one by one from the exact incoming transmittance with Algorithm 5's rule, so the
// stop position, n_contrib and n_eval follow the sequential rule (the composed products
// differ from the sequential chain by float32 reassociation only).
constexpr int kGwChunk = 8;                          // entries a lane blends serially per round
constexpr int kGwIdx = 32 * kGwChunk + 32;           // staged indices of the largest round, skewed

template <int P>
struct GwShape {
    static constexpr int PPL = P >= 2 ? 2 : 1;  // pixels per lane
    static constexpr int PXL = P / PPL;         // pixel-lanes
    static_assert(PXL * PPL == P && 32 % PXL == 0, "pixels per Gaussian-wise item: 1, 2, 4, 8 or 16");
};

// Lanes pl, pl + PXL, pl + 2 PXL, ...: the chunk-lanes of pixel-lane pl.
template <int PXL>
__device__ __forceinline__ unsigned gw_group_mask(int pl) {
    constexpr unsigned pat = PXL == 1 ? 0xffffffffu
                           : PXL == 2 ? 0x55555555u
                           : PXL == 4 ? 0x11111111u
                           : PXL == 8 ? 0x01010101u
                                      : 0x00010001u;
    return pat << pl;
}

__device__ __forceinline__ void gw_item_pixel(const TileGeom &tg, int group, int P, int p, bool &ok, float &pxf,
                                              float &pyf) {
    const int npix = tg.vw * tg.vh;
    const int q = group * P + p;
    ok = q < npix;
    const int qq = ok ? q : 0;
    pxf = (float)(tg.x0 + qq % tg.vw);
    pyf = (float)(tg.y0 + qq / tg.vw);
}

// Walks entries [e0, e1) of a tile's list (which starts at list0) for a lane's PPL pixels of
// a Gaussian-wise item laid out as PXL pixel-lanes x (32 / PXL) chunk-lanes.  Per pixel p, on
// entry: Ts = transmittance in front of e0, live = still walking (both the same on the
// chunk-lanes of a pixel); the lane accumulators (c0, c1, c2, d: this lane's share of colour
// and depth; nacc: its contributing pairs) add to what they hold, last (the same on the
// pixel's lanes) is the latest contributor so far.  Per round each chunk-lane blends kGwChunk
// consecutive entries from a local transmittance of 1; a shuffle prefix product over the
// pixel's chunk-lanes gives the transmittance in front of each chunk.  When the round's
// composed transmittance falls below 1e-4:
//   resolve = true (Ts exact): the chunk-lanes in front of the first one whose product falls
//     below 1e-4 compose as usual, and that lane walks the rest of the round entry by entry
//     with Algorithm 5's rule from the transmittance in front of its chunk; the pixel stops
//     at the first entry whose next transmittance is below 1e-4 (stop = entries up to and
//     including it) -- if none does (float32 reassociation), the walk goes on;
//   resolve = false: the pixel is left saturated (live = false, Ts < 1e-4), for the merge.
template <int PXL, int PPL>
__device__ __forceinline__ void gw_walk(const FwdArgs &a, uint32_t e0, uint32_t e1, uint32_t list0, const float *pxf,
                                        const float *pyf, bool resolve, uint32_t *idx_s, int lane, float *Ts,
                                        float *ca0, float *ca1, float *ca2, float *da, int *last, int *nacc,
                                        int *stop, bool *live) {
    constexpr int NCH = 32 / PXL, RND = NCH * kGwChunk;
    const int pl = lane % PXL, ch = lane / PXL;
    const unsigned gmask = gw_group_mask<PXL>(pl);
    const int src_last = (NCH - 1) * PXL + pl;  // the pixel's last chunk-lane
    for (uint32_t base = e0; base < e1; base += (uint32_t)RND) {
        bool any = false;
#pragma unroll
        for (int p = 0; p < PPL; ++p) any = any || live[p];
        if (!__any_sync(kFull, any)) break;
        const uint32_t rend = (uint32_t)min((unsigned long long)e1, (unsigned long long)base + RND);
        // stage the round's indices (coalesced); entry m of the round sits at m + m / kGwChunk
        __syncwarp();
#pragma unroll
        for (int m = lane; m < RND; m += 32) {
            const uint32_t j = base + (uint32_t)m;
            idx_s[m + m / kGwChunk] = j < rend ? a.point_list[j] : 0u;
        }
        __syncwarp();
        float Tl[PPL], c0[PPL], c1[PPL], c2[PPL], dl[PPL];
        int ll[PPL], nl[PPL];
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
            Tl[p] = 1.f;
            c0[p] = c1[p] = c2[p] = dl[p] = 0.f;
            ll[p] = -1;
            nl[p] = 0;
        }
        const uint32_t jc = base + (uint32_t)(kGwChunk * ch);
        for (int k = 0; k < kGwChunk; ++k) {
            const uint32_t j = jc + (uint32_t)k;
            if (j >= rend) break;
            const uint32_t g = idx_s[kGwChunk * ch + k + ch];
            if ((long long)g >= a.N) {
                raise_check(a.ctrl, BGS_CHECK_INDEX);  // a transparent entry
                continue;
            }
            const Rec r = a.recs[g];
#pragma unroll
            for (int p = 0; p < PPL; ++p) {
                float dx, dy;
                const float p2 = pair_power2(r.a, r.b.x, pxf[p], pyf[p], dx, dy);
                const float oG = pair_oG(p2, r.b.y);
                if (live[p] && p2 <= 0.f && oG >= kAlphaMin) {
                    const float al = fminf(kAlphaMax, oG);
                    const float w = al * Tl[p];
                    c0[p] += w * r.c.x;
                    c1[p] += w * r.c.y;
                    c2[p] += w * r.c.z;
                    dl[p] += w * r.c.w;
                    Tl[p] = next_T(Tl[p], al);
                    ll[p] = (int)(j - list0);
                    ++nl[p];
                }
            }
        }
#pragma unroll
        for (int p = 0; p < PPL; ++p) {
            float incl = Tl[p];
#pragma unroll
            for (int off = 1; off < NCH; off <<= 1) {
                const float v = __shfl_up_sync(kFull, incl, off * PXL);
                if (ch >= off) incl *= v;
            }
            float excl = __shfl_up_sync(kFull, incl, PXL);
            if (ch == 0) excl = 1.f;
            const float Tb = Ts[p] * excl;
            const float Tround = Ts[p] * __shfl_sync(kFull, incl, src_last);
            // the same on the pixel's chunk-lanes
            const bool cross = resolve && live[p] && Tround < kTMin;
            const unsigned bal = __ballot_sync(kFull, cross && Ts[p] * incl < kTMin) & gmask;
            const int lam = cross ? __ffs(bal) - 1 : lane;
            const bool front = live[p] && (!cross || lane < lam);
            if (front) {
                ca0[p] += Tb * c0[p];
                ca1[p] += Tb * c1[p];
                ca2[p] += Tb * c2[p];
                da[p] += Tb * dl[p];
                nacc[p] += nl[p];
            }
            int lmax = front ? ll[p] : -1;
#pragma unroll
            for (int off = PXL; off < 32; off <<= 1) lmax = max(lmax, __shfl_xor_sync(kFull, lmax, off));
            last[p] = max(last[p], lmax);
            // the crossing chunk-lane walks the rest of the round for this pixel
            float T = Tb;
            int st = 0, lw = -1;
            if (cross && lane == lam) {
                for (uint32_t j = jc; j < rend; ++j) {
                    const uint32_t m = j - base;
                    const uint32_t g = idx_s[m + m / kGwChunk];
                    if ((long long)g >= a.N) continue;  // raised above
                    const Rec r = a.recs[g];
                    float dx, dy;
                    const float p2 = pair_power2(r.a, r.b.x, pxf[p], pyf[p], dx, dy);
                    const float oG = pair_oG(p2, r.b.y);
                    if (!(p2 <= 0.f && oG >= kAlphaMin)) continue;
                    const float al = fminf(kAlphaMax, oG);
                    const float tt = next_T(T, al);
                    if (tt < kTMin) {
                        st = (int)(j - list0 + 1u);
                        break;
                    }
                    const float w = al * T;
                    ca0[p] += w * r.c.x;
                    ca1[p] += w * r.c.y;
                    ca2[p] += w * r.c.z;
                    da[p] += w * r.c.w;
                    T = tt;
                    lw = (int)(j - list0);
                    ++nacc[p];
                }
            }
            const float Tn = __shfl_sync(kFull, T, lam);
            const int lwn = __shfl_sync(kFull, lw, lam);
            const int stn = __shfl_sync(kFull, st, lam);
            if (cross) {
                Ts[p] = Tn;
                last[p] = max(last[p], lwn);
                if (stn) {
                    stop[p] = stn;
                    live[p] = false;
                }
            } else if (live[p]) {
                Ts[p] = Tround;
                // a pixel below 1e-4 from a transmittance of at most 1 stops within this
                // segment: the rest of it is not needed
                if (Tround < kTMin) live[p] = false;
            }
        }
    }
}

// Sum over the chunk-lanes of each pixel-lane (xor offsets that keep lane % PXL).
template <int PXL>
__device__ __forceinline__ void gw_group_sum5(float &x0, float &x1, float &x2, float &x3, int &n) {
#pragma unroll
    for (int o = PXL; o < 32; o <<= 1) {
        x0 += __shfl_xor_sync(kFull, x0, o);
        x1 += __shfl_xor_sync(kFull, x1, o);
        x2 += __shfl_xor_sync(kFull, x2, o);
        x3 += __shfl_xor_sync(kFull, x3, o);
        n += __shfl_xor_sync(kFull, n, o);
    }
}

// A Gaussian-wise segment item: P pixels of a tile over one segment of its list.  The first
// segment starts from transmittance 1, which is exact, so its stops are resolved here; later
// segments leave saturated pixels to the merge.
template <int P>
__device__ __forceinline__ void gw_segment_item(const FwdArgs &a, int tile, int sub, unsigned item, uint32_t *idx_s,
                                                int lane) {
    constexpr int PPL = GwShape<P>::PPL, PXL = GwShape<P>::PXL;
    const TileGeom tg = tile_geom(a, tile);
    const int groups = (tg.vw * tg.vh + P - 1) / P;
    const int group = sub % groups, seg = sub / groups;
    const uint2 rg = load_range(a, tile);
    // segment size 0: the list is not split (one segment)
    const unsigned int seg_len = *((volatile unsigned int *)&a.ctrl->gw_seg);
    const unsigned long long L = seg_len ? (unsigned long long)seg_len : (1ull << 32);
    const unsigned long long s0 = (unsigned long long)rg.x + (unsigned long long)seg * L;
    const uint32_t e0 = (uint32_t)min((unsigned long long)rg.y, s0);
    const uint32_t e1 = (uint32_t)min((unsigned long long)rg.y, s0 + L);
    const int pl = lane % PXL;
    float pxf[PPL], pyf[PPL], Ts[PPL], ca0[PPL], ca1[PPL], ca2[PPL], da[PPL];
    int last[PPL], nacc[PPL], stop[PPL];
    bool live[PPL];
#pragma unroll
    for (int p = 0; p < PPL; ++p) {
        bool ok;
        gw_item_pixel(tg, group, P, pl * PPL + p, ok, pxf[p], pyf[p]);
        Ts[p] = 1.f;
        ca0[p] = ca1[p] = ca2[p] = da[p] = 0.f;
        last[p] = -1;
        nacc[p] = stop[p] = 0;
        live[p] = ok;
    }
    gw_walk<PXL, PPL>(a, e0, e1, rg.x, pxf, pyf, seg == 0, idx_s, lane, Ts, ca0, ca1, ca2, da, last, nacc, stop,
                      live);
    GwSum *out = reinterpret_cast<GwSum *>(a.gw_sum) + (size_t)item * P;
#pragma unroll
    for (int p = 0; p < PPL; ++p) {
        gw_group_sum5<PXL>(ca0[p], ca1[p], ca2[p], da[p], nacc[p]);
        if (lane < PXL) {  // chunk-lane 0 of each pixel-lane
            GwSum sm;
            sm.cd = make_float4(ca0[p], ca1[p], ca2[p], da[p]);
            sm.t = make_float4(Ts[p], __int_as_float(last[p]), __int_as_float(nacc[p]), __int_as_float(stop[p]));
            out[pl * PPL + p] = sm;
        }
    }
}

__device__ __forceinline__ void flush_stats(const FwdArgs &a, int lane, unsigned long long st_eval,
                                            unsigned long long st_acc, unsigned long long st_items) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        st_eval += __shfl_xor_sync(kFull, st_eval, o);
        st_acc += __shfl_xor_sync(kFull, st_acc, o);
    }
    if (lane == 0) {
        atomicAdd(&a.ctrl->eval_pairs, st_eval);
        atomicAdd(&a.ctrl->contrib_pairs, st_acc);
        atomicAdd(&a.ctrl->items_done, st_items);
    }
}

// Gaussian-wise segment items [0, num_gauss) of the work list.  Launched first; lets the
// pixel-wise kernel launch as soon as all its blocks are resident (programmatic dependent
// launch), so that pixel-wise blocks take over SMs as Gaussian-wise blocks run out of items.
template <int P>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_forward_gauss(FwdArgs a) {
    asm volatile("griddepcontrol.launch_dependents;");
    __shared__ unsigned int blk[2];
    __shared__ uint32_t idx_s[kWarpsPerBlock][kGwIdx];
    if (threadIdx.x == 0) blk[0] = blk[1] = 0u;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned num_items = a.ctrl->num_gauss;
    const unsigned chunk = (unsigned)a.chunk;
    unsigned long long st_items = 0;
    while (true) {
        unsigned first = 0;
        if (lane == 0) first = atomicAdd(&a.ctrl->queue_head_g, chunk);
        first = __shfl_sync(kFull, first, 0);
        if (first >= num_items) break;
        const unsigned end = min(first + chunk, num_items);
        for (unsigned it = first; it < end; ++it) {
            const uint2 item = a.items[it];
            gw_segment_item<P>(a, (int)item.x, (int)(item.y & ~kKindGauss), it, idx_s[warp], lane);
            ++st_items;
        }
    }
    if (lane == 0) atomicAdd(&a.ctrl->items_done, st_items);
    if (lane == 0) finish_pass(a.ctrl, st_items, blk, kWarpsPerBlock, a.pass_blocks);
}

// A warp per first-segment item: for each of its P pixels, composes the segment summaries
// in list order with (C1, T1) o (C2, T2) = (C1 + T1 C2, T1 T2) while the composed
// transmittance stays >= 1e-4; a segment in which it would fall below is walked again from
// the exact incoming transmittance with the stop resolved (gw_walk), after which the
// composition goes on if the walk did not stop.  Writes the pixel's outputs and counts its
// evaluated and contributing pairs.
template <int P>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_forward_gw_merge(FwdArgs a) {
    __shared__ uint32_t idx_s[kWarpsPerBlock][kGwIdx];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned num_first = a.ctrl->num_gauss0;
    GwSum *sums = reinterpret_cast<GwSum *>(a.gw_sum);  // rewritten in place, see below
    const uint32_t L = a.ctrl->gw_seg;
    unsigned long long st_eval = 0, st_acc = 0;
    for (unsigned it = blockIdx.x * kWarpsPerBlock + warp; it < num_first; it += gridDim.x * kWarpsPerBlock) {
        const uint2 item = a.items[it];
        const int tile = (int)item.x, sub = (int)(item.y & ~kKindGauss);
        const TileGeom tg = tile_geom(a, tile);
        const int groups = (tg.vw * tg.vh + P - 1) / P;
        const uint2 rg = load_range(a, tile);
        const uint32_t n = rg.y - rg.x;
        const uint32_t S = (n == 0u || L == 0u) ? 1u : (n - 1u) / L + 1u;
        // summary of segment sg >= 1: the tile's later-segment items, segment-major
        const size_t later = S > 1u ? (size_t)num_first + a.gw_exoff[tile] + (size_t)sub : 0;
        for (int p = 0; p < P; ++p) {
            bool ok;
            float pxf, pyf;
            gw_item_pixel(tg, sub, P, p, ok, pxf, pyf);
            if (!ok) break;
            float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, D = 0.f;
            int last = -1, nacc = 0, stop = 0;
            uint32_t s_end = S - 1u;  // the last segment the pixel reaches
            for (uint32_t sg = 0; sg < S; ++sg) {
                const size_t si = sg == 0u ? (size_t)it : later + (size_t)(sg - 1u) * groups;
                GwSum *slot = sums + si * P + p;
                const GwSum sm = *slot;
                const int sst = __float_as_int(sm.t.w);
                if (sg == 0u && sst) {  // stopped in the first segment, resolved there
                    T = sm.t.x;
                    c0 = sm.cd.x, c1 = sm.cd.y, c2 = sm.cd.z, D = sm.cd.w;
                    last = __float_as_int(sm.t.y);
                    nacc = __float_as_int(sm.t.z);
                    stop = sst;
                    s_end = 0u;
                    break;
                }
                const float T_in = T;
                float a0, a1, a2, ad;  // the segment's colour and depth with absolute weights
                bool stopped = false;
                if (T * sm.t.x >= kTMin) {
                    a0 = T * sm.cd.x, a1 = T * sm.cd.y, a2 = T * sm.cd.z, ad = T * sm.cd.w;
                    T *= sm.t.x;
                    last = max(last, __float_as_int(sm.t.y));
                    nacc += __float_as_int(sm.t.z);
                } else {
                    const uint32_t e0 = S > 1u ? rg.x + sg * L : rg.x;
                    const uint32_t e1 =
                        S > 1u ? (uint32_t)min((unsigned long long)rg.y, (unsigned long long)e0 + L) : rg.y;
                    float Tw = T, w0 = 0.f, w1 = 0.f, w2 = 0.f, wd = 0.f;
                    int lw = last, nw = 0, sw = 0;
                    bool live = true;
                    gw_walk<1, 1>(a, e0, e1, rg.x, &pxf, &pyf, true, idx_s[warp], lane, &Tw, &w0, &w1, &w2, &wd, &lw,
                                  &nw, &sw, &live);
                    gw_group_sum5<1>(w0, w1, w2, wd, nw);
                    a0 = w0, a1 = w1, a2 = w2, ad = wd;
                    T = Tw;
                    last = lw;
                    nacc += nw;
                    if (sw) {
                        stop = sw;
                        stopped = true;
                    }
                }
                c0 += a0, c1 += a1, c2 += a2, D += ad;
                // the slot now holds the segment's absolute contribution and entry T (the
                // backward's boundary states are formed from them below); every lane has read it
                __syncwarp();
                if (S > 1u && lane == 0) {
                    GwSum o;
                    o.cd = make_float4(a0, a1, a2, ad);
                    o.t = make_float4(T_in, 0.f, 0.f, 0.f);
                    *slot = o;
                }
                if (stopped) {
                    s_end = sg;
                    break;
                }
            }
            // Boundary states for a segmented backward: per segment u the pixel reaches, the
            // transmittance behind it (in front of segment u + 1, or the final T) and the
            // colour and depth accumulated behind it with absolute weights, background
            // included -- summed from the back, so no difference of two sums is formed.
            if (S > 1u && lane == 0 && s_end > 0u) {
                float b0 = T * a.bg[0], b1 = T * a.bg[1], b2 = T * a.bg[2], bd = 0.f, Tnext = T;
                for (int u = (int)s_end; u >= 0; --u) {
                    GwSum *slot = sums + ((u == 0 ? (size_t)it : later + (size_t)(u - 1) * groups) * P + p);
                    const GwSum sm = *slot;
                    GwSum o;
                    o.cd = make_float4(b0, b1, b2, bd);
                    o.t = make_float4(Tnext, 0.f, 0.f, 0.f);
                    *slot = o;
                    b0 += sm.cd.x, b1 += sm.cd.y, b2 += sm.cd.z, bd += sm.cd.w;
                    Tnext = sm.t.x;
                }
            }
            const int neval = stop ? stop : (int)n;
            if (lane == 0) {
                write_pixel(a, tg.v, (int)pxf, (int)pyf, T, c0, c1, c2, D, last + 1, neval);
                if (a.tile_cost && last >= 0) atomicMax(a.tile_cost + tile, (unsigned int)(last + 1));
                st_eval += (unsigned long long)neval;
                st_acc += (unsigned long long)nacc;
            }
        }
    }
    if (lane == 0 && (st_eval | st_acc)) {
        atomicAdd(&a.ctrl->eval_pairs, st_eval);
        atomicAdd(&a.ctrl->contrib_pairs, st_acc);
    }
}

// Pixel-wise items [num_gauss, num_items) of the work list.
template <int Q>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_forward_pixel(FwdArgs a) {
    __shared__ Rec sbuf[kWarpsPerBlock][32];
    __shared__ unsigned int blk[2];
    if (threadIdx.x == 0) blk[0] = blk[1] = 0u;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Rec *buf = sbuf[warp];
    const unsigned num_items = a.ctrl->num_items;
    const unsigned chunk = (unsigned)a.chunk;
    unsigned long long st_eval = 0, st_acc = 0, st_items = 0;
    while (true) {
        unsigned first = 0;
        if (lane == 0) first = atomicAdd(&a.ctrl->queue_head, chunk);
        first = __shfl_sync(kFull, first, 0);
        if (first >= num_items) break;
        const unsigned end = min(first + chunk, num_items);
        for (unsigned it = first; it < end; ++it) {
            const uint2 item = a.items[it];
            pixel_item<Q>(a, (int)item.x, (int)(item.y & ~kKindGauss), buf, lane, st_eval, st_acc);
            ++st_items;
        }
    }
    flush_stats(a, lane, st_eval, st_acc, st_items);
    if (lane == 0) finish_pass(a.ctrl, st_items, blk, kWarpsPerBlock, a.pass_blocks);
    // launched after k_forward_gauss with programmatic serialisation: complete only once the
    // Gaussian-wise grid has (so that whatever follows on the stream, the merge included,
    // sees its summaries); a no-op for an ordinary launch
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

int forward_balanced_block_threads() { return kWarpsPerBlock * 32; }

const void *forward_gauss_kernel(int gw_pixels) {
    switch (gw_pixels) {
        case 1: return (const void *)k_forward_gauss<1>;
        case 2: return (const void *)k_forward_gauss<2>;
        case 4: return (const void *)k_forward_gauss<4>;
        case 8: return (const void *)k_forward_gauss<8>;
        case 16: return (const void *)k_forward_gauss<16>;
        default: return nullptr;
    }
}

const void *forward_gw_merge_kernel(int gw_pixels) {
    switch (gw_pixels) {
        case 1: return (const void *)k_forward_gw_merge<1>;
        case 2: return (const void *)k_forward_gw_merge<2>;
        case 4: return (const void *)k_forward_gw_merge<4>;
        case 8: return (const void *)k_forward_gw_merge<8>;
        case 16: return (const void *)k_forward_gw_merge<16>;
        default: return nullptr;
    }
}

const void *forward_pixel_kernel(int pixel_rows) {
    switch (pixel_rows) {
        case 1: return (const void *)k_forward_pixel<1>;
        case 2: return (const void *)k_forward_pixel<2>;
        case 4: return (const void *)k_forward_pixel<4>;
        case 8: return (const void *)k_forward_pixel<8>;
        default: return nullptr;
    }
}

cudaError_t launch_forward_gauss(const FwdArgs &a, int grid, cudaStream_t s) {
    const int threads = kWarpsPerBlock * 32;
    switch (a.gw_pixels) {
        case 1: k_forward_gauss<1><<<grid, threads, 0, s>>>(a); break;
        case 2: k_forward_gauss<2><<<grid, threads, 0, s>>>(a); break;
        case 4: k_forward_gauss<4><<<grid, threads, 0, s>>>(a); break;
        case 8: k_forward_gauss<8><<<grid, threads, 0, s>>>(a); break;
        case 16: k_forward_gauss<16><<<grid, threads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_forward_gw_merge(const FwdArgs &a, int grid, cudaStream_t s) {
    switch (a.gw_pixels) {
        case 1: k_forward_gw_merge<1><<<grid, kWarpsPerBlock * 32, 0, s>>>(a); break;
        case 2: k_forward_gw_merge<2><<<grid, kWarpsPerBlock * 32, 0, s>>>(a); break;
        case 4: k_forward_gw_merge<4><<<grid, kWarpsPerBlock * 32, 0, s>>>(a); break;
        case 8: k_forward_gw_merge<8><<<grid, kWarpsPerBlock * 32, 0, s>>>(a); break;
        case 16: k_forward_gw_merge<16><<<grid, kWarpsPerBlock * 32, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// after_gauss: launched right after k_forward_gauss on the same stream, with programmatic
// stream serialisation (the two kernels touch disjoint pixels and k_forward_gauss started
// after the work list was complete, so no wait is needed).  Otherwise an ordinary launch:
// the kernel has no grid-dependency wait, so it must not overlap the kernels that build
// its work list.
cudaError_t launch_forward_pixel(const FwdArgs &a, int grid, bool after_gauss, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kWarpsPerBlock * 32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = after_gauss ? 1 : 0;
    switch (a.pixel_rows) {
        case 1: return cudaLaunchKernelEx(&cfg, k_forward_pixel<1>, a);
        case 2: return cudaLaunchKernelEx(&cfg, k_forward_pixel<2>, a);
        case 4: return cudaLaunchKernelEx(&cfg, k_forward_pixel<4>, a);
        case 8: return cudaLaunchKernelEx(&cfg, k_forward_pixel<8>, a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bgs
