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
//                          Sec. 4.3): P pixels of a tile processed one after another by
//                          the whole warp, lanes splitting the list 32 entries at a time
//                          and combining transmittance with a shuffle prefix product;
//                        - pixel-wise: an 8x8 sub-block of a tile, two pixels per lane,
//                          walking the tile's list through a warp-private shared memory
//                          window of 32 records.
//
// All evaluate each (pixel, entry) pair with the same code (pair_power2 / pair_alpha), so
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
            float dx, dy, G;
            const float p2 = pair_power2(ra, rb.x, pxf, pyf, dx, dy);
            const float al = pair_alpha(p2, rb.y, G);
            if (p2 > 0.f || al < kAlphaMin) continue;
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
                float dy, G;
                const float p2 = pair_power2_y(px2, ra.y, rb.x, pyf[q], dy);
                const float al = pair_alpha(p2, rb.y, G);
                if (!done[q] && p2 <= 0.f && al >= kAlphaMin) {
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
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (inside[q]) {
            write_pixel(a, tg.v, px, py0 + kRowStep * q, T[q], c0[q], c1[q], c2[q], D[q], last[q], neval[q]);
            st_eval += (unsigned long long)neval[q];
            st_acc += (unsigned long long)nacc[q];
        }
    }
}

// Gaussian-wise item: P pixels, lanes split the list 32 entries at a time.
template <int P>
__device__ __forceinline__ void gauss_item(const FwdArgs &a, int tile, int sub, int lane,
                                           unsigned long long &st_eval, unsigned long long &st_acc) {
    const TileGeom tg = tile_geom(a, tile);
    const int npix = tg.vw * tg.vh;
    const uint2 rg = load_range(a, tile);
    const int n = (int)(rg.y - rg.x);
    float pxf[P], pyf[P], T[P], c0[P], c1[P], c2[P], D[P];
    int last[P], neval[P], nacc[P];
    bool done[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int q = sub * P + p;
        const bool ok = q < npix;
        const int qq = ok ? q : 0;
        pxf[p] = (float)(tg.x0 + qq % tg.vw);
        pyf[p] = (float)(tg.y0 + qq / tg.vw);
        T[p] = 1.f;
        c0[p] = c1[p] = c2[p] = D[p] = 0.f;
        last[p] = 0;
        neval[p] = n;
        nacc[p] = 0;
        done[p] = !ok;
    }
    for (uint32_t base = rg.x; base < rg.y; base += 32) {
        bool all_done = true;
#pragma unroll
        for (int p = 0; p < P; ++p) all_done = all_done && done[p];
        if (all_done) break;
        const uint32_t j = base + lane;
        const bool inb = j < rg.y;
        Rec r;
        if (inb) {
            r = load_rec(a, j);
        } else {
            r.a = make_float4(0.f, 0.f, 0.f, 0.f);
            r.b = r.a;
            r.c = r.a;
        }
        const int pos0 = (int)(base - rg.x);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (done[p]) continue;  // warp-uniform
            float dx, dy, G;
            const float p2 = pair_power2(r.a, r.b.x, pxf[p], pyf[p], dx, dy);
            const float al = pair_alpha(p2, r.b.y, G);
            const bool valid = inb && p2 <= 0.f && al >= kAlphaMin;
            const unsigned vmask = __ballot_sync(kFull, valid);
            if (vmask == 0u) continue;  // no lane contributes: skip the scan (Algorithm 6's all-invalid test)
            // inclusive prefix product of (1 - alpha) over the lanes (skipped lanes contribute 1)
            float incl = valid ? 1.f - al : 1.f;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float v = __shfl_up_sync(kFull, incl, off);
                if (lane >= off) incl *= v;
            }
            float excl = __shfl_up_sync(kFull, incl, 1);
            if (lane == 0) excl = 1.f;
            const float Tp = T[p];
            const float tt = Tp * incl;  // transmittance after this lane's entry
            // early stop (Algorithm 5's rule on the prefix-product T'): the first valid lane
            // whose T' falls below 1e-4 stops the pixel and is not accumulated; the lanes
            // before it are.  T' differs from the sequential FMA chain of the pixel-wise
            // kernels by rounding only.
            const unsigned smask = __ballot_sync(kFull, valid && tt < kTMin);
            const int kstop = smask ? __ffs(smask) - 1 : 32;
            const unsigned below = kstop >= 32 ? kFull : ((1u << kstop) - 1u);
            const unsigned amask = vmask & below;
            if (valid && lane < kstop) {
                const float w = al * (Tp * excl);
                c0[p] += w * r.c.x;
                c1[p] += w * r.c.y;
                c2[p] += w * r.c.z;
                D[p] += w * r.c.w;
            }
            const float tnew = __shfl_sync(kFull, tt, kstop > 0 ? kstop - 1 : 0);
            if (kstop > 0) T[p] = tnew;
            if (amask) {
                last[p] = pos0 + (32 - __clz(amask));
                nacc[p] += __popc(amask);
            }
            if (smask) {
                done[p] = true;
                neval[p] = pos0 + kstop + 1;
            }
        }
    }
    // combine the lanes' partial sums and write the P pixels
#pragma unroll
    for (int p = 0; p < P; ++p) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c0[p] += __shfl_xor_sync(kFull, c0[p], o);
            c1[p] += __shfl_xor_sync(kFull, c1[p], o);
            c2[p] += __shfl_xor_sync(kFull, c2[p], o);
            D[p] += __shfl_xor_sync(kFull, D[p], o);
        }
        const int q = sub * P + p;
        if (q < npix) {
            if (lane == p)
                write_pixel(a, tg.v, (int)pxf[p], (int)pyf[p], T[p], c0[p], c1[p], c2[p], D[p], last[p],
                            neval[p]);
            if (lane == 0) {
                st_eval += (unsigned long long)neval[p];
                st_acc += (unsigned long long)nacc[p];
            }
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

// Gaussian-wise items [0, num_gauss) of the work list.  Launched first; lets the pixel-wise
// kernel launch as soon as all its blocks are resident (programmatic dependent launch),
// so that pixel-wise blocks take over SMs as Gaussian-wise blocks run out of items.
template <int P>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_forward_gauss(FwdArgs a) {
    asm volatile("griddepcontrol.launch_dependents;");
    __shared__ unsigned int blk[2];
    if (threadIdx.x == 0) blk[0] = blk[1] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned num_items = a.ctrl->num_gauss;
    const unsigned chunk = (unsigned)a.chunk;
    unsigned long long st_eval = 0, st_acc = 0, st_items = 0;
    while (true) {
        unsigned first = 0;
        if (lane == 0) first = atomicAdd(&a.ctrl->queue_head_g, chunk);
        first = __shfl_sync(kFull, first, 0);
        if (first >= num_items) break;
        const unsigned end = min(first + chunk, num_items);
        for (unsigned it = first; it < end; ++it) {
            const uint2 item = a.items[it];
            gauss_item<P>(a, (int)item.x, (int)(item.y & ~kKindGauss), lane, st_eval, st_acc);
            ++st_items;
        }
    }
    flush_stats(a, lane, st_eval, st_acc, st_items);
    if (lane == 0) finish_pass(a.ctrl, st_items, blk, kWarpsPerBlock, a.pass_blocks);
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
}

int forward_balanced_block_threads() { return kWarpsPerBlock * 32; }

const void *forward_gauss_kernel(int gw_pixels) {
    switch (gw_pixels) {
        case 1: return (const void *)k_forward_gauss<1>;
        case 2: return (const void *)k_forward_gauss<2>;
        case 4: return (const void *)k_forward_gauss<4>;
        case 8: return (const void *)k_forward_gauss<8>;
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
