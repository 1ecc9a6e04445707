// noalloc.cu -- an allocation-free variant of the balanced forward render.
//
// bgs_render_forward keeps its scratch (packed records, the work list, queue counters) in
// the plan's workspace, which the library allocates with cudaMalloc on first use.  Some
// callers cannot allow that: a host application that owns every byte of device memory
// under a fixed budget (a game engine, an inference server), a plugin loaded into such a
// process, or a runtime that forbids device allocations after start-up.  For them,
// bgs_render_forward_noalloc runs the persistent pixel-wise forward with its scratch in
// one fixed-size array that lives in this library's own device memory (a file-scope
// __device__ array, present on every GPU that loads the library until the process
// exits).  The caller still provides every input and output buffer.
//
// The scratch array is shared by all calls: each call first resets the parts that must
// start at zero, so consecutive calls on one stream are independent, but calls that
// overlap on the GPU (different streams, or concurrent host threads) race on it.
// Entries with an out-of-range index or tile span are rendered as transparent and raise a
// check bit in the scratch array; a caller that passes a host word for the bits gets them
// back (the call then waits for its own work), otherwise they are not reported.
#include <mutex>

#include "bgs_internal.cuh"

namespace {

using namespace bgs;

constexpr int kNaMaxTiles = 65536;  // largest tile grid the scratch array holds
constexpr int kNaBuckets = 33;      // list-length classes: 0 for n = 0, 1 + floor(log2 n) otherwise
constexpr int kNaWarps = 8;

struct NaScratch {
    unsigned int queue_head;   // next work item
    unsigned int num_items;    // work items of this call
    unsigned int check_bits;   // BGS_CHECK_* raised by this call
    unsigned int pad;
    unsigned int tile_order[kNaMaxTiles];  // tiles, longest lists first (by length class)
};

// The scratch: 256-byte aligned, about 256 KiB, one copy per device.
static __device__ __align__(256) NaScratch g_na_scratch;

struct NaArgs {
    const float *means2D, *conic_opacity, *colors, *depths;
    const uint32_t *point_list;
    const uint2 *ranges;
    long long N, num_entries;
    int W, H, tile_w, tile_h, tiles_x, tiles_y, items_per_tile;
    float bg[3];
    float *out_color, *out_depth, *out_alpha, *final_T;
    int *n_contrib, *n_eval;
};

__device__ __forceinline__ int length_class(uint32_t n) { return n == 0 ? 0 : 32 - __clz(n); }

// One block: resets the queue, orders the tiles by descending list-length class (a
// counting sort over 33 classes) and publishes the item count.  The order inside a class
// is arbitrary; it does not change any pixel's result.
__global__ void __launch_bounds__(1024) k_na_prepare(NaArgs a, NaScratch *sc) {
    __shared__ unsigned int hist[kNaBuckets], base[kNaBuckets];
    const int T = a.tiles_x * a.tiles_y;
    if (threadIdx.x < kNaBuckets) hist[threadIdx.x] = 0u;
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const uint2 rg = a.ranges[t];
        atomicAdd(&hist[length_class(rg.y >= rg.x ? rg.y - rg.x : 0u)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int run = 0;
        for (int c = kNaBuckets - 1; c >= 0; --c) {  // longest class first
            base[c] = run;
            run += hist[c];
        }
        sc->queue_head = 0u;
        sc->num_items = (unsigned int)T * (unsigned int)a.items_per_tile;
        sc->check_bits = 0u;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const uint2 rg = a.ranges[t];
        const unsigned int slot = atomicAdd(&base[length_class(rg.y >= rg.x ? rg.y - rg.x : 0u)], 1u);
        sc->tile_order[slot] = (unsigned int)t;
    }
}

// Persistent pixel-wise forward: warps pull items (tile slot, 8x4 sub-block) from the
// queue in the scratch array; records are read from the caller's arrays and staged in a
// warp-private shared-memory window.  Same per-pair arithmetic as the other kernels.
__global__ void __launch_bounds__(kNaWarps * 32) k_na_forward(NaArgs a, NaScratch *sc) {
    __shared__ Rec sbuf[kNaWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Rec *buf = sbuf[warp];
    const unsigned int num_items = sc->num_items;
    while (true) {
        unsigned int it = 0;
        if (lane == 0) it = atomicAdd(&sc->queue_head, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= num_items) break;
        const int tile = (int)sc->tile_order[it / a.items_per_tile];
        const int sub = (int)(it % a.items_per_tile);
        const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
        const int x0 = tx * a.tile_w, y0 = ty * a.tile_h;
        const int subs_x = a.tile_w / 8;
        const int px = x0 + (sub % subs_x) * 8 + (lane & 7), py = y0 + (sub / subs_x) * 4 + (lane >> 3);
        const bool inside = px < a.W && py < a.H;
        uint2 rg = a.ranges[tile];
        if (rg.y < rg.x || (long long)rg.y > a.num_entries) {
            if (lane == 0) atomicOr(&sc->check_bits, (unsigned int)BGS_CHECK_RANGE);
            rg = make_uint2(0u, 0u);
        }
        const float pxf = (float)px, pyf = (float)py;
        float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, D = 0.f;
        int last = 0, neval = (int)(rg.y - rg.x);
        bool done = !inside;
        for (uint32_t base = rg.x; base < rg.y; base += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            const uint32_t j = base + lane;
            __syncwarp();
            if (j < rg.y) {
                const uint32_t g = a.point_list[j];
                if ((long long)g < a.N) {
                    buf[lane] = make_rec(a.means2D, a.conic_opacity, a.colors, a.depths, g);
                } else {
                    atomicOr(&sc->check_bits, (unsigned int)BGS_CHECK_INDEX);
                    buf[lane].a = make_float4(0.f, 0.f, 0.f, 0.f);
                    buf[lane].b = make_float4(0.f, 0.f, 0.f, 0.f);
                    buf[lane].c = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            __syncwarp();
            const int cnt = min(32, (int)(rg.y - base));
            for (int k = 0; k < cnt; ++k) {
                const float4 ra = buf[k].a;
                const float4 rb = buf[k].b;
                float dx, dy;
                const float p2 = pair_power2(ra, rb.x, pxf, pyf, dx, dy);
                const float oG = pair_oG(p2, rb.y);
                if (!done && p2 <= 0.f && oG >= kAlphaMin) {
                    const float al = fminf(kAlphaMax, oG);
                    const float tt = next_T(T, al);
                    if (tt < kTMin) {
                        done = true;
                        neval = (int)(base + k + 1 - rg.x);
                    } else {
                        const float4 rc = buf[k].c;
                        const float w = al * T;
                        c0 += w * rc.x;
                        c1 += w * rc.y;
                        c2 += w * rc.z;
                        D += w * rc.w;
                        T = tt;
                        last = (int)(base + k + 1 - rg.x);
                    }
                }
            }
        }
        if (inside) {
            const long long HW = (long long)a.W * a.H, pid = (long long)py * a.W + px;
            a.out_color[pid] = c0 + T * a.bg[0];
            a.out_color[HW + pid] = c1 + T * a.bg[1];
            a.out_color[2 * HW + pid] = c2 + T * a.bg[2];
            a.out_depth[pid] = D;
            a.out_alpha[pid] = 1.f - T;  // sum of alpha_i T_i telescopes to 1 - T
            a.final_T[pid] = T;
            a.n_contrib[pid] = last;
            if (a.n_eval) a.n_eval[pid] = neval;
        }
    }
}

// Device address of the scratch array, looked up once per device (with that device
// current) and cached.  In host code the array's name is only a host-side stand-in.
std::mutex g_na_mutex;
NaScratch *g_na_ptr[64] = {};
int g_na_blocks[64] = {};

int na_fail(int code, const char *msg) { return bgs::set_error(code, msg); }

}  // namespace

extern "C" int bgs_render_forward_noalloc(int64_t N, const float *means2D, const float *conic_opacity,
                                          const float *colors, const float *depths, const uint32_t *point_list,
                                          int64_t num_entries, const uint32_t *ranges, int32_t W, int32_t H,
                                          int32_t tile_w, int32_t tile_h, const float *bg, float *out_color,
                                          float *out_depth, float *out_alpha, float *final_T, int32_t *n_contrib,
                                          int32_t *n_eval, uint32_t *check_bits, void *stream) {
    if (N < 0 || N >= (1ll << 32) || num_entries < 0 || num_entries > BGS_MAX_ENTRIES)
        return na_fail(BGS_ERR_INVALID, "bgs_render_forward_noalloc: N or num_entries out of range");
    if (W <= 0 || H <= 0 || (long long)W * H > (1ll << 31) - 1)
        return na_fail(BGS_ERR_INVALID, "bgs_render_forward_noalloc: bad image size");
    if (tile_w <= 0 || tile_h <= 0 || tile_w % 8 != 0 || tile_h % 4 != 0 || tile_w * tile_h > 1024)
        return na_fail(BGS_ERR_INVALID, "bgs_render_forward_noalloc: tile_w must be a multiple of 8, tile_h of 4");
    if (!ranges || !bg || !out_color || !out_depth || !out_alpha || !final_T || !n_contrib ||
        (num_entries > 0 && !point_list) || (N > 0 && (!means2D || !conic_opacity || !colors || !depths)))
        return na_fail(BGS_ERR_INVALID, "bgs_render_forward_noalloc: NULL array");
    const int tiles_x = (W + tile_w - 1) / tile_w, tiles_y = (H + tile_h - 1) / tile_h;
    if ((long long)tiles_x * tiles_y > kNaMaxTiles)
        return na_fail(BGS_ERR_CAPACITY, "bgs_render_forward_noalloc: more than 65536 tiles (the fixed scratch "
                                         "array's limit); use bgs_render_forward");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return na_fail(BGS_ERR_CUDA, "bgs_render_forward_noalloc: no current CUDA device");
    NaScratch *sc = nullptr;
    int blocks = 0;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p)
                return na_fail(BGS_ERR_CUDA, "bgs_render_forward_noalloc: cudaGetSymbolAddress failed");
            int sms = 0, per_sm = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_na_forward, kNaWarps * 32, 0) !=
                    cudaSuccess)
                return na_fail(BGS_ERR_CUDA, "bgs_render_forward_noalloc: device query failed");
            g_na_blocks[dev] = sms * (per_sm > 0 ? per_sm : 1);
            g_na_ptr[dev] = (NaScratch *)p;
        }
        sc = g_na_ptr[dev];
        blocks = g_na_blocks[dev];
    }
    NaArgs a;
    a.means2D = means2D;
    a.conic_opacity = conic_opacity;
    a.colors = colors;
    a.depths = depths;
    a.point_list = point_list;
    a.ranges = reinterpret_cast<const uint2 *>(ranges);
    a.N = N;
    a.num_entries = num_entries;
    a.W = W;
    a.H = H;
    a.tile_w = tile_w;
    a.tile_h = tile_h;
    a.tiles_x = tiles_x;
    a.tiles_y = tiles_y;
    a.items_per_tile = (tile_w / 8) * (tile_h / 4);
    a.bg[0] = bg[0];
    a.bg[1] = bg[1];
    a.bg[2] = bg[2];
    a.out_color = out_color;
    a.out_depth = out_depth;
    a.out_alpha = out_alpha;
    a.final_T = final_T;
    a.n_contrib = n_contrib;
    a.n_eval = n_eval;
    cudaStream_t s = (cudaStream_t)stream;
    k_na_prepare<<<1, 1024, 0, s>>>(a, sc);
    k_na_forward<<<blocks, kNaWarps * 32, 0, s>>>(a, sc);
    if (cudaGetLastError() != cudaSuccess) return na_fail(BGS_ERR_CUDA, "bgs_render_forward_noalloc: launch failed");
    if (check_bits) {
        // this call's bits, read after its kernels (a copy into the caller's host word)
        if (cudaMemcpyAsync(check_bits, &sc->check_bits, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return na_fail(BGS_ERR_CUDA, "bgs_render_forward_noalloc: reading the check bits failed");
        if (*check_bits)
            return na_fail(BGS_ERR_DEVICE_CHECK, "bgs_render_forward_noalloc: device check tripped (an index >= N "
                                                 "or a tile span past num_entries was rendered transparent)");
    }
    return BGS_OK;
}
