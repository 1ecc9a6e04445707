// capi.cu -- the C ABI (include/bgs.h): plan, workspace, argument checks and the
// host-side sequencing of the kernels of each entry point.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "bgs_internal.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(BGS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BGS_CUDA(call, what)                         \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

int bits_for(long long v) {
    int b = 1;
    while ((1ll << b) <= v) ++b;
    return b;
}

}  // namespace

namespace bgs {
// Records a message for bgs_last_error() (used by entry points defined in other files).
int set_error(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace bgs

constexpr int kSortStreams = 4;

struct bgs_plan {
    bgs_plan_desc desc;
    int device = 0;
    int num_sms = 0;
    bgs::DevCtrl *ctrl = nullptr;
    // optional CUDA-event timing of the two render kernels (forward, backward)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_fwd, ev_bwd;
    unsigned long long host_launches = 0;
    // binning
    Buf touched, touched_sorted, dkey, dkey_sorted, gidx, order, offsets, keys_in, keys_out, vals_in, cub_tmp;
    // counting-sort binning, one buffer set per concurrent view (stream slot): tile histogram,
    // totals, starts, packed rectangles, masks; list truncation (credits, last block per
    // tile); the scatter's work items per tile group; the tile scan's temporaries
    struct BinSlot {
        Buf h, total, start, rect, mask, credit, sat, items, scan_tmp, stopped;
    } bin_slot[kSortStreams];
    cudaEvent_t view_done[bgs::kMaxViews] = {};  // a view's entry count is known
    int smem_optin = 0;
    // render
    Buf recs, tile_idx, items, grad_acc, warp_items;  // tile_idx: each tile's slot in its work-list bucket
    Buf gw_exoff, gw_sum, gw_tile;  // Gaussian-wise segments: per-tile later-segment offsets, per-item
                                    // summaries, per-tile segment item positions
    Buf tile_cost;                  // per-tile largest n_contrib, from the last forward (the
                                    // backward's work-list order); valid for cost_key's tiles
    // batched binning: depth keys of every view
    Buf vkey_sorted;
    long long iota_n = 0;  // gidx[0, iota_n) holds 0, 1, ... (the batched depth sort's values)
    // the views' depth sorts run concurrently on kSortStreams streams forked from the caller's
    cudaStream_t sort_stream[kSortStreams] = {};
    cudaEvent_t sort_fork = nullptr, sort_join[kSortStreams] = {};
    Buf sort_tmp[kSortStreams];
    // captured CUDA graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    // what the packed records and the work list currently hold (a backward on the arrays of
    // the last forward reuses both instead of rebuilding them)
    struct RecKey {
        const void *means2D, *conic_opacity, *colors, *depths;
        int64_t n_records, n_colors;
    } rec_key;
    struct WlKey {
        const void *ranges;
        bgs::ViewTable vt;
        int tw, th, mode, heavy_threshold, gw_pixels, pixel_rows, lpt_order, gw_segment, bseg_mode, costed;
    } wl_key;
    // the last forward split Gaussian-wise lists into segments on the list of this key: a
    // backward on the same arrays walks those tiles segment by segment from the boundary
    // states the forward left in gw_sum (per tile: gw_tile)
    WlKey gw_fwd_key;
    bool gw_fwd_valid = false;
    WlKey cost_key;  // the tiles tile_cost describes
    bool cost_valid = false;
    bool rec_valid = false, wl_valid = false;
    unsigned int inject = 0;  // BGS_CHECK_* fault to inject into the next persistent pass
    // BGS_MODE_SELECT (Sec. 4.4)
    bool sel_switched = false;
    long long sel_calls = 0, sel_measurements = 0;
    double sel_last_balanced = 0.0, sel_last_static = 0.0;
};

namespace {

// A fault requested by bgs_plan_inject_fault, applied once before the next persistent pass.
int inject_pending_fault(bgs_plan *p, cudaStream_t s) {
    if (p->inject & BGS_CHECK_QUEUE) BGS_CUDA(bgs::launch_exhaust_queue(p->ctrl, s), "inject queue fault");
    p->inject = 0;
    return BGS_OK;
}

int ensure(bgs_plan *p, Buf &b, size_t bytes, cudaStream_t s, const char *what) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return BGS_OK;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone)
        return fail(BGS_ERR_CAPACITY, "workspace '%s' needs %zu bytes while the stream is being captured; "
                                      "call bgs_plan_reserve before capture", what, bytes);
    if (&b == &p->recs) p->rec_valid = false;
    if (&b == &p->items) p->wl_valid = false;
    if (&b == &p->gidx) p->iota_n = 0;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree(workspace)");
    }
    const size_t grown = bytes + bytes / 8 + 256;
    cudaError_t e = cudaMalloc(&b.p, grown);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return fail(BGS_ERR_CUDA, "cudaMalloc(%zu) for workspace '%s': %s", grown, what, cudaGetErrorString(e));
    }
    b.bytes = grown;
    return BGS_OK;
}

cudaEvent_t take_event(bgs_plan *p) {
    if (!p->ev_pool.empty()) {
        cudaEvent_t e = p->ev_pool.back();
        p->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone;
}

// Records an event pair around one render-kernel launch when timing is on.
struct KernelTimer {
    bgs_plan *p;
    cudaStream_t s;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *dst;
    cudaEvent_t a = nullptr, b = nullptr;
    KernelTimer(bgs_plan *p_, cudaStream_t s_, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *d)
        : p(p_), s(s_), dst(d) {
        if (p->timing && !capturing(s)) {
            a = take_event(p);
            b = take_event(p);
            if (a && b) cudaEventRecord(a, s);
        }
    }
    void stop() {
        if (a && b) {
            cudaEventRecord(b, s);
            dst->emplace_back(a, b);
            a = b = nullptr;
        }
    }
};

#define BGS_TRY(x)                 \
    do {                           \
        int r_ = (x);              \
        if (r_ != BGS_OK) return r_; \
    } while (0)

int check_tile(int tw, int th, bool balanced) {
    if (tw <= 0 || th <= 0 || tw * th > 1024 || (tw * th) % 32 != 0)
        return fail(BGS_ERR_INVALID, "tile %dx%d: need 32 <= tile_w*tile_h <= 1024, a multiple of 32", tw, th);
    if (balanced && (tw % 8 != 0 || th % 4 != 0))
        return fail(BGS_ERR_INVALID, "tile %dx%d: the persistent kernels need tile_w %% 8 == 0 and tile_h %% 4 == 0",
                    tw, th);
    return BGS_OK;
}

int check_image(int W, int H) {
    if (W <= 0 || H <= 0 || (long long)W * H > (1ll << 31) - 1)
        return fail(BGS_ERR_INVALID, "image %dx%d: need 0 < W*H < 2^31", W, H);
    return BGS_OK;
}

int grid_for(const bgs_plan *p, const void *kernel, int threads) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    if (p->desc.blocks_per_sm > 0) per_sm = std::min(per_sm, (int)p->desc.blocks_per_sm);
    return p->num_sms * per_sm;
}

// Builds the work list of the persistent kernels over the global tile space of the views (a3).
bgs_plan::WlKey worklist_key(const bgs_plan *p, const uint32_t *ranges, const bgs::ViewTable &vt, int tw, int th,
                             int mode, int bseg_mode = -1, int costed = 0) {
    bgs_plan::WlKey k;
    memset(&k, 0, sizeof k);  // padding included: keys are compared with memcmp
    k.ranges = ranges;
    k.vt = vt;
    k.tw = tw;
    k.th = th;
    k.mode = mode;
    k.heavy_threshold = p->desc.heavy_threshold;
    k.gw_pixels = p->desc.gw_pixels;
    k.pixel_rows = p->desc.pixel_rows;
    k.lpt_order = p->desc.lpt_order;
    k.gw_segment = p->desc.gw_segment;
    k.bseg_mode = bseg_mode;
    k.costed = costed;
    return k;
}

bgs_plan::RecKey records_key(const float *means2D, const float *conic_opacity, const float *colors,
                             const float *depths, int64_t n_records, int64_t n_colors) {
    bgs_plan::RecKey k;
    memset(&k, 0, sizeof k);
    k.means2D = means2D;
    k.conic_opacity = conic_opacity;
    k.colors = colors;
    k.depths = depths;
    k.n_records = n_records;
    k.n_colors = n_colors;
    return k;
}

// Gaussian-wise items can be queued in this mode (AUTO: some list may pass the threshold).
bool gauss_possible(const bgs_plan *p, int mode, int64_t num_entries) {
    return mode == BGS_MODE_GAUSSIAN || (mode == BGS_MODE_AUTO && p->desc.heavy_threshold != INT32_MAX &&
                                         (int64_t)p->desc.heavy_threshold < num_entries);
}

// Pixel groups of a Gaussian-wise item over a whole tile.
long long gw_groups(const bgs_plan *p, int tw, int th) {
    return ((long long)tw * th + p->desc.gw_pixels - 1) / p->desc.gw_pixels;
}

// Most later-segment items a list over num_entries entries is given: one per (segment after
// a tile's first, pixel group) when the tile ranges do not overlap, at most 2^24; beyond it
// no list is split.
long long gw_extra_cap(const bgs_plan *p, int tw, int th, int64_t num_entries) {
    const long long L = p->desc.gw_segment;
    return std::min<long long>(gw_groups(p, tw, th) * (num_entries / L + 1), 1ll << 24);
}

// mode: the render mode; AUTO with a threshold no list can exceed queues every tile
// pixel-wise and builds the same list as PIXEL (so a backward can reuse it).  bseg_mode >= 0
// (with mode PIXEL, for a backward): the render mode of the last forward on these arrays,
// whose split Gaussian-wise tiles get their pixel-wise items once per segment.
int build_worklist(bgs_plan *p, const uint32_t *ranges, const bgs::ViewTable &vt, int tw, int th, int mode,
                   int64_t num_entries, cudaStream_t s, int bseg_mode = -1, const uint32_t *cost = nullptr) {
    if (mode == BGS_MODE_AUTO && (p->desc.heavy_threshold == INT32_MAX ||
                                  (int64_t)p->desc.heavy_threshold >= num_entries))
        mode = BGS_MODE_PIXEL;
    const int T = vt.tile_base[vt.V];
    const int P = p->desc.gw_pixels;
    const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
    const int item_w = bgs::pix_item_w(p->desc.pixel_rows), item_h = bgs::pix_item_h(p->desc.pixel_rows);
    const long long per_tile = std::max<long long>(((tw + item_w - 1) / item_w) * ((th + item_h - 1) / item_h),
                                                   (tw * th + P - 1) / P);
    const bool gauss = gauss_possible(p, mode, num_entries);
    const long long extra_cap = gauss ? gw_extra_cap(p, tw, th, num_entries) : 0;
    // a segmented backward list: the tiles' pixel-wise items once per segment, at most as many
    // more segments as the forward's split (which fit its budget) had
    const long long pix_per_tile = ((tw + item_w - 1) / item_w) * ((th + item_h - 1) / item_h);
    const long long bseg_extra =
        bseg_mode >= 0 ? pix_per_tile * (gw_extra_cap(p, tw, th, num_entries) / gw_groups(p, tw, th) + 1) : 0;
    const long long max_items = (long long)T * per_tile + extra_cap + bseg_extra;
    if (max_items >= (1ll << 31)) return fail(BGS_ERR_INVALID, "too many work items (%lld)", max_items);
    BGS_TRY(ensure(p, p->tile_idx, sizeof(uint32_t) * T, s, "tile_idx"));
    BGS_TRY(ensure(p, p->items, sizeof(uint2) * max_items, s, "items"));
    if (gauss) {
        BGS_TRY(ensure(p, p->gw_exoff, sizeof(uint32_t) * T, s, "gw_exoff"));
        // summaries of the Gaussian-wise items: first segments of at most every tile, plus
        // the later segments
        const long long gw_items = (long long)T * gw_groups(p, tw, th) + extra_cap;
        BGS_TRY(ensure(p, p->gw_sum, (size_t)gw_items * P * 2 * sizeof(float4), s, "gw_sum"));
        BGS_TRY(ensure(p, p->gw_tile, sizeof(uint2) * T, s, "gw_tile"));
    }
    BGS_CUDA(bgs::launch_worklist_buckets(rg, T, vt, tw, th, mode, p->desc.heavy_threshold, p->desc.lpt_order, P,
                                          p->desc.pixel_rows, gauss ? p->desc.gw_segment : 0, extra_cap,
                                          (uint32_t *)p->tile_idx.p, gauss ? (uint32_t *)p->gw_exoff.p : nullptr,
                                          (uint2 *)p->items.p, (long long)(p->items.bytes / sizeof(uint2)), bseg_mode,
                                          gauss ? (uint2 *)p->gw_tile.p : nullptr, cost, p->ctrl, s),
             "build_worklist");
    p->host_launches += T > 0 ? 2 : 1;
    p->wl_key = worklist_key(p, ranges, vt, tw, th, mode, bseg_mode, cost ? 1 : 0);
    p->wl_valid = true;
    return BGS_OK;
}

bool valid_desc(const bgs_plan_desc *d) {
    return d->heavy_threshold >= 0 && (d->gw_pixels == 1 || d->gw_pixels == 2 || d->gw_pixels == 4 ||
                                       d->gw_pixels == 8 || d->gw_pixels == 16) &&
           d->queue_chunk >= 1 && d->queue_chunk <= 1024 && d->blocks_per_sm >= 0 && d->blocks_per_sm <= 64 &&
           (d->pixel_rows == 1 || d->pixel_rows == 2 || d->pixel_rows == 4 || d->pixel_rows == 8) &&
           d->select_period >= 1 && d->bin_block >= 0 && d->bin_block % 32 == 0 && d->gw_segment >= 256 &&
           d->gw_segment <= (1 << 30) && d->gw_segment % 256 == 0;
}

}  // namespace

extern "C" {

const char *bgs_last_error(void) { return g_last_error.c_str(); }

void bgs_plan_desc_default(bgs_plan_desc *d) {
    if (!d) return;
    d->heavy_threshold = 512;
    d->gw_pixels = 4;
    d->queue_chunk = 1;
    d->blocks_per_sm = 0;
    d->lpt_order = 1;
    d->device = -1;
    d->pixel_rows = 2;
    d->select_period = 1000;
    d->bin_block = 0;
    d->gw_segment = 2048;
}

int bgs_plan_create(const bgs_plan_desc *desc, bgs_plan **out) {
    if (!out) return fail(BGS_ERR_INVALID, "bgs_plan_create: out is NULL");
    *out = nullptr;
    bgs_plan_desc d;
    bgs_plan_desc_default(&d);
    if (desc) d = *desc;
    if (!valid_desc(&d)) return fail(BGS_ERR_INVALID, "bgs_plan_create: invalid tuning knobs");
    int dev = d.device;
    if (dev < 0) BGS_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    int ndev = 0;
    BGS_CUDA(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (dev >= ndev) return fail(BGS_ERR_INVALID, "device %d of %d", dev, ndev);
    DeviceGuard g(dev);
    bgs_plan *p = new bgs_plan();
    p->desc = d;
    p->desc.device = dev;
    p->device = dev;
    cudaError_t e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->ctrl, sizeof(bgs::DevCtrl));
    if (e == cudaSuccess) e = cudaMemset(p->ctrl, 0, sizeof(bgs::DevCtrl));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->sort_fork, cudaEventDisableTiming);
    for (int i = 0; i < kSortStreams && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&p->sort_stream[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->sort_join[i], cudaEventDisableTiming);
    }
    for (int v = 0; v < bgs::kMaxViews && e == cudaSuccess; ++v)
        e = cudaEventCreateWithFlags(&p->view_done[v], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        bgs_plan_destroy(p);
        return cuda_fail(e, "bgs_plan_create");
    }
    *out = p;
    return BGS_OK;
}

int bgs_plan_destroy(bgs_plan *p) {
    if (!p) return BGS_OK;
    DeviceGuard g(p->device);
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (int i = 0; i < kSortStreams; ++i) {
        if (p->sort_stream[i]) cudaStreamDestroy(p->sort_stream[i]);
        if (p->sort_join[i]) cudaEventDestroy(p->sort_join[i]);
        if (p->sort_tmp[i].p) cudaFree(p->sort_tmp[i].p);
    }
    if (p->sort_fork) cudaEventDestroy(p->sort_fork);
    for (cudaEvent_t e : p->view_done)
        if (e) cudaEventDestroy(e);
    for (auto &sl : p->bin_slot) {
        Buf *sb[] = {&sl.h,     &sl.total, &sl.start, &sl.rect,     &sl.mask,
                     &sl.credit, &sl.sat,  &sl.items, &sl.scan_tmp, &sl.stopped};
        for (Buf *b : sb)
            if (b->p) cudaFree(b->p);
    }
    Buf *bufs[] = {&p->gw_exoff, &p->gw_sum, &p->gw_tile, &p->tile_cost, &p->vkey_sorted, &p->touched, &p->touched_sorted, &p->dkey,
                   &p->dkey_sorted, &p->gidx, &p->order, &p->offsets,
                   &p->keys_in, &p->keys_out, &p->vals_in, &p->cub_tmp, &p->recs,
                   &p->tile_idx, &p->items, &p->warp_items,
                   &p->grad_acc};
    for (Buf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (p->ctrl) cudaFree(p->ctrl);
    for (auto &e : p->ev_fwd) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    for (auto &e : p->ev_bwd) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    delete p;
    return BGS_OK;
}

int bgs_plan_timing(bgs_plan *p, int enable) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_plan_timing: NULL plan");
    p->timing = enable != 0;
    return BGS_OK;
}

int bgs_plan_kernel_ms(bgs_plan *p, double *fwd_ms, int32_t *fwd_n, double *bwd_ms, int32_t *bwd_n) {
    if (!p || !fwd_ms || !fwd_n || !bwd_ms || !bwd_n) return fail(BGS_ERR_INVALID, "bgs_plan_kernel_ms: NULL argument");
    DeviceGuard g(p->device);
    double sums[2] = {0.0, 0.0};
    int counts[2] = {0, 0};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *lists[2] = {&p->ev_fwd, &p->ev_bwd};
    for (int k = 0; k < 2; ++k) {
        for (auto &e : *lists[k]) {
            BGS_CUDA(cudaEventSynchronize(e.second), "kernel timing sync");
            float ms = 0.f;
            BGS_CUDA(cudaEventElapsedTime(&ms, e.first, e.second), "kernel timing");
            sums[k] += ms;
            counts[k] += 1;
            p->ev_pool.push_back(e.first);
            p->ev_pool.push_back(e.second);
        }
        lists[k]->clear();
    }
    *fwd_ms = sums[0];
    *fwd_n = counts[0];
    *bwd_ms = sums[1];
    *bwd_n = counts[1];
    return BGS_OK;
}

int bgs_plan_set(bgs_plan *p, const bgs_plan_desc *d) {
    if (!p || !d) return fail(BGS_ERR_INVALID, "bgs_plan_set: NULL argument");
    if (!valid_desc(d)) return fail(BGS_ERR_INVALID, "bgs_plan_set: invalid tuning knobs");
    const int dev = p->device;
    p->desc = *d;
    p->desc.device = dev;
    return BGS_OK;
}

int bgs_plan_get(const bgs_plan *p, bgs_plan_desc *d) {
    if (!p || !d) return fail(BGS_ERR_INVALID, "bgs_plan_get: NULL argument");
    *d = p->desc;
    return BGS_OK;
}

int bgs_plan_num_sms(const bgs_plan *p) { return p ? p->num_sms : 0; }

size_t bgs_workspace_size(const bgs_plan *p, int64_t N, int64_t K, int64_t T, int64_t /*pixels*/) {
    if (!p || N < 0 || K < 0 || T < 0) return 0;
    const int P = p->desc.gw_pixels > 0 ? p->desc.gw_pixels : 1;
    size_t s = 0;
    s += 4 * N + 8 * N;                 // touched, offsets
    s += 8 * K * 2 + 4 * K;             // keys in/out, values in
    s += 48 * N * 2;                    // packed records, gradient accumulators
    s += 4 * T;                         // work-list bucket slots
    s += 8 * T * (size_t)std::max(8, (256 + P - 1) / P);  // work items (16x16 tiles)
    if ((int64_t)p->desc.heavy_threshold < K) {  // Gaussian-wise segments (AUTO)
        const size_t groups = (256 + P - 1) / P;
        const size_t extra = std::min<size_t>(groups * ((size_t)K / p->desc.gw_segment + 1), (size_t)1 << 24);
        s += 8 * extra + 4 * T + (groups * T + extra) * P * 32;
    }
    s += 64 << 20;                      // CUB temporaries (upper estimate)
    return s;
}

int bgs_plan_selector(const bgs_plan *p, int32_t *switched, int64_t *calls, int64_t *measurements,
                      double *last_balanced_ms, double *last_static_ms) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_plan_selector: NULL plan");
    if (switched) *switched = p->sel_switched ? 1 : 0;
    if (calls) *calls = p->sel_calls;
    if (measurements) *measurements = p->sel_measurements;
    if (last_balanced_ms) *last_balanced_ms = p->sel_last_balanced;
    if (last_static_ms) *last_static_ms = p->sel_last_static;
    return BGS_OK;
}

int bgs_plan_selector_restore(bgs_plan *p, int32_t switched, int64_t calls, int64_t measurements,
                              double last_balanced_ms, double last_static_ms) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_plan_selector_restore: NULL plan");
    if ((switched != 0 && switched != 1) || calls < 0 || measurements < 0 || measurements > calls ||
        !(last_balanced_ms >= 0.0) || !(last_static_ms >= 0.0))
        return fail(BGS_ERR_INVALID, "bgs_plan_selector_restore: inconsistent state");
    p->sel_switched = switched != 0;
    p->sel_calls = calls;
    p->sel_measurements = measurements;
    p->sel_last_balanced = last_balanced_ms;
    p->sel_last_static = last_static_ms;
    return BGS_OK;
}

int bgs_plan_inject_fault(bgs_plan *p, uint32_t which) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_plan_inject_fault: NULL plan");
    if (which & ~(unsigned)BGS_CHECK_QUEUE) return fail(BGS_ERR_INVALID, "bgs_plan_inject_fault: unsupported fault");
    p->inject |= which;
    return BGS_OK;
}

int bgs_plan_selector_reset(bgs_plan *p) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_plan_selector_reset: NULL plan");
    p->sel_switched = false;
    p->sel_calls = p->sel_measurements = 0;
    p->sel_last_balanced = p->sel_last_static = 0.0;
    return BGS_OK;
}

int bgs_plan_reserve(bgs_plan *p, int64_t N, int64_t K, int64_t T, int64_t pixels) {
    if (!p || N < 0 || K < 0 || T < 0 || pixels < 0) return fail(BGS_ERR_INVALID, "bgs_plan_reserve: bad sizes");
    DeviceGuard g(p->device);
    cudaStream_t s = 0;
    Buf *n4[] = {&p->touched, &p->touched_sorted, &p->dkey, &p->dkey_sorted, &p->gidx, &p->order};
    for (Buf *b : n4) BGS_TRY(ensure(p, *b, 4 * N, s, "per-Gaussian"));
    BGS_TRY(ensure(p, p->offsets, 8 * N, s, "offsets"));
    BGS_TRY(ensure(p, p->keys_in, 4 * K, s, "keys_in"));
    BGS_TRY(ensure(p, p->keys_out, 4 * K, s, "keys_out"));
    BGS_TRY(ensure(p, p->vals_in, 4 * K, s, "vals_in"));
    BGS_TRY(ensure(p, p->recs, sizeof(bgs::Rec) * N, s, "recs"));
    BGS_TRY(ensure(p, p->grad_acc, sizeof(bgs::Rec) * N, s, "grad_acc"));
    const int P = p->desc.gw_pixels;
    BGS_TRY(ensure(p, p->tile_idx, 4 * T, s, "per-tile"));
    // work items (16 x 16 tiles); with Gaussian-wise items possible in AUTO mode, the segment
    // items and summaries too
    const bool gauss = (int64_t)p->desc.heavy_threshold < K;
    const long long extra = gauss ? gw_extra_cap(p, 16, 16, K) : 0;
    BGS_TRY(ensure(p, p->items, 8 * (T * (size_t)std::max(8, (256 + P - 1) / P) + (size_t)extra), s, "items"));
    if (gauss) {
        BGS_TRY(ensure(p, p->gw_exoff, 4 * T, s, "gw_exoff"));
        BGS_TRY(ensure(p, p->gw_sum, ((size_t)T * gw_groups(p, 16, 16) + (size_t)extra) * P * 32, s, "gw_sum"));
    }
    // CUB temporaries: the largest of the depth sort, the N-scan, the tile sort and the tile scan
    size_t t[4] = {0, 0, 0, 0};
    const int64_t n1 = std::max<int64_t>(N, 1), k1 = std::max<int64_t>(K, 1);
    const int tt = (int)std::max<int64_t>(T, 1);
    uint32_t *u = nullptr;
    unsigned long long *ul = nullptr;
    BGS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, t[0], u, u, u, u, n1, 0, 32, s), "sort size");
    BGS_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, t[1], u, ul, n1, s), "scan size");
    BGS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, t[2], u, u, u, u, k1, 0, 32, s), "tile sort size");
    BGS_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, t[3], u, u, tt, s), "tile scan size");
    BGS_TRY(ensure(p, p->cub_tmp, *std::max_element(t, t + 4), s, "cub_tmp"));
    for (int i = 0; i < kSortStreams; ++i) BGS_TRY(ensure(p, p->sort_tmp[i], t[0], s, "sort_tmp"));
    return BGS_OK;
}

int bgs_check(bgs_plan *p, void *stream) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_check: NULL plan");
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int bits = 0;
    BGS_CUDA(cudaMemcpyAsync(&bits, &p->ctrl->check_bits, sizeof bits, cudaMemcpyDeviceToHost, s), "bgs_check copy");
    BGS_CUDA(cudaStreamSynchronize(s), "bgs_check sync");
    if (bits) {
        BGS_CUDA(cudaMemsetAsync(&p->ctrl->check_bits, 0, sizeof bits, s), "bgs_check clear");
        BGS_CUDA(cudaStreamSynchronize(s), "bgs_check sync");
        return fail(BGS_ERR_DEVICE_CHECK, "device check tripped: bits 0x%x (%s%s%s%s)", bits,
                    (bits & BGS_CHECK_INDEX) ? "index " : "", (bits & BGS_CHECK_RANGE) ? "range " : "",
                    (bits & BGS_CHECK_OVERFLOW) ? "overflow " : "", (bits & BGS_CHECK_QUEUE) ? "queue" : "");
    }
    return BGS_OK;
}

int bgs_plan_stats(bgs_plan *p, bgs_stats *out, void *stream) {
    if (!p || !out) return fail(BGS_ERR_INVALID, "bgs_plan_stats: NULL argument");
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    bgs::DevCtrl c;
    BGS_CUDA(cudaMemcpyAsync(&c, p->ctrl, offsetof(bgs::DevCtrl, wl_cnt), cudaMemcpyDeviceToHost, s), "stats copy");
    BGS_CUDA(cudaStreamSynchronize(s), "stats sync");
    out->eval_pairs = c.eval_pairs;
    out->contrib_pairs = c.contrib_pairs;
    out->items = c.items_done;
    out->check_bits = c.check_bits;
    out->last_num_items = c.num_items;
    out->host_launches = p->host_launches;
    return BGS_OK;
}

int bgs_plan_reset_stats(bgs_plan *p, void *stream) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_plan_reset_stats: NULL plan");
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    BGS_CUDA(cudaMemsetAsync(&p->ctrl->eval_pairs, 0, 3 * sizeof(unsigned long long), s), "reset stats");
    return BGS_OK;
}

int bgs_preprocess(bgs_plan *p, int64_t N, const float *means3D, const float *log_scales, const float *quats,
                   const float *opacities, const bgs_camera *cam, int32_t tw, int32_t th, float *means2D,
                   float *conic_opacity, float *depths, int32_t *radii, uint32_t *tiles_touched, void *stream) {
    if (!p || !cam) return fail(BGS_ERR_INVALID, "bgs_preprocess: NULL plan or camera");
    if (N < 0 || N >= (1ll << 32)) return fail(BGS_ERR_INVALID, "bgs_preprocess: N=%lld out of range", (long long)N);
    if (N > 0 && (!means3D || !log_scales || !quats || !opacities || !means2D || !conic_opacity || !depths || !radii ||
                  !tiles_touched))
        return fail(BGS_ERR_INVALID, "bgs_preprocess: NULL array");
    BGS_TRY(check_image(cam->width, cam->height));
    BGS_TRY(check_tile(tw, th, false));
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return fail(BGS_ERR_INVALID, "bgs_preprocess: focal lengths must be > 0");
    DeviceGuard g(p->device);
    BGS_CUDA(bgs::launch_preprocess(N, 1, means3D, log_scales, quats, opacities, cam, tw, th, means2D, conic_opacity,
                                    depths, radii, tiles_touched, (cudaStream_t)stream),
             "preprocess");
    if (N > 0) p->host_launches += 1;
    return BGS_OK;
}

int bgs_preprocess_backward(bgs_plan *p, int64_t N, const float *means3D, const float *log_scales,
                            const float *quats, const bgs_camera *cam, const int32_t *radii, const float *dL_dmeans2D,
                            const float *dL_dconic, const float *dL_ddepths, float *dL_dmeans3D,
                            float *dL_dlog_scales, float *dL_dquats, void *stream) {
    if (!p || !cam) return fail(BGS_ERR_INVALID, "bgs_preprocess_backward: NULL plan or camera");
    if (N < 0 || N >= (1ll << 32)) return fail(BGS_ERR_INVALID, "bgs_preprocess_backward: N out of range");
    if (N > 0 && (!means3D || !log_scales || !quats || !radii || !dL_dmeans2D || !dL_dconic || !dL_dmeans3D ||
                  !dL_dlog_scales || !dL_dquats))
        return fail(BGS_ERR_INVALID, "bgs_preprocess_backward: NULL array");
    if (((uintptr_t)dL_dmeans2D) & 7) return fail(BGS_ERR_INVALID, "bgs_preprocess_backward: dL_dmeans2D alignment");
    BGS_TRY(check_image(cam->width, cam->height));
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f))
        return fail(BGS_ERR_INVALID, "bgs_preprocess_backward: focal lengths must be > 0");
    DeviceGuard g(p->device);
    BGS_CUDA(bgs::launch_preprocess_backward(N, 1, means3D, log_scales, quats, cam, radii, dL_dmeans2D, dL_dconic,
                                             dL_ddepths, dL_dmeans3D, dL_dlog_scales, dL_dquats, (cudaStream_t)stream),
             "preprocess_backward");
    if (N > 0) p->host_launches += 1;
    return BGS_OK;
}

}  // extern "C"

namespace {

// Counting-sort binning of one view (binning.cu), in two halves on stream s with the buffer
// set `slot`.  order holds the view's records in depth order (global record indices);
// ranges points at the view's first tile.  bin_view_a counts (tile histogram, masks,
// credits, truncated totals, tile starts) and stores the view's entry count in
// ctrl->view_k[v]; bin_view_b writes the ranges and the lists from the view's first
// point_list slot (the counts of views 0..v-1, which must be stored by then) on.  No host
// synchronisation; bgs::launch_bin_finish then totals the call's views.
// depth-order fractions 1 / d at which truncated binning starts its second and third passes
constexpr long long kBinPassDiv[2] = {8, 2};

struct BinView {
    int tiles_x, tiles_y;
    long long T, G, B, W32, nC;
    bool trunc;
};

int bin_view_a(bgs_plan *p, int slot, int v, long long n, const uint32_t *order, const float *means2D,
               const int32_t *radii, const float *conic_opacity, int W, int H, int tw, int th, BinView &bv,
               cudaStream_t s) {
    bgs_plan::BinSlot &sl = p->bin_slot[slot];
    bv.tiles_x = (W + tw - 1) / tw;
    bv.tiles_y = (H + th - 1) / th;
    const long long T = bv.T = (long long)bv.tiles_x * bv.tiles_y;
    const size_t smem = bgs::bin_count_smem(bv.tiles_x, bv.tiles_y);
    if (smem > (size_t)p->smem_optin) return fail(BGS_ERR_INVALID, "tile grid too large for counting-sort binning");
    // G: a multiple of 32.  Automatic: at least 2048, about 4 counting blocks per SM (fewer,
    // longer blocks keep the scatter's per-(block, tile group) overhead down), and large
    // enough that B T stays below 2^24
    long long G = p->desc.bin_block;
    if (G <= 0) {
        G = std::max<long long>(2048, (n + 4ll * p->num_sms - 1) / (4ll * std::max(1, p->num_sms)));
        G = std::max<long long>(G, (n * T + (1ll << 24) - 1) >> 24);
    }
    G = bv.G = (G + 31) & ~31ll;
    const long long B = bv.B = std::max<long long>(1, (n + G - 1) / G);
    const long long W32 = bv.W32 = ((G + 511) / 512) * 16;  // mask words per (block, tile group)
    const long long nC = bv.nC = bgs::bin_mask_groups(bv.tiles_x, bv.tiles_y);
    if (B * T >= (1ll << 31) || B * nC * W32 >= (1ll << 40)) return fail(BGS_ERR_INVALID, "tile histogram too large");
    BGS_TRY(ensure(p, sl.h, sizeof(uint32_t) * B * T, s, "bin_h"));
    BGS_TRY(ensure(p, sl.total, sizeof(uint32_t) * T, s, "bin_total"));
    BGS_TRY(ensure(p, sl.start, sizeof(uint32_t) * T, s, "bin_start"));
    BGS_TRY(ensure(p, sl.rect, sizeof(uint4) * n, s, "bin_rect"));
    BGS_TRY(ensure(p, sl.mask, sizeof(uint32_t) * B * nC * W32, s, "bin_mask"));
    uint32_t *Hm = (uint32_t *)sl.h.p, *tot = (uint32_t *)sl.total.p, *start = (uint32_t *)sl.start.p;
    uint4 *rect = (uint4 *)sl.rect.p;
    if (smem > 48 * 1024) BGS_CUDA(bgs::setup_bin_kernels(bv.tiles_x, bv.tiles_y), "bin smem attribute");
    // list truncation: per-block credits toward the certificate that a tile's pixels have all
    // stopped (needs the conics, and the credit counters of one block in shared memory)
    bv.trunc = conic_opacity && bgs::bin_credit_smem(bv.tiles_x, bv.tiles_y) <= (size_t)p->smem_optin;
    uint16_t *credit = nullptr;
    uint32_t *bsat = nullptr;
    if (bv.trunc) {
        BGS_TRY(ensure(p, sl.credit, sizeof(uint16_t) * B * T, s, "bin_credit"));
        BGS_TRY(ensure(p, sl.sat, sizeof(uint32_t) * T, s, "bin_sat"));
        credit = (uint16_t *)sl.credit.p;
        bsat = (uint32_t *)sl.sat.p;
    }
    // With truncation, in passes over the depth order ([0, B / 8), [B / 8, B / 2), [B / 2, B)):
    // a later pass leaves out the Gaussians all of whose tiles the earlier passes' credits
    // already certify as stopped (their entries lie past the ends of all their lists, so the
    // lists are the same)
    long long bounds[4] = {0, B, B, B};
    int passes = 1;
    if (bv.trunc && B >= 32) {
        bounds[1] = B / kBinPassDiv[0];
        bounds[2] = B / kBinPassDiv[1];
        bounds[3] = B;
        passes = 3;
    }
    uint32_t *masks = (uint32_t *)sl.mask.p;
    int *P = nullptr;
    if (passes > 1) {
        BGS_TRY(ensure(p, sl.stopped, sizeof(int) * ((bv.tiles_x + 1) * (bv.tiles_y + 1) + bv.T), s, "bin_stopped"));
        P = (int *)sl.stopped.p;
    }
    for (int k = 0; k < passes; ++k) {
        const int lo = (int)bounds[k], hi = (int)bounds[k + 1];
        if (k > 0) BGS_CUDA(bgs::launch_bin_stopped(lo, bv.tiles_x, bv.tiles_y, credit, P, s), "bin_stopped");
        BGS_CUDA(bgs::launch_bin_count(n, (int)G, lo, hi, order, means2D, radii, W, H, tw, th, Hm, rect, masks,
                                       (int)W32, k > 0 ? P : nullptr, s),
                 "bin_count");
        if (bv.trunc)
            BGS_CUDA(bgs::launch_bin_credit(n, (int)G, lo, hi, rect, means2D, conic_opacity, W, H, tw, th, credit, s),
                     "bin_credit");
        p->host_launches += k > 0 ? 4 : 1;
    }
    if (bv.trunc) p->host_launches += 1;
    BGS_CUDA(bgs::launch_bin_colscan((int)B, (int)T, Hm, credit, tot, bsat, s), "bin_colscan");
    size_t tmp = 0;
    BGS_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp, tot, start, (int)T, s), "tile scan (size)");
    BGS_TRY(ensure(p, sl.scan_tmp, tmp, s, "scan_tmp"));
    tmp = sl.scan_tmp.bytes;
    BGS_CUDA(cub::DeviceScan::ExclusiveSum(sl.scan_tmp.p, tmp, tot, start, (int)T, s), "tile scan");
    BGS_CUDA(bgs::launch_bin_view_total((int)T, tot, v, p->ctrl, s), "bin_view_total");
    p->host_launches += 3;  // count, colscan, view total
    return BGS_OK;
}

int bin_view_b(bgs_plan *p, int slot, int v, long long n, const BinView &bv, int W, int H, int tw, int th,
               uint32_t *point_list, long long capacity, uint32_t *ranges, cudaStream_t s) {
    bgs_plan::BinSlot &sl = p->bin_slot[slot];
    const uint32_t *Hm = (const uint32_t *)sl.h.p, *tot = (const uint32_t *)sl.total.p;
    const uint32_t *start = (const uint32_t *)sl.start.p;
    BGS_CUDA(bgs::launch_bin_ranges((int)bv.T, start, tot, reinterpret_cast<uint2 *>(ranges), v, p->ctrl, s),
             "bin_ranges");
    BGS_TRY(ensure(p, sl.items, sizeof(uint32_t) * (bv.nC + 1), s, "bin_items"));
    BGS_CUDA(bgs::launch_bin_scatter(n, (int)bv.G, (int)bv.B, (int)bv.W32, (const uint4 *)sl.rect.p, W, H, tw, th, Hm,
                                     start, (const uint32_t *)sl.mask.p, point_list, capacity,
                                     bv.trunc ? (const uint32_t *)sl.sat.p : nullptr, (uint32_t *)sl.items.p,
                                     p->num_sms, v, p->ctrl, s),
             "bin_scatter");
    p->host_launches += bv.trunc ? 3 : 2;  // ranges, (work list), scatter
    return BGS_OK;
}

template <typename KeyT>
int sort_and_range(bgs_plan *p, long long N, const float *means2D, const int32_t *radii, int W, int H, int tw,
                   int th, long long K, long long T, uint32_t *point_list, uint32_t *ranges, cudaStream_t s) {
    const uint32_t *order = (const uint32_t *)p->order.p;
    const unsigned long long *off = (const unsigned long long *)p->offsets.p;
    BGS_TRY(ensure(p, p->keys_in, sizeof(KeyT) * K, s, "keys_in"));
    BGS_TRY(ensure(p, p->keys_out, sizeof(KeyT) * K, s, "keys_out"));
    BGS_TRY(ensure(p, p->vals_in, 4 * K, s, "vals_in"));
    KeyT *kin = (KeyT *)p->keys_in.p, *kout = (KeyT *)p->keys_out.p;
    uint32_t *vin = (uint32_t *)p->vals_in.p;
    BGS_CUDA(bgs::launch_duplicate<KeyT>(N, order, means2D, radii, off, W, H, tw, th, kin, vin, K, s), "duplicate");
    // tile ids are < T: sort on the bits of T - 1 only (never more than the key type holds)
    const int end_bit = bits_for(T - 1);
    if (end_bit > (int)(8 * sizeof(KeyT))) return fail(BGS_ERR_INVALID, "tile id does not fit the sort key");
    size_t tmp = 0;
    BGS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, kin, kout, vin, point_list, (int64_t)K, 0, end_bit, s),
             "tile sort (size)");
    BGS_TRY(ensure(p, p->cub_tmp, tmp, s, "cub_tmp"));
    tmp = p->cub_tmp.bytes;
    BGS_CUDA(cub::DeviceRadixSort::SortPairs(p->cub_tmp.p, tmp, kin, kout, vin, point_list, (int64_t)K, 0, end_bit, s),
             "tile sort");
    BGS_CUDA(bgs::launch_ranges<KeyT>(kout, K, reinterpret_cast<uint2 *>(ranges), s), "ranges");
    p->host_launches += 2;  // duplicate, ranges
    return BGS_OK;
}

}  // namespace

extern "C" {

int bgs_bin_and_sort(bgs_plan *p, int64_t N, const float *means2D, const int32_t *radii, const float *depths,
                     const float *conic_opacity, int32_t W, int32_t H, int32_t tw, int32_t th, uint32_t *point_list,
                     int64_t capacity, uint32_t *ranges, int64_t *num_rendered, int64_t *needed, void *stream) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_bin_and_sort: NULL plan");
    if (N < 0 || N >= (1ll << 32)) return fail(BGS_ERR_INVALID, "bgs_bin_and_sort: N out of range");
    if (capacity < 0) return fail(BGS_ERR_INVALID, "bgs_bin_and_sort: negative capacity");
    BGS_TRY(check_image(W, H));
    BGS_TRY(check_tile(tw, th, false));
    if (!ranges || (N > 0 && (!means2D || !radii || !depths)) || (capacity > 0 && !point_list))
        return fail(BGS_ERR_INVALID, "bgs_bin_and_sort: NULL array");
    if (((uintptr_t)conic_opacity) & 15) return fail(BGS_ERR_INVALID, "bgs_bin_and_sort: conic_opacity alignment");
    const int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    const long long T = (long long)tiles_x * tiles_y;
    if (T >= (1ll << 31)) return fail(BGS_ERR_INVALID, "bgs_bin_and_sort: too many tiles");
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    BGS_CUDA(cudaMemsetAsync(ranges, 0, sizeof(uint2) * T, s), "clear ranges");
    if (num_rendered) *num_rendered = 0;
    if (needed) *needed = 0;
    if (N == 0) return BGS_OK;
    // (1) entry counts and the depth order of the Gaussians (stable: ties keep index order)
    BGS_TRY(ensure(p, p->touched, 4 * N, s, "touched"));
    BGS_TRY(ensure(p, p->touched_sorted, 4 * N, s, "touched_sorted"));
    BGS_TRY(ensure(p, p->dkey, 4 * N, s, "dkey"));
    BGS_TRY(ensure(p, p->dkey_sorted, 4 * N, s, "dkey_sorted"));
    BGS_TRY(ensure(p, p->gidx, 4 * N, s, "gidx"));
    BGS_TRY(ensure(p, p->order, 4 * N, s, "order"));
    BGS_TRY(ensure(p, p->offsets, 8 * N, s, "offsets"));
    uint32_t *touched = (uint32_t *)p->touched.p, *tsorted = (uint32_t *)p->touched_sorted.p;
    uint32_t *dkey = (uint32_t *)p->dkey.p, *dkey2 = (uint32_t *)p->dkey_sorted.p;
    uint32_t *gidx = (uint32_t *)p->gidx.p, *order = (uint32_t *)p->order.p;
    unsigned long long *off = (unsigned long long *)p->offsets.p;
    BGS_CUDA(bgs::launch_touched(N, means2D, radii, depths, W, H, tw, th, touched, dkey, gidx, s), "touched");
    size_t tmp = 0;
    BGS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, dkey, dkey2, gidx, order, (int64_t)N, 0, 32, s),
             "depth sort (size)");
    BGS_TRY(ensure(p, p->cub_tmp, tmp, s, "cub_tmp"));
    tmp = p->cub_tmp.bytes;
    BGS_CUDA(cub::DeviceRadixSort::SortPairs(p->cub_tmp.p, tmp, dkey, dkey2, gidx, order, (int64_t)N, 0, 32, s),
             "depth sort");
    // (2) counting sort over tile rectangles when the per-tile counters fit in shared memory
    if (bgs::bin_count_smem(tiles_x, tiles_y) <= (size_t)p->smem_optin) {
        BinView bv;
        BGS_TRY(bin_view_a(p, 0, 0, N, order, means2D, radii, conic_opacity, W, H, tw, th, bv, s));
        BGS_TRY(bin_view_b(p, 0, 0, N, bv, W, H, tw, th, point_list, capacity, ranges, s));
        BGS_CUDA(bgs::launch_bin_finish(1, 1ll << 62, p->ctrl, s), "bin_finish");  // the host checks K
        unsigned long long K = 0;
        BGS_CUDA(cudaMemcpyAsync(&K, &p->ctrl->num_entries, sizeof K, cudaMemcpyDeviceToHost, s), "read K");
        BGS_CUDA(cudaStreamSynchronize(s), "sync K");
        if (needed) *needed = (int64_t)K;
        if ((long long)K > capacity || (long long)K > BGS_MAX_ENTRIES)
            return fail(BGS_ERR_CAPACITY, "bgs_bin_and_sort: %llu entries exceed capacity %lld (or BGS_MAX_ENTRIES)",
                        K, (long long)capacity);
        if (num_rendered) *num_rendered = (int64_t)K;
        return BGS_OK;
    }
    // (2') otherwise: entry offsets in depth order, emit, stable radix sort on the tile id
    BGS_CUDA(bgs::launch_gather_u32(N, touched, order, tsorted, s), "gather counts");
    tmp = 0;
    BGS_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp, tsorted, off, (int64_t)N, s), "scan (size)");
    BGS_TRY(ensure(p, p->cub_tmp, tmp, s, "cub_tmp"));
    tmp = p->cub_tmp.bytes;
    BGS_CUDA(cub::DeviceScan::ExclusiveSum(p->cub_tmp.p, tmp, tsorted, off, (int64_t)N, s), "scan");
    BGS_CUDA(bgs::launch_count_total(N, tsorted, off, p->ctrl, s), "count_total");
    p->host_launches += 3;  // touched, gather, count_total
    unsigned long long K = 0;
    BGS_CUDA(cudaMemcpyAsync(&K, &p->ctrl->num_entries, sizeof K, cudaMemcpyDeviceToHost, s), "read K");
    BGS_CUDA(cudaStreamSynchronize(s), "sync K");
    if (needed) *needed = (int64_t)K;
    if ((long long)K > capacity)
        return fail(BGS_ERR_CAPACITY, "bgs_bin_and_sort: %llu entries exceed capacity %lld", K, (long long)capacity);
    if ((long long)K > BGS_MAX_ENTRIES)
        return fail(BGS_ERR_CAPACITY, "bgs_bin_and_sort: %llu entries exceed BGS_MAX_ENTRIES", K);
    if (num_rendered) *num_rendered = (int64_t)K;
    if (K == 0) return BGS_OK;
    // emit entries in depth order and group them per tile with a stable sort on the tile id
    if (T <= 65536)
        return sort_and_range<uint16_t>(p, N, means2D, radii, W, H, tw, th, (long long)K, T, point_list, ranges, s);
    return sort_and_range<uint32_t>(p, N, means2D, radii, W, H, tw, th, (long long)K, T, point_list, ranges, s);
}

}  // extern "C"

namespace {

int check_render_arrays(int64_t N, const float *means2D, const float *conic_opacity, const float *colors,
                        const float *depths, const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges,
                        int tw, int th, const float *bg, int mode, const char *who) {
    if (N < 0 || N >= (1ll << 32)) return fail(BGS_ERR_INVALID, "%s: N out of range", who);
    if (num_entries < 0 || num_entries > BGS_MAX_ENTRIES)
        return fail(BGS_ERR_INVALID, "%s: num_entries out of range (<= BGS_MAX_ENTRIES)", who);
    if (mode < BGS_MODE_AUTO || mode > BGS_MODE_SELECT) return fail(BGS_ERR_INVALID, "%s: unknown mode %d", who, mode);
    BGS_TRY(check_tile(tw, th, mode != BGS_MODE_STATIC));
    if (!ranges || !bg || (num_entries > 0 && !point_list) ||
        (N > 0 && (!means2D || !conic_opacity || !colors || !depths)))
        return fail(BGS_ERR_INVALID, "%s: NULL array", who);
    if ((((uintptr_t)means2D) & 7) || (((uintptr_t)conic_opacity) & 15) || (((uintptr_t)ranges) & 7))
        return fail(BGS_ERR_INVALID, "%s: means2D must be 8-byte, conic_opacity 16-byte aligned", who);
    return BGS_OK;
}

// View table of V views of the given sizes (tile grids laid out one after the other).
int make_view_table(int V, const int *W, const int *H, int tw, int th, bgs::ViewTable &vt) {
    if (V < 1 || V > bgs::kMaxViews) return fail(BGS_ERR_INVALID, "number of views %d outside [1, %d]", V, bgs::kMaxViews);
    memset(&vt, 0, sizeof vt);
    vt.V = V;
    long long base = 0;
    for (int v = 0; v < V; ++v) {
        BGS_TRY(check_image(W[v], H[v]));
        vt.W[v] = W[v];
        vt.H[v] = H[v];
        vt.tiles_x[v] = (W[v] + tw - 1) / tw;
        vt.tiles_y[v] = (H[v] + th - 1) / th;
        vt.tile_base[v] = (int)base;
        base += (long long)vt.tiles_x[v] * vt.tiles_y[v];
        if (base >= (1ll << 30)) return fail(BGS_ERR_INVALID, "too many tiles over the views");
    }
    vt.tile_base[V] = (int)base;
    return BGS_OK;
}

// Forward over the views of vt; records are n_records = V * n_per_view, colours n_colors rows.
int render_forward_impl(bgs_plan *p, const bgs::ViewTable &vt, const bgs::ViewOut &io, int64_t n_records,
                        int64_t n_colors, const float *means2D, const float *conic_opacity, const float *colors,
                        const float *depths, const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges,
                        int tw, int th, const float *bg, int mode, cudaStream_t s) {
    bgs::FwdArgs a;
    memset(&a, 0, sizeof a);
    a.means2D = means2D;
    a.conic_opacity = conic_opacity;
    a.colors = colors;
    a.depths = depths;
    a.point_list = point_list;
    a.ranges = reinterpret_cast<const uint2 *>(ranges);
    a.N = n_records;
    a.num_entries = num_entries;
    a.tile_w = tw;
    a.tile_h = th;
    a.num_tiles = vt.tile_base[vt.V];
    a.bg[0] = bg[0];
    a.bg[1] = bg[1];
    a.bg[2] = bg[2];
    a.vt = vt;
    a.io = io;
    a.ctrl = p->ctrl;
    a.gw_pixels = p->desc.gw_pixels;
    a.pixel_rows = p->desc.pixel_rows;
    a.chunk = p->desc.queue_chunk;
    if (mode == BGS_MODE_STATIC) {
        if (vt.V != 1) return fail(BGS_ERR_INVALID, "the static kernel renders one view");
        KernelTimer kt(p, s, &p->ev_fwd);
        BGS_CUDA(bgs::launch_forward_static(a, s), "forward_static");
        kt.stop();
        p->host_launches += 1;
        p->cost_valid = false;  // no per-tile cost gathered
        return BGS_OK;
    }
    BGS_TRY(ensure(p, p->recs, sizeof(bgs::Rec) * std::max<int64_t>(n_records, 1), s, "recs"));
    BGS_CUDA(bgs::launch_pack(n_records, means2D, conic_opacity, colors, n_colors, depths, (bgs::Rec *)p->recs.p, s),
             "pack");
    p->host_launches += 1;
    p->rec_key = records_key(means2D, conic_opacity, colors, depths, n_records, n_colors);
    p->rec_valid = true;
    a.recs = (const bgs::Rec *)p->recs.p;
    BGS_TRY(build_worklist(p, ranges, vt, tw, th, mode, num_entries, s));
    a.items = (const uint2 *)p->items.p;
    const int threads = bgs::forward_balanced_block_threads();
    const int grid_g = grid_for(p, bgs::forward_gauss_kernel(a.gw_pixels), threads);
    const int grid_p = grid_for(p, bgs::forward_pixel_kernel(a.pixel_rows), threads);
    // AUTO with a threshold no list can exceed queues no Gaussian-wise item
    const bool gauss = gauss_possible(p, mode, num_entries);
    a.gw_exoff = gauss ? (const uint32_t *)p->gw_exoff.p : nullptr;
    a.gw_sum = gauss ? (float4 *)p->gw_sum.p : nullptr;
    {  // the backward's per-tile cost, gathered by the forward kernels
        const int T = vt.tile_base[vt.V];
        BGS_TRY(ensure(p, p->tile_cost, sizeof(uint32_t) * std::max(T, 1), s, "tile_cost"));
        BGS_CUDA(cudaMemsetAsync(p->tile_cost.p, 0, sizeof(uint32_t) * std::max(T, 1), s), "clear tile_cost");
        a.tile_cost = (unsigned int *)p->tile_cost.p;
        p->cost_key = worklist_key(p, ranges, vt, tw, th, BGS_MODE_PIXEL);
        p->cost_valid = true;
    }
    a.pass_blocks = (gauss ? grid_g : 0) + (mode != BGS_MODE_GAUSSIAN ? grid_p : 0);
    BGS_TRY(inject_pending_fault(p, s));
    KernelTimer kt(p, s, &p->ev_fwd);
    if (gauss) BGS_CUDA(bgs::launch_forward_gauss(a, grid_g, s), "forward_gauss");
    if (mode != BGS_MODE_GAUSSIAN) BGS_CUDA(bgs::launch_forward_pixel(a, grid_p, gauss, s), "forward_pixel");
    if (gauss) BGS_CUDA(bgs::launch_forward_gw_merge(a, grid_for(p, bgs::forward_gw_merge_kernel(a.gw_pixels), threads), s),
                        "forward_gw_merge");
    p->gw_fwd_valid = gauss;
    p->gw_fwd_key = p->wl_key;
    kt.stop();
    p->host_launches += (gauss && mode != BGS_MODE_GAUSSIAN) ? 3 : (gauss ? 2 : 1);
    return BGS_OK;
}

int render_backward_impl(bgs_plan *p, const bgs::ViewTable &vt, const bgs::ViewGradIn &gi, int64_t n_records,
                         int64_t n_colors, const float *means2D, const float *conic_opacity, const float *colors,
                         const float *depths, const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges,
                         int tw, int th, const float *bg, int mode, float *dL_dmeans2D, float *dL_dconic,
                         float *dL_dopacity, float *dL_dcolors, float *dL_ddepths, cudaStream_t s) {
    if (n_records == 0) return BGS_OK;
    BGS_TRY(ensure(p, p->grad_acc, sizeof(bgs::Rec) * n_records, s, "grad_acc"));
    BGS_CUDA(cudaMemsetAsync(p->grad_acc.p, 0, sizeof(bgs::Rec) * n_records, s), "clear grad_acc");
    bgs::BwdArgs a;
    memset(&a, 0, sizeof a);
    a.bseg_mode = -1;
    a.means2D = means2D;
    a.conic_opacity = conic_opacity;
    a.colors = colors;
    a.depths = depths;
    a.point_list = point_list;
    a.ranges = reinterpret_cast<const uint2 *>(ranges);
    a.N = n_records;
    a.num_entries = num_entries;
    a.tile_w = tw;
    a.tile_h = th;
    a.num_tiles = vt.tile_base[vt.V];
    a.bg[0] = bg[0];
    a.bg[1] = bg[1];
    a.bg[2] = bg[2];
    a.vt = vt;
    a.gi = gi;
    a.grad_acc = (float *)p->grad_acc.p;
    a.ctrl = p->ctrl;
    a.pixel_rows = p->desc.pixel_rows;
    a.chunk = p->desc.queue_chunk;
    int n_warps = 0;  // warps of the persistent pass whose item counts finalize checks
    if (mode == BGS_MODE_STATIC) {
        if (vt.V != 1) return fail(BGS_ERR_INVALID, "the static kernel renders one view");
        KernelTimer kt(p, s, &p->ev_bwd);
        BGS_CUDA(bgs::launch_backward_static(a, s), "backward_static");
        kt.stop();
        p->host_launches += 1;
    } else {
        // the packed records and the pixel-wise work list of the last forward, when it ran on
        // these arrays (the backward needs the forward's inputs unchanged in any case)
        const bgs_plan::RecKey rk = records_key(means2D, conic_opacity, colors, depths, n_records, n_colors);
        if (!(p->rec_valid && memcmp(&rk, &p->rec_key, sizeof rk) == 0)) {
            BGS_TRY(ensure(p, p->recs, sizeof(bgs::Rec) * n_records, s, "recs"));
            BGS_CUDA(bgs::launch_pack(n_records, means2D, conic_opacity, colors, n_colors, depths,
                                      (bgs::Rec *)p->recs.p, s),
                     "pack");
            p->host_launches += 1;
            p->rec_key = rk;
            p->rec_valid = true;
        }
        a.recs = (const bgs::Rec *)p->recs.p;
        // the last forward on these arrays split Gaussian-wise lists: walk those tiles per segment
        const bgs_plan::WlKey fk = worklist_key(p, ranges, vt, tw, th, mode);
        const int bseg = (p->gw_fwd_valid && memcmp(&fk, &p->gw_fwd_key, sizeof fk) == 0) ? mode : -1;
        a.bseg_mode = bseg;
        a.heavy_threshold = p->desc.heavy_threshold;
        a.gw_pixels = p->desc.gw_pixels;
        a.gw_tile = bseg >= 0 ? (const uint2 *)p->gw_tile.p : nullptr;
        a.gw_sum = bseg >= 0 ? (const bgs::GwSum *)p->gw_sum.p : nullptr;
        // heaviest first by what the backward walks: each tile's largest n_contrib, which the
        // last forward on these tiles gathered (its list length overstates the walk where
        // pixels stop early); the order changes no result
        const bgs_plan::WlKey ck = worklist_key(p, ranges, vt, tw, th, BGS_MODE_PIXEL);
        const bool costed = p->cost_valid && memcmp(&ck, &p->cost_key, sizeof ck) == 0;
        const bgs_plan::WlKey wk = worklist_key(p, ranges, vt, tw, th, BGS_MODE_PIXEL, bseg, costed ? 1 : 0);
        if (p->wl_valid && memcmp(&wk, &p->wl_key, sizeof wk) == 0) {
            // same list: rewind its queue
            BGS_CUDA(bgs::launch_rewind_queue(p->ctrl, s), "rewind queue");
            p->host_launches += 1;
        } else {
            BGS_TRY(build_worklist(p, ranges, vt, tw, th, BGS_MODE_PIXEL, num_entries, s, bseg,
                                   costed ? (const uint32_t *)p->tile_cost.p : nullptr));
        }
        a.items = (const uint2 *)p->items.p;
        const int grid = grid_for(p, bgs::backward_balanced_kernel(a), bgs::backward_balanced_block_threads());
        n_warps = grid * (bgs::backward_balanced_block_threads() / 32);
        BGS_TRY(ensure(p, p->warp_items, sizeof(unsigned int) * n_warps, s, "warp_items"));
        a.warp_items = (unsigned int *)p->warp_items.p;
        BGS_TRY(inject_pending_fault(p, s));
        KernelTimer kt(p, s, &p->ev_bwd);
        BGS_CUDA(bgs::launch_backward_balanced(a, grid, s), "backward_balanced");
        kt.stop();
        p->host_launches += 1;  // kernel
    }
    BGS_CUDA(bgs::launch_grad_finalize(n_records, n_colors, (const float4 *)p->grad_acc.p, conic_opacity, dL_dmeans2D,
                                       dL_dconic, dL_dopacity, dL_dcolors, dL_ddepths,
                                       (const unsigned int *)p->warp_items.p, n_warps, p->ctrl, s),
             "grad_finalize");
    p->host_launches += 1;  // finalize
    return BGS_OK;
}

}  // namespace

extern "C" {

int bgs_render_forward(bgs_plan *p, int64_t N, const float *means2D, const float *conic_opacity, const float *colors,
                       const float *depths, const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges,
                       int32_t W, int32_t H, int32_t tw, int32_t th, const float *bg, int32_t mode, float *out_color,
                       float *out_depth, float *out_alpha, float *final_T, int32_t *n_contrib, int32_t *n_eval,
                       void *stream) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_render_forward: NULL plan");
    BGS_TRY(check_render_arrays(N, means2D, conic_opacity, colors, depths, point_list, num_entries, ranges, tw, th, bg,
                                mode, "bgs_render_forward"));
    if (!out_color || !out_depth || !out_alpha || !final_T || !n_contrib)
        return fail(BGS_ERR_INVALID, "bgs_render_forward: NULL output");
    bgs::ViewTable vt;
    BGS_TRY(make_view_table(1, &W, &H, tw, th, vt));
    bgs::ViewOut io;
    memset(&io, 0, sizeof io);
    io.out_color[0] = out_color;
    io.out_depth[0] = out_depth;
    io.out_alpha[0] = out_alpha;
    io.final_T[0] = final_T;
    io.n_contrib[0] = n_contrib;
    io.n_eval[0] = n_eval;
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (mode != BGS_MODE_SELECT)
        return render_forward_impl(p, vt, io, N, N, means2D, conic_opacity, colors, depths, point_list, num_entries,
                                   ranges, tw, th, bg, mode, s);
    // Sec. 4.4: balanced kernels until a timing finds the static pixel-wise forward faster
    const long long call = p->sel_calls++;
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    BGS_CUDA(cudaStreamIsCapturing(s, &cst), "cudaStreamIsCapturing");
    const bool measure = !p->sel_switched && call % p->desc.select_period == 0 && cst == cudaStreamCaptureStatusNone;
    if (!measure)
        return render_forward_impl(p, vt, io, N, N, means2D, conic_opacity, colors, depths, point_list, num_entries,
                                   ranges, tw, th, bg, p->sel_switched ? BGS_MODE_STATIC : BGS_MODE_AUTO, s);
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    for (auto &e : ev) BGS_CUDA(cudaEventCreate(&e), "cudaEventCreate");
    int rc = BGS_OK;
    if (cudaEventRecord(ev[0], s) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "cudaEventRecord");
    if (rc == BGS_OK)
        rc = render_forward_impl(p, vt, io, N, N, means2D, conic_opacity, colors, depths, point_list, num_entries,
                                 ranges, tw, th, bg, BGS_MODE_AUTO, s);
    if (rc == BGS_OK && cudaEventRecord(ev[1], s) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "cudaEventRecord");
    if (rc == BGS_OK)
        rc = render_forward_impl(p, vt, io, N, N, means2D, conic_opacity, colors, depths, point_list, num_entries,
                                 ranges, tw, th, bg, BGS_MODE_STATIC, s);
    if (rc == BGS_OK && cudaEventRecord(ev[2], s) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "cudaEventRecord");
    float t_bal = 0.f, t_sta = 0.f;
    if (rc == BGS_OK) {
        cudaError_t e = cudaEventSynchronize(ev[2]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t_bal, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t_sta, ev[1], ev[2]);
        if (e != cudaSuccess) rc = cuda_fail(e, "selector timing");
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (rc != BGS_OK) return rc;
    p->sel_measurements += 1;
    p->sel_last_balanced = t_bal;
    p->sel_last_static = t_sta;
    if (t_sta < t_bal) p->sel_switched = true;
    return BGS_OK;
}

int bgs_render_backward(bgs_plan *p, int64_t N, const float *means2D, const float *conic_opacity, const float *colors,
                        const float *depths, const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges,
                        int32_t W, int32_t H, int32_t tw, int32_t th, const float *bg, int32_t mode,
                        const float *final_T, const int32_t *n_contrib, const float *dL_dcolor, const float *dL_ddepth,
                        const float *dL_dalpha, float *dL_dmeans2D, float *dL_dconic, float *dL_dopacity,
                        float *dL_dcolors, float *dL_ddepths, void *stream) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_render_backward: NULL plan");
    BGS_TRY(check_render_arrays(N, means2D, conic_opacity, colors, depths, point_list, num_entries, ranges, tw, th, bg,
                                mode, "bgs_render_backward"));
    if (!final_T || !n_contrib || !dL_dcolor)
        return fail(BGS_ERR_INVALID, "bgs_render_backward: NULL final_T / n_contrib / dL_dcolor");
    if (N > 0 && (!dL_dmeans2D || !dL_dconic || !dL_dopacity || !dL_dcolors))
        return fail(BGS_ERR_INVALID, "bgs_render_backward: NULL gradient output");
    bgs::ViewTable vt;
    BGS_TRY(make_view_table(1, &W, &H, tw, th, vt));
    bgs::ViewGradIn gi;
    memset(&gi, 0, sizeof gi);
    gi.final_T[0] = final_T;
    gi.n_contrib[0] = n_contrib;
    gi.dL_dcolor[0] = dL_dcolor;
    gi.dL_ddepth[0] = dL_ddepth;
    gi.dL_dalpha[0] = dL_dalpha;
    DeviceGuard g(p->device);
    if (mode == BGS_MODE_SELECT) mode = p->sel_switched ? BGS_MODE_STATIC : BGS_MODE_AUTO;
    return render_backward_impl(p, vt, gi, N, N, means2D, conic_opacity, colors, depths, point_list, num_entries,
                                ranges, tw, th, bg, mode, dL_dmeans2D, dL_dconic, dL_dopacity, dL_dcolors, dL_ddepths,
                                (cudaStream_t)stream);
}


// ---- a7: batched views and graph capture ----------------------------------------------

int bgs_preprocess_batched(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, const float *means3D,
                           const float *log_scales, const float *quats, const float *opacities, int32_t tw, int32_t th,
                           float *means2D, float *conic_opacity, float *depths, int32_t *radii,
                           uint32_t *tiles_touched, void *stream) {
    if (!p || !views) return fail(BGS_ERR_INVALID, "bgs_preprocess_batched: NULL plan or views");
    if (V < 1 || V > bgs::kMaxViews) return fail(BGS_ERR_INVALID, "bgs_preprocess_batched: V=%d", V);
    if (N < 0 || N * V >= (1ll << 32)) return fail(BGS_ERR_INVALID, "bgs_preprocess_batched: N out of range");
    if (N > 0 && (!means3D || !log_scales || !quats || !opacities || !means2D || !conic_opacity || !depths || !radii ||
                  !tiles_touched))
        return fail(BGS_ERR_INVALID, "bgs_preprocess_batched: NULL array");
    BGS_TRY(check_tile(tw, th, false));
    bgs_camera cams[bgs::kMaxViews];
    for (int v = 0; v < V; ++v) {
        BGS_TRY(check_image(views[v].cam.width, views[v].cam.height));
        if (!(views[v].cam.fx > 0.f) || !(views[v].cam.fy > 0.f))
            return fail(BGS_ERR_INVALID, "bgs_preprocess_batched: focal lengths must be > 0");
        cams[v] = views[v].cam;
    }
    DeviceGuard g(p->device);
    BGS_CUDA(bgs::launch_preprocess(N, V, means3D, log_scales, quats, opacities, cams, tw, th, means2D, conic_opacity,
                                    depths, radii, tiles_touched, (cudaStream_t)stream),
             "preprocess_batched");
    if (N > 0) p->host_launches += 1;
    return BGS_OK;
}

int bgs_preprocess_backward_batched(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, const float *means3D,
                                    const float *log_scales, const float *quats, const int32_t *radii,
                                    const float *dL_dmeans2D, const float *dL_dconic, const float *dL_ddepths,
                                    float *dL_dmeans3D, float *dL_dlog_scales, float *dL_dquats, void *stream) {
    if (!p || !views) return fail(BGS_ERR_INVALID, "bgs_preprocess_backward_batched: NULL plan or views");
    if (V < 1 || V > bgs::kMaxViews) return fail(BGS_ERR_INVALID, "bgs_preprocess_backward_batched: V=%d", V);
    if (N < 0 || N * V >= (1ll << 32)) return fail(BGS_ERR_INVALID, "bgs_preprocess_backward_batched: N out of range");
    if (N > 0 && (!means3D || !log_scales || !quats || !radii || !dL_dmeans2D || !dL_dconic || !dL_dmeans3D ||
                  !dL_dlog_scales || !dL_dquats))
        return fail(BGS_ERR_INVALID, "bgs_preprocess_backward_batched: NULL array");
    if (((uintptr_t)dL_dmeans2D) & 7)
        return fail(BGS_ERR_INVALID, "bgs_preprocess_backward_batched: dL_dmeans2D alignment");
    bgs_camera cams[bgs::kMaxViews];
    for (int v = 0; v < V; ++v) {
        BGS_TRY(check_image(views[v].cam.width, views[v].cam.height));
        if (!(views[v].cam.fx > 0.f) || !(views[v].cam.fy > 0.f))
            return fail(BGS_ERR_INVALID, "bgs_preprocess_backward_batched: focal lengths must be > 0");
        cams[v] = views[v].cam;
    }
    DeviceGuard g(p->device);
    BGS_CUDA(bgs::launch_preprocess_backward(N, V, means3D, log_scales, quats, cams, radii, dL_dmeans2D, dL_dconic,
                                             dL_ddepths, dL_dmeans3D, dL_dlog_scales, dL_dquats, (cudaStream_t)stream),
             "preprocess_backward_batched");
    if (N > 0) p->host_launches += 1;
    return BGS_OK;
}

int bgs_bin_and_sort_batched(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                             const int32_t *radii, const float *depths, const float *conic_opacity, int32_t tw,
                             int32_t th, uint32_t *point_list, int64_t capacity, uint32_t *ranges, int32_t flags,
                             int64_t *num_rendered, int64_t *needed, void *stream) {
    if (!p || !views) return fail(BGS_ERR_INVALID, "bgs_bin_and_sort_batched: NULL plan or views");
    if (V < 1 || V > bgs::kMaxViews) return fail(BGS_ERR_INVALID, "bgs_bin_and_sort_batched: V=%d", V);
    if (N < 0 || N * V >= (1ll << 32)) return fail(BGS_ERR_INVALID, "bgs_bin_and_sort_batched: N out of range");
    if (capacity < 0) return fail(BGS_ERR_INVALID, "bgs_bin_and_sort_batched: negative capacity");
    if (!ranges || (N > 0 && (!means2D || !radii || !depths)) || (capacity > 0 && !point_list))
        return fail(BGS_ERR_INVALID, "bgs_bin_and_sort_batched: NULL array");
    if (((uintptr_t)conic_opacity) & 15)
        return fail(BGS_ERR_INVALID, "bgs_bin_and_sort_batched: conic_opacity alignment");
    BGS_TRY(check_tile(tw, th, false));
    int Ws[bgs::kMaxViews], Hs[bgs::kMaxViews];
    for (int v = 0; v < V; ++v) {
        Ws[v] = views[v].cam.width;
        Hs[v] = views[v].cam.height;
    }
    bgs::ViewTable vt;
    BGS_TRY(make_view_table(V, Ws, Hs, tw, th, vt));
    for (int v = 0; v < V; ++v)
        if (bgs::bin_count_smem(vt.tiles_x[v], vt.tiles_y[v]) > (size_t)p->smem_optin)
            return fail(BGS_ERR_INVALID, "bgs_bin_and_sort_batched: view %d has too many tiles", v);
    const bool sync = (flags & BGS_BIN_NO_SYNC) == 0;
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    const long long T = vt.tile_base[V];
    BGS_CUDA(cudaMemsetAsync(ranges, 0, sizeof(uint2) * T, s), "clear ranges");
    BGS_CUDA(cudaMemsetAsync(&p->ctrl->bin_base, 0, sizeof(unsigned long long), s), "clear bin base");
    if (num_rendered) *num_rendered = 0;
    if (needed) *needed = 0;
    const long long R = N * V;
    if (R > 0) {
        // depth order of every view's records: one 32-bit key sort per view slice (a single
        // sort of 64-bit (view, depth) keys over all V N records was measured slower)
        BGS_TRY(ensure(p, p->vkey_sorted, 4 * R, s, "dkey_sorted"));
        BGS_TRY(ensure(p, p->gidx, 4 * R, s, "gidx"));
        BGS_TRY(ensure(p, p->order, 4 * R, s, "order"));
        // keys: the depths' float32 bit patterns (the order both sides sort on); values: record
        // indices, kept in gidx from one call to the next (a call under stream capture records
        // the fill without counting it as done, so that its graph fills them on every replay)
        const uint32_t *k0 = reinterpret_cast<const uint32_t *>(depths);
        uint32_t *k1 = (uint32_t *)p->vkey_sorted.p;
        uint32_t *gidx = (uint32_t *)p->gidx.p, *order = (uint32_t *)p->order.p;
        if (p->iota_n < R) {
            BGS_CUDA(bgs::launch_iota(p->iota_n, R, gidx, s), "record indices");
            p->host_launches += 1;
            cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusNone) p->iota_n = R;
        }
        size_t tmp = 0;
        BGS_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp, k0, k1, gidx, order, (int64_t)N, 0, 32, s),
                 "view depth sort (size)");
        // the views' sorts are independent: fork them over the side streams (a fork-join of
        // events, which a graph capture records as such) and join before the binning
        // (one view: no fork, everything on the caller's stream)
        const int NS = std::min<int>(V, kSortStreams);
        auto stream_of = [&](int i) { return NS > 1 ? p->sort_stream[i] : s; };
        for (int i = 0; i < NS; ++i) BGS_TRY(ensure(p, p->sort_tmp[i], tmp, s, "sort_tmp"));
        if (NS > 1) {
            BGS_CUDA(cudaEventRecord(p->sort_fork, s), "sort fork");
            for (int i = 0; i < NS; ++i)
                BGS_CUDA(cudaStreamWaitEvent(p->sort_stream[i], p->sort_fork, 0), "sort fork wait");
        }
        for (int v = 0; v < V; ++v) {
            const size_t o = (size_t)v * N;
            const int i = v % NS;
            size_t t = p->sort_tmp[i].bytes;
            BGS_CUDA(cub::DeviceRadixSort::SortPairs(p->sort_tmp[i].p, t, k0 + o, k1 + o, gidx + o, order + o,
                                                     (int64_t)N, 0, 32, stream_of(i)),
                     "view depth sort");
        }
        // then each view's binning on its sort's stream (view v's records are positions
        // [v N, (v+1) N) of the order; views v, v + NS, ... share the stream's buffer set):
        // counts, then -- once the counts of the views before it are stored -- its lists
        for (int v = 0; v < V; ++v) {
            const int i = v % NS;
            cudaStream_t si = stream_of(i);
            BinView bv;
            BGS_TRY(bin_view_a(p, i, v, N, order + (size_t)v * N, means2D, radii, conic_opacity, Ws[v], Hs[v], tw, th,
                               bv, si));
            if (NS > 1) {
                BGS_CUDA(cudaEventRecord(p->view_done[v], si), "view count done");
                for (int u = 0; u < v; ++u)
                    if (u % NS != i) BGS_CUDA(cudaStreamWaitEvent(si, p->view_done[u], 0), "earlier view counts");
            }
            BGS_TRY(bin_view_b(p, i, v, N, bv, Ws[v], Hs[v], tw, th, point_list, capacity,
                               ranges + 2ull * vt.tile_base[v], si));
        }
        for (int i = 0; i < NS && NS > 1; ++i) {
            BGS_CUDA(cudaEventRecord(p->sort_join[i], p->sort_stream[i]), "binning join");
            BGS_CUDA(cudaStreamWaitEvent(s, p->sort_join[i], 0), "binning join wait");
        }
        BGS_CUDA(bgs::launch_bin_finish(V, sync ? (1ll << 62) : capacity, p->ctrl, s), "bin_finish");
        p->host_launches += 1;
    }
    if (!sync) return BGS_OK;
    unsigned long long K = 0;
    if (R > 0) {
        BGS_CUDA(cudaMemcpyAsync(&K, &p->ctrl->num_entries, sizeof K, cudaMemcpyDeviceToHost, s), "read K");
        BGS_CUDA(cudaStreamSynchronize(s), "sync K");
    }
    if (needed) *needed = (int64_t)K;
    if ((long long)K > capacity || (long long)K > BGS_MAX_ENTRIES)
        return fail(BGS_ERR_CAPACITY, "bgs_bin_and_sort_batched: %llu entries exceed capacity %lld (or "
                                      "BGS_MAX_ENTRIES)", K, (long long)capacity);
    if (num_rendered) *num_rendered = (int64_t)K;
    return BGS_OK;
}

static int batched_tables(int V, const bgs_view *views, int tw, int th, bgs::ViewTable &vt) {
    if (!views) return fail(BGS_ERR_INVALID, "NULL views");
    if (V < 1 || V > bgs::kMaxViews) return fail(BGS_ERR_INVALID, "V=%d outside [1, %d]", V, bgs::kMaxViews);
    int Ws[bgs::kMaxViews], Hs[bgs::kMaxViews];
    for (int v = 0; v < V; ++v) {
        Ws[v] = views[v].cam.width;
        Hs[v] = views[v].cam.height;
    }
    return make_view_table(V, Ws, Hs, tw, th, vt);
}

// Batched forward; colours [N,3] shared by the views (per_view false) or [V*N,3] per record.
static int render_forward_batched(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                                  const float *conic_opacity, const float *colors, const float *depths,
                                  const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges, int32_t tw,
                                  int32_t th, const float *bg, int32_t mode, bool per_view, void *stream) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_render_forward_batched: NULL plan");
    if (mode == BGS_MODE_STATIC || mode == BGS_MODE_SELECT)
        return fail(BGS_ERR_INVALID, "bgs_render_forward_batched: the static kernel (and the selector) is single-view");
    bgs::ViewTable vt;
    BGS_TRY(batched_tables(V, views, tw, th, vt));
    if (N < 0 || N * V >= (1ll << 32)) return fail(BGS_ERR_INVALID, "bgs_render_forward_batched: N out of range");
    BGS_TRY(check_render_arrays(N * V, means2D, conic_opacity, colors, depths, point_list, num_entries, ranges, tw, th,
                                bg, mode, "bgs_render_forward_batched"));
    bgs::ViewOut io;
    memset(&io, 0, sizeof io);
    for (int v = 0; v < V; ++v) {
        const bgs_view &w = views[v];
        if (!w.out_color || !w.out_depth || !w.out_alpha || !w.final_T || !w.n_contrib)
            return fail(BGS_ERR_INVALID, "bgs_render_forward_batched: NULL output of view %d", v);
        io.out_color[v] = w.out_color;
        io.out_depth[v] = w.out_depth;
        io.out_alpha[v] = w.out_alpha;
        io.final_T[v] = w.final_T;
        io.n_contrib[v] = w.n_contrib;
        io.n_eval[v] = w.n_eval;
    }
    DeviceGuard g(p->device);
    return render_forward_impl(p, vt, io, N * V, per_view ? N * V : N, means2D, conic_opacity, colors, depths,
                               point_list, num_entries, ranges, tw, th, bg, mode, (cudaStream_t)stream);
}

int bgs_render_forward_batched(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                               const float *conic_opacity, const float *colors, const float *depths,
                               const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges, int32_t tw,
                               int32_t th, const float *bg, int32_t mode, void *stream) {
    return render_forward_batched(p, V, views, N, means2D, conic_opacity, colors, depths, point_list, num_entries,
                                  ranges, tw, th, bg, mode, false, stream);
}

int bgs_render_forward_batched_vc(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                                  const float *conic_opacity, const float *colors, const float *depths,
                                  const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges, int32_t tw,
                                  int32_t th, const float *bg, int32_t mode, void *stream) {
    return render_forward_batched(p, V, views, N, means2D, conic_opacity, colors, depths, point_list, num_entries,
                                  ranges, tw, th, bg, mode, true, stream);
}

// Batched backward; colours and dL_dcolors [N,3] shared by the views (per_view false) or
// [V*N,3] per record.
static int render_backward_batched(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                                   const float *conic_opacity, const float *colors, const float *depths,
                                   const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges,
                                   int32_t tw, int32_t th, const float *bg, int32_t mode, float *dL_dmeans2D,
                                   float *dL_dconic, float *dL_dopacity, float *dL_dcolors, float *dL_ddepths,
                                   bool per_view, void *stream) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_render_backward_batched: NULL plan");
    if (mode == BGS_MODE_STATIC || mode == BGS_MODE_SELECT)
        return fail(BGS_ERR_INVALID, "bgs_render_backward_batched: the static kernel (and the selector) is single-view");
    bgs::ViewTable vt;
    BGS_TRY(batched_tables(V, views, tw, th, vt));
    if (N < 0 || N * V >= (1ll << 32)) return fail(BGS_ERR_INVALID, "bgs_render_backward_batched: N out of range");
    BGS_TRY(check_render_arrays(N * V, means2D, conic_opacity, colors, depths, point_list, num_entries, ranges, tw, th,
                                bg, mode, "bgs_render_backward_batched"));
    if (N > 0 && (!dL_dmeans2D || !dL_dconic || !dL_dopacity || !dL_dcolors))
        return fail(BGS_ERR_INVALID, "bgs_render_backward_batched: NULL gradient output");
    bgs::ViewGradIn gi;
    memset(&gi, 0, sizeof gi);
    for (int v = 0; v < V; ++v) {
        const bgs_view &w = views[v];
        if (!w.final_T || !w.n_contrib || !w.dL_dcolor)
            return fail(BGS_ERR_INVALID, "bgs_render_backward_batched: NULL final_T / n_contrib / dL_dcolor of view %d", v);
        gi.final_T[v] = w.final_T;
        gi.n_contrib[v] = w.n_contrib;
        gi.dL_dcolor[v] = w.dL_dcolor;
        gi.dL_ddepth[v] = w.dL_ddepth;
        gi.dL_dalpha[v] = w.dL_dalpha;
    }
    DeviceGuard g(p->device);
    return render_backward_impl(p, vt, gi, N * V, per_view ? N * V : N, means2D, conic_opacity, colors, depths,
                                point_list, num_entries, ranges, tw, th, bg, mode, dL_dmeans2D, dL_dconic,
                                dL_dopacity, dL_dcolors, dL_ddepths, (cudaStream_t)stream);
}

int bgs_render_backward_batched(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                                const float *conic_opacity, const float *colors, const float *depths,
                                const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges, int32_t tw,
                                int32_t th, const float *bg, int32_t mode, float *dL_dmeans2D, float *dL_dconic,
                                float *dL_dopacity, float *dL_dcolors, float *dL_ddepths, void *stream) {
    return render_backward_batched(p, V, views, N, means2D, conic_opacity, colors, depths, point_list, num_entries,
                                   ranges, tw, th, bg, mode, dL_dmeans2D, dL_dconic, dL_dopacity, dL_dcolors,
                                   dL_ddepths, false, stream);
}

int bgs_render_backward_batched_vc(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                                   const float *conic_opacity, const float *colors, const float *depths,
                                   const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges,
                                   int32_t tw, int32_t th, const float *bg, int32_t mode, float *dL_dmeans2D,
                                   float *dL_dconic, float *dL_dopacity, float *dL_dcolors, float *dL_ddepths,
                                   void *stream) {
    return render_backward_batched(p, V, views, N, means2D, conic_opacity, colors, depths, point_list, num_entries,
                                   ranges, tw, th, bg, mode, dL_dmeans2D, dL_dconic, dL_dopacity, dL_dcolors,
                                   dL_ddepths, true, stream);
}

// Camera centre of a world -> camera viewmat (row-major [A t; 0 1]): A c + t = 0, solved in
// double by the adjugate of A (A is a rotation for a rigid camera, then c = -A^T t).
static bool camera_centre(const bgs_camera &cam, float *c) {
    const float *M = cam.viewmat;
    const double a[3][3] = {{M[0], M[1], M[2]}, {M[4], M[5], M[6]}, {M[8], M[9], M[10]}};
    const double t[3] = {M[3], M[7], M[11]};
    const double co[3][3] = {{a[1][1] * a[2][2] - a[1][2] * a[2][1], a[1][2] * a[2][0] - a[1][0] * a[2][2],
                              a[1][0] * a[2][1] - a[1][1] * a[2][0]},
                             {a[0][2] * a[2][1] - a[0][1] * a[2][2], a[0][0] * a[2][2] - a[0][2] * a[2][0],
                              a[0][1] * a[2][0] - a[0][0] * a[2][1]},
                             {a[0][1] * a[1][2] - a[0][2] * a[1][1], a[0][2] * a[1][0] - a[0][0] * a[1][2],
                              a[0][0] * a[1][1] - a[0][1] * a[1][0]}};
    const double det = a[0][0] * co[0][0] + a[0][1] * co[0][1] + a[0][2] * co[0][2];
    if (!(fabs(det) > 1e-30)) return false;
    // inverse = co^T / det; c = -inverse t
    for (int r = 0; r < 3; ++r) c[r] = (float)(-(co[0][r] * t[0] + co[1][r] * t[1] + co[2][r] * t[2]) / det);
    return true;
}

static int sh_args(const char *fn, bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, int32_t degree,
                   int32_t stride, float *campos) {
    if (!p || !views) return fail(BGS_ERR_INVALID, "%s: NULL plan or views", fn);
    if (V < 1 || V > bgs::kMaxViews) return fail(BGS_ERR_INVALID, "%s: V=%d", fn, V);
    if (N < 0 || N * V >= (1ll << 40)) return fail(BGS_ERR_INVALID, "%s: N out of range", fn);
    if (degree < 0 || degree > 3) return fail(BGS_ERR_INVALID, "%s: degree %d not in 0..3", fn, degree);
    if (stride < (degree + 1) * (degree + 1)) return fail(BGS_ERR_INVALID, "%s: stride %d < (degree+1)^2", fn, stride);
    for (int v = 0; v < V; ++v)
        if (!camera_centre(views[v].cam, campos + 3 * v))
            return fail(BGS_ERR_INVALID, "%s: singular viewmat of view %d", fn, v);
    return BGS_OK;
}

int bgs_sh_to_rgb(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, int32_t degree, int32_t stride,
                  const float *sh, const float *means3D, float *rgb, uint8_t *clamped, void *stream) {
    float campos[3 * bgs::kMaxViews];
    BGS_TRY(sh_args("bgs_sh_to_rgb", p, V, views, N, degree, stride, campos));
    if (N > 0 && (!sh || !means3D || !rgb)) return fail(BGS_ERR_INVALID, "bgs_sh_to_rgb: NULL array");
    DeviceGuard g(p->device);
    BGS_CUDA(bgs::launch_sh(false, N, degree, stride, sh, means3D, V, campos, rgb, clamped, nullptr, nullptr, nullptr,
                            (cudaStream_t)stream),
             "sh_to_rgb");
    if (N > 0) p->host_launches += 1;
    return BGS_OK;
}

int bgs_sh_to_rgb_backward(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, int32_t degree, int32_t stride,
                           const float *sh, const float *means3D, const float *dL_drgb, float *dL_dsh,
                           float *dL_dmeans3D, void *stream) {
    float campos[3 * bgs::kMaxViews];
    BGS_TRY(sh_args("bgs_sh_to_rgb_backward", p, V, views, N, degree, stride, campos));
    if (N > 0 && (!sh || !means3D || !dL_drgb || !dL_dsh || !dL_dmeans3D))
        return fail(BGS_ERR_INVALID, "bgs_sh_to_rgb_backward: NULL array");
    DeviceGuard g(p->device);
    BGS_CUDA(bgs::launch_sh(true, N, degree, stride, sh, means3D, V, campos, nullptr, nullptr, dL_drgb, dL_dsh,
                            dL_dmeans3D, (cudaStream_t)stream),
             "sh_to_rgb_backward");
    if (N > 0) p->host_launches += 1;
    return BGS_OK;
}

int bgs_graph_begin(bgs_plan *p, void *stream) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_graph_begin: NULL plan");
    DeviceGuard g(p->device);
    BGS_CUDA(cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    return BGS_OK;
}

int bgs_graph_end(bgs_plan *p, void *stream) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_graph_end: NULL plan");
    DeviceGuard g(p->device);
    cudaGraph_t graph = nullptr;
    BGS_CUDA(cudaStreamEndCapture((cudaStream_t)stream, &graph), "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->graph = graph;
    p->graph_exec = exec;
    return BGS_OK;
}

int bgs_graph_launch(bgs_plan *p, void *stream) {
    if (!p) return fail(BGS_ERR_INVALID, "bgs_graph_launch: NULL plan");
    if (!p->graph_exec) return fail(BGS_ERR_INVALID, "bgs_graph_launch: no captured graph");
    DeviceGuard g(p->device);
    BGS_CUDA(cudaGraphLaunch(p->graph_exec, (cudaStream_t)stream), "cudaGraphLaunch");
    return BGS_OK;
}


int bgs_autotune_render(bgs_plan *p, int32_t V, const bgs_view *views, int64_t N, const float *means2D,
                        const float *conic_opacity, const float *colors, const float *depths,
                        const uint32_t *point_list, int64_t num_entries, const uint32_t *ranges, int32_t tw, int32_t th,
                        const float *bg, int32_t backward, float *dL_dmeans2D, float *dL_dconic, float *dL_dopacity,
                        float *dL_dcolors, double *best_ms, void *stream) {
    if (!p || !views) return fail(BGS_ERR_INVALID, "bgs_autotune_render: NULL plan or views");
    DeviceGuard g(p->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BGS_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    const bgs_plan_desc start = p->desc;
    const bool was_timing = p->timing;
    p->timing = false;
    // one candidate: 1 untimed + 2 timed passes of forward (+ backward); best of the two
    auto run = [&](const bgs_plan_desc &d, double &ms) -> int {
        p->desc = d;
        ms = 1e30;
        for (int rep = 0; rep < 3; ++rep) {
            BGS_CUDA(cudaEventRecord(e0, s), "event");
            BGS_TRY(bgs_render_forward_batched(p, V, views, N, means2D, conic_opacity, colors, depths, point_list,
                                               num_entries, ranges, tw, th, bg, BGS_MODE_AUTO, stream));
            if (backward)
                BGS_TRY(bgs_render_backward_batched(p, V, views, N, means2D, conic_opacity, colors, depths,
                                                    point_list, num_entries, ranges, tw, th, bg, BGS_MODE_AUTO,
                                                    dL_dmeans2D, dL_dconic, dL_dopacity, dL_dcolors, nullptr, stream));
            BGS_CUDA(cudaEventRecord(e1, s), "event");
            BGS_CUDA(cudaEventSynchronize(e1), "event sync");
            float t = 0.f;
            BGS_CUDA(cudaEventElapsedTime(&t, e0, e1), "elapsed");
            if (rep > 0) ms = std::min(ms, (double)t);
        }
        return BGS_OK;
    };
    bgs_plan_desc best = start, d = start;
    double best_t = 1e30, t = 0.0;
    int rc = BGS_OK;
    // stage 1: sub-tile (pixel rows per lane) with pixel-wise items only
    d.heavy_threshold = 0x7fffffff;
    d.queue_chunk = 1;
    for (int q : {1, 2, 4, 8}) {
        d.pixel_rows = q;
        if ((rc = run(d, t)) != BGS_OK) break;
        if (t < best_t) best_t = t, best = d;
    }
    // stage 2: heavy-tile threshold and pixels per Gaussian-wise item; Gaussian-wise items are
    // kept only when they gain more than 1 % over the best without them (a threshold above
    // every list queues none and would win or lose on timing noise alone)
    const bgs_plan_desc no_gw = best;
    const double no_gw_t = best_t;
    for (int thr : {256, 1024, 4096, 16384}) {
        if (rc != BGS_OK) break;
        for (int P : {4, 8, 16}) {
            d = no_gw;
            d.heavy_threshold = thr;
            d.gw_pixels = P;
            if ((rc = run(d, t)) != BGS_OK) break;
            if (t < best_t && t < 0.99 * no_gw_t) best_t = t, best = d;
        }
    }
    // stage 2b: segment length of the Gaussian-wise items, when the best uses them
    for (int L : {512, 8192}) {
        if (rc != BGS_OK || best.heavy_threshold == INT32_MAX || (int64_t)best.heavy_threshold >= num_entries) break;
        d = best;
        d.gw_segment = L;
        if ((rc = run(d, t)) != BGS_OK) break;
        if (t < best_t) best_t = t, best = d;
    }
    // stage 3: queue granularity
    for (int c : {2, 4}) {
        if (rc != BGS_OK) break;
        d = best;
        d.queue_chunk = c;
        if ((rc = run(d, t)) != BGS_OK) break;
        if (t < best_t) best_t = t, best = d;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->timing = was_timing;
    p->desc = (rc == BGS_OK) ? best : start;
    if (best_ms) *best_ms = best_t;
    return rc;
}

}  // extern "C"
