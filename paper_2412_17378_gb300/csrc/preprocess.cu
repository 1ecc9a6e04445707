// preprocess.cu -- a1: per-Gaussian projection (Eq. 1-3 of the paper, Sec. 2.1).
//
// One thread per Gaussian.  The work is ~80 bytes of HBM traffic and ~150 FP32
// operations per Gaussian: a few microseconds per million Gaussians, far below the
// render kernels, so the kernel is written for clarity with coalesced scalar loads.
#include "bgs_internal.cuh"

namespace bgs {

struct CamDev {
    float V[12];  // rows 0..2 of the world->camera matrix
    float fx, fy, cx, cy, near_plane, lowpass, lim_x, lim_y;
    int W, H, tile_w, tile_h, tiles_x, tiles_y;
};

struct CamTable {
    int V;
    CamDev cam[kMaxViews];
};

// Tile rectangle of a Gaussian: x in [floor((u-r)/tw), floor((u+(r+tw-1))/tw)), clamped.
// Float32 with one IEEE rounding per operation (no contraction), the same operations the
// binning kernel and the host-side checks use.
__device__ __forceinline__ void tile_rect(float u, float v, int r, int tw, int th, int tx, int ty, int &x0,
                                          int &x1, int &y0, int &y1) {
    x0 = (int)floorf(__fdiv_rn(__fsub_rn(u, (float)r), (float)tw));
    x1 = (int)floorf(__fdiv_rn(__fadd_rn(u, (float)(r + tw - 1)), (float)tw));
    y0 = (int)floorf(__fdiv_rn(__fsub_rn(v, (float)r), (float)th));
    y1 = (int)floorf(__fdiv_rn(__fadd_rn(v, (float)(r + th - 1)), (float)th));
    x0 = min(max(x0, 0), tx);
    x1 = min(max(x1, 0), tx);
    y0 = min(max(y0, 0), ty);
    y1 = min(max(y1, 0), ty);
}

// Record i = v * N + g projects Gaussian g into view v (one view for the single-view call).
__global__ void __launch_bounds__(256) k_preprocess(long long N, const float *__restrict__ means3D,
                                                    const float *__restrict__ log_scales,
                                                    const float *__restrict__ quats,
                                                    const float *__restrict__ opacities, const CamTable ct,
                                                    float2 *__restrict__ means2D, float4 *__restrict__ conic_opacity,
                                                    float *__restrict__ depths, int *__restrict__ radii,
                                                    uint32_t *__restrict__ tiles_touched) {
    const long long rec = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (rec >= N * ct.V) return;
    const int view = (int)(rec / N);
    const long long g = rec - (long long)view * N;
    const CamDev &cam = ct.cam[view];
    const float px = means3D[3 * g], py = means3D[3 * g + 1], pz = means3D[3 * g + 2];
    const float *V = cam.V;
    const float tx = V[0] * px + V[1] * py + V[2] * pz + V[3];
    const float ty = V[4] * px + V[5] * py + V[6] * pz + V[7];
    const float tz = V[8] * px + V[9] * py + V[10] * pz + V[11];
    float2 m2 = make_float2(0.f, 0.f);
    float4 co = make_float4(0.f, 0.f, 0.f, 0.f);
    int radius = 0;
    uint32_t touched = 0;
    depths[rec] = tz;
    if (tz > cam.near_plane) {
        // R from the normalised quaternion (w, x, y, z)
        float qw = quats[4 * g], qx = quats[4 * g + 1], qy = quats[4 * g + 2], qz = quats[4 * g + 3];
        const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        qw /= qn; qx /= qn; qy /= qn; qz /= qn;
        const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz), R02 = 2.f * (qx * qz + qw * qy);
        const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz), R12 = 2.f * (qy * qz - qw * qx);
        const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx), R22 = 1.f - 2.f * (qx * qx + qy * qy);
        const float s0 = expf(log_scales[3 * g]), s1 = expf(log_scales[3 * g + 1]), s2 = expf(log_scales[3 * g + 2]);
        // M = R S ; Sigma = M M^T (symmetric, 6 entries)
        const float M00 = R00 * s0, M01 = R01 * s1, M02 = R02 * s2;
        const float M10 = R10 * s0, M11 = R11 * s1, M12 = R12 * s2;
        const float M20 = R20 * s0, M21 = R21 * s1, M22 = R22 * s2;
        const float S00 = M00 * M00 + M01 * M01 + M02 * M02;
        const float S01 = M00 * M10 + M01 * M11 + M02 * M12;
        const float S02 = M00 * M20 + M01 * M21 + M02 * M22;
        const float S11 = M10 * M10 + M11 * M11 + M12 * M12;
        const float S12 = M10 * M20 + M11 * M21 + M12 * M22;
        const float S22 = M20 * M20 + M21 * M21 + M22 * M22;
        // Jacobian of the pinhole map at the tangent-clamped point
        const float iz = 1.f / tz;
        const float xc = fminf(cam.lim_x, fmaxf(-cam.lim_x, tx * iz)) * tz;
        const float yc = fminf(cam.lim_y, fmaxf(-cam.lim_y, ty * iz)) * tz;
        const float J00 = cam.fx * iz, J02 = -cam.fx * xc * iz * iz;
        const float J11 = cam.fy * iz, J12 = -cam.fy * yc * iz * iz;
        // T = J W (2x3)
        const float T00 = J00 * V[0] + J02 * V[8], T01 = J00 * V[1] + J02 * V[9], T02 = J00 * V[2] + J02 * V[10];
        const float T10 = J11 * V[4] + J12 * V[8], T11 = J11 * V[5] + J12 * V[9], T12 = J11 * V[6] + J12 * V[10];
        // Sigma' = T Sigma T^T
        const float U00 = S00 * T00 + S01 * T01 + S02 * T02;  // (Sigma T^T) column 0
        const float U10 = S01 * T00 + S11 * T01 + S12 * T02;
        const float U20 = S02 * T00 + S12 * T01 + S22 * T02;
        const float U01 = S00 * T10 + S01 * T11 + S02 * T12;  // column 1
        const float U11 = S01 * T10 + S11 * T11 + S12 * T12;
        const float U21 = S02 * T10 + S12 * T11 + S22 * T12;
        const float c00 = T00 * U00 + T01 * U10 + T02 * U20 + cam.lowpass;
        const float c01 = T00 * U01 + T01 * U11 + T02 * U21;
        const float c11 = T10 * U01 + T11 * U11 + T12 * U21 + cam.lowpass;
        const float det = c00 * c11 - c01 * c01;
        if (det > 0.f) {
            const float mid = 0.5f * (c00 + c11);
            const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
            const int r = (int)ceilf(3.f * sqrtf(lam));
            const float idet = 1.f / det;
            const float u = cam.fx * tx * iz + cam.cx, v = cam.fy * ty * iz + cam.cy;
            m2 = make_float2(u, v);
            co = make_float4(c11 * idet, -c01 * idet, c00 * idet, opacities[g]);
            int x0, x1, y0, y1;
            tile_rect(u, v, r, cam.tile_w, cam.tile_h, cam.tiles_x, cam.tiles_y, x0, x1, y0, y1);
            const long long area = (long long)(x1 - x0) * (long long)(y1 - y0);
            if (area > 0) {
                radius = r;
                touched = (uint32_t)area;
            }
        }
    }
    means2D[rec] = m2;
    conic_opacity[rec] = co;
    radii[rec] = radius;
    tiles_touched[rec] = touched;
}

static CamDev cam_dev(const bgs_camera &c, int tile_w, int tile_h) {
    CamDev cam;
    for (int k = 0; k < 12; ++k) cam.V[k] = c.viewmat[k];
    cam.fx = c.fx; cam.fy = c.fy; cam.cx = c.cx; cam.cy = c.cy;
    cam.near_plane = c.near_plane;
    cam.lowpass = c.lowpass;
    cam.lim_x = 1.3f * (float)((double)c.width / (2.0 * (double)c.fx));
    cam.lim_y = 1.3f * (float)((double)c.height / (2.0 * (double)c.fy));
    cam.W = c.width; cam.H = c.height;
    cam.tile_w = tile_w; cam.tile_h = tile_h;
    cam.tiles_x = (c.width + tile_w - 1) / tile_w;
    cam.tiles_y = (c.height + tile_h - 1) / tile_h;
    return cam;
}

cudaError_t launch_preprocess(long long N, int V, const float *means3D, const float *log_scales, const float *quats,
                              const float *opacities, const bgs_camera *cams, int tile_w, int tile_h,
                              float *means2D, float *conic_opacity, float *depths, int *radii,
                              uint32_t *tiles_touched, cudaStream_t s) {
    if (V < 1 || V > kMaxViews) return cudaErrorInvalidValue;
    CamTable ct;
    ct.V = V;
    for (int v = 0; v < V; ++v) ct.cam[v] = cam_dev(cams[v], tile_w, tile_h);
    if (N == 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (N * V + threads - 1) / threads;
    k_preprocess<<<(unsigned)blocks, threads, 0, s>>>(N, means3D, log_scales, quats, opacities, ct,
                                                       reinterpret_cast<float2 *>(means2D),
                                                       reinterpret_cast<float4 *>(conic_opacity), depths, radii,
                                                       tiles_touched);
    return cudaGetLastError();
}

// Depth sort keys of a batched binning: (view << 32 | float bits of depth), value = record.
__global__ void __launch_bounds__(256) k_depth_keys64(long long N, int V, const float *__restrict__ depths,
                                                      unsigned long long *__restrict__ keys, uint32_t *__restrict__ idx) {
    const long long rec = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (rec >= N * V) return;
    const unsigned long long view = (unsigned long long)(rec / N);
    keys[rec] = (view << 32) | (unsigned long long)__float_as_uint(depths[rec]);
    idx[rec] = (uint32_t)rec;
}

cudaError_t launch_depth_keys64(long long N, int V, const float *depths, unsigned long long *keys, uint32_t *idx,
                                cudaStream_t s) {
    if (N * V == 0) return cudaSuccess;
    k_depth_keys64<<<(unsigned)((N * V + 255) / 256), 256, 0, s>>>(N, V, depths, keys, idx);
    return cudaGetLastError();
}

// ---- a2: binning -----------------------------------------------------------------------
// The per-tile lists must be ordered by (float32 depth, Gaussian index).  Instead of one
// radix sort of 64-bit (tile, depth) keys over all K duplicated entries, the Gaussians are
// first sorted by depth (N keys of 32 bits), the entries are then emitted in that order,
// and a stable radix sort on the tile id alone (13-17 bits) groups them per tile while
// keeping the depth order.  This moves the multi-pass work from K 12-byte records over
// 45 key bits to K 6- or 8-byte records over the tile bits only.

// Entry count (rectangle area) and depth sort key of each Gaussian.
__global__ void __launch_bounds__(256) k_touched(long long N, const float2 *__restrict__ means2D,
                                                 const int *__restrict__ radii, const float *__restrict__ depths,
                                                 int tw, int th, int tx, int ty, uint32_t *__restrict__ touched,
                                                 uint32_t *__restrict__ dkey, uint32_t *__restrict__ idx) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int r = radii[i];
    uint32_t c = 0;
    if (r > 0) {
        const float2 m = means2D[i];
        int x0, x1, y0, y1;
        tile_rect(m.x, m.y, r, tw, th, tx, ty, x0, x1, y0, y1);
        if (x1 > x0 && y1 > y0) c = (uint32_t)((x1 - x0) * (y1 - y0));
    }
    touched[i] = c;
    dkey[i] = __float_as_uint(depths[i]);
    idx[i] = (uint32_t)i;
}

cudaError_t launch_touched(long long N, const float *means2D, const int *radii, const float *depths, int W, int H,
                           int tile_w, int tile_h, uint32_t *touched, uint32_t *dkey, uint32_t *idx, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const int tx = (W + tile_w - 1) / tile_w, ty = (H + tile_h - 1) / tile_h;
    k_touched<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, reinterpret_cast<const float2 *>(means2D), radii, depths,
                                                          tile_w, tile_h, tx, ty, touched, dkey, idx);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_gather_u32(long long N, const uint32_t *__restrict__ src,
                                                    const uint32_t *__restrict__ order, uint32_t *__restrict__ dst) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) dst[i] = src[order[i]];
}

cudaError_t launch_gather_u32(long long N, const uint32_t *src, const uint32_t *order, uint32_t *dst, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    k_gather_u32<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, src, order, dst);
    return cudaGetLastError();
}

// Emits the entries of the depth-ordered Gaussians: position s of the depth order writes
// one (tile id, Gaussian index) pair per covered tile at offsets[s], row-major over its
// rectangle.  A warp takes 32 consecutive positions and writes their runs one after the
// other, the 32 lanes storing consecutive entries of a run (coalesced stores).
template <typename KeyT>
__global__ void __launch_bounds__(256) k_duplicate(long long N, const uint32_t *__restrict__ order,
                                                   const float2 *__restrict__ means2D, const int *__restrict__ radii,
                                                   const unsigned long long *__restrict__ offsets, int tw, int th,
                                                   int tx, int ty, KeyT *__restrict__ keys, uint32_t *__restrict__ vals,
                                                   long long capacity) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint32_t i = 0;
    int x0 = 0, y0 = 0, w = 1, cnt = 0;
    long long off = 0;
    if (s < N) {
        i = order[s];
        const int r = radii[i];
        if (r > 0) {
            const float2 m = means2D[i];
            int x1, y1;
            tile_rect(m.x, m.y, r, tw, th, tx, ty, x0, x1, y0, y1);
            if (x1 > x0 && y1 > y0) {
                w = x1 - x0;
                cnt = w * (y1 - y0);
                off = (long long)offsets[s];
            }
        }
    }
    unsigned pending = __ballot_sync(0xffffffffu, cnt > 0);
    while (pending) {
        const int q = __ffs(pending) - 1;
        pending &= pending - 1;
        const int cq = __shfl_sync(0xffffffffu, cnt, q);
        const int wq = __shfl_sync(0xffffffffu, w, q);
        const int xq = __shfl_sync(0xffffffffu, x0, q);
        const int yq = __shfl_sync(0xffffffffu, y0, q);
        const uint32_t iq = __shfl_sync(0xffffffffu, i, q);
        const long long oq = __shfl_sync(0xffffffffu, off, q);
        for (int k = lane; k < cq; k += 32) {
            const long long o = oq + k;
            if (o < capacity) {
                const int dy = k / wq;
                keys[o] = (KeyT)((yq + dy) * tx + xq + (k - dy * wq));
                vals[o] = iq;
            }
        }
    }
}

template <typename KeyT>
cudaError_t launch_duplicate(long long N, const uint32_t *order, const float *means2D, const int *radii,
                             const unsigned long long *offsets, int W, int H, int tile_w, int tile_h, KeyT *keys,
                             uint32_t *vals, long long capacity, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const int tx = (W + tile_w - 1) / tile_w, ty = (H + tile_h - 1) / tile_h;
    k_duplicate<KeyT><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, order, reinterpret_cast<const float2 *>(means2D),
                                                                  radii, offsets, tile_w, tile_h, tx, ty, keys, vals,
                                                                  capacity);
    return cudaGetLastError();
}
template cudaError_t launch_duplicate<uint16_t>(long long, const uint32_t *, const float *, const int *,
                                                const unsigned long long *, int, int, int, int, uint16_t *, uint32_t *,
                                                long long, cudaStream_t);
template cudaError_t launch_duplicate<uint32_t>(long long, const uint32_t *, const float *, const int *,
                                                const unsigned long long *, int, int, int, int, uint32_t *, uint32_t *,
                                                long long, cudaStream_t);

__global__ void k_count_total(long long N, const uint32_t *touched, const unsigned long long *offsets,
                              DevCtrl *ctrl) {
    ctrl->num_entries = N > 0 ? offsets[N - 1] + touched[N - 1] : 0ull;
}

cudaError_t launch_count_total(long long N, const uint32_t *touched, const unsigned long long *offsets, DevCtrl *ctrl,
                               cudaStream_t s) {
    k_count_total<<<1, 1, 0, s>>>(N, touched, offsets, ctrl);
    return cudaGetLastError();
}

// ranges[t] = [first, last+1) of tile t in the sorted tile keys (ranges zeroed beforehand).
// Each thread inspects 8 consecutive keys and their right neighbour.
template <typename KeyT>
__global__ void __launch_bounds__(256) k_ranges(const KeyT *__restrict__ keys, long long K, uint2 *__restrict__ ranges) {
    const long long j0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 8;
    if (j0 >= K) return;
    const int n = (int)min(8ll, K - j0);
    uint32_t k[9];
#pragma unroll
    for (int q = 0; q < 8; ++q) k[q] = q < n ? (uint32_t)keys[j0 + q] : 0u;
    k[8] = (j0 + 8 < K) ? (uint32_t)keys[j0 + 8] : 0xffffffffu;
    const uint32_t prev = j0 > 0 ? (uint32_t)keys[j0 - 1] : 0xffffffffu;
    if (prev != k[0]) ranges[k[0]].x = (uint32_t)j0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (q >= n) break;
        const uint32_t nxt = (q + 1 < n) ? k[q + 1] : k[8];
        if (nxt != k[q]) {
            ranges[k[q]].y = (uint32_t)(j0 + q + 1);
            if (q + 1 < n) ranges[k[q + 1]].x = (uint32_t)(j0 + q + 1);
        }
    }
}

template <typename KeyT>
cudaError_t launch_ranges(const KeyT *keys, long long K, uint2 *ranges, cudaStream_t s) {
    if (K == 0) return cudaSuccess;
    const long long threads = (K + 7) / 8;
    k_ranges<KeyT><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(keys, K, ranges);
    return cudaGetLastError();
}
template cudaError_t launch_ranges<uint16_t>(const uint16_t *, long long, uint2 *, cudaStream_t);
template cudaError_t launch_ranges<uint32_t>(const uint32_t *, long long, uint2 *, cudaStream_t);

// ---- render input packing ------------------------------------------------------------------
// recs[i] packs record i; the colour comes from Gaussian i % n_colors (views share colours).
__global__ void __launch_bounds__(256) k_pack(long long N, const float *__restrict__ means2D,
                                              const float *__restrict__ conic_opacity,
                                              const float *__restrict__ colors, long long n_colors,
                                              const float *__restrict__ depths, Rec *__restrict__ recs) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long long c = (n_colors == N) ? i : i % n_colors;
    recs[i] = make_rec(means2D, conic_opacity, colors, depths, (unsigned int)i, (unsigned int)c);
}

cudaError_t launch_pack(long long N, const float *means2D, const float *conic_opacity, const float *colors,
                        long long n_colors, const float *depths, Rec *recs, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    k_pack<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, means2D, conic_opacity, colors, n_colors, depths, recs);
    return cudaGetLastError();
}

}  // namespace bgs
