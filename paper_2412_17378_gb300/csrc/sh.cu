// sh.cu -- view-dependent colour from spherical harmonics (Sec. 2.1: a Gaussian's colour is
// represented by spherical harmonics) and its gradient.
//
// Basis: the real orthonormal spherical harmonics of degree l <= 3 with the Condon-Shortley
// phase, as homogeneous harmonic polynomials of the unit direction d = (x, y, z) from the
// camera centre to the Gaussian's mean, coefficients ordered (l, m) = (0,0), (1,-1), (1,0),
// (1,1), (2,-2), ..., (3,3).  Colour channel c = sum_k Y_k(d) sh[k][c] + 1/2, clamped below at
// 0; a clamped channel passes no gradient.
//
// Both kernels are HBM-bound (degree 3: 192 bytes of coefficients per Gaussian against ~60
// flops forward, ~250 backward).  One thread per Gaussian loops over the views, so the
// coefficients are read once whatever the number of views, and the backward sums the
// views' gradients (no atomics).
// Staged single-view backward (the coefficient array holds exactly the used rows, 3 (D+1)^2
// a multiple of 4 floats, 16-byte aligned -- degree 1 or 3 in rows of 4 or 16; degree 3 on 1M
// Gaussians: 75 us against 119 us unstaged): each warp copies its 32
// Gaussians' contiguous coefficients into a warp-private shared buffer with coalesced float4
// loads, into rows padded to 3 (D+1)^2 + 1 floats so that each lane's reads of its own row
// are bank-conflict free; the single-view backward writes its dL/dsh into the same row and
// the warp stores it with coalesced float4 stores.  Warps synchronise only with themselves,
// so loading and arithmetic of different warps overlap freely.  (Staging the forward the
// same way measured slower than its direct loads, 73 vs 69 us, so every forward is direct.)  Otherwise each thread reads its row block
// directly (float4 when 16-byte aligned) and the multi-view backward sums in registers.
#include <algorithm>

#include "bgs_internal.cuh"

namespace bgs {

// Normalisation constants of the basis (closed forms in the comments).
constexpr float kY00 = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
constexpr float kY2a = 1.0925484305920792f;   // sqrt(15 / pi) / 2
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5 / pi) / 4
constexpr float kY2c = 0.54627421529603959f;  // sqrt(15 / pi) / 4
constexpr float kY3a = 0.59004358992664352f;  // sqrt(35 / (2 pi)) / 4
constexpr float kY3b = 2.8906114426405538f;   // sqrt(105 / pi) / 2
constexpr float kY3c = 0.45704579946446572f;  // sqrt(21 / (2 pi)) / 4
constexpr float kY3d = 0.37317633259011540f;  // sqrt(7 / pi) / 4
constexpr float kY3e = 1.4453057213202769f;   // sqrt(105 / pi) / 4

// Y[k], k < (D+1)^2, at the unit direction (x, y, z).
template <int D>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float *Y) {
    Y[0] = kY00;
    if (D >= 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (D >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;
        Y[5] = -kY2a * y * z;
        Y[6] = kY2b * (2.f * zz - xx - yy);
        Y[7] = -kY2a * x * z;
        Y[8] = kY2c * (xx - yy);
        if (D >= 3) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            Y[10] = kY3b * x * y * z;
            Y[11] = -kY3c * y * (4.f * zz - xx - yy);
            Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kY3c * x * (4.f * zz - xx - yy);
            Y[14] = kY3e * z * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
        }
    }
}

// Adds w_k * grad Y_k (the polynomial's gradient, x, y, z independent) to g for k < (D+1)^2.
template <int D>
__device__ __forceinline__ void sh_grad_acc(float x, float y, float z, const float *w, float3 &g) {
    if (D >= 1) {
        g.y -= kY1 * w[1];
        g.z += kY1 * w[2];
        g.x -= kY1 * w[3];
    }
    if (D >= 2) {
        g.x += kY2a * y * w[4];
        g.y += kY2a * x * w[4];
        g.y -= kY2a * z * w[5];
        g.z -= kY2a * y * w[5];
        g.x -= 2.f * kY2b * x * w[6];
        g.y -= 2.f * kY2b * y * w[6];
        g.z += 4.f * kY2b * z * w[6];
        g.x -= kY2a * z * w[7];
        g.z -= kY2a * x * w[7];
        g.x += 2.f * kY2c * x * w[8];
        g.y -= 2.f * kY2c * y * w[8];
        if (D >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            // Y9 = -a (3 x^2 y - y^3)
            g.x -= 6.f * kY3a * x * y * w[9];
            g.y -= 3.f * kY3a * (xx - yy) * w[9];
            // Y10 = b x y z
            g.x += kY3b * y * z * w[10];
            g.y += kY3b * x * z * w[10];
            g.z += kY3b * x * y * w[10];
            // Y11 = -c (4 y z^2 - x^2 y - y^3)
            g.x += 2.f * kY3c * x * y * w[11];
            g.y -= kY3c * (4.f * zz - xx - 3.f * yy) * w[11];
            g.z -= 8.f * kY3c * y * z * w[11];
            // Y12 = d (2 z^3 - 3 x^2 z - 3 y^2 z)
            g.x -= 6.f * kY3d * x * z * w[12];
            g.y -= 6.f * kY3d * y * z * w[12];
            g.z += 3.f * kY3d * (2.f * zz - xx - yy) * w[12];
            // Y13 = -c (4 x z^2 - x^3 - x y^2)
            g.x -= kY3c * (4.f * zz - 3.f * xx - yy) * w[13];
            g.y += 2.f * kY3c * x * y * w[13];
            g.z -= 8.f * kY3c * x * z * w[13];
            // Y14 = e z (x^2 - y^2)
            g.x += 2.f * kY3e * x * z * w[14];
            g.y -= 2.f * kY3e * y * z * w[14];
            g.z += kY3e * (xx - yy) * w[14];
            // Y15 = -a (x^3 - 3 x y^2)
            g.x -= 3.f * kY3a * (xx - yy) * w[15];
            g.y += 6.f * kY3a * x * y * w[15];
        }
    }
}

struct ShViews {
    int V;
    float cx[kMaxViews], cy[kMaxViews], cz[kMaxViews];  // camera centres
};

// The K = (D+1)^2 coefficient rows of Gaussian i (row stride `stride` rows of 3 floats).
template <int D, bool Vec>
__device__ __forceinline__ void load_sh(const float *__restrict__ sh, long long i, int stride, float *c) {
    constexpr int K = (D + 1) * (D + 1);
    const float *p = sh + (size_t)i * stride * 3;
    if (Vec) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int j = 0; j < (3 * K) / 4; ++j) {
            const float4 v = __ldg(q + j);
            c[4 * j] = v.x;
            c[4 * j + 1] = v.y;
            c[4 * j + 2] = v.z;
            c[4 * j + 3] = v.w;
        }
#pragma unroll
        for (int j = (3 * K) / 4 * 4; j < 3 * K; ++j) c[j] = __ldg(p + j);
    } else {
#pragma unroll
        for (int j = 0; j < 3 * K; ++j) c[j] = __ldg(p + j);
    }
}

__device__ __forceinline__ float3 unit_dir(float3 m, const ShViews &cv, int v, float &len) {
    const float ux = m.x - cv.cx[v], uy = m.y - cv.cy[v], uz = m.z - cv.cz[v];
    len = sqrtf(ux * ux + uy * uy + uz * uz);
    const float il = 1.f / len;
    return make_float3(ux * il, uy * il, uz * il);
}

template <int D, bool Vec>
__global__ void __launch_bounds__(256) k_sh_forward(long long N, int stride, const float *__restrict__ sh,
                                                    const float *__restrict__ means3D, ShViews cv,
                                                    float *__restrict__ rgb, uint8_t *__restrict__ clamped) {
    constexpr int K = (D + 1) * (D + 1);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float c[3 * K];
    load_sh<D, Vec>(sh, i, stride, c);
    const float3 m = make_float3(means3D[3 * i], means3D[3 * i + 1], means3D[3 * i + 2]);
    for (int v = 0; v < cv.V; ++v) {
        float len;
        const float3 d = unit_dir(m, cv, v, len);
        float Y[K];
        sh_eval<D>(d.x, d.y, d.z, Y);
        const size_t o = ((size_t)v * N + i) * 3;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float s = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) s = fmaf(Y[k], c[3 * k + ch], s);
            rgb[o + ch] = fmaxf(s, 0.f);
            if (clamped) clamped[o + ch] = s < 0.f ? 1 : 0;
        }
    }
}

// dL/dsh [N, stride, 3] (rows K .. stride-1 zeroed) and dL/dmeans3D [N, 3], summed over the
// views: dL/dsh[k][c] = Y_k g_c and dL/du = (dL/dd - (dL/dd . d) d) / |u| with
// dL/dd = sum_k (sum_c sh[k][c] g_c) grad Y_k, u = mean - campos, d = u / |u|, and
// g_c = dL/drgb_c unless the channel was clamped.
template <int D, bool Vec>
__global__ void __launch_bounds__(256) k_sh_backward(long long N, int stride, const float *__restrict__ sh,
                                                     const float *__restrict__ means3D, ShViews cv,
                                                     const float *__restrict__ dL_drgb, float *__restrict__ dL_dsh,
                                                     float *__restrict__ dL_dmeans3D) {
    constexpr int K = (D + 1) * (D + 1);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float c[3 * K], acc[3 * K];
    load_sh<D, Vec>(sh, i, stride, c);
#pragma unroll
    for (int j = 0; j < 3 * K; ++j) acc[j] = 0.f;
    const float3 m = make_float3(means3D[3 * i], means3D[3 * i + 1], means3D[3 * i + 2]);
    float3 gm = make_float3(0.f, 0.f, 0.f);
    for (int v = 0; v < cv.V; ++v) {
        float len;
        const float3 d = unit_dir(m, cv, v, len);
        float Y[K];
        sh_eval<D>(d.x, d.y, d.z, Y);
        const size_t o = ((size_t)v * N + i) * 3;
        float g[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float s = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) s = fmaf(Y[k], c[3 * k + ch], s);
            g[ch] = s < 0.f ? 0.f : dL_drgb[o + ch];
        }
        float w[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            w[k] = c[3 * k] * g[0] + c[3 * k + 1] * g[1] + c[3 * k + 2] * g[2];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) acc[3 * k + ch] = fmaf(Y[k], g[ch], acc[3 * k + ch]);
        }
        float3 gd = make_float3(0.f, 0.f, 0.f);
        sh_grad_acc<D>(d.x, d.y, d.z, w, gd);
        const float dot = gd.x * d.x + gd.y * d.y + gd.z * d.z;
        const float il = 1.f / len;
        gm.x += (gd.x - dot * d.x) * il;
        gm.y += (gd.y - dot * d.y) * il;
        gm.z += (gd.z - dot * d.z) * il;
    }
    float *q = dL_dsh + (size_t)i * stride * 3;
    if (Vec) {
        float4 *q4 = reinterpret_cast<float4 *>(q);
#pragma unroll
        for (int j = 0; j < (3 * K) / 4; ++j)
            q4[j] = make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]);
#pragma unroll
        for (int j = (3 * K) / 4 * 4; j < 3 * K; ++j) q[j] = acc[j];
    } else {
#pragma unroll
        for (int j = 0; j < 3 * K; ++j) q[j] = acc[j];
    }
    for (int j = 3 * K; j < 3 * stride; ++j) q[j] = 0.f;
    dL_dmeans3D[3 * i] = gm.x;
    dL_dmeans3D[3 * i + 1] = gm.y;
    dL_dmeans3D[3 * i + 2] = gm.z;
}

// ---- staged kernels ----------------------------------------------------------------------
constexpr int kShBlock = 256;

template <int D>
__host__ __device__ constexpr int sh_row_pad() { return 3 * (D + 1) * (D + 1) + 1; }

// Copies the warp's nG Gaussians' coefficients (nG * F contiguous floats from Gaussian g0,
// F = 3 (D+1)^2 a multiple of 4, 16-byte aligned) into rows of F + 1 floats.
template <int D>
__device__ __forceinline__ void stage_sh(const float *__restrict__ sh, long long g0, int nG, float *s_sh, int lane) {
    constexpr int F = 3 * (D + 1) * (D + 1), P = sh_row_pad<D>();
    const float4 *src = reinterpret_cast<const float4 *>(sh + g0 * F);
    const int n4 = nG * F / 4;
    for (int c = lane; c < n4; c += 32) {
        const float4 v = __ldg(src + c);
        const int f = 4 * c, g = f / F, w = f - g * F;
        float *d = s_sh + g * P + w;
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
    }
    __syncwarp();
}

// Single view: dL/dsh overwrites the lane's staged row, then the warp stores its rows.
template <int D>
__global__ void __launch_bounds__(kShBlock) k_sh_backward_staged(long long N, const float *__restrict__ sh,
                                                                 const float *__restrict__ means3D, ShViews cv,
                                                                 const float *__restrict__ dL_drgb,
                                                                 float *__restrict__ dL_dsh,
                                                                 float *__restrict__ dL_dmeans3D) {
    constexpr int K = (D + 1) * (D + 1), F = 3 * K, P = sh_row_pad<D>();
    extern __shared__ float s_sh[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long g0 = (long long)blockIdx.x * kShBlock + 32 * warp;
    if (g0 >= N) return;  // whole warp
    const int nG = (int)min(32ll, N - g0);
    float *buf = s_sh + warp * 32 * P;
    stage_sh<D>(sh, g0, nG, buf, lane);
    if (lane < nG) {
        const long long i = g0 + lane;
        float *c = buf + lane * P;
        const float3 m = make_float3(means3D[3 * i], means3D[3 * i + 1], means3D[3 * i + 2]);
        float len;
        const float3 d = unit_dir(m, cv, 0, len);
        float Y[K];
        sh_eval<D>(d.x, d.y, d.z, Y);
        float g[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float s = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) s = fmaf(Y[k], c[3 * k + ch], s);
            g[ch] = s < 0.f ? 0.f : dL_drgb[3 * i + ch];
        }
        float w[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            w[k] = c[3 * k] * g[0] + c[3 * k + 1] * g[1] + c[3 * k + 2] * g[2];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) c[3 * k + ch] = Y[k] * g[ch];
        }
        float3 gd = make_float3(0.f, 0.f, 0.f);
        sh_grad_acc<D>(d.x, d.y, d.z, w, gd);
        const float dot = gd.x * d.x + gd.y * d.y + gd.z * d.z;
        const float il = 1.f / len;
        dL_dmeans3D[3 * i] = (gd.x - dot * d.x) * il;
        dL_dmeans3D[3 * i + 1] = (gd.y - dot * d.y) * il;
        dL_dmeans3D[3 * i + 2] = (gd.z - dot * d.z) * il;
    }
    __syncwarp();
    float4 *dst = reinterpret_cast<float4 *>(dL_dsh + g0 * F);
    const int n4 = nG * F / 4;
    for (int q = lane; q < n4; q += 32) {
        const int f = 4 * q, g = f / F, w = f - g * F;
        const float *r = buf + g * P + w;
        dst[q] = make_float4(r[0], r[1], r[2], r[3]);
    }
}

template <int D>
static cudaError_t launch_sh_d(bool backward, long long N, int stride, const float *sh, const float *means3D,
                               const ShViews &cv, float *rgb, uint8_t *clamped, const float *dL_drgb,
                               float *dL_dsh, float *dL_dmeans3D, cudaStream_t s) {
    const unsigned blocks = (unsigned)((N + 255) / 256);
    // float4 rows: the sh pointer and every Gaussian's block of 3 * stride floats 16-byte aligned
    const bool vec = (reinterpret_cast<uintptr_t>(sh) & 15u) == 0u && (3 * stride) % 4 == 0 &&
                     (!backward || (reinterpret_cast<uintptr_t>(dL_dsh) & 15u) == 0u);
    // staged: exactly the used rows (contiguous blocks of Gaussians), float4-able
    constexpr int K = (D + 1) * (D + 1);
    if (vec && stride == K && (3 * K) % 4 == 0 && backward && cv.V == 1) {
        const size_t smem = sizeof(float) * kShBlock * sh_row_pad<D>();
        cudaError_t e = cudaFuncSetAttribute((const void *)k_sh_backward_staged<D>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_sh_backward_staged<D><<<blocks, kShBlock, smem, s>>>(N, sh, means3D, cv, dL_drgb, dL_dsh, dL_dmeans3D);
        return cudaGetLastError();
    }
    if (!backward) {
        if (vec) k_sh_forward<D, true><<<blocks, 256, 0, s>>>(N, stride, sh, means3D, cv, rgb, clamped);
        else k_sh_forward<D, false><<<blocks, 256, 0, s>>>(N, stride, sh, means3D, cv, rgb, clamped);
    } else {
        if (vec)
            k_sh_backward<D, true><<<blocks, 256, 0, s>>>(N, stride, sh, means3D, cv, dL_drgb, dL_dsh, dL_dmeans3D);
        else
            k_sh_backward<D, false><<<blocks, 256, 0, s>>>(N, stride, sh, means3D, cv, dL_drgb, dL_dsh, dL_dmeans3D);
    }
    return cudaGetLastError();
}

cudaError_t launch_sh(bool backward, long long N, int degree, int stride, const float *sh, const float *means3D,
                      int V, const float *campos, float *rgb, uint8_t *clamped, const float *dL_drgb, float *dL_dsh,
                      float *dL_dmeans3D, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    if (V < 1 || V > kMaxViews) return cudaErrorInvalidValue;
    ShViews cv;
    cv.V = V;
    for (int v = 0; v < V; ++v) {
        cv.cx[v] = campos[3 * v];
        cv.cy[v] = campos[3 * v + 1];
        cv.cz[v] = campos[3 * v + 2];
    }
    switch (degree) {
        case 0: return launch_sh_d<0>(backward, N, stride, sh, means3D, cv, rgb, clamped, dL_drgb, dL_dsh, dL_dmeans3D, s);
        case 1: return launch_sh_d<1>(backward, N, stride, sh, means3D, cv, rgb, clamped, dL_drgb, dL_dsh, dL_dmeans3D, s);
        case 2: return launch_sh_d<2>(backward, N, stride, sh, means3D, cv, rgb, clamped, dL_drgb, dL_dsh, dL_dmeans3D, s);
        case 3: return launch_sh_d<3>(backward, N, stride, sh, means3D, cv, rgb, clamped, dL_drgb, dL_dsh, dL_dmeans3D, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bgs
