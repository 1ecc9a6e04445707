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
// For a power-of-two tile side the quotient is the product by its exact reciprocal.
__device__ __forceinline__ float tile_quot(float a, int t) {
    return (t & (t - 1)) == 0 ? __fmul_rn(a, 1.f / (float)t) : __fdiv_rn(a, (float)t);
}

__device__ __forceinline__ void tile_rect(float u, float v, int r, int tw, int th, int tx, int ty, int &x0,
                                          int &x1, int &y0, int &y1) {
    x0 = (int)floorf(tile_quot(__fsub_rn(u, (float)r), tw));
    x1 = (int)floorf(tile_quot(__fadd_rn(u, (float)(r + tw - 1)), tw));
    y0 = (int)floorf(tile_quot(__fsub_rn(v, (float)r), th));
    y1 = (int)floorf(tile_quot(__fadd_rn(v, (float)(r + th - 1)), th));
    x0 = min(max(x0, 0), tx);
    x1 = min(max(x1, 0), tx);
    y0 = min(max(y0, 0), ty);
    y1 = min(max(y1, 0), ty);
}

// FP32 intermediates of one Gaussian's projection into one view (Eq. 1-3): the forward
// kernel reads the outputs, the backward kernel recomputes them to apply the chain rule.
struct Proj {
    float tx, ty, tz, iz;          // camera-space centre, 1 / z
    float qw, qx, qy, qz, qn;      // normalised quaternion and the input's norm
    float R[3][3], s[3];           // rotation, scales
    float M[3][3];                 // R S
    float clx, cly;                // tangents of the centre, clamped
    bool in_x, in_y;               // ... and whether the clamp is inactive
    float J00, J02, J11, J12;      // pinhole Jacobian at the clamped centre
    float T[2][3];                 // J W
    float Q[2][3];                 // T R
    float P[2][3];                 // T R S = Q S: Sigma' (before the low-pass) = P P^T
    float c00, c01, c11, det;      // 2D covariance (+ low-pass) and its determinant
};

// The view-independent part of a Gaussian's projection: the normalised quaternion, R, the
// scales and M = R S (computed once per Gaussian, then shared by its views).
__device__ __forceinline__ void gauss_frame(const float *__restrict__ log_scales, const float *__restrict__ quats,
                                            long long g, Proj &o) {
    // R from the normalised quaternion (w, x, y, z)
    float qw = quats[4 * g], qx = quats[4 * g + 1], qy = quats[4 * g + 2], qz = quats[4 * g + 3];
    o.qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw /= o.qn; qx /= o.qn; qy /= o.qn; qz /= o.qn;
    o.qw = qw; o.qx = qx; o.qy = qy; o.qz = qz;
    o.R[0][0] = 1.f - 2.f * (qy * qy + qz * qz); o.R[0][1] = 2.f * (qx * qy - qw * qz); o.R[0][2] = 2.f * (qx * qz + qw * qy);
    o.R[1][0] = 2.f * (qx * qy + qw * qz); o.R[1][1] = 1.f - 2.f * (qx * qx + qz * qz); o.R[1][2] = 2.f * (qy * qz - qw * qx);
    o.R[2][0] = 2.f * (qx * qz - qw * qy); o.R[2][1] = 2.f * (qy * qz + qw * qx); o.R[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
    o.s[0] = expf(log_scales[3 * g]);
    o.s[1] = expf(log_scales[3 * g + 1]);
    o.s[2] = expf(log_scales[3 * g + 2]);
    // M = R S (Sigma = M M^T is never formed: Sigma' = T M (T M)^T below)
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) o.M[r][k] = o.R[r][k] * o.s[k];
}

// The projection of a Gaussian with centre p (world space) and frame o (gauss_frame) into one
// view.  Returns false when the Gaussian is culled (z <= near or det <= 0); tz is always set.
__device__ __forceinline__ bool project(const CamDev &cam, float px, float py, float pz, Proj &o) {
    const float *V = cam.V;
    o.tx = V[0] * px + V[1] * py + V[2] * pz + V[3];
    o.ty = V[4] * px + V[5] * py + V[6] * pz + V[7];
    o.tz = V[8] * px + V[9] * py + V[10] * pz + V[11];
    if (!(o.tz > cam.near_plane)) return false;
    // Jacobian of the pinhole map at the tangent-clamped point
    o.iz = 1.f / o.tz;
    const float ux = o.tx * o.iz, uy = o.ty * o.iz;
    o.in_x = ux >= -cam.lim_x && ux <= cam.lim_x;
    o.in_y = uy >= -cam.lim_y && uy <= cam.lim_y;
    o.clx = fminf(cam.lim_x, fmaxf(-cam.lim_x, ux));
    o.cly = fminf(cam.lim_y, fmaxf(-cam.lim_y, uy));
    const float xc = o.clx * o.tz, yc = o.cly * o.tz;
    o.J00 = cam.fx * o.iz;
    o.J02 = -cam.fx * xc * o.iz * o.iz;
    o.J11 = cam.fy * o.iz;
    o.J12 = -cam.fy * yc * o.iz * o.iz;
    // T = J W (2x3)
    o.T[0][0] = o.J00 * V[0] + o.J02 * V[8];
    o.T[0][1] = o.J00 * V[1] + o.J02 * V[9];
    o.T[0][2] = o.J00 * V[2] + o.J02 * V[10];
    o.T[1][0] = o.J11 * V[4] + o.J12 * V[8];
    o.T[1][1] = o.J11 * V[5] + o.J12 * V[9];
    o.T[1][2] = o.J11 * V[6] + o.J12 * V[10];
    const float (&T)[2][3] = o.T;
    // Sigma' = T Sigma T^T = P P^T with P = T R S, written without cancellation: the diagonal
    // entries are sums of squares, and the determinant comes from the Cauchy-Binet formula
    // det(P P^T) = sum of the squared 2x2 minors of P.  The minors of P = Q S are s_i s_j
    // times those of Q = T R, i.e. the components of R^T (t0 x t1) for the rows t0, t1 of
    // T.  So det(Sigma' + l I) = det(P P^T) + l (A + C) + l^2 is a sum of positive terms,
    // accurate to a few ulp even for long, thin Gaussians (A C - B^2 computed directly
    // cancels by a factor of up to ~10^4 there).
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o.Q[r][k] = T[r][0] * o.R[0][k] + T[r][1] * o.R[1][k] + T[r][2] * o.R[2][k];
            o.P[r][k] = o.Q[r][k] * o.s[k];
        }
    const float (&P)[2][3] = o.P;
    const float A0 = P[0][0] * P[0][0] + P[0][1] * P[0][1] + P[0][2] * P[0][2];
    const float C0 = P[1][0] * P[1][0] + P[1][1] * P[1][1] + P[1][2] * P[1][2];
    o.c01 = P[0][0] * P[1][0] + P[0][1] * P[1][1] + P[0][2] * P[1][2];
    o.c00 = A0 + cam.lowpass;
    o.c11 = C0 + cam.lowpass;
    const float n0 = T[0][1] * T[1][2] - T[0][2] * T[1][1];  // t0 x t1
    const float n1 = T[0][2] * T[1][0] - T[0][0] * T[1][2];
    const float n2 = T[0][0] * T[1][1] - T[0][1] * T[1][0];
    const float m0 = o.R[0][0] * n0 + o.R[1][0] * n1 + o.R[2][0] * n2;  // R^T (t0 x t1)
    const float m1 = o.R[0][1] * n0 + o.R[1][1] * n1 + o.R[2][1] * n2;
    const float m2 = o.R[0][2] * n0 + o.R[1][2] * n1 + o.R[2][2] * n2;
    const float d0 = o.s[1] * o.s[2] * m0, d1 = o.s[0] * o.s[2] * m1, d2 = o.s[0] * o.s[1] * m2;
    o.det = (d0 * d0 + d1 * d1 + d2 * d2) + cam.lowpass * (A0 + C0) + cam.lowpass * cam.lowpass;
    return o.det > 0.f;
}

// Record i = v * N + g projects Gaussian g into view v (one view for the single-view call).
// A thread per Gaussian, over the views: the Gaussian's parameters are read from DRAM once
// (the views' later reads hit L1), and record v N + g of every view is written (coalesced
// per view).
__global__ void __launch_bounds__(256) k_preprocess(long long N, const float *__restrict__ means3D,
                                                    const float *__restrict__ log_scales,
                                                    const float *__restrict__ quats,
                                                    const float *__restrict__ opacities, const CamTable ct,
                                                    float2 *__restrict__ means2D, float4 *__restrict__ conic_opacity,
                                                    float *__restrict__ depths, int *__restrict__ radii,
                                                    uint32_t *__restrict__ tiles_touched) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    const float op = opacities[g];
    const float px = means3D[3 * g], py = means3D[3 * g + 1], pz = means3D[3 * g + 2];
    Proj frame;
    gauss_frame(log_scales, quats, g, frame);
    for (int view = 0; view < ct.V; ++view) {
        const long long rec = (long long)view * N + g;
        const CamDev &cam = ct.cam[view];
        Proj o = frame;
        const bool ok = project(cam, px, py, pz, o);
        float2 m2 = make_float2(0.f, 0.f);
        float4 co = make_float4(0.f, 0.f, 0.f, 0.f);
        int radius = 0;
        uint32_t touched = 0;
        depths[rec] = o.tz;
        if (ok) {
            const float mid = 0.5f * (o.c00 + o.c11);
            // mid^2 - det = ((A - C) / 2)^2 + B^2, written without cancellation
            const float hd = 0.5f * (o.c00 - o.c11);
            const float lam = mid + sqrtf(fmaxf(0.1f, hd * hd + o.c01 * o.c01));
            const int r = (int)ceilf(3.f * sqrtf(lam));
            const float idet = 1.f / o.det;
            const float u = cam.fx * o.tx * o.iz + cam.cx, v = cam.fy * o.ty * o.iz + cam.cy;
            m2 = make_float2(u, v);
            co = make_float4(o.c11 * idet, -o.c01 * idet, o.c00 * idet, op);
            int x0, x1, y0, y1;
            tile_rect(u, v, r, cam.tile_w, cam.tile_h, cam.tiles_x, cam.tiles_y, x0, x1, y0, y1);
            const long long area = (long long)(x1 - x0) * (long long)(y1 - y0);
            if (area > 0) {
                radius = r;
                touched = (uint32_t)area;
            }
        }
        means2D[rec] = m2;
        conic_opacity[rec] = co;
        radii[rec] = radius;
        tiles_touched[rec] = touched;
    }
}

// Projection backward: thread per Gaussian, summing its records over the views.  Records
// with radius 0 pass no gradient.  The chain rule through the projection above:
//   conic = (C, -B, A) / det of C2 = (A B; B C), det = A C - B^2;
//   C2 = T Sigma T^T + lowpass I with T = J W: dL/dSigma = T^T G T, dL/dT = 2 G T Sigma
//     (G = dL/dC2, its off-diagonal entry half of dL/dB);
//   J(t) at the clamped tangent (the clamped coordinate carries no x / y gradient);
//   means2D = (fx x / z + cx, fy y / z + cy), depth = z, t = W p + w;
//   Sigma = M M^T, M = R S: dL/dM = 2 dL/dSigma M, dL/dlog s_k = s_k sum_r dL/dM_rk R_rk,
//   dL/dR = dL/dM S, then R(q) and the Jacobian of q / |q|.
__global__ void __launch_bounds__(256) k_preprocess_backward(long long N, const float *__restrict__ means3D,
                                                             const float *__restrict__ log_scales,
                                                             const float *__restrict__ quats, const CamTable ct,
                                                             const int *__restrict__ radii,
                                                             const float2 *__restrict__ dL_dmeans2D,
                                                             const float *__restrict__ dL_dconic,
                                                             const float *__restrict__ dL_ddepths,
                                                             float *__restrict__ dL_dmeans3D,
                                                             float *__restrict__ dL_dlog_scales,
                                                             float *__restrict__ dL_dquats) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    float gp[3] = {0.f, 0.f, 0.f}, gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
    const float px = means3D[3 * g], py = means3D[3 * g + 1], pz = means3D[3 * g + 2];
    Proj frame;
    gauss_frame(log_scales, quats, g, frame);
    for (int view = 0; view < ct.V; ++view) {
        const long long rec = (long long)view * N + g;
        if (radii[rec] <= 0) continue;
        const CamDev &cam = ct.cam[view];
        Proj o = frame;
        if (!project(cam, px, py, pz, o)) continue;
        const float *V = cam.V;
        const float2 gm = dL_dmeans2D[rec];
        const float ga = dL_dconic[3 * rec], gb = dL_dconic[3 * rec + 1], gc = dL_dconic[3 * rec + 2];
        const float iz2 = o.iz * o.iz;
        // means2D and depth
        float gtx = gm.x * cam.fx * o.iz, gty = gm.y * cam.fy * o.iz;
        float gtz = (dL_ddepths ? dL_ddepths[rec] : 0.f) - (gm.x * cam.fx * o.tx + gm.y * cam.fy * o.ty) * iz2;
        // conic -> G = dL/dC2
        const float A = o.c00, B = o.c01, C = o.c11;
        const float idet = 1.f / o.det, id2 = idet * idet;
        const float dA = (-C * C * ga + B * C * gb - B * B * gc) * id2;
        const float dC = (-B * B * ga + A * B * gb - A * A * gc) * id2;
        const float hB = (B * C * ga - B * B * gb + A * B * gc) * id2 - 0.5f * gb * idet;  // dL/dB / 2
        // with G = dL/dC2 and Sigma' = P P^T, P = T R S = Q S (no Sigma formed):
        //   dL/dT = 2 G T Sigma = 2 (G P) M^T,
        //   dL/dM = 2 T^T G T M, so dL/dlog s_k = 2 s_k^2 q_k^T G q_k (q_k: column k of Q)
        //   and dL/dR_rk = 2 s_k^2 (T^T G q_k)_r
        const float (&T)[2][3] = o.T;
        const float (&P)[2][3] = o.P;
        const float (&Q)[2][3] = o.Q;
        float GP[2][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            GP[0][k] = dA * P[0][k] + hB * P[1][k];
            GP[1][k] = hB * P[0][k] + dC * P[1][k];
        }
        float gT[2][3];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                gT[r][k] = 2.f * (GP[r][0] * o.M[k][0] + GP[r][1] * o.M[k][1] + GP[r][2] * o.M[k][2]);
        // T = J W: the four nonzero entries of J
        const float gJ00 = gT[0][0] * V[0] + gT[0][1] * V[1] + gT[0][2] * V[2];
        const float gJ02 = gT[0][0] * V[8] + gT[0][1] * V[9] + gT[0][2] * V[10];
        const float gJ11 = gT[1][0] * V[4] + gT[1][1] * V[5] + gT[1][2] * V[6];
        const float gJ12 = gT[1][0] * V[8] + gT[1][1] * V[9] + gT[1][2] * V[10];
        // J00 = fx / z, J02 = -fx cl(x / z) / z, J11 = fy / z, J12 = -fy cl(y / z) / z
        gtz += (-gJ00 * cam.fx - gJ11 * cam.fy + gJ02 * cam.fx * o.clx + gJ12 * cam.fy * o.cly) * iz2;
        if (o.in_x) {
            gtx -= gJ02 * cam.fx * iz2;
            gtz += gJ02 * cam.fx * o.tx * iz2 * o.iz;
        }
        if (o.in_y) {
            gty -= gJ12 * cam.fy * iz2;
            gtz += gJ12 * cam.fy * o.ty * iz2 * o.iz;
        }
        // t = W p + w
#pragma unroll
        for (int k = 0; k < 3; ++k) gp[k] += V[k] * gtx + V[4 + k] * gty + V[8 + k] * gtz;
        // Sigma = M M^T, M = R S
        float gR[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float g0 = dA * Q[0][k] + hB * Q[1][k], g1 = hB * Q[0][k] + dC * Q[1][k];  // G q_k
            const float s2 = 2.f * o.s[k] * o.s[k];
            gls[k] += s2 * (Q[0][k] * g0 + Q[1][k] * g1);
#pragma unroll
            for (int r = 0; r < 3; ++r) gR[r][k] = s2 * (T[0][r] * g0 + T[1][r] * g1);
        }
        // R(q) of the normalised quaternion, then d(q / |q|)
        const float w = o.qw, x = o.qx, y = o.qy, z = o.qz;
        float dq[4];
        dq[0] = 2.f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
        dq[1] = 2.f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.f * x * gR[1][1] - w * gR[1][2] + z * gR[2][0] +
                       w * gR[2][1] - 2.f * x * gR[2][2]);
        dq[2] = 2.f * (-2.f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] -
                       w * gR[2][0] + z * gR[2][1] - 2.f * y * gR[2][2]);
        dq[3] = 2.f * (-2.f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2.f * z * gR[1][1] +
                       y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
        const float dot = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
        const float iqn = 1.f / o.qn;
        gq[0] += (dq[0] - w * dot) * iqn;
        gq[1] += (dq[1] - x * dot) * iqn;
        gq[2] += (dq[2] - y * dot) * iqn;
        gq[3] += (dq[3] - z * dot) * iqn;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dL_dmeans3D[3 * g + k] = gp[k];
        dL_dlog_scales[3 * g + k] = gls[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) dL_dquats[4 * g + k] = gq[k];
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
    const long long blocks = (N + threads - 1) / threads;
    k_preprocess<<<(unsigned)blocks, threads, 0, s>>>(N, means3D, log_scales, quats, opacities, ct,
                                                       reinterpret_cast<float2 *>(means2D),
                                                       reinterpret_cast<float4 *>(conic_opacity), depths, radii,
                                                       tiles_touched);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_backward(long long N, int V, const float *means3D, const float *log_scales,
                                       const float *quats, const bgs_camera *cams, const int *radii,
                                       const float *dL_dmeans2D, const float *dL_dconic, const float *dL_ddepths,
                                       float *dL_dmeans3D, float *dL_dlog_scales, float *dL_dquats, cudaStream_t s) {
    if (V < 1 || V > kMaxViews) return cudaErrorInvalidValue;
    CamTable ct;
    ct.V = V;
    for (int v = 0; v < V; ++v) ct.cam[v] = cam_dev(cams[v], 16, 16);
    if (N == 0) return cudaSuccess;
    k_preprocess_backward<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
        N, means3D, log_scales, quats, ct, radii, reinterpret_cast<const float2 *>(dL_dmeans2D), dL_dconic,
        dL_ddepths, dL_dmeans3D, dL_dlog_scales, dL_dquats);
    return cudaGetLastError();
}

// idx[i] = i for i in [lo, hi): the values of the batched depth sort (its keys are the depths'
// float32 bit patterns themselves), filled once and kept by the plan.
__global__ void __launch_bounds__(256) k_iota(long long lo, long long hi, uint32_t *__restrict__ idx) {
    const long long i = lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < hi) idx[i] = (uint32_t)i;
}

cudaError_t launch_iota(long long lo, long long hi, uint32_t *idx, cudaStream_t s) {
    if (hi <= lo) return cudaSuccess;
    k_iota<<<(unsigned)((hi - lo + 255) / 256), 256, 0, s>>>(lo, hi, idx);
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
// A thread per record on a grid of (colour rows, views): record v n_colors + c of view
// blockIdx.y = v takes colour row c, with no division.
__global__ void __launch_bounds__(256) k_pack(long long n_colors, const float *__restrict__ means2D,
                                              const float *__restrict__ conic_opacity,
                                              const float *__restrict__ colors, const float *__restrict__ depths,
                                              Rec *__restrict__ recs) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_colors) return;
    const long long i = (long long)blockIdx.y * n_colors + c;
    recs[i] = make_rec(means2D, conic_opacity, colors, depths, (unsigned int)i, (unsigned int)c);
}

cudaError_t launch_pack(long long N, const float *means2D, const float *conic_opacity, const float *colors,
                        long long n_colors, const float *depths, Rec *recs, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    if (n_colors <= 0 || N % n_colors != 0 || N / n_colors > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((n_colors + 255) / 256), (unsigned)(N / n_colors));
    k_pack<<<grid, 256, 0, s>>>(n_colors, means2D, conic_opacity, colors, depths, recs);
    return cudaGetLastError();
}

}  // namespace bgs
