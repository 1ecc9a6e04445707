/*
 * oracle/orc.c -- plain, slow, FP64 CPU reference of the tile-based 3D Gaussian
 * Splatting rasterizer (projection, tile binning, front-to-back blending and
 * its analytic gradient).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * do.  It shares no code, header, table or constant generator with the CUDA
 * library: every formula here is written out again from the paper's equations
 * and the reading of them stated beside each function.
 *
 * Sources (Balanced 3DGS, arXiv 2412.17378):
 *   Eq. 1  3D Gaussian G(x) = exp(-1/2 (x-mu)^T Sigma^-1 (x-mu))         (Sec. 2.1)
 *   Eq. 2  EWA projection Sigma' = J W Sigma W^T J^T                     (Sec. 2.1)
 *   Eq. 3  2D Gaussian with the inverse of Sigma' (the "conic")          (Sec. 2.1)
 *   Eq. 4  front-to-back blending C = sum_i c_i a_i prod_{j<i} (1-a_j)   (Sec. 2.1)
 *   Algorithm 5 (Appendix A): the per-pixel sequential rule -- skip a pair whose
 *          power is > 0 or whose alpha is < 1/255; stop (without accumulating)
 *          at the first pair whose updated transmittance would fall below 1e-4.
 * Constants the paper leaves out ("computation details of power, alpha and t"
 * are omitted in Appendix A) follow standard 3DGS: alpha = min(0.99, o*G'),
 * radius = ceil(3 sqrt(lambda_max)) with the discriminant floored at 0.1, a
 * +lowpass term on the 2D covariance diagonal, near cull at z <= near, and the
 * Jacobian tangent clamp at 1.3 tan(fov/2).
 *
 * Precision: every continuous quantity is computed in double.  Integer
 * decisions that the GPU takes in float32 (the tile rectangle of a Gaussian)
 * are taken here in float32 as well, with the same operation order, so that
 * binning can be compared bit for bit.  Build with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_ALPHA_MIN (1.0 / 255.0)
#define ORC_ALPHA_MAX 0.99
#define ORC_T_MIN 1e-4

/* ambiguity flags written per pixel by the forward (see orc_render) */
#define ORC_FLAG_ALPHA_EDGE 1u   /* a visited pair has |alpha - 1/255| < 1e-6       */
#define ORC_FLAG_T_EDGE 2u       /* a visited pair has |T' - 1e-4| < 1e-9           */
#define ORC_FLAG_CLAMP_EDGE 4u   /* an accepted pair has |o*G - 0.99| < 1e-6        */
#define ORC_FLAG_POWER_EDGE 8u   /* a visited pair has |power| < 1e-9               */

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* Tile rectangle of a projected Gaussian (the binning step that Sec. 4.3's   */
/* footnote calls the "patch" pre-processing).  Reading: a Gaussian of       */
/* integer radius r centred at (u, v) covers tiles                           */
/*   x in [floor((u - r)/tw), floor((u + (r + tw - 1))/tw)) clamped to        */
/*   [0, tiles_x], likewise for y.  Float32 arithmetic, one rounding per op.  */
/* ------------------------------------------------------------------------- */
static void tile_rect(float u, float v, int r, int tiles_x, int tiles_y, int tw, int th,
                      int *x0, int *x1, int *y0, int *y1) {
    volatile float lo_x = u - (float)r;
    volatile float hi_x = u + (float)(r + tw - 1);
    volatile float lo_y = v - (float)r;
    volatile float hi_y = v + (float)(r + th - 1);
    volatile float qx0 = lo_x / (float)tw, qx1 = hi_x / (float)tw;
    volatile float qy0 = lo_y / (float)th, qy1 = hi_y / (float)th;
    int a = (int)floorf(qx0), b = (int)floorf(qx1);
    int c = (int)floorf(qy0), d = (int)floorf(qy1);
    if (a < 0) a = 0;
    if (a > tiles_x) a = tiles_x;
    if (b < 0) b = 0;
    if (b > tiles_x) b = tiles_x;
    if (c < 0) c = 0;
    if (c > tiles_y) c = tiles_y;
    if (d < 0) d = 0;
    if (d > tiles_y) d = tiles_y;
    *x0 = a; *x1 = b; *y0 = c; *y1 = d;
}

void orc_tile_rect(float u, float v, int r, int W, int H, int tw, int th, int32_t *out4) {
    int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    int a, b, c, d;
    tile_rect(u, v, r, tx, ty, tw, th, &a, &b, &c, &d);
    out4[0] = a; out4[1] = b; out4[2] = c; out4[3] = d;
}

/* Camera of the projection: rows 0..2 of the 4x4 row-major world->camera matrix V,
   intrinsics, near plane, low-pass and the tangent clamp lim = 1.3 tan(fov / 2). */
typedef struct {
    const double *V;
    double fx, fy, cx, cy, near_z, lowpass, lim_x, lim_y;
} orc_cam;

static orc_cam make_cam(const double *V, int W, int H, double fx, double fy, double cx, double cy, double near_z,
                        double lowpass) {
    orc_cam c;
    c.V = V;
    c.fx = fx; c.fy = fy; c.cx = cx; c.cy = cy;
    c.near_z = near_z;
    c.lowpass = lowpass;
    c.lim_x = 1.3 * ((double)W / (2.0 * fx));
    c.lim_y = 1.3 * ((double)H / (2.0 * fy));
    return c;
}

/* The intermediate values of one Gaussian's projection (Eq. 1-3).  Returns 0 when the
   Gaussian is culled (z <= near or a non-positive-definite 2D covariance). */
typedef struct {
    double t[3];          /* camera-space centre */
    double q[4], qn;      /* normalised quaternion (w, x, y, z) and the input's norm */
    double R[3][3], s[3]; /* rotation, scales */
    double M[3][3];       /* R S */
    double Sig[3][3];     /* 3D covariance (R S)(R S)^T */
    double J[2][3];       /* Jacobian of the pinhole map at the tangent-clamped point */
    int in_x, in_y;       /* tangent of the centre within the clamp */
    double Tm[2][3];      /* J W */
    double C2[2][2];      /* 2D covariance + low-pass */
    double det;
    double u, v, conic[3], rr;
} orc_proj;

static int project_one(const orc_cam *c, const double p[3], const double log_s[3], const double quat[4],
                       orc_proj *o) {
    const double *V = c->V;
    for (int r = 0; r < 3; ++r) o->t[r] = V[4 * r] * p[0] + V[4 * r + 1] * p[1] + V[4 * r + 2] * p[2] + V[4 * r + 3];
    if (!(o->t[2] > c->near_z)) return 0;
    o->qn = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    for (int k = 0; k < 4; ++k) o->q[k] = quat[k] / o->qn;
    const double qw = o->q[0], qx = o->q[1], qy = o->q[2], qz = o->q[3];
    const double R[3][3] = {
        {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
        {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
        {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
    memcpy(o->R, R, sizeof R);
    for (int k = 0; k < 3; ++k) o->s[k] = exp(log_s[k]);
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) o->M[r][k] = R[r][k] * o->s[k];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k)
            o->Sig[r][k] = o->M[r][0] * o->M[k][0] + o->M[r][1] * o->M[k][1] + o->M[r][2] * o->M[k][2];
    const double z = o->t[2];
    const double txz = o->t[0] / z, tyz = o->t[1] / z;
    o->in_x = txz >= -c->lim_x && txz <= c->lim_x;
    o->in_y = tyz >= -c->lim_y && tyz <= c->lim_y;
    const double xc = (txz < -c->lim_x ? -c->lim_x : (txz > c->lim_x ? c->lim_x : txz)) * z;
    const double yc = (tyz < -c->lim_y ? -c->lim_y : (tyz > c->lim_y ? c->lim_y : tyz)) * z;
    const double J[2][3] = {{c->fx / z, 0.0, -c->fx * xc / (z * z)}, {0.0, c->fy / z, -c->fy * yc / (z * z)}};
    memcpy(o->J, J, sizeof J);
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) o->Tm[r][k] = J[r][0] * V[k] + J[r][1] * V[4 + k] + J[r][2] * V[8 + k];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 2; ++k) {
            double acc = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += o->Tm[r][a] * o->Sig[a][b] * o->Tm[k][b];
            o->C2[r][k] = acc;
        }
    o->C2[0][0] += c->lowpass;
    o->C2[1][1] += c->lowpass;
    o->det = o->C2[0][0] * o->C2[1][1] - o->C2[0][1] * o->C2[1][0];
    if (!(o->det > 0.0)) return 0;
    double mid = 0.5 * (o->C2[0][0] + o->C2[1][1]);
    double disc = mid * mid - o->det;
    if (disc < 0.1) disc = 0.1;
    o->rr = 3.0 * sqrt(mid + sqrt(disc));
    o->u = c->fx * o->t[0] / z + c->cx;
    o->v = c->fy * o->t[1] / z + c->cy;
    o->conic[0] = o->C2[1][1] / o->det;
    o->conic[1] = -o->C2[0][1] / o->det;
    o->conic[2] = o->C2[0][0] / o->det;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Projection (Eq. 1-3, Sec. 2.1): camera-space centre t = W p + w, 3D        */
/* covariance Sigma = R S S^T R^T from the normalised quaternion (w, x, y, z) */
/* and exp(log_scale), 2D covariance J W Sigma W^T J^T (+ low-pass on the     */
/* diagonal) with J the pinhole Jacobian at the tangent-clamped centre, conic */
/* = its inverse (a, b, c), radius = ceil(3 sqrt(lambda_max)) with the        */
/* discriminant floored at 0.1, means2D = (fx x/z + cx, fy y/z + cy).        */
/* ------------------------------------------------------------------------- */
void orc_preprocess(int64_t N, const float *means3D, const float *log_scales, const float *quats,
                    const float *opacities, int W, int H, double fx, double fy, double cx, double cy,
                    const double *V, double near_z, double lowpass, int tw, int th,
                    double *means2D, double *conic_opacity, double *depth, int32_t *radius,
                    double *radius_raw, int32_t *tiles_touched) {
    const int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    const orc_cam cam = make_cam(V, W, H, fx, fy, cx, cy, near_z, lowpass);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        const double p[3] = {means3D[3 * i], means3D[3 * i + 1], means3D[3 * i + 2]};
        const double ls[3] = {log_scales[3 * i], log_scales[3 * i + 1], log_scales[3 * i + 2]};
        const double q[4] = {quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3]};
        orc_proj o;
        const int ok = project_one(&cam, p, ls, q, &o);
        means2D[2 * i] = means2D[2 * i + 1] = 0.0;
        for (int k = 0; k < 4; ++k) conic_opacity[4 * i + k] = 0.0;
        depth[i] = o.t[2];
        radius[i] = 0;
        radius_raw[i] = 0.0;
        tiles_touched[i] = 0;
        if (!ok) continue;
        const int r = (int)ceil(o.rr);
        means2D[2 * i] = o.u;
        means2D[2 * i + 1] = o.v;
        for (int k = 0; k < 3; ++k) conic_opacity[4 * i + k] = o.conic[k];
        conic_opacity[4 * i + 3] = opacities[i];
        radius_raw[i] = o.rr;
        int x0, x1, y0, y1;
        tile_rect((float)o.u, (float)o.v, r, tiles_x, tiles_y, tw, th, &x0, &x1, &y0, &y1);
        int64_t area = (int64_t)(x1 - x0) * (int64_t)(y1 - y0);
        if (area <= 0) continue;
        radius[i] = r;
        tiles_touched[i] = (int32_t)area;
    }
}

/* The same projection from FP64 inputs (means2D, conic (a, b, c), depth; valid = not
   culled), for finite differences of the projection backward. */
void orc_project64(int64_t N, const double *means3D, const double *log_scales, const double *quats, int W, int H,
                   double fx, double fy, double cx, double cy, const double *V, double near_z, double lowpass,
                   double *means2D, double *conic, double *depth, int32_t *valid) {
    const orc_cam cam = make_cam(V, W, H, fx, fy, cx, cy, near_z, lowpass);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        orc_proj o;
        valid[i] = project_one(&cam, means3D + 3 * i, log_scales + 3 * i, quats + 4 * i, &o);
        depth[i] = o.t[2];
        means2D[2 * i] = valid[i] ? o.u : 0.0;
        means2D[2 * i + 1] = valid[i] ? o.v : 0.0;
        for (int k = 0; k < 3; ++k) conic[3 * i + k] = valid[i] ? o.conic[k] : 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* Projection backward (not printed in the paper; the chain rule through     */
/* Eq. 2-3 as written above): given dL/d(means2D, conic a b c, depth) of     */
/* each Gaussian, dL/d(means3D, log_scales, quats).  Gaussians with          */
/* radius 0 (culled or off-screen) get zero.                                  */
/*   conic = inv(C2): with A, B, C the entries of C2 and det = AC - B^2,       */
/*     a = C/det, b = -B/det, c = A/det;                                      */
/*   C2 = T Sigma T^T + lowpass I, T = J W: dL/dSigma = T^T G T,               */
/*     dL/dT = 2 G T Sigma (G = dL/dC2 symmetric, off-diagonal = dL/dB / 2);   */
/*   J from the clamped centre: d/dx of the clamped tangent is 0 outside;     */
/*   Sigma = M M^T, M = R S: dL/dM = 2 dL/dSigma M; dL/ds = column sums of     */
/*     dL/dM * R; dL/dR = dL/dM S; R(q) from the normalised quaternion, then  */
/*     the normalisation's Jacobian; t = W p + w: dL/dp = W^T dL/dt.          */
/* ------------------------------------------------------------------------- */
void orc_preprocess_backward(int64_t N, const double *means3D, const double *log_scales, const double *quats,
                             int W, int H, double fx, double fy, double cx, double cy, const double *V,
                             double near_z, double lowpass, const int32_t *radius, const double *g_means2D,
                             const double *g_conic, const double *g_depth, double *g_means3D,
                             double *g_log_scales, double *g_quats) {
    const orc_cam cam = make_cam(V, W, H, fx, fy, cx, cy, near_z, lowpass);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int k = 0; k < 3; ++k) g_means3D[3 * i + k] = g_log_scales[3 * i + k] = 0.0;
        for (int k = 0; k < 4; ++k) g_quats[4 * i + k] = 0.0;
        if (radius && radius[i] <= 0) continue;
        orc_proj o;
        if (!project_one(&cam, means3D + 3 * i, log_scales + 3 * i, quats + 4 * i, &o)) continue;
        const double z = o.t[2];
        double gt[3] = {0.0, 0.0, g_depth ? g_depth[i] : 0.0};
        /* means2D */
        const double gu = g_means2D[2 * i], gv = g_means2D[2 * i + 1];
        gt[0] += gu * fx / z;
        gt[1] += gv * fy / z;
        gt[2] += -gu * fx * o.t[0] / (z * z) - gv * fy * o.t[1] / (z * z);
        /* conic -> C2 */
        const double A = o.C2[0][0], B = o.C2[0][1], C = o.C2[1][1], d2 = o.det * o.det;
        const double ga = g_conic[3 * i], gb = g_conic[3 * i + 1], gc = g_conic[3 * i + 2];
        const double dA = ga * (-C * C / d2) + gb * (B * C / d2) + gc * (-B * B / d2);
        const double dC = ga * (-B * B / d2) + gb * (A * B / d2) + gc * (-A * A / d2);
        const double dB = ga * (2.0 * B * C / d2) + gb * (-1.0 / o.det - 2.0 * B * B / d2) + gc * (2.0 * A * B / d2);
        const double G[2][2] = {{dA, 0.5 * dB}, {0.5 * dB, dC}};
        /* C2 = T Sigma T^T */
        double gSig[3][3], gT[2][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int r = 0; r < 2; ++r)
                    for (int k = 0; k < 2; ++k) acc += o.Tm[r][a] * G[r][k] * o.Tm[k][b];
                gSig[a][b] = acc;
            }
        for (int r = 0; r < 2; ++r)
            for (int a = 0; a < 3; ++a) {
                double acc = 0.0;
                for (int k = 0; k < 2; ++k)
                    for (int b = 0; b < 3; ++b) acc += G[r][k] * o.Tm[k][b] * o.Sig[b][a];
                gT[r][a] = 2.0 * acc;
            }
        /* T = J W: dL/dJ[r][k] = sum_c dL/dT[r][c] W[k][c] */
        double gJ[2][3];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k) gJ[r][k] = gT[r][0] * V[4 * k] + gT[r][1] * V[4 * k + 1] + gT[r][2] * V[4 * k + 2];
        /* J(t): J00 = fx/z, J02 = -fx cl(x/z)/z, J11 = fy/z, J12 = -fy cl(y/z)/z */
        const double clx = -o.J[0][2] * z / fx, cly = -o.J[1][2] * z / fy; /* clamped tangents */
        gt[2] += gJ[0][0] * (-fx / (z * z)) + gJ[1][1] * (-fy / (z * z));
        gt[2] += gJ[0][2] * (fx * clx / (z * z)) + gJ[1][2] * (fy * cly / (z * z));
        if (o.in_x) {
            gt[0] += gJ[0][2] * (-fx / (z * z));
            gt[2] += gJ[0][2] * (fx * o.t[0] / (z * z * z));
        }
        if (o.in_y) {
            gt[1] += gJ[1][2] * (-fy / (z * z));
            gt[2] += gJ[1][2] * (fy * o.t[1] / (z * z * z));
        }
        /* t = W p + w */
        for (int k = 0; k < 3; ++k) g_means3D[3 * i + k] = V[k] * gt[0] + V[4 + k] * gt[1] + V[8 + k] * gt[2];
        /* Sigma = M M^T, M = R S */
        double gM[3][3];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k)
                gM[r][k] = 2.0 * (gSig[r][0] * o.M[0][k] + gSig[r][1] * o.M[1][k] + gSig[r][2] * o.M[2][k]);
        double gR[3][3];
        for (int k = 0; k < 3; ++k) {
            double gs = 0.0;
            for (int r = 0; r < 3; ++r) {
                gs += gM[r][k] * o.R[r][k];
                gR[r][k] = gM[r][k] * o.s[k];
            }
            g_log_scales[3 * i + k] = gs * o.s[k];
        }
        /* R(q), q normalised (w, x, y, z) */
        const double w = o.q[0], x = o.q[1], y = o.q[2], zq = o.q[3];
        double gq[4];
        gq[0] = 2.0 * (-zq * gR[0][1] + y * gR[0][2] + zq * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
        gq[1] = 2.0 * (y * gR[0][1] + zq * gR[0][2] + y * gR[1][0] - 2.0 * x * gR[1][1] - w * gR[1][2] + zq * gR[2][0] +
                       w * gR[2][1] - 2.0 * x * gR[2][2]);
        gq[2] = 2.0 * (-2.0 * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + zq * gR[1][2] - w * gR[2][0] +
                       zq * gR[2][1] - 2.0 * y * gR[2][2]);
        gq[3] = 2.0 * (-2.0 * zq * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2.0 * zq * gR[1][1] +
                       y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
        const double dot = o.q[0] * gq[0] + o.q[1] * gq[1] + o.q[2] * gq[2] + o.q[3] * gq[3];
        for (int k = 0; k < 4; ++k) g_quats[4 * i + k] = (gq[k] - o.q[k] * dot) / o.qn;
    }
}

/* ------------------------------------------------------------------------- */
/* Binning: for every tile, the list of Gaussians whose rectangle covers it,  */
/* ordered by (float32 depth bit pattern, Gaussian index).  Written as the    */
/* plain definition: emit one (tile, depth bits, index) record per covered    */
/* tile, then sort the records.                                                */
/* point_list receives the Gaussian indices; ranges[2t], ranges[2t+1] is the  */
/* half-open span of tile t.  Returns K, or -K if K > capacity (nothing       */
/* written to point_list then).                                                */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint32_t tile, depth_bits, idx;
} orc_entry;

static int cmp_entry(const void *pa, const void *pb) {
    const orc_entry *a = (const orc_entry *)pa, *b = (const orc_entry *)pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->depth_bits != b->depth_bits) return a->depth_bits < b->depth_bits ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

int64_t orc_bin(int64_t N, const float *means2D, const int32_t *radius, const float *depth, int W, int H,
                int tw, int th, int64_t capacity, uint32_t *point_list, uint32_t *ranges) {
    const int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    const int64_t T = (int64_t)tiles_x * tiles_y;
    int64_t K = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (radius[i] <= 0) continue;
        int x0, x1, y0, y1;
        tile_rect(means2D[2 * i], means2D[2 * i + 1], radius[i], tiles_x, tiles_y, tw, th, &x0, &x1, &y0, &y1);
        if (x1 > x0 && y1 > y0) K += (int64_t)(x1 - x0) * (y1 - y0);
    }
    for (int64_t t = 0; t < T; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
    if (K > capacity) return -K;
    if (K == 0) return 0;
    orc_entry *e = (orc_entry *)malloc((size_t)K * sizeof(orc_entry));
    if (!e) return -K;
    int64_t k = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (radius[i] <= 0) continue;
        int x0, x1, y0, y1;
        tile_rect(means2D[2 * i], means2D[2 * i + 1], radius[i], tiles_x, tiles_y, tw, th, &x0, &x1, &y0, &y1);
        uint32_t bits;
        memcpy(&bits, &depth[i], 4);
        for (int y = y0; y < y1; ++y)
            for (int x = x0; x < x1; ++x) {
                e[k].tile = (uint32_t)(y * tiles_x + x);
                e[k].depth_bits = bits;
                e[k].idx = (uint32_t)i;
                ++k;
            }
    }
    qsort(e, (size_t)K, sizeof(orc_entry), cmp_entry);
    for (int64_t j = 0; j < K; ++j) {
        point_list[j] = e[j].idx;
        uint32_t t = e[j].tile;
        if (j == 0 || e[j - 1].tile != t) ranges[2 * t] = (uint32_t)j;
        ranges[2 * t + 1] = (uint32_t)(j + 1);
    }
    free(e);
    return K;
}

/* Visible Gaussians (radius > 0) in the stable depth order of the per-tile lists: by float32
   depth bits, ties by index.  Writes them to order and returns their count. */
typedef struct {
    uint32_t depth_bits, idx;
} orc_key;

static int cmp_key(const void *pa, const void *pb) {
    const orc_key *a = (const orc_key *)pa, *b = (const orc_key *)pb;
    if (a->depth_bits != b->depth_bits) return a->depth_bits < b->depth_bits ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

int64_t orc_depth_order(int64_t N, const int32_t *radius, const float *depth, uint32_t *order) {
    int64_t n = 0;
    for (int64_t i = 0; i < N; ++i) n += radius[i] > 0;
    orc_key *k = (orc_key *)malloc((size_t)(n > 0 ? n : 1) * sizeof(orc_key));
    n = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (radius[i] <= 0) continue;
        memcpy(&k[n].depth_bits, &depth[i], 4);
        k[n].idx = (uint32_t)i;
        ++n;
    }
    qsort(k, (size_t)n, sizeof(orc_key), cmp_key);
    for (int64_t j = 0; j < n; ++j) order[j] = k[j].idx;
    free(k);
    return n;
}

/* The same per-tile lists for a subset of the tiles only: `sel` lists ns distinct tile ids;
   their lists (same tile rectangles, same stable (depth bits, index) order as orc_bin) are
   written one after the other to point_list, and ranges [T][2] gets their spans (every
   other tile empty).  Every tile's list is the subsequence of the depth order of all
   visible Gaussians whose rectangles cover the tile, so the lists are filled by one walk
   over that order (`order`, from orc_depth_order, n_order entries).  Returns the entry
   count, or -count when it exceeds capacity (nothing written).  For sampling large frames
   without materialising every tile's list. */
int64_t orc_bin_subset(int64_t N, const float *means2D, const int32_t *radius, int W, int H, int tw, int th,
                       int64_t ns, const int64_t *sel, const uint32_t *order, int64_t n_order, int64_t capacity,
                       uint32_t *point_list, uint32_t *ranges) {
    (void)N;
    const int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    const int64_t T = (int64_t)tiles_x * tiles_y;
    for (int64_t t = 0; t < T; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
    /* the selected tiles of every tile row, and each selected tile's fill position */
    int64_t *row_start = (int64_t *)calloc((size_t)tiles_y + 1, sizeof(int64_t));
    int32_t *row_x = (int32_t *)malloc((size_t)(ns > 0 ? ns : 1) * sizeof(int32_t));
    int64_t *cnt = (int64_t *)calloc((size_t)(ns > 0 ? ns : 1), sizeof(int64_t));
    for (int64_t q = 0; q < ns; ++q) row_start[sel[q] / tiles_x + 1] += 1;
    for (int y = 0; y < tiles_y; ++y) row_start[y + 1] += row_start[y];
    int64_t *fill = (int64_t *)malloc((size_t)(tiles_y + 1) * sizeof(int64_t));
    memcpy(fill, row_start, (size_t)(tiles_y + 1) * sizeof(int64_t));
    for (int64_t q = 0; q < ns; ++q) row_x[fill[sel[q] / tiles_x]++] = (int32_t)(sel[q] % tiles_x);
    free(fill);
    int64_t K = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t j = 0; j < n_order; ++j) {
            const uint32_t i = order[j];
            int x0, x1, y0, y1;
            tile_rect(means2D[2 * i], means2D[2 * i + 1], radius[i], tiles_x, tiles_y, tw, th, &x0, &x1, &y0, &y1);
            for (int y = y0; y < y1; ++y)
                for (int64_t q = row_start[y]; q < row_start[y + 1]; ++q) {
                    const int x = row_x[q];
                    if (x < x0 || x >= x1) continue;
                    if (pass == 1) point_list[cnt[q]] = i;
                    ++cnt[q];
                }
        }
        if (pass == 0) {
            K = 0;
            for (int64_t q = 0; q < ns; ++q) K += cnt[q];
            if (K > capacity || K == 0) break;
            /* tiles in sel order, each list contiguous */
            int64_t run = 0;
            for (int y = 0; y < tiles_y; ++y)
                for (int64_t q = row_start[y]; q < row_start[y + 1]; ++q) {
                    const int64_t t = (int64_t)y * tiles_x + row_x[q];
                    const int64_t c = cnt[q];
                    cnt[q] = run;
                    if (c) {
                        ranges[2 * t] = (uint32_t)run;
                        ranges[2 * t + 1] = (uint32_t)(run + c);
                    }
                    run += c;
                }
        }
    }
    free(row_start);
    free(row_x);
    free(cnt);
    if (K > capacity) return -K;
    return K;
}

/* ------------------------------------------------------------------------- */
/* One pixel of the forward (Eq. 4 under Algorithm 5's rules).                */
/* Walks the tile's depth-sorted list front to back:                           */
/*   d = mu - (px, py); power = -1/2 (a dx^2 + c dy^2) - b dx dy;             */
/*   skip if power > 0; alpha = min(0.99, o exp(power)); skip if alpha<1/255; */
/*   T' = T (1 - alpha); stop (not accumulated) if T' < 1e-4;                 */
/*   else w = alpha T, C += w c, D += w depth, A += w, T = T'.                 */
/* n_contrib = list position + 1 of the last accumulated pair (0 if none);     */
/* n_eval = pairs the rule visits (stop position + 1, or the list length);    */
/* n_acc = pairs accumulated (the "contributing" pairs).                       */
/* ------------------------------------------------------------------------- */
typedef struct {
    double C[3], D, A, T;
    int32_t n_contrib, n_eval, n_acc;
    uint8_t flags;
} orc_pix;

static void render_pixel(int px, int py, uint32_t start, uint32_t end, const uint32_t *point_list,
                         const double *means2D, const double *co, const double *colors, const double *depth,
                         const double bg[3], orc_pix *out) {
    double T = 1.0, C[3] = {0, 0, 0}, D = 0.0, A = 0.0;
    int32_t last = 0, n_eval = (int32_t)(end - start), n_acc = 0;
    uint8_t flags = 0;
    for (uint32_t j = start; j < end; ++j) {
        uint32_t g = point_list[j];
        double dx = means2D[2 * g] - (double)px, dy = means2D[2 * g + 1] - (double)py;
        double a = co[4 * g], b = co[4 * g + 1], c = co[4 * g + 2], o = co[4 * g + 3];
        double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
        if (fabs(power) < 1e-9 && o >= ORC_ALPHA_MIN) flags |= ORC_FLAG_POWER_EDGE;
        if (power > 0.0) continue;
        double og = o * exp(power);
        double alpha = og < ORC_ALPHA_MAX ? og : ORC_ALPHA_MAX;
        if (fabs(alpha - ORC_ALPHA_MIN) < 1e-6) flags |= ORC_FLAG_ALPHA_EDGE;
        if (alpha < ORC_ALPHA_MIN) continue;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - ORC_T_MIN) < 1e-9) flags |= ORC_FLAG_T_EDGE;
        if (Tn < ORC_T_MIN) {
            n_eval = (int32_t)(j - start + 1);
            break;
        }
        if (fabs(og - ORC_ALPHA_MAX) < 1e-6) flags |= ORC_FLAG_CLAMP_EDGE;
        double w = alpha * T;
        C[0] += w * colors[3 * g];
        C[1] += w * colors[3 * g + 1];
        C[2] += w * colors[3 * g + 2];
        D += w * depth[g];
        A += w;
        T = Tn;
        last = (int32_t)(j - start + 1);
        ++n_acc;
    }
    for (int ch = 0; ch < 3; ++ch) out->C[ch] = C[ch] + T * bg[ch];
    out->D = D;
    out->A = A;
    out->T = T;
    out->n_contrib = last;
    out->n_eval = n_eval;
    out->n_acc = n_acc;
    out->flags = flags;
}

/* Forward over all pixels (pix == NULL, outputs planar [3,H,W] / [H,W]) or    */
/* over npix listed pixels (linear ids y*W+x; outputs [3,npix] / [npix]).      */
void orc_render(int W, int H, int tw, int th, const double *means2D, const double *conic_opacity,
                const double *colors, const double *depth, const uint32_t *point_list, const uint32_t *ranges,
                const double *bg, int64_t npix, const int64_t *pix, double *out_color, double *out_depth,
                double *out_alpha, double *final_T, int32_t *n_contrib, int32_t *n_eval, int32_t *n_acc,
                uint8_t *flags) {
    const int tiles_x = (W + tw - 1) / tw;
    const int64_t P = pix ? npix : (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < P; ++q) {
        int64_t id = pix ? pix[q] : q;
        int px = (int)(id % W), py = (int)(id / W);
        int64_t t = (int64_t)(py / th) * tiles_x + px / tw;
        orc_pix r;
        render_pixel(px, py, ranges[2 * t], ranges[2 * t + 1], point_list, means2D, conic_opacity, colors, depth,
                     bg, &r);
        for (int ch = 0; ch < 3; ++ch) out_color[ch * P + q] = r.C[ch];
        out_depth[q] = r.D;
        out_alpha[q] = r.A;
        final_T[q] = r.T;
        n_contrib[q] = r.n_contrib;
        n_eval[q] = r.n_eval;
        n_acc[q] = r.n_acc;
        flags[q] = r.flags;
    }
}

/* ------------------------------------------------------------------------- */
/* Analytic gradient of the forward, from its definition.                      */
/* With T_i = prod_{j<i, accepted} (1 - alpha_j) and T_f the final            */
/* transmittance, the pixel outputs are                                        */
/*   C = sum_i c_i alpha_i T_i + T_f bg,  D = sum_i d_i alpha_i T_i,           */
/*   A = sum_i alpha_i T_i = 1 - T_f.                                          */
/* Every accepted pair's alpha_i enters T_j (j > i) and T_f through one factor */
/* (1 - alpha_i), so                                                           */
/*   dC/dalpha_i = c_i T_i - (sum_{j>i} c_j alpha_j T_j + T_f bg)/(1-alpha_i)  */
/*   dD/dalpha_i = d_i T_i - (sum_{j>i} d_j alpha_j T_j)/(1-alpha_i)           */
/*   dA/dalpha_i = T_f / (1 - alpha_i)                                        */
/*   dC/dc_i = alpha_i T_i,  dD/dd_i = alpha_i T_i.                            */
/* alpha = min(0.99, o G): d alpha/do = G, d alpha/dG = o where o G <= 0.99,   */
/* both 0 where the clamp is active.  G = exp(power):                          */
/*   dG/dmu_x = G (-a dx - b dy), dG/dmu_y = G (-c dy - b dx),                 */
/*   dG/da = -G dx^2 / 2, dG/db = -G dx dy, dG/dc = -G dy^2 / 2.               */
/* Gradients are summed over pixels.  Only tiles listed in `tiles` (or all    */
/* tiles when tiles == NULL) are visited, and only Gaussians with mask[g] != 0 */
/* (or all when mask == NULL) receive gradients.  dL_ddepth / dL_dalpha may be */
/* NULL (treated as zero).  Outputs are overwritten.  When abs_terms is not   */
/* NULL it receives, per Gaussian, the sum of the absolute values of the same */
/* per-pair terms ([N][10]: mean x, y, conic a, b, c, opacity, colour r, g, b, */
/* depth) -- the condition of each gradient sum, which bounds the rounding    */
/* error any summation order of those terms can make (test tolerances only).  */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint32_t g;
    double alpha, G, T, dx, dy;
    int clamped;
} orc_acc;

void orc_render_backward(int W, int H, int tw, int th, int64_t N, const double *means2D, const double *co,
                         const double *colors, const double *depth, const uint32_t *point_list,
                         const uint32_t *ranges, const double *bg, const double *dL_dcolor, const double *dL_ddepth,
                         const double *dL_dalpha, int64_t ntiles_sel, const int64_t *tiles, const uint8_t *mask,
                         double *dL_dmeans2D, double *dL_dconic, double *dL_dopacity, double *dL_dcolors,
                         double *dL_ddepths, double *abs_terms) {
    const int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    const int64_t HW = (int64_t)W * H;
    memset(dL_dmeans2D, 0, sizeof(double) * 2 * N);
    memset(dL_dconic, 0, sizeof(double) * 3 * N);
    memset(dL_dopacity, 0, sizeof(double) * N);
    memset(dL_dcolors, 0, sizeof(double) * 3 * N);
    memset(dL_ddepths, 0, sizeof(double) * N);
    if (abs_terms) memset(abs_terms, 0, sizeof(double) * 10 * N);
    const int64_t TT = tiles ? ntiles_sel : (int64_t)tiles_x * tiles_y;
#pragma omp parallel
    {
        size_t cap = 1024;
        orc_acc *acc = (orc_acc *)malloc(cap * sizeof(orc_acc));
        double *suf = (double *)malloc(cap * 4 * sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < TT; ++q) {
            int64_t t = tiles ? tiles[q] : q;
            int tx = (int)(t % tiles_x), ty = (int)(t / tiles_x);
            uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
            for (int py = ty * th; py < (ty + 1) * th && py < H; ++py)
                for (int px = tx * tw; px < (tx + 1) * tw && px < W; ++px) {
                    int64_t pid = (int64_t)py * W + px;
                    double gC[3] = {dL_dcolor[pid], dL_dcolor[HW + pid], dL_dcolor[2 * HW + pid]};
                    double gD = dL_ddepth ? dL_ddepth[pid] : 0.0;
                    double gA = dL_dalpha ? dL_dalpha[pid] : 0.0;
                    /* forward walk, recording accepted pairs */
                    size_t m = 0;
                    double T = 1.0;
                    for (uint32_t j = start; j < end; ++j) {
                        uint32_t g = point_list[j];
                        double dx = means2D[2 * g] - (double)px, dy = means2D[2 * g + 1] - (double)py;
                        double a = co[4 * g], b = co[4 * g + 1], c = co[4 * g + 2], o = co[4 * g + 3];
                        double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
                        if (power > 0.0) continue;
                        double G = exp(power);
                        double og = o * G;
                        double alpha = og < ORC_ALPHA_MAX ? og : ORC_ALPHA_MAX;
                        if (alpha < ORC_ALPHA_MIN) continue;
                        double Tn = T * (1.0 - alpha);
                        if (Tn < ORC_T_MIN) break;
                        if (m == cap) {
                            cap *= 2;
                            acc = (orc_acc *)realloc(acc, cap * sizeof(orc_acc));
                            suf = (double *)realloc(suf, cap * 4 * sizeof(double));
                        }
                        acc[m].g = g;
                        acc[m].alpha = alpha;
                        acc[m].G = G;
                        acc[m].T = T;
                        acc[m].dx = dx;
                        acc[m].dy = dy;
                        acc[m].clamped = og > ORC_ALPHA_MAX;
                        ++m;
                        T = Tn;
                    }
                    const double Tf = T;
                    /* suffix sums S[i] = sum_{j>i} (c_j, d_j) alpha_j T_j */
                    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
                    for (size_t i = m; i-- > 0;) {
                        suf[4 * i] = s0;
                        suf[4 * i + 1] = s1;
                        suf[4 * i + 2] = s2;
                        suf[4 * i + 3] = s3;
                        double w = acc[i].alpha * acc[i].T;
                        uint32_t g = acc[i].g;
                        s0 += colors[3 * g] * w;
                        s1 += colors[3 * g + 1] * w;
                        s2 += colors[3 * g + 2] * w;
                        s3 += depth[g] * w;
                    }
                    for (size_t i = 0; i < m; ++i) {
                        uint32_t g = acc[i].g;
                        if (mask && !mask[g]) continue;
                        double al = acc[i].alpha, Ti = acc[i].T, om = 1.0 - al;
                        double dLda = 0.0;
                        for (int ch = 0; ch < 3; ++ch)
                            dLda += gC[ch] * (colors[3 * g + ch] * Ti - (suf[4 * i + ch] + Tf * bg[ch]) / om);
                        dLda += gD * (depth[g] * Ti - suf[4 * i + 3] / om);
                        dLda += gA * (Tf / om);
                        double w = al * Ti;
                        double o = co[4 * g + 3], a = co[4 * g], b = co[4 * g + 1], c = co[4 * g + 2];
                        double dLdo = 0.0, dLdpow = 0.0;
                        if (!acc[i].clamped) {
                            dLdo = acc[i].G * dLda;
                            dLdpow = o * dLda * acc[i].G; /* dL/dG * dG/dpower */
                        }
                        double dx = acc[i].dx, dy = acc[i].dy;
                        double gmx = dLdpow * (-a * dx - b * dy);
                        double gmy = dLdpow * (-c * dy - b * dx);
                        double ga = dLdpow * (-0.5 * dx * dx);
                        double gb = dLdpow * (-dx * dy);
                        double gc = dLdpow * (-0.5 * dy * dy);
#pragma omp atomic
                        dL_dmeans2D[2 * g] += gmx;
#pragma omp atomic
                        dL_dmeans2D[2 * g + 1] += gmy;
#pragma omp atomic
                        dL_dconic[3 * g] += ga;
#pragma omp atomic
                        dL_dconic[3 * g + 1] += gb;
#pragma omp atomic
                        dL_dconic[3 * g + 2] += gc;
#pragma omp atomic
                        dL_dopacity[g] += dLdo;
#pragma omp atomic
                        dL_dcolors[3 * g] += w * gC[0];
#pragma omp atomic
                        dL_dcolors[3 * g + 1] += w * gC[1];
#pragma omp atomic
                        dL_dcolors[3 * g + 2] += w * gC[2];
#pragma omp atomic
                        dL_ddepths[g] += w * gD;
                        if (abs_terms) {
                            /* magnitudes of the same per-pair terms (the condition of each sum) */
                            const double t[10] = {gmx, gmy, ga, gb, gc, dLdo, w * gC[0], w * gC[1], w * gC[2], w * gD};
                            for (int k = 0; k < 10; ++k) {
#pragma omp atomic
                                abs_terms[10 * g + k] += fabs(t[k]);
                            }
                        }
                    }
                }
        }
        free(acc);
        free(suf);
    }
}

/* ---- view-dependent colour from spherical harmonics (Sec. 2.1) -------------------------
 * The paper represents a Gaussian's colour by spherical harmonics (Sec. 2.1) and fixes no
 * basis.  Reading: the real orthonormal spherical harmonics of degree l <= 3 with the
 * Condon-Shortley phase, written as homogeneous harmonic polynomials of the unit
 * direction d = (x, y, z) from the camera centre to the Gaussian's mean, in the order
 * (l, m) = (0,0), (1,-1), (1,0), (1,1), (2,-2), ..., (2,2), (3,-3), ..., (3,3).  Colour
 * channel c = sum_k Y_k(d) sh[k][c] + 1/2, clamped below at 0; a clamped channel passes no
 * gradient.  Normalisation constants are the closed forms sqrt((2l+1)/(4 pi) ...) below.
 *
 * Y[k] and, when grad is not NULL, the gradient of the polynomial Y_k(x, y, z) (x, y, z
 * taken as independent variables) in grad[3k .. 3k+2]. */
static void orc_sh_basis(int degree, double x, double y, double z, double *Y, double *grad) {
    const double pi = 3.14159265358979323846;
    const double c0 = 0.5 / sqrt(pi);                  /* Y_00                       */
    const double c1 = sqrt(3.0 / (4.0 * pi));          /* |Y_1m| / |coordinate|      */
    const double c2a = 0.5 * sqrt(15.0 / pi);          /* xy, yz, xz terms           */
    const double c2b = 0.25 * sqrt(5.0 / pi);          /* 2z^2 - x^2 - y^2           */
    const double c2c = 0.25 * sqrt(15.0 / pi);         /* x^2 - y^2                  */
    const double c3a = 0.25 * sqrt(35.0 / (2.0 * pi)); /* y(3x^2 - y^2), x(x^2 - 3y^2) */
    const double c3b = 0.5 * sqrt(105.0 / pi);         /* xyz                        */
    const double c3c = 0.25 * sqrt(21.0 / (2.0 * pi)); /* y(4z^2 - x^2 - y^2), x(...) */
    const double c3d = 0.25 * sqrt(7.0 / pi);          /* z(2z^2 - 3x^2 - 3y^2)       */
    const double c3e = 0.25 * sqrt(105.0 / pi);        /* z(x^2 - y^2)               */
    double g[16][3];
    memset(g, 0, sizeof g);
    Y[0] = c0;
    if (degree >= 1) {
        Y[1] = -c1 * y;  g[1][1] = -c1;
        Y[2] = c1 * z;   g[2][2] = c1;
        Y[3] = -c1 * x;  g[3][0] = -c1;
    }
    if (degree >= 2) {
        Y[4] = c2a * x * y;
        g[4][0] = c2a * y; g[4][1] = c2a * x;
        Y[5] = -c2a * y * z;
        g[5][1] = -c2a * z; g[5][2] = -c2a * y;
        Y[6] = c2b * (2.0 * z * z - x * x - y * y);
        g[6][0] = -2.0 * c2b * x; g[6][1] = -2.0 * c2b * y; g[6][2] = 4.0 * c2b * z;
        Y[7] = -c2a * x * z;
        g[7][0] = -c2a * z; g[7][2] = -c2a * x;
        Y[8] = c2c * (x * x - y * y);
        g[8][0] = 2.0 * c2c * x; g[8][1] = -2.0 * c2c * y;
    }
    if (degree >= 3) {
        Y[9] = -c3a * y * (3.0 * x * x - y * y);
        g[9][0] = -6.0 * c3a * x * y; g[9][1] = -c3a * (3.0 * x * x - 3.0 * y * y);
        Y[10] = c3b * x * y * z;
        g[10][0] = c3b * y * z; g[10][1] = c3b * x * z; g[10][2] = c3b * x * y;
        Y[11] = -c3c * y * (4.0 * z * z - x * x - y * y);
        g[11][0] = 2.0 * c3c * x * y; g[11][1] = -c3c * (4.0 * z * z - x * x - 3.0 * y * y);
        g[11][2] = -8.0 * c3c * y * z;
        Y[12] = c3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
        g[12][0] = -6.0 * c3d * x * z; g[12][1] = -6.0 * c3d * y * z;
        g[12][2] = c3d * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
        Y[13] = -c3c * x * (4.0 * z * z - x * x - y * y);
        g[13][0] = -c3c * (4.0 * z * z - 3.0 * x * x - y * y); g[13][1] = 2.0 * c3c * x * y;
        g[13][2] = -8.0 * c3c * x * z;
        Y[14] = c3e * z * (x * x - y * y);
        g[14][0] = 2.0 * c3e * x * z; g[14][1] = -2.0 * c3e * y * z; g[14][2] = c3e * (x * x - y * y);
        Y[15] = -c3a * x * (x * x - 3.0 * y * y);
        g[15][0] = -c3a * (3.0 * x * x - 3.0 * y * y); g[15][1] = 6.0 * c3a * x * y;
    }
    if (grad) memcpy(grad, g, sizeof(double) * 3 * (degree + 1) * (degree + 1));
}

/* Unit direction from campos to the mean and its length. */
static double orc_sh_dir(const double *mean, const double *campos, double *d) {
    const double v[3] = {mean[0] - campos[0], mean[1] - campos[1], mean[2] - campos[2]};
    const double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int a = 0; a < 3; ++a) d[a] = v[a] / len;
    return len;
}

/* rgb [V,N,3] and clamped [V,N,3] (nullable; 1 where the channel was clamped at 0) of N
 * Gaussians with coefficients sh [N, stride, 3] (stride >= (degree+1)^2 rows) seen from V
 * camera centres campos [V,3]. */
void orc_sh_to_rgb(int64_t N, int V, int degree, int stride, const double *sh, const double *means3D,
                   const double *campos, double *rgb, uint8_t *clamped) {
    const int nk = (degree + 1) * (degree + 1);
    for (int v = 0; v < V; ++v)
        for (int64_t i = 0; i < N; ++i) {
            double d[3], Y[16];
            orc_sh_dir(means3D + 3 * i, campos + 3 * v, d);
            orc_sh_basis(degree, d[0], d[1], d[2], Y, NULL);
            for (int c = 0; c < 3; ++c) {
                double s = 0.5;
                for (int k = 0; k < nk; ++k) s += Y[k] * sh[(i * stride + k) * 3 + c];
                const int64_t o = ((int64_t)v * N + i) * 3 + c;
                rgb[o] = s < 0.0 ? 0.0 : s;
                if (clamped) clamped[o] = s < 0.0 ? 1 : 0;
            }
        }
}

/* Gradients of orc_sh_to_rgb: dL_drgb [V,N,3] -> dL_dsh [N, stride, 3] and dL_dmeans3D
 * [N,3], summed over the views (overwritten).  With u = mean - campos and d = u / |u|,
 * dL/du = (dL/dd - (dL/dd . d) d) / |u|, and dL/dd = sum_k (sum_c sh[k][c] g_c) grad Y_k
 * with g_c = dL/drgb_c for an unclamped channel, 0 for a clamped one. */
void orc_sh_to_rgb_backward(int64_t N, int V, int degree, int stride, const double *sh, const double *means3D,
                            const double *campos, const double *dL_drgb, double *dL_dsh, double *dL_dmeans3D) {
    const int nk = (degree + 1) * (degree + 1);
    memset(dL_dsh, 0, sizeof(double) * N * stride * 3);
    memset(dL_dmeans3D, 0, sizeof(double) * N * 3);
    for (int v = 0; v < V; ++v)
        for (int64_t i = 0; i < N; ++i) {
            double d[3], Y[16], gY[48];
            const double len = orc_sh_dir(means3D + 3 * i, campos + 3 * v, d);
            orc_sh_basis(degree, d[0], d[1], d[2], Y, gY);
            double g[3];
            for (int c = 0; c < 3; ++c) {
                double s = 0.5;
                for (int k = 0; k < nk; ++k) s += Y[k] * sh[(i * stride + k) * 3 + c];
                g[c] = s < 0.0 ? 0.0 : dL_drgb[((int64_t)v * N + i) * 3 + c];
            }
            double dd[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < nk; ++k) {
                double w = 0.0;
                for (int c = 0; c < 3; ++c) {
                    dL_dsh[(i * stride + k) * 3 + c] += Y[k] * g[c];
                    w += sh[(i * stride + k) * 3 + c] * g[c];
                }
                for (int a = 0; a < 3; ++a) dd[a] += w * gY[3 * k + a];
            }
            const double dot = dd[0] * d[0] + dd[1] * d[1] + dd[2] * d[2];
            for (int a = 0; a < 3; ++a) dL_dmeans3D[3 * i + a] += (dd[a] - dot * d[a]) / len;
        }
}
