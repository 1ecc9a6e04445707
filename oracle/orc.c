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

/* ------------------------------------------------------------------------- */
/* Projection (Eq. 1-3).                                                      */
/*   camera: fx fy cx cy, row-major 4x4 world->camera matrix V, near plane,   */
/*   lowpass added to the diagonal of Sigma'.                                 */
/*   Sigma = R S S^T R^T, R from the normalised quaternion (w,x,y,z), S =     */
/*   diag(exp(log_scale)).  J is the Jacobian of (fx x/z + cx, fy y/z + cy)   */
/*   at the (tangent-clamped) camera-space point; W is V's rotation block.    */
/* Outputs: means2D [N,2], conic_opacity [N,4] (a,b,c,o with                   */
/*   power = -1/2 (a dx^2 + c dy^2) - b dx dy), depth [N], radius [N] (int),   */
/*   radius_raw [N] = 3 sqrt(lambda_max) before the ceil, tiles_touched [N]    */
/*   (rectangle area, computed from the float32-rounded mean).                */
/* A culled Gaussian gets radius 0 and tiles_touched 0.                        */
/* ------------------------------------------------------------------------- */
void orc_preprocess(int64_t N, const float *means3D, const float *log_scales, const float *quats,
                    const float *opacities, int W, int H, double fx, double fy, double cx, double cy,
                    const double *V, double near_z, double lowpass, int tw, int th,
                    double *means2D, double *conic_opacity, double *depth, int32_t *radius,
                    double *radius_raw, int32_t *tiles_touched) {
    const int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    const double tan_x = (double)W / (2.0 * fx), tan_y = (double)H / (2.0 * fy);
    const double lim_x = 1.3 * tan_x, lim_y = 1.3 * tan_y;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double p[3] = {means3D[3 * i], means3D[3 * i + 1], means3D[3 * i + 2]};
        double t[3];
        for (int r = 0; r < 3; ++r) t[r] = V[4 * r] * p[0] + V[4 * r + 1] * p[1] + V[4 * r + 2] * p[2] + V[4 * r + 3];
        means2D[2 * i] = means2D[2 * i + 1] = 0.0;
        for (int k = 0; k < 4; ++k) conic_opacity[4 * i + k] = 0.0;
        depth[i] = t[2];
        radius[i] = 0;
        radius_raw[i] = 0.0;
        tiles_touched[i] = 0;
        if (!(t[2] > near_z)) continue;

        /* rotation from the normalised quaternion q = (w, x, y, z) */
        double qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
        double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
        qw /= qn; qx /= qn; qy /= qn; qz /= qn;
        double R[3][3] = {
            {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
            {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
            {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
        double s[3] = {exp(log_scales[3 * i]), exp(log_scales[3 * i + 1]), exp(log_scales[3 * i + 2])};
        /* Sigma = (R S)(R S)^T */
        double M[3][3], Sig[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) M[r][c] = R[r][c] * s[c];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) Sig[r][c] = M[r][0] * M[c][0] + M[r][1] * M[c][1] + M[r][2] * M[c][2];

        /* Jacobian at the tangent-clamped point */
        double z = t[2];
        double txz = t[0] / z, tyz = t[1] / z;
        double xc = (txz < -lim_x ? -lim_x : (txz > lim_x ? lim_x : txz)) * z;
        double yc = (tyz < -lim_y ? -lim_y : (tyz > lim_y ? lim_y : tyz)) * z;
        double J[2][3] = {{fx / z, 0.0, -fx * xc / (z * z)}, {0.0, fy / z, -fy * yc / (z * z)}};
        /* T = J W (2x3), W = rotation block of V */
        double Tm[2][3];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) Tm[r][c] = J[r][0] * V[c] + J[r][1] * V[4 + c] + J[r][2] * V[8 + c];
        double C2[2][2];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += Tm[r][k] * Sig[k][l] * Tm[c][l];
                C2[r][c] = acc;
            }
        C2[0][0] += lowpass;
        C2[1][1] += lowpass;
        double det = C2[0][0] * C2[1][1] - C2[0][1] * C2[1][0];
        if (!(det > 0.0)) continue;
        double mid = 0.5 * (C2[0][0] + C2[1][1]);
        double disc = mid * mid - det;
        if (disc < 0.1) disc = 0.1;
        double lam = mid + sqrt(disc);
        double rr = 3.0 * sqrt(lam);
        int r = (int)ceil(rr);

        double u = fx * t[0] / z + cx, v = fy * t[1] / z + cy;
        means2D[2 * i] = u;
        means2D[2 * i + 1] = v;
        conic_opacity[4 * i + 0] = C2[1][1] / det;
        conic_opacity[4 * i + 1] = -C2[0][1] / det;
        conic_opacity[4 * i + 2] = C2[0][0] / det;
        conic_opacity[4 * i + 3] = opacities[i];
        radius_raw[i] = rr;
        int x0, x1, y0, y1;
        tile_rect((float)u, (float)v, r, tiles_x, tiles_y, tw, th, &x0, &x1, &y0, &y1);
        int64_t area = (int64_t)(x1 - x0) * (int64_t)(y1 - y0);
        if (area <= 0) continue;
        radius[i] = r;
        tiles_touched[i] = (int32_t)area;
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
/* NULL (treated as zero).  Outputs are overwritten.                           */
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
                         double *dL_ddepths) {
    const int tiles_x = (W + tw - 1) / tw, tiles_y = (H + th - 1) / th;
    const int64_t HW = (int64_t)W * H;
    memset(dL_dmeans2D, 0, sizeof(double) * 2 * N);
    memset(dL_dconic, 0, sizeof(double) * 3 * N);
    memset(dL_dopacity, 0, sizeof(double) * N);
    memset(dL_dcolors, 0, sizeof(double) * 3 * N);
    memset(dL_ddepths, 0, sizeof(double) * N);
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
                    }
                }
        }
        free(acc);
        free(suf);
    }
}
