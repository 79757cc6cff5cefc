/*
 * FP64 CPU oracle for the GS3LAM semantic-splatting rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product path never calls it
 * and there is no CPU fallback.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Everything is written out step by step in double precision, in the order
 * the paper states the method (GS3LAM, Sec. 3.2-3.4 and supplementary B.1):
 *
 *   Eq. 2   Sigma = R S S^T R^T (quaternion (w,x,y,z), S = diag(exp(log_s)))
 *   Eq. 3   Sigma2D = J R_cw Sigma R_cw^T J^T, J = perspective Jacobian at p
 *   B.1     g_i = K T_cw mu / d_i (projected centre), d_i = camera-frame z
 *   Eq. 5   alpha_i = o_i exp(-1/2 sigma^T Sigma2D^-1 sigma)
 *   Eq. 4,6,7,10  front-to-back blend of colour, depth, feature and opacity
 *   Eq. 8   softmax decoder (read as a per-pixel linear map, see below)
 *   Eq. 12  depth-adaptive scale regularisation (DSR)
 *   Eq. 15-18, 21  L1 colour/depth, semantic cross-entropy, tracking mask
 *   B.1     analytic Jacobian of the loss w.r.t. the camera pose
 *
 * Readings of points the paper leaves open (pixel centres at +0.5, the
 * thresholds alpha_min / alpha_max / T_min, z_near, the low-pass term, the
 * 3-sigma radius, 16x16 tiles, sort ties by Gaussian index, cross-entropy in
 * place of BCE, L1 normalised by the pixel count, DSR pooled over the three
 * axis scales with detached statistics) are listed with the tests that pin
 * them; every one is a parameter or a single, visible line here.
 *
 * One decision is taken in single precision on purpose: the depth-sort key.
 * "Sorting the Gaussians in depth order" (Sec. 3.2.1) needs an ordering;
 * ordering by a float32 key computed as an explicit fused multiply-add chain
 * makes that order identical, bit for bit, on any IEEE-754 machine, so the
 * integer decision is the same on both sides.  All blended values remain
 * double precision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Raster parameters, passed as a double array in this order. */
enum {
    P_TILE = 0, P_ALPHA_MIN, P_ALPHA_MAX, P_T_MIN, P_Z_NEAR, P_LOWPASS,
    P_RADIUS_SIGMA, P_BG_R, P_BG_G, P_BG_B, P_EXACT_J, P_COUNT
};

/* Camera intrinsics, passed as a double array: width, height, fx, fy, cx, cy. */
enum { C_W = 0, C_H, C_FX, C_FY, C_CX, C_CY };

int or_param_count(void) { return P_COUNT; }

/* Threads of the per-Gaussian and per-pixel loops (projection, blend, their
 * backwards), which are parallel over Gaussians or image rows when built with
 * OpenMP; 1 thread otherwise.  The per-Gaussian gradient sums of the blend
 * backward are then added atomically, so their order (and last bits) varies. */
void or_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ helpers */
static int64_t floordiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Rotation matrix of a unit quaternion (w,x,y,z), row-major. */
static void quat_to_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* C = A B for 3x3 row-major. */
static void mm3(const double A[9], const double B[9], double C[9]) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static void transpose3(const double A[9], double T[9]) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[3 * j + i] = A[3 * i + j];
}

/* Half-open tile rectangle of a splat centred at (u, v) with integer radius r.
 * floor((u - r) / tile) equals floordiv(floor(u) - r, tile) exactly because r is
 * an integer, so the rectangle is an exact function of (floor(u), floor(v), r). */
static void tile_rect(double u, double v, int64_t r, int tile, int tx, int ty, int32_t rect[4]) {
    double fu = floor(u), fv = floor(v);
    const double lim = 1099511627776.0; /* 2^40: keeps the integer arithmetic in range */
    fu = fu < -lim ? -lim : (fu > lim ? lim : fu);
    fv = fv < -lim ? -lim : (fv > lim ? lim : fv);
    int64_t iu = (int64_t)fu, iv = (int64_t)fv;
    rect[0] = (int32_t)clampi(floordiv(iu - r, tile), 0, tx);
    rect[1] = (int32_t)clampi(floordiv(iv - r, tile), 0, ty);
    rect[2] = (int32_t)clampi(floordiv(iu + r, tile) + 1, 0, tx);
    rect[3] = (int32_t)clampi(floordiv(iv + r, tile) + 1, 0, ty);
}

/* Camera-frame depth as the float32 sort key: fma(r20, x, fma(r21, y, fma(r22, z, tz))). */
static float depth_key(const double T[16], const double mu[3]) {
    float r20 = (float)T[8], r21 = (float)T[9], r22 = (float)T[10], tz = (float)T[11];
    float x = (float)mu[0], y = (float)mu[1], z = (float)mu[2];
    return fmaf(r20, x, fmaf(r21, y, fmaf(r22, z, tz)));
}

/* Point at which the EWA Jacobian J of Eq. 3 is evaluated: (x/z, y/z) of the
 * camera-frame centre.  With prm[P_EXACT_J] = 0 (the default) it is clamped to
 * the view's extent widened by 15% of the image size on each side (for a
 * centred principal point: 1.3 x the half field of view, the convention of the
 * 3DGS rasterizer that GS3LAM renders with); with prm[P_EXACT_J] != 0 it is not
 * clamped, which is the literal perspective Jacobian of Eq. 3.  The projected
 * centre itself is never clamped.  in_x / in_y report whether the coordinate is
 * inside the clamp interval (its derivative is 0 outside). */
static void jacobian_point(const double p[3], const double *cam, const double *prm, double *tx, double *ty,
                           int *in_x, int *in_y) {
    double W = cam[C_W], H = cam[C_H], fx = cam[C_FX], fy = cam[C_FY], cx = cam[C_CX], cy = cam[C_CY];
    double x = p[0] / p[2], y = p[1] / p[2];
    if (prm[P_EXACT_J] != 0) {
        *tx = x;
        *ty = y;
        if (in_x) *in_x = 1;
        if (in_y) *in_y = 1;
        return;
    }
    double lox = (-cx - 0.15 * W) / fx, hix = (W - cx + 0.15 * W) / fx;
    double loy = (-cy - 0.15 * H) / fy, hiy = (H - cy + 0.15 * H) / fy;
    *tx = x < lox ? lox : (x > hix ? hix : x);
    *ty = y < loy ? loy : (y > hiy ? hiy : y);
    if (in_x) *in_x = (x >= lox && x <= hix);
    if (in_y) *in_y = (y >= loy && y <= hiy);
}

/* ------------------------------------------------- A1-A2: projection (Eq. 2, 3) */
/*
 * For each Gaussian: activate the parameters, build Sigma (Eq. 2), move the
 * mean into the camera frame, project it (supp. B.1: g = K T_cw mu / d), form
 * Sigma2D by the EWA approximation (Eq. 3) with J evaluated at the clamped
 * point of jacobian_point(), add the low-pass term, invert it
 * to the conic, and bound the splat by radius_sigma standard deviations of the
 * larger eigenvalue.  Culled Gaussians (z <= z_near, singular or non-finite
 * Sigma2D) get radius 0 and touch no tile.
 *
 * Outputs (per Gaussian): uv[2], depth (camera z, double), depth_key (float32
 * sort key), conic[3] = (A, B, C) of Sigma2D^-1, opacity = sigmoid(logit),
 * radius (int), rect[4] = (x0, y0, x1, y1) half-open in tiles, touched,
 * radius_real = radius_sigma * sqrt(lambda_max) before the ceiling, and
 * cov2d[3] = (a, b, c) of Sigma2D including the low-pass term.
 */
void or_project(int64_t n, const double *means, const double *quats, const double *log_scales,
                const double *logits, const double *cam, const double *T, const double *prm,
                double *uv, double *depth, float *depth_key_out, double *conic, double *opacity,
                int32_t *radius, int32_t *rect, int32_t *touched, double *radius_real, double *cov2d) {
    int tile = (int)prm[P_TILE];
    int W = (int)cam[C_W], H = (int)cam[C_H];
    int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    double fx = cam[C_FX], fy = cam[C_FY], cx = cam[C_CX], cy = cam[C_CY];
    double Rcw[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    double tcw[3] = {T[3], T[7], T[11]};
    double RcwT[9];
    transpose3(Rcw, RcwT);

    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        const double *mu = means + 3 * i;
        uv[2 * i] = uv[2 * i + 1] = 0;
        conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0;
        cov2d[3 * i] = cov2d[3 * i + 1] = cov2d[3 * i + 2] = 0;
        radius[i] = 0;
        touched[i] = 0;
        radius_real[i] = 0;
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        opacity[i] = 1.0 / (1.0 + exp(-logits[i]));
        depth_key_out[i] = depth_key(T, mu);

        /* camera-frame centre p = R_cw mu + t_cw */
        double p[3];
        for (int r = 0; r < 3; r++) p[r] = Rcw[3 * r] * mu[0] + Rcw[3 * r + 1] * mu[1] + Rcw[3 * r + 2] * mu[2] + tcw[r];
        depth[i] = p[2];
        if (!(p[2] > prm[P_Z_NEAR])) continue;

        /* Eq. 2: Sigma = (R S)(R S)^T */
        double q[4] = {quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3]};
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        if (!(qn > 0)) continue;
        for (int k = 0; k < 4; k++) q[k] /= qn;
        double Rq[9], M[9], MT[9], Sig[9];
        quat_to_rot(q, Rq);
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) M[3 * r + c] = Rq[3 * r + c] * exp(log_scales[3 * i + c]);
        transpose3(M, MT);
        mm3(M, MT, Sig);

        /* Eq. 3: Sigma2D = J R_cw Sigma R_cw^T J^T */
        double tmp[9], Sc[9];
        mm3(Rcw, Sig, tmp);
        mm3(tmp, RcwT, Sc);
        double z = p[2];
        double tx_, ty_;
        jacobian_point(p, cam, prm, &tx_, &ty_, NULL, NULL);
        double J[6] = {fx / z, 0, -fx * tx_ / z, 0, fy / z, -fy * ty_ / z};
        double JS[6];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++)
                JS[3 * r + c] = J[3 * r] * Sc[c] + J[3 * r + 1] * Sc[3 + c] + J[3 * r + 2] * Sc[6 + c];
        double a = JS[0] * J[0] + JS[1] * J[1] + JS[2] * J[2] + prm[P_LOWPASS];
        double b = JS[0] * J[3] + JS[1] * J[4] + JS[2] * J[5];
        double c = JS[3] * J[3] + JS[4] * J[4] + JS[5] * J[5] + prm[P_LOWPASS];

        double u = fx * p[0] / z + cx, v = fy * p[1] / z + cy;
        uv[2 * i] = u;
        uv[2 * i + 1] = v;
        cov2d[3 * i] = a; cov2d[3 * i + 1] = b; cov2d[3 * i + 2] = c;

        double det = a * c - b * b;
        if (!(det > 0) || !isfinite(det) || !isfinite(u) || !isfinite(v)) continue;
        conic[3 * i] = c / det;
        conic[3 * i + 1] = -b / det;
        conic[3 * i + 2] = a / det;

        double mid = 0.5 * (a + c);
        double disc = mid * mid - det;
        double lmax = mid + sqrt(disc > 0 ? disc : 0);
        double rr = prm[P_RADIUS_SIGMA] * sqrt(lmax);
        radius_real[i] = rr;
        if (!(rr < 16777216.0)) rr = 16777216.0;
        int64_t r = (int64_t)ceil(rr);
        radius[i] = (int32_t)r;
        if (r <= 0) continue;
        tile_rect(u, v, r, tile, tx, ty, rect + 4 * i);
        touched[i] = (rect[4 * i + 2] - rect[4 * i]) * (rect[4 * i + 3] - rect[4 * i + 1]);
    }
}

/* Tile rectangles from given centres and radii (the same exact integer rule
 * as inside or_project), for binning records produced elsewhere. */
void or_rects(int64_t n, const double *uv, const int32_t *radius, int width, int height, int tile,
              int32_t *rect, int32_t *touched) {
    int tx = (width + tile - 1) / tile, ty = (height + tile - 1) / tile;
    for (int64_t i = 0; i < n; i++) {
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        touched[i] = 0;
        if (radius[i] <= 0) continue;
        tile_rect(uv[2 * i], uv[2 * i + 1], radius[i], tile, tx, ty, rect + 4 * i);
        touched[i] = (rect[4 * i + 2] - rect[4 * i]) * (rect[4 * i + 3] - rect[4 * i + 1]);
    }
}

/* -------------------------------------- A3-A5: binning and depth sort (Sec. 3.2.1) */
typedef struct { uint64_t key; uint32_t val; } kv_t;

static int kv_cmp(const void *pa, const void *pb) {
    const kv_t *a = (const kv_t *)pa, *b = (const kv_t *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->val < b->val ? -1 : (a->val > b->val);
}

int64_t or_count_instances(int64_t n, const int32_t *touched) {
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) m += touched[i];
    return m;
}

/*
 * One (key, value) instance per tile a splat touches; key = tile << 32 |
 * bits(depth_key), value = the splat's index (offset by view * n_per_view for
 * view v, whose tiles are numbered after those of views 0..v-1).  Instances are
 * ordered by key and then by value, which is the unique stable order.  ranges
 * receives [start, end) per tile.  Returns the instance count.
 *
 * n_views views of n_per_view splats each; tiles_per_view[v] = tx*ty of view v;
 * tx_per_view[v] = its tile columns.
 */
int64_t or_bin_sort(int n_views, int64_t n_per_view, const int32_t *rect, const float *depth_key,
                    const int32_t *tx_per_view, const int32_t *tiles_per_view,
                    uint64_t *keys, uint32_t *vals, uint32_t *ranges) {
    int64_t total_tiles = 0;
    for (int v = 0; v < n_views; v++) total_tiles += tiles_per_view[v];
    int64_t m = 0;
    for (int64_t i = 0; i < n_per_view * n_views; i++)
        m += (int64_t)(rect[4 * i + 2] - rect[4 * i]) * (rect[4 * i + 3] - rect[4 * i + 1]);
    kv_t *buf = (kv_t *)malloc(sizeof(kv_t) * (size_t)(m > 0 ? m : 1));
    int64_t k = 0, tile_base = 0;
    for (int v = 0; v < n_views; v++) {
        for (int64_t g = 0; g < n_per_view; g++) {
            int64_t i = (int64_t)v * n_per_view + g;
            uint32_t bits;
            memcpy(&bits, depth_key + i, 4);
            for (int y = rect[4 * i + 1]; y < rect[4 * i + 3]; y++)
                for (int x = rect[4 * i]; x < rect[4 * i + 2]; x++) {
                    uint64_t t = (uint64_t)(tile_base + (int64_t)y * tx_per_view[v] + x);
                    buf[k].key = (t << 32) | bits;
                    buf[k].val = (uint32_t)i;
                    k++;
                }
        }
        tile_base += tiles_per_view[v];
    }
    qsort(buf, (size_t)m, sizeof(kv_t), kv_cmp);
    for (int64_t t = 0; t < total_tiles; t++) ranges[2 * t] = ranges[2 * t + 1] = 0;
    for (int64_t j = 0; j < m; j++) {
        keys[j] = buf[j].key;
        vals[j] = buf[j].val;
        uint64_t t = buf[j].key >> 32;
        if (j == 0 || (buf[j - 1].key >> 32) != t) ranges[2 * t] = (uint32_t)j;
        ranges[2 * t + 1] = (uint32_t)(j + 1);
    }
    free(buf);
    return m;
}

/* ------------------------------------------- A6: front-to-back blend (Eq. 4-7, 10) */
/*
 * Splat j of a pixel's tile list, visited in sorted order:
 *   power = -1/2 (A dx^2 + C dy^2) - B dx dy, dx = px + 0.5 - u (Eq. 5)
 *   skip if power > 0 (numerical guard); alpha = min(alpha_max, o e^power)
 *   skip if alpha < alpha_min; stop (without blending) if T (1 - alpha) < T_min
 *   w = alpha T; accumulate w c, w d, w f, w; T <- T (1 - alpha)
 * Outputs: rgb = sum w c + T bg, depth = sum w d, sil = sum w (Eq. 10),
 * feat = sum w f, T_final, n_contrib = 1-based list position of the last
 * blended splat.
 *
 * Two further per-pixel figures say how well single-precision inputs determine
 * the pixel (they are not part of the method; the parity tests use them to
 * tell rounding from error).  The unit is a relative rounding eps of 1e-7.
 * Model: each splat's 2D covariance Sigma2D is known to within eps * lambda_max
 * per entry (it is formed in single precision from a 3D covariance), and its
 * alpha carries a further relative rounding of 4 eps (opacity, exponential,
 * product).  To first order a perturbation dSigma changes the exponent by
 * 1/2 y^T dSigma y with y = Sigma2D^-1 (dx, dy), so splat j's alpha moves by
 * at most r_j eps relative, r_j = 1/2 lambda_max (|y1| + |y2|)^2 + 4 (0 where
 * alpha is clamped at alpha_max).
 *   margin = the smallest gap of any threshold decision taken at the pixel
 *     over that decision's rounding bound (alpha against alpha_min and
 *     alpha_max: |ln(alpha / threshold)| over eps r_j; the transmittance stop:
 *     |ln(T (1 - alpha) / T_min)| over eps times the accumulated sensitivity of
 *     T (1 - alpha), sum of alpha_k r_k / (1 - alpha_k) + 1 per blended splat):
 *     a decision can flip only where margin < 1.
 *   sens = the first-order bound, in units of eps, of the absolute change of
 *     any of the pixel's colour, silhouette and feature values: for an output
 *     x, d out / d alpha_j = T_j (x_j - S_j) with S_j the blended value behind
 *     splat j, so |d out| <= eps sum_j w_j r_j |x_j - S_j|; the maximum over
 *     the channels.
 *   sens_depth = the same bound for the depth divided by |depth| (relative;
 *     0 where nothing is blended).
 *
 * Gaussian attributes are indexed by vals[j] (a view-local index after
 * subtracting view_offset); images are planar [C, H, W].
 */
typedef struct {
    int W, H, tile, tx, D;
    const double *uv, *conic, *opacity, *depth, *rgb, *feat;
    const uint32_t *vals, *ranges;
    const double *prm;
    int64_t view_offset, tile_offset;
    int conditioning; /* compute r_j and the decision margins (forward images only) */
} raster_ctx;

/* Blended splats of one pixel, front to back (scratch sized by the longest tile list). */
typedef struct {
    int64_t *pos;   /* view-local Gaussian index */
    double *alpha;  /* alpha_j */
    double *T;      /* transmittance in front of j */
    double *G;      /* e^power */
    int *clamped;   /* alpha clamped at alpha_max */
    double *r;      /* rounding sensitivity r_j of alpha_j (0 where clamped) */
} blend_list;

static int blend_list_alloc(blend_list *l, int64_t n) {
    size_t m = (size_t)(n > 0 ? n : 1);
    l->pos = (int64_t *)malloc(sizeof(int64_t) * m);
    l->alpha = (double *)malloc(sizeof(double) * m);
    l->T = (double *)malloc(sizeof(double) * m);
    l->G = (double *)malloc(sizeof(double) * m);
    l->clamped = (int *)malloc(sizeof(int) * m);
    l->r = (double *)malloc(sizeof(double) * m);
    return l->pos && l->alpha && l->T && l->G && l->clamped && l->r;
}

static void blend_list_free(blend_list *l) {
    free(l->pos); free(l->alpha); free(l->T); free(l->G); free(l->clamped); free(l->r);
}

/* Longest tile list of a view (scratch size of the per-pixel lists). */
static int64_t longest_tile(const uint32_t *ranges, int64_t tile_offset, int64_t n_tiles) {
    int64_t maxlen = 1;
    for (int64_t t = 0; t < n_tiles; t++) {
        int64_t len = (int64_t)ranges[2 * (tile_offset + t) + 1] - ranges[2 * (tile_offset + t)];
        if (len > maxlen) maxlen = len;
    }
    return maxlen;
}

/* Gap between a positive value and a threshold as |ln(a / b)|: a relative change
 * of a by e flips a < b only if |e| reaches it (to first order; the relative gap
 * |a - b| / b for a near b).  0 < a: underflow to 0 counts as an infinite gap. */
static double log_gap(double a, double b) { return a > 0 ? fabs(log(a / b)) : INFINITY; }

/* The unit eps of the rounding figures: a relative rounding of 1e-7 (about two
 * units in the last place of a single-precision value). */
#define COND_EPS 1e-7

/* Relative rounding sensitivity of alpha for a splat with conic cn evaluated at
 * offset (dx, dy), in units of eps (see the comment above): lambda_max of
 * Sigma2D = cn^-1 is 1 / lambda_min(cn) = (m + sqrt(m^2 - det)) / det. */
static double alpha_sensitivity(const double cn[3], double dx, double dy) {
    double det = cn[0] * cn[2] - cn[1] * cn[1];
    double m = 0.5 * (cn[0] + cn[2]);
    double disc = m * m - det;
    double lam = (m + sqrt(disc > 0 ? disc : 0)) / det;
    double y1 = cn[0] * dx + cn[1] * dy, y2 = cn[1] * dx + cn[2] * dy;
    double q = fabs(y1) + fabs(y2);
    return 0.5 * lam * q * q + 4.0;
}

/* Visit the splats of pixel (px, py) front to back; writes the blended list
 * into l and returns the number of blended splats. */
static int64_t blend_pixel(const raster_ctx *c, int px, int py, double *acc_rgb, double *acc_depth,
                           double *acc_sil, double *acc_feat, double *T_out, int64_t *last_out,
                           double *margin_out, blend_list *l) {
    const double *prm = c->prm;
    int64_t t = c->tile_offset + (int64_t)(py / c->tile) * c->tx + px / c->tile;
    uint32_t start = c->ranges[2 * t], end = c->ranges[2 * t + 1];
    double T = 1.0, margin = INFINITY, cT = 0.0;
    double pxc = px + 0.5, pyc = py + 0.5;
    int64_t nb = 0, last = 0;
    for (int d = 0; d < 3; d++) acc_rgb[d] = 0;
    *acc_depth = 0;
    *acc_sil = 0;
    for (int d = 0; d < c->D; d++) acc_feat[d] = 0;
    for (uint32_t j = start; j < end; j++) {
        int64_t g = (int64_t)c->vals[j] - c->view_offset;
        const double *cn = c->conic + 3 * g;
        double dx = pxc - c->uv[2 * g], dy = pyc - c->uv[2 * g + 1];
        double power = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
        if (power > 0) continue;
        double G = exp(power);
        double oG = c->opacity[g] * G;
        double alpha = oG < prm[P_ALPHA_MAX] ? oG : prm[P_ALPHA_MAX];
        int clamped = !(oG < prm[P_ALPHA_MAX]);
        double r = c->conditioning ? alpha_sensitivity(cn, dx, dy) : 1.0;
        if (c->conditioning) {
            double m1 = log_gap(oG, prm[P_ALPHA_MAX]) / (COND_EPS * r);
            if (m1 < margin) margin = m1;
            if (prm[P_ALPHA_MIN] > 0) {
                double m2 = log_gap(alpha, prm[P_ALPHA_MIN]) / (COND_EPS * r);
                if (m2 < margin) margin = m2;
            }
        }
        if (alpha < prm[P_ALPHA_MIN]) continue;
        double Tn = T * (1.0 - alpha);
        double r_alpha = clamped ? 0.0 : r;
        /* relative sensitivity of T (1 - alpha): the splats in front, this one, one rounding */
        double cTn = cT + alpha * r_alpha / (1.0 - alpha) + 1.0;
        if (c->conditioning && prm[P_T_MIN] > 0) {
            double m3 = log_gap(Tn, prm[P_T_MIN]) / (COND_EPS * cTn);
            if (m3 < margin) margin = m3;
        }
        if (Tn < prm[P_T_MIN]) break;
        double w = alpha * T;
        for (int d = 0; d < 3; d++) acc_rgb[d] += w * c->rgb[3 * g + d];
        *acc_depth += w * c->depth[g];
        *acc_sil += w;
        for (int d = 0; d < c->D; d++) acc_feat[d] += w * c->feat[(int64_t)c->D * g + d];
        l->pos[nb] = g;
        l->alpha[nb] = alpha;
        l->T[nb] = T;
        l->G[nb] = G;
        l->clamped[nb] = clamped;
        l->r[nb] = r_alpha;
        nb++;
        T = Tn;
        cT = cTn;
        last = (int64_t)(j - start) + 1;
    }
    *T_out = T;
    *last_out = last;
    *margin_out = margin;
    return nb;
}

/* First-order rounding bounds of a blended pixel (sens, sens_depth above):
 * walks the blended list back to front with the value S behind each splat of
 * every channel (background bg for colour, 0 for depth, silhouette and
 * features). */
static void pixel_sensitivity(const raster_ctx *c, const blend_list *l, int64_t nb, double depth,
                              double *S, double *kap, double *sens_out, double *sens_depth_out) {
    const double *prm = c->prm;
    int nch = 5 + c->D; /* r, g, b, depth, sil, features */
    for (int d = 0; d < 3; d++) S[d] = prm[P_BG_R + d];
    for (int ch = 3; ch < nch; ch++) S[ch] = 0;
    for (int ch = 0; ch < nch; ch++) kap[ch] = 0;
    for (int64_t k = nb - 1; k >= 0; k--) {
        int64_t g = l->pos[k];
        double alpha = l->alpha[k], wr = alpha * l->T[k] * l->r[k];
        for (int ch = 0; ch < nch; ch++) {
            double x = ch < 3 ? c->rgb[3 * g + ch]
                     : ch == 3 ? c->depth[g]
                     : ch == 4 ? 1.0
                     : c->feat[(int64_t)c->D * g + (ch - 5)];
            kap[ch] += wr * fabs(x - S[ch]);
            S[ch] = alpha * x + (1.0 - alpha) * S[ch];
        }
    }
    double m = 0;
    for (int ch = 0; ch < nch; ch++)
        if (ch != 3 && kap[ch] > m) m = kap[ch];
    *sens_out = m;
    *sens_depth_out = depth != 0 ? kap[3] / fabs(depth) : 0.0;
}

/* Renders one view.  Arrays out_* are planar [C, H, W] for that view; out_margin,
 * out_sens and out_sens_depth may be NULL (the rounding figures are then not computed). */
void or_render_fwd(int W, int H, int tile, int D, int64_t view_offset, int64_t tile_offset,
                   const double *uv, const double *conic, const double *opacity, const double *depth,
                   const double *rgb, const double *feat, const uint32_t *vals, const uint32_t *ranges,
                   const double *prm, double *out_rgb, double *out_depth, double *out_sil,
                   double *out_feat, double *out_T, int32_t *out_ncontrib, double *out_margin,
                   double *out_sens, double *out_sens_depth) {
    /* the rounding figures only when asked for (out_margin, out_sens, out_sens_depth not NULL) */
    int cond = out_margin && out_sens && out_sens_depth;
    raster_ctx c = {W, H, tile, (W + tile - 1) / tile, D, uv, conic, opacity, depth, rgb, feat,
                    vals, ranges, prm, view_offset, tile_offset, cond};
    int64_t P = (int64_t)W * H;
    int64_t maxlen = longest_tile(ranges, tile_offset, (int64_t)c.tx * ((H + tile - 1) / tile));
    #pragma omp parallel
    {
    blend_list l;
    int ok = blend_list_alloc(&l, maxlen);
    double *acc_feat = (double *)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));
    double *S = (double *)malloc(sizeof(double) * (size_t)(5 + D));
    double *kap = (double *)malloc(sizeof(double) * (size_t)(5 + D));
    #pragma omp for schedule(dynamic, 4)
        for (int py = 0; py < H; py++)
            for (int px = 0; ok && acc_feat && S && kap && px < W; px++) {
                int64_t pix = (int64_t)py * W + px;
                double acc_rgb[3], acc_depth, acc_sil, T, margin, sens, sens_depth;
                int64_t last;
                int64_t nb = blend_pixel(&c, px, py, acc_rgb, &acc_depth, &acc_sil, acc_feat, &T, &last, &margin,
                                         &l);
                if (cond) pixel_sensitivity(&c, &l, nb, acc_depth, S, kap, &sens, &sens_depth);
                for (int d = 0; d < 3; d++) out_rgb[d * P + pix] = acc_rgb[d] + T * prm[P_BG_R + d];
                out_depth[pix] = acc_depth;
                out_sil[pix] = acc_sil;
                for (int d = 0; d < D; d++) out_feat[d * P + pix] = acc_feat[d];
                out_T[pix] = T;
                out_ncontrib[pix] = (int32_t)last;
                if (cond) {
                    out_margin[pix] = margin;
                    out_sens[pix] = sens;
                    out_sens_depth[pix] = sens_depth;
                }
            }
    blend_list_free(&l);
    free(acc_feat); free(S); free(kap);
    }
}

/* ------------------------------------------------------- A8: blend backward */
/*
 * Gradient of the blended images w.r.t. each splat's 2D attributes, for one
 * view.  For each pixel the forward visit is repeated to list the blended
 * splats with their alpha and transmittance T_k (product of (1 - alpha) of the
 * splats in front).  Walking the list back to front with the value S_k of
 * everything behind splat k (S = background after the last splat):
 *   d out / d alpha_k = T_k (x_k - S_k),  S_{k-1} = alpha_k x_k + (1 - alpha_k) S_k
 *   d out / d x_k     = alpha_k T_k
 * for x in {rgb (background bg), depth, each feature, silhouette (x = 1)}.
 * Then alpha = o G (no gradient where clamped at alpha_max), G = e^power:
 *   d/do = G dalpha, d/dpower = o G dalpha,
 *   dpower/d(A,B,C) = (-dx^2/2, -dx dy, -dy^2/2), dpower/d(u,v) = (A dx + B dy, B dx + C dy).
 * Gradients are accumulated (+=) into per-splat outputs indexed view-locally.
 */
void or_render_bwd(int W, int H, int tile, int D, int64_t view_offset, int64_t tile_offset,
                   const double *uv, const double *conic, const double *opacity, const double *depth,
                   const double *rgb, const double *feat, const uint32_t *vals, const uint32_t *ranges,
                   const double *prm, const double *g_rgb, const double *g_depth, const double *g_sil,
                   const double *g_feat, double *d_uv, double *d_conic, double *d_opacity,
                   double *d_depth, double *d_rgb, double *d_feat) {
    raster_ctx c = {W, H, tile, (W + tile - 1) / tile, D, uv, conic, opacity, depth, rgb, feat,
                    vals, ranges, prm, view_offset, tile_offset, 0};
    int64_t P = (int64_t)W * H;
    int64_t maxlen = longest_tile(ranges, tile_offset, (int64_t)c.tx * ((H + tile - 1) / tile));
    int nch = 5 + D;
    #pragma omp parallel
    {
    blend_list l;
    int ok = blend_list_alloc(&l, maxlen);
    double *S = (double *)malloc(sizeof(double) * (size_t)nch);
    double *gx = (double *)malloc(sizeof(double) * (size_t)nch);
    double *x = (double *)malloc(sizeof(double) * (size_t)nch);
    double *acc_feat = (double *)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));

    #pragma omp for schedule(dynamic, 4)
    for (int py = 0; py < H; py++)
        for (int px = 0; ok && S && gx && x && acc_feat && px < W; px++) {
            int64_t pix = (int64_t)py * W + px;
            double acc_rgb[3], acc_depth, acc_sil, T, margin;
            int64_t last;
            int64_t nb = blend_pixel(&c, px, py, acc_rgb, &acc_depth, &acc_sil, acc_feat, &T, &last, &margin, &l);
            /* channel order: r, g, b, depth, sil, feat[0..D) */
            for (int d = 0; d < 3; d++) { gx[d] = g_rgb[d * P + pix]; S[d] = prm[P_BG_R + d]; }
            gx[3] = g_depth[pix]; S[3] = 0;
            gx[4] = g_sil[pix]; S[4] = 0;
            for (int d = 0; d < D; d++) { gx[5 + d] = g_feat[d * P + pix]; S[5 + d] = 0; }
            double pxc = px + 0.5, pyc = py + 0.5;
            for (int64_t k = nb - 1; k >= 0; k--) {
                int64_t g = l.pos[k];
                double alpha = l.alpha[k], Tk = l.T[k], w = alpha * Tk;
                for (int d = 0; d < 3; d++) x[d] = rgb[3 * g + d];
                x[3] = depth[g];
                x[4] = 1.0;
                for (int d = 0; d < D; d++) x[5 + d] = feat[(int64_t)D * g + d];
                double dalpha = 0;
                for (int ch = 0; ch < nch; ch++) {
                    dalpha += gx[ch] * Tk * (x[ch] - S[ch]);
                    S[ch] = alpha * x[ch] + (1.0 - alpha) * S[ch];
                }
                for (int d = 0; d < 3; d++) {
                    #pragma omp atomic
                    d_rgb[3 * g + d] += w * gx[d];
                }
                #pragma omp atomic
                d_depth[g] += w * gx[3];
                for (int d = 0; d < D; d++) {
                    #pragma omp atomic
                    d_feat[(int64_t)D * g + d] += w * gx[5 + d];
                }
                if (l.clamped[k]) continue; /* alpha clamped at alpha_max: flat in o and G */
                double G = l.G[k], o = opacity[g];
                #pragma omp atomic
                d_opacity[g] += G * dalpha;
                double dpow = o * G * dalpha;
                const double *cn = conic + 3 * g;
                double dx = pxc - uv[2 * g], dy = pyc - uv[2 * g + 1];
                #pragma omp atomic
                d_conic[3 * g] += -0.5 * dx * dx * dpow;
                #pragma omp atomic
                d_conic[3 * g + 1] += -dx * dy * dpow;
                #pragma omp atomic
                d_conic[3 * g + 2] += -0.5 * dy * dy * dpow;
                #pragma omp atomic
                d_uv[2 * g] += (cn[0] * dx + cn[1] * dy) * dpow;
                #pragma omp atomic
                d_uv[2 * g + 1] += (cn[1] * dx + cn[2] * dy) * dpow;
            }
        }
    blend_list_free(&l);
    free(S); free(gx); free(x); free(acc_feat);
    }
}

/* ------------------------------------ A9-A10: projection backward and pose (B.1) */
/*
 * Chain rule from the splat's 2D attributes back to the 3D parameters, and the
 * pose gradient as an SE(3) twist xi = (rho, phi) applied on the left,
 * T(xi) = Exp(xi) T_cw, at xi = 0 (supp. B.1 expands dL/dT_cw through Sigma2D
 * and the projected centre g_i; here the same chain is written per factor):
 *
 *   conic = Sigma2D^-1:      G2 = -conic Ghat conic, Ghat = [[dA, dB/2], [dB/2, dC]]
 *   Sigma2D = J Sc J^T:      Gc = J^T G2 J,  dJ = 2 G2 J Sc
 *   Sc = R_cw Sigma R_cw^T:  GSigma = R_cw^T Gc R_cw
 *   J(p) (through the clamped evaluation point), u(p), v(p), d = p_z give g_p;
 *   g_mu = R_cw^T g_p
 *   Sigma = M M^T, M = Rq diag(s): dM = 2 GSigma M -> ds, dRq -> dq_hat -> dq
 *   o = sigmoid(logit): dlogit = o (1 - o) do
 *   pose: p' = p + phi x p + rho, Sc' = Sc + [phi]x Sc - Sc [phi]x, so
 *         g_rho = sum g_p,  g_phi = sum p x g_p + 2 (A12, A20, A01), A = Sc Gc - Gc Sc
 *
 * d_* outputs are overwritten; twist receives the sum over all Gaussians.
 */
void or_project_bwd(int64_t n, const double *means, const double *quats, const double *log_scales,
                    const double *logits, const double *cam, const double *T, const double *prm,
                    const double *d_uv, const double *d_conic, const double *d_opacity,
                    const double *d_depth, double *d_means, double *d_quats, double *d_log_scales,
                    double *d_logits, double *twist) {
    double fx = cam[C_FX], fy = cam[C_FY];
    double Rcw[9] = {T[0], T[1], T[2], T[4], T[5], T[6], T[8], T[9], T[10]};
    double tcw[3] = {T[3], T[7], T[11]};
    double RcwT[9];
    transpose3(Rcw, RcwT);
    for (int k = 0; k < 6; k++) twist[k] = 0;
    double tw[6] = {0, 0, 0, 0, 0, 0};

    #pragma omp parallel for schedule(static) reduction(+ : tw[:6])
    for (int64_t i = 0; i < n; i++) {
        double *gm = d_means + 3 * i, *gq = d_quats + 4 * i, *gs = d_log_scales + 3 * i;
        for (int k = 0; k < 3; k++) gm[k] = gs[k] = 0;
        for (int k = 0; k < 4; k++) gq[k] = 0;
        double o = 1.0 / (1.0 + exp(-logits[i]));
        d_logits[i] = o * (1.0 - o) * d_opacity[i];

        const double *mu = means + 3 * i;
        double p[3];
        for (int r = 0; r < 3; r++) p[r] = Rcw[3 * r] * mu[0] + Rcw[3 * r + 1] * mu[1] + Rcw[3 * r + 2] * mu[2] + tcw[r];
        if (!(p[2] > prm[P_Z_NEAR])) continue;
        double q[4] = {quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3]};
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        if (!(qn > 0)) continue;
        double qh[4];
        for (int k = 0; k < 4; k++) qh[k] = q[k] / qn;
        double s[3] = {exp(log_scales[3 * i]), exp(log_scales[3 * i + 1]), exp(log_scales[3 * i + 2])};
        double Rq[9], M[9], MT[9], Sig[9], tmp[9], Sc[9];
        quat_to_rot(qh, Rq);
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) M[3 * r + c] = Rq[3 * r + c] * s[c];
        transpose3(M, MT);
        mm3(M, MT, Sig);
        mm3(Rcw, Sig, tmp);
        mm3(tmp, RcwT, Sc);
        double x = p[0], y = p[1], z = p[2], z2 = z * z;
        double tx_, ty_;
        int in_x, in_y;
        jacobian_point(p, cam, prm, &tx_, &ty_, &in_x, &in_y);
        double J[6] = {fx / z, 0, -fx * tx_ / z, 0, fy / z, -fy * ty_ / z};
        double JS[6];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++)
                JS[3 * r + c] = J[3 * r] * Sc[c] + J[3 * r + 1] * Sc[3 + c] + J[3 * r + 2] * Sc[6 + c];
        double a = JS[0] * J[0] + JS[1] * J[1] + JS[2] * J[2] + prm[P_LOWPASS];
        double b = JS[0] * J[3] + JS[1] * J[4] + JS[2] * J[5];
        double c = JS[3] * J[3] + JS[4] * J[4] + JS[5] * J[5] + prm[P_LOWPASS];
        double det = a * c - b * b;
        if (!(det > 0) || !isfinite(det)) continue;
        double A = c / det, B = -b / det, C = a / det;
        double Cn[4] = {A, B, B, C};

        /* conic -> Sigma2D */
        double Gh[4] = {d_conic[3 * i], 0.5 * d_conic[3 * i + 1], 0.5 * d_conic[3 * i + 1], d_conic[3 * i + 2]};
        double t2[4], G2[4];
        for (int r = 0; r < 2; r++)
            for (int cc = 0; cc < 2; cc++) t2[2 * r + cc] = Cn[2 * r] * Gh[cc] + Cn[2 * r + 1] * Gh[2 + cc];
        for (int r = 0; r < 2; r++)
            for (int cc = 0; cc < 2; cc++) G2[2 * r + cc] = -(t2[2 * r] * Cn[cc] + t2[2 * r + 1] * Cn[2 + cc]);

        /* Sigma2D -> Sc (Gc = J^T G2 J) and J (dJ = 2 G2 J Sc) */
        double Gc[9];
        for (int r = 0; r < 3; r++)
            for (int cc = 0; cc < 3; cc++) {
                double sacc = 0;
                for (int k = 0; k < 2; k++)
                    for (int l = 0; l < 2; l++) sacc += J[3 * k + r] * G2[2 * k + l] * J[3 * l + cc];
                Gc[3 * r + cc] = sacc;
            }
        double dJ[6];
        for (int r = 0; r < 2; r++)
            for (int cc = 0; cc < 3; cc++) {
                double sacc = 0;
                for (int l = 0; l < 2; l++) sacc += G2[2 * r + l] * JS[3 * l + cc];
                dJ[3 * r + cc] = 2.0 * sacc;
            }

        /* camera-frame centre: J(p), u(p), v(p), depth */
        double gp[3] = {0, 0, 0};
        double du = d_uv[2 * i], dv = d_uv[2 * i + 1];
        gp[0] += du * fx / z;
        gp[2] += -du * fx * x / z2;
        gp[1] += dv * fy / z;
        gp[2] += -dv * fy * y / z2;
        gp[2] += d_depth[i];
        /* J02 = -fx t_x / z, t_x = clamp(x / z): dt_x/dx = 1/z, dt_x/dz = -x/z^2 inside, 0 outside */
        double dtx_dx = in_x ? 1.0 / z : 0.0, dtx_dz = in_x ? -x / z2 : 0.0;
        double dty_dy = in_y ? 1.0 / z : 0.0, dty_dz = in_y ? -y / z2 : 0.0;
        gp[2] += dJ[0] * (-fx / z2);
        gp[0] += dJ[2] * (-fx / z) * dtx_dx;
        gp[2] += dJ[2] * (-fx * dtx_dz / z + fx * tx_ / z2);
        gp[2] += dJ[4] * (-fy / z2);
        gp[1] += dJ[5] * (-fy / z) * dty_dy;
        gp[2] += dJ[5] * (-fy * dty_dz / z + fy * ty_ / z2);
        for (int k = 0; k < 3; k++) gm[k] = RcwT[3 * k] * gp[0] + RcwT[3 * k + 1] * gp[1] + RcwT[3 * k + 2] * gp[2];

        /* Sc -> Sigma -> M -> (s, Rq) */
        double GS[9];
        mm3(RcwT, Gc, tmp);
        mm3(tmp, Rcw, GS);
        double dM[9];
        mm3(GS, M, dM);
        for (int k = 0; k < 9; k++) dM[k] *= 2.0;
        double dRq[9];
        for (int cc = 0; cc < 3; cc++) {
            double ds = 0;
            for (int r = 0; r < 3; r++) {
                ds += dM[3 * r + cc] * Rq[3 * r + cc];
                dRq[3 * r + cc] = dM[3 * r + cc] * s[cc];
            }
            gs[cc] = ds * s[cc];
        }
        /* Rq(w,x,y,z) -> q_hat */
        double w_ = qh[0], x_ = qh[1], y_ = qh[2], z_ = qh[3];
        double gw = 2 * (-z_ * dRq[1] + y_ * dRq[2] + z_ * dRq[3] - x_ * dRq[5] - y_ * dRq[6] + x_ * dRq[7]);
        double gx = 2 * (y_ * dRq[1] + z_ * dRq[2] + y_ * dRq[3] - 2 * x_ * dRq[4] - w_ * dRq[5] + z_ * dRq[6] + w_ * dRq[7] - 2 * x_ * dRq[8]);
        double gy = 2 * (-2 * y_ * dRq[0] + x_ * dRq[1] + w_ * dRq[2] + x_ * dRq[3] + z_ * dRq[5] - w_ * dRq[6] + z_ * dRq[7] - 2 * y_ * dRq[8]);
        double gz = 2 * (-2 * z_ * dRq[0] - w_ * dRq[1] + x_ * dRq[2] + w_ * dRq[3] - 2 * z_ * dRq[4] + y_ * dRq[5] + x_ * dRq[6] + y_ * dRq[7]);
        double gqh[4] = {gw, gx, gy, gz};
        double dot = gqh[0] * qh[0] + gqh[1] * qh[1] + gqh[2] * qh[2] + gqh[3] * qh[3];
        for (int k = 0; k < 4; k++) gq[k] = (gqh[k] - qh[k] * dot) / qn;

        /* pose twist */
        double Am[9], SG[9], GSc[9];
        mm3(Sc, Gc, SG);
        mm3(Gc, Sc, GSc);
        for (int k = 0; k < 9; k++) Am[k] = SG[k] - GSc[k];
        tw[0] += gp[0];
        tw[1] += gp[1];
        tw[2] += gp[2];
        tw[3] += y * gp[2] - z * gp[1] + 2.0 * Am[5];
        tw[4] += z * gp[0] - x * gp[2] + 2.0 * Am[6];
        tw[5] += x * gp[1] - y * gp[0] + 2.0 * Am[1];
    }
    for (int k = 0; k < 6; k++) twist[k] = tw[k];
}

/* -------------------------------------------------- A7: decoder and losses */
/*
 * Lower median (element floor((n-1)/2) of the sorted values), the statistic
 * behind the depth-error threshold of the tracking mask (Eq. 21).
 */
static int dbl_cmp(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : (x > y);
}

double or_lower_median(int64_t n, const double *values) {
    if (n <= 0) return 0.0;
    double *c = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(c, values, sizeof(double) * (size_t)n);
    qsort(c, (size_t)n, sizeof(double), dbl_cmp);
    double m = c[(n - 1) / 2];
    free(c);
    return m;
}

/*
 * Per-pixel loss of one view and its gradient w.r.t. the rendered images and
 * the decoder.  The decoder F_cnn of Eq. 8 is read as a 1x1 convolution, i.e.
 * logits z = W f + b per pixel (W is K x D).  Per pixel with mask m:
 *   colour   lc |c - c_gt|_1                      (Eq. 15 L1 part / tracking L1)
 *   depth    ld |d - d_gt|        where d_gt > 0  (Eq. 17)
 *   semantic ls (logsumexp(z) - z_label)  where label != 255 (cross-entropy, Eq. 16 reading)
 * each summed over pixels and divided by the pixel count P.
 * mask_mode 0: m = 1 (mapping).  mask_mode 1 (tracking, Eq. 21):
 *   m = [sil > tau_obs] [d_gt > 0] [|d - d_gt| < 10 median], the median being
 *   the lower median of |d - d_gt| over pixels with d_gt > 0; m is a constant
 *   for differentiation.  The L1 subgradient at 0 is 0.
 * Writes dL/d{rgb, depth, sil, feat}, accumulates (+=) dW, db; mask_out gets m;
 * terms[0..2] = colour, depth and semantic sums already divided by P and
 * weighted; returns the total.  median_out gets the median (0 if unused).
 */
double or_loss(int64_t P, int D, int K, const double *rgb, const double *depth, const double *sil,
               const double *feat, const double *t_rgb, const double *t_depth, const uint8_t *label,
               const double *Wd, const double *bd, double lc, double ld, double ls, int mask_mode,
               double tau_obs, double *g_rgb, double *g_depth, double *g_sil, double *g_feat,
               double *dW, double *db, double *mask_out, double *terms, double *median_out) {
    double med = 0.0;
    if (mask_mode == 1) {
        int64_t nv = 0;
        double *e = (double *)malloc(sizeof(double) * (size_t)(P > 0 ? P : 1));
        for (int64_t i = 0; i < P; i++)
            if (t_depth[i] > 0) e[nv++] = fabs(depth[i] - t_depth[i]);
        med = or_lower_median(nv, e);
        free(e);
    }
    *median_out = med;
    double *z = (double *)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
    double sc = 0, sd = 0, ss = 0;
    for (int64_t i = 0; i < P; i++) {
        double m = 1.0;
        if (mask_mode == 1)
            m = (sil[i] > tau_obs && t_depth[i] > 0 && fabs(depth[i] - t_depth[i]) < 10.0 * med) ? 1.0 : 0.0;
        mask_out[i] = m;
        for (int ch = 0; ch < 3; ch++) {
            double r = rgb[ch * P + i] - t_rgb[ch * P + i];
            sc += m * fabs(r);
            g_rgb[ch * P + i] = m * lc * (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / (double)P;
        }
        g_depth[i] = 0;
        if (t_depth[i] > 0) {
            double r = depth[i] - t_depth[i];
            sd += m * fabs(r);
            g_depth[i] = m * ld * (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / (double)P;
        }
        g_sil[i] = 0;
        for (int d = 0; d < D; d++) g_feat[(int64_t)d * P + i] = 0;
        if (K > 0 && label[i] != 255 && label[i] < K) {
            double zmax = -INFINITY;
            for (int k = 0; k < K; k++) {
                double s = bd[k];
                for (int d = 0; d < D; d++) s += Wd[k * D + d] * feat[(int64_t)d * P + i];
                z[k] = s;
                if (s > zmax) zmax = s;
            }
            double se = 0;
            for (int k = 0; k < K; k++) se += exp(z[k] - zmax);
            double lse = zmax + log(se);
            ss += m * (lse - z[label[i]]);
            for (int k = 0; k < K; k++) {
                double dz = m * ls * (exp(z[k] - lse) - (k == label[i] ? 1.0 : 0.0)) / (double)P;
                db[k] += dz;
                for (int d = 0; d < D; d++) {
                    dW[k * D + d] += dz * feat[(int64_t)d * P + i];
                    g_feat[(int64_t)d * P + i] += Wd[k * D + d] * dz;
                }
            }
        }
    }
    free(z);
    terms[0] = lc * sc / (double)P;
    terms[1] = ld * sd / (double)P;
    terms[2] = ls * ss / (double)P;
    return terms[0] + terms[1] + terms[2];
}

/* ---------------------------------------------------------- A11: DSR (Eq. 12) */
/*
 * s runs over the three axis scales exp(log_s) of every Gaussian (3N values).
 * mu_s, sigma_s = population mean and standard deviation (treated as constants
 * for differentiation); s_big = mu + 2 sigma, s_small = mu - 2 sigma.
 *   L_big = mean of s over {s > s_big}, L_small = mean of -log s over {s < s_small}
 * (an empty set gives 0).  Returns lb L_big + lsm L_small and accumulates its
 * gradient w.r.t. log_s into d_log_scales (+=): lb s / n_big on the big set,
 * -lsm / n_small on the small set.  stats = (mu, sigma, n_big, n_small, L_big, L_small).
 */
double or_dsr(int64_t n, const double *log_scales, double lb, double lsm, double *d_log_scales,
              double *stats) {
    int64_t m = 3 * n;
    double sum = 0;
    for (int64_t i = 0; i < m; i++) sum += exp(log_scales[i]);
    double mu = m > 0 ? sum / (double)m : 0.0;
    double var = 0;
    for (int64_t i = 0; i < m; i++) {
        double e = exp(log_scales[i]) - mu;
        var += e * e;
    }
    double sigma = m > 0 ? sqrt(var / (double)m) : 0.0;
    double hi = mu + 2 * sigma, lo = mu - 2 * sigma;
    double sb = 0, ssm = 0;
    int64_t nb = 0, ns = 0;
    for (int64_t i = 0; i < m; i++) {
        double s = exp(log_scales[i]);
        if (s > hi) { sb += s; nb++; }
        if (s < lo) { ssm += -log_scales[i]; ns++; }
    }
    double Lb = nb ? sb / (double)nb : 0.0, Ls = ns ? ssm / (double)ns : 0.0;
    for (int64_t i = 0; i < m; i++) {
        double s = exp(log_scales[i]);
        if (s > hi) d_log_scales[i] += lb * s / (double)nb;
        if (s < lo) d_log_scales[i] += -lsm / (double)ns;
    }
    stats[0] = mu; stats[1] = sigma; stats[2] = (double)nb; stats[3] = (double)ns;
    stats[4] = Lb; stats[5] = Ls;
    return lb * Lb + lsm * Ls;
}

/* --------------------------------------------------- A12: pose step (Sec. 3.4) */
/*
 * Adam step on the left twist xi = (rho, phi) with per-component learning
 * rates, then T <- Exp(delta) T with delta = -lr * mhat / (sqrt(vhat) + eps).
 * Exp is the SE(3) exponential: R = I + a [phi] + b [phi]^2,
 * V = I + b [phi] + c [phi]^2, t = V rho, with a = sin(t)/t, b = (1-cos t)/t^2,
 * c = (t - sin t)/t^3, t = |phi|.  state = m[6], v[6]; step is 1-based.
 */
void or_pose_step(double *T, const double *grad, double *m, double *v, int step, const double *lr,
                  double b1, double b2, double eps) {
    double delta[6];
    for (int k = 0; k < 6; k++) {
        m[k] = b1 * m[k] + (1 - b1) * grad[k];
        v[k] = b2 * v[k] + (1 - b2) * grad[k] * grad[k];
        double mh = m[k] / (1 - pow(b1, step)), vh = v[k] / (1 - pow(b2, step));
        delta[k] = -lr[k] * mh / (sqrt(vh) + eps);
    }
    double ph[3] = {delta[3], delta[4], delta[5]};
    double th = sqrt(ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2]);
    double a, b, c;
    if (th < 1e-8) { a = 1 - th * th / 6; b = 0.5 - th * th / 24; c = 1.0 / 6 - th * th / 120; }
    else { a = sin(th) / th; b = (1 - cos(th)) / (th * th); c = (th - sin(th)) / (th * th * th); }
    double K[9] = {0, -ph[2], ph[1], ph[2], 0, -ph[0], -ph[1], ph[0], 0};
    double K2[9];
    mm3(K, K, K2);
    double R[9], V[9];
    for (int k = 0; k < 9; k++) {
        double id = (k % 4 == 0) ? 1.0 : 0.0;
        R[k] = id + a * K[k] + b * K2[k];
        V[k] = id + b * K[k] + c * K2[k];
    }
    double t[3];
    for (int r = 0; r < 3; r++) t[r] = V[3 * r] * delta[0] + V[3 * r + 1] * delta[1] + V[3 * r + 2] * delta[2];
    double E[16] = {R[0], R[1], R[2], t[0], R[3], R[4], R[5], t[1], R[6], R[7], R[8], t[2], 0, 0, 0, 1};
    double out[16];
    for (int r = 0; r < 4; r++)
        for (int cc = 0; cc < 4; cc++) {
            double s = 0;
            for (int k = 0; k < 4; k++) s += E[4 * r + k] * T[4 * k + cc];
            out[4 * r + cc] = s;
        }
    memcpy(T, out, sizeof(out));
}

/* ------------------------------------------------------------------ SSIM
 * Structural similarity (Wang et al. 2004) of the rendered and observed colour,
 * the D-SSIM part of the mapping colour loss (Eq. 15, read as 1 - SSIM):
 * per channel and pixel p, the window moments over an 11x11 Gaussian window
 * (sigma 1.5, weights summing to one; pixels outside the image count as zero)
 *   mx = sum w x, my = sum w y, sx = sum w x^2 - mx^2, sy = sum w y^2 - my^2,
 *   sxy = sum w x y - mx my,
 *   S(p) = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx + sy + C2)),
 * C1 = 0.01^2, C2 = 0.03^2 (intensities in [0, 1]).  Returns the mean of S over
 * the 3 H W positions; grad (may be NULL) receives d(mean)/dx.  With the window
 * symmetric, dS(p)/dx(q) = w(q - p) (A(p) + 2 B(p) x(q) + C(p) y(q)) where
 * A = dS/dmx - 2 mx dS/dsx - my dS/dsxy, B = dS/dsx, C = dS/dsxy, so the
 * gradient is one more pass of the window over the maps A, B, C. */
double or_ssim(int64_t H, int64_t W, const double *x, const double *y, double *grad) {
    double g[11], gs = 0.0;
    for (int k = 0; k < 11; k++) {
        g[k] = exp(-(double)((k - 5) * (k - 5)) / (2.0 * 1.5 * 1.5));
        gs += g[k];
    }
    for (int k = 0; k < 11; k++) g[k] /= gs;
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    const int64_t P = H * W;
    double *A = NULL, *B = NULL, *Cm = NULL;
    if (grad) {
        A = (double *)calloc((size_t)P, sizeof(double));
        B = (double *)calloc((size_t)P, sizeof(double));
        Cm = (double *)calloc((size_t)P, sizeof(double));
    }
    double total = 0.0;
    for (int ch = 0; ch < 3; ch++) {
        const double *xc = x + ch * P, *yc = y + ch * P;
        for (int64_t py = 0; py < H; py++)
            for (int64_t px = 0; px < W; px++) {
                double mx = 0, my = 0, mxx = 0, myy = 0, mxy = 0;
                for (int dy = -5; dy <= 5; dy++)
                    for (int dx = -5; dx <= 5; dx++) {
                        const int64_t qy = py + dy, qx = px + dx;
                        if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;
                        const double w = g[dy + 5] * g[dx + 5];
                        const double a = xc[qy * W + qx], b = yc[qy * W + qx];
                        mx += w * a;
                        my += w * b;
                        mxx += w * a * a;
                        myy += w * b * b;
                        mxy += w * a * b;
                    }
                const double sx = mxx - mx * mx, sy = myy - my * my, sxy = mxy - mx * my;
                const double N1 = 2 * mx * my + C1, N2 = 2 * sxy + C2;
                const double D1 = mx * mx + my * my + C1, D2 = sx + sy + C2;
                const double S = N1 * N2 / (D1 * D2);
                total += S;
                if (grad) {
                    const double dS_dmx = 2 * my * N2 / (D1 * D2) - S * 2 * mx / D1;
                    const double dS_dsx = -S / D2;
                    const double dS_dsxy = 2 * N1 / (D1 * D2);
                    A[py * W + px] = dS_dmx - 2 * mx * dS_dsx - my * dS_dsxy;
                    B[py * W + px] = dS_dsx;
                    Cm[py * W + px] = dS_dsxy;
                }
            }
        if (!grad) continue;
        for (int64_t qy = 0; qy < H; qy++)
            for (int64_t qx = 0; qx < W; qx++) {
                double s = 0.0;
                const double a = xc[qy * W + qx], b = yc[qy * W + qx];
                for (int dy = -5; dy <= 5; dy++)
                    for (int dx = -5; dx <= 5; dx++) {
                        const int64_t py = qy + dy, px = qx + dx;
                        if (py < 0 || py >= H || px < 0 || px >= W) continue;
                        const double w = g[dy + 5] * g[dx + 5];
                        const int64_t p = py * W + px;
                        s += w * (A[p] + 2 * B[p] * a + Cm[p] * b);
                    }
                grad[ch * P + qy * W + qx] = s / (double)(3 * P);
            }
    }
    free(A);
    free(B);
    free(Cm);
    return total / (double)(3 * P);
}
