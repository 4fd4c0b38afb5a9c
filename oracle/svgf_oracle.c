/*
 * svgf_oracle.c -- plain, slow FP64 CPU statement of the spatiotemporal variance-guided
 * denoiser of "Hybrid-Rendering Techniques in GPU" (Granja & Pereira, 2021): Reinhard tone
 * mapping (Sec. 3.4), temporal accumulation with backward reprojection and moment/variance
 * estimation (Sec. 2, Sec. 3 step 4), history rectification by variance colour clamping or
 * clipping (Sec. 3.1), the adaptive start of the blur (Sec. 3.2), the edge-avoiding a-trous
 * wavelet passes with depth/normal/luminance-variance edge stopping (Sec. 2, Fig. 1, Sec. 3
 * step 5), the separable variant (Sec. 3.3), the inverse tone map (Sec. 3.4) and the
 * roughness-adapted number of a-trous passes (Sec. 3.5).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or constant table with
 * the CUDA path, and the CUDA path never calls it.
 *
 * Every stage is one plain loop nest over pixels (OpenMP over rows only), in FP64, in the
 * order the method states it.  The paper cites SVGF for the temporal filter and the a-trous
 * edge functions but prints none of their formulas; where it is silent the published SVGF
 * form is used, and each such reading is stated at the function that takes it.
 *
 * Layouts: images are row-major [H][W][C] doubles, pixel (x, y) at index y*W + x.
 *   colour          C=3  RGB
 *   gbuf            C=4  world unit normal (x, y, z), linear view-axis depth z
 *   motion          C=2  mv = p_cur - p_prev in pixels
 *   cv (colour+var) C=4  RGB, luminance variance
 *   moments         C=3  mu1 = E[l], mu2 = E[l^2], history length n
 *
 * Pins (what fixes each function independently of this file) are listed in the test suite.
 * The composition of all stages over a frame sequence (ora_denoise_frame) is pinned by its
 * closed form with the edge functions off on a static scene: every stage is then a linear map
 * (tone map, copy-reprojection, accumulation, dilated B3 correlations), the history is the
 * pass-0 output and the result the inverse map of the fifth pass.
 */
#include <float.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double alpha;              /* colour accumulation factor (0.2) */
    double alpha_moments;      /* moment accumulation factor (0.2) */
    double clamp_gamma;        /* clamp box half-width in std-devs (1.0) */
    int atrous_iters;          /* number of a-trous iterations (5) */
    double sigma_z, sigma_n, sigma_l; /* edge-stopping parameters (1, 128, 4) */
    int separable;             /* 0: 5x5 kernel, 1: horizontal then vertical 5-tap passes */
    int clamp_enable;          /* history rectification on/off */
    int adaptive_start;        /* start one scale higher above the roughness threshold */
    double roughness_threshold;/* 0.2 */
    int tonemap;               /* Reinhard before, inverse after */
    double luma_k;             /* lumaMultiplier of the forward map (1) */
    double inv_weight;         /* reinhardToneMappingWeight of the printed inverse (1) */
    int inverse_mode;          /* 0: exact inverse, 1: the printed (paper-literal) form */
    int history_from_pass;     /* a-trous pass whose output is the colour history; -1: the accumulated colour */
    double depth_rel_tol;      /* reprojection depth test: |z_prev - z| <= tol * z (0.1) */
    double normal_cos_tol;     /* reprojection normal test: cos angle >= tol (0.9) */
    double disocclusion_weight;/* bilinear weight sum below which history is dropped (1e-4) */
    int max_history;           /* history length cap (255) */
    int min_temporal_frames;   /* temporal variance once n >= this (4) */
    int spatial_var_radius;    /* spatial variance window radius (3 -> 7x7) */
    double eps;                /* guard in edge-stopping denominators (1e-10) */
    int rectify_mode;          /* history rectification: 0 variance colour clamping, 1 variance
                                  colour clipping (Sec. 3.1) */
    int iter_by_roughness;     /* per-pixel a-trous pass budget from the roughness (Sec. 3.5) */
    double iter_rough_t0, iter_rough_t1; /* budget thresholds (0, 0.05) */
    int iter_count0, iter_count1;        /* passes for roughness <= t0, <= t1 (0, 1); otherwise
                                            all atrous_iters */
} ora_config;

/* Threads the OpenMP loops use (1 without OpenMP). */
int ora_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Rec. 709 luma (the paper's luma() is not defined; Rec. 709 is the reading taken). */
double ora_luma(const double* c) { return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2]; }

/* B3-spline taps [1 4 6 4 1]/16 of the a-trous wavelet (Sec. 2, Fig. 1), and the [1 2 1]/4
 * taps of the 3x3 Gaussian that prefilters the variance guide. */
static const double B3[5] = {1.0 / 16.0, 4.0 / 16.0, 6.0 / 16.0, 4.0 / 16.0, 1.0 / 16.0};
static const double G3[3] = {0.25, 0.5, 0.25};

/* Number of neighbour visits of one a-trous iteration: 25 for the 5x5 kernel, 5 + 5 for the
 * separable variant (Sec. 3.3). */
int ora_atrous_taps(int separable) { return separable ? 10 : 25; }

/* ---------------------------------------------------------------- Sec. 3.4: Reinhard */

/* Forward tone map as printed: c /= (1 + luma(c) * k). */
void ora_tonemap(long n, const double* in, double* out, const ora_config* cf) {
    for (long i = 0; i < n; ++i) {
        double d = 1.0 + ora_luma(in + 3 * i) * cf->luma_k;
        for (int c = 0; c < 3; ++c) out[3 * i + c] = in[3 * i + c] / d;
    }
}

/* Inverse tone map.  Exact mode solves the forward map for c: luma(c') = L/(1+kL) gives
 * 1 + kL = 1/(1 - k luma(c')), so c = c' / (1 - k luma(c')) (denominator floored at 1e-6).
 * Paper-literal mode is the printed line: c = c' * (1 + luma(c')) * w. */
void ora_inverse_tonemap(long n, const double* in, double* out, const ora_config* cf) {
    for (long i = 0; i < n; ++i) {
        double l = ora_luma(in + 3 * i);
        double f;
        if (cf->inverse_mode == 1) {
            f = (1.0 + l) * cf->inv_weight;
        } else {
            double d = 1.0 - cf->luma_k * l;
            if (d < 1e-6) d = 1e-6;
            f = 1.0 / d;
        }
        for (int c = 0; c < 3; ++c) out[3 * i + c] = in[3 * i + c] * f;
    }
}

/* ------------------------------------------------------------ depth gradient (helper) */

/* Screen-space depth gradient: central differences inside, one-sided at the borders, zero
 * along an axis of extent 1.  Used by the depth edge-stopping function as the expected
 * depth change per pixel of offset. */
void ora_depth_gradient(int W, int H, const double* gbuf, double* grad) {
#pragma omp parallel for
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
#define Z(xx, yy) gbuf[4 * ((long)(yy) * W + (xx)) + 3]
            double gx, gy;
            if (W == 1) gx = 0.0;
            else if (x == 0) gx = Z(1, y) - Z(0, y);
            else if (x == W - 1) gx = Z(W - 1, y) - Z(W - 2, y);
            else gx = 0.5 * (Z(x + 1, y) - Z(x - 1, y));
            if (H == 1) gy = 0.0;
            else if (y == 0) gy = Z(x, 1) - Z(x, 0);
            else if (y == H - 1) gy = Z(x, H - 1) - Z(x, H - 2);
            else gy = 0.5 * (Z(x, y + 1) - Z(x, y - 1));
#undef Z
            grad[2 * ((long)y * W + x) + 0] = gx;
            grad[2 * ((long)y * W + x) + 1] = gy;
        }
}

/* ------------------------------------------------------- edge-stopping functions (Sec. 2) */

/* Depth: exp(-|z_q - z_p| / (sigma_z |grad z_p . (p - q)| + eps)). */
static double w_depth(double zp, double zq, const double* gp, double dx, double dy,
                      const ora_config* cf) {
    double den = cf->sigma_z * fabs(gp[0] * dx + gp[1] * dy) + cf->eps;
    return exp(-fabs(zq - zp) / den);
}

/* Normal: max(0, 1 - |n_p - n_q|^2 / 2) ^ sigma_n.  For unit normals 1 - |n_p - n_q|^2/2 is
 * n_p . n_q, i.e. this is SVGF's max(0, n_p . n_q)^sigma_n written in the form that does not
 * depend on the normals being unit to more than storage precision. */
static double w_normal(const double* np, const double* nq, const ora_config* cf) {
    double dx = np[0] - nq[0], dy = np[1] - nq[1], dz = np[2] - nq[2];
    double c = 1.0 - 0.5 * (dx * dx + dy * dy + dz * dz);
    if (c <= 0.0) return 0.0;
    return pow(c, cf->sigma_n);
}

/* Luminance: exp(-|l_p - l_q| / (sigma_l sqrt(g(var)_p) + eps)), g = 3x3 Gaussian prefilter
 * of the variance at the centre pixel (SVGF's variance-guided edge function, Sec. 2). */
static double w_luma(double lp, double lq, double den_l) { return exp(-fabs(lp - lq) / den_l); }

/* 3x3 [1 2 1]x[1 2 1]/16 blur of the variance channel of cv at (x, y), in-image taps only and
 * renormalised, always at unit step. */
static double var_prefilter(int W, int H, const double* cv, int x, int y) {
    double s = 0.0, ws = 0.0;
    for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
            int xx = x + a, yy = y + b;
            if (xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
            double k = G3[a + 1] * G3[b + 1];
            s += k * cv[4 * ((long)yy * W + xx) + 3];
            ws += k;
        }
    return s / ws;
}

/* Adaptive start level (Sec. 3.2): a pixel whose roughness is above the threshold starts the
 * a-trous iterations one scale higher.  The comparison is taken in FP32, the precision of the
 * roughness input, so that both implementations take the same decision. */
static int start_level(const double* rough, long p, const ora_config* cf) {
    if (!cf->adaptive_start || !rough) return 0;
    return (float)rough[p] > (float)cf->roughness_threshold ? 1 : 0;
}

/* Number of a-trous passes pixel p takes part in (Sec. 3.5, the roughness-adapted iteration
 * count): roughness <= t0 -> iter_count0, roughness <= t1 -> iter_count1, otherwise all
 * atrous_iters.  In a pass beyond its budget the pixel keeps its input colour and variance
 * (and is still read as a tap by its neighbours).  The comparisons are taken in FP32, the
 * precision of the roughness input. */
static int pass_budget(const double* rough, long p, const ora_config* cf) {
    if (!cf->iter_by_roughness || !rough) return cf->atrous_iters;
    float r = (float)rough[p];
    if (r <= (float)cf->iter_rough_t0) return cf->iter_count0;
    if (r <= (float)cf->iter_rough_t1) return cf->iter_count1;
    return cf->atrous_iters;
}

/* ------------------------------------------- Sec. 2 / Sec. 3 step 5: one a-trous pass */

/* One 5x5 edge-avoiding a-trous iteration `iter` at step 2^(iter + start level).
 * Weights w = h_j h_k w_z w_n w_l, colour out = sum w c / sum w, variance out =
 * sum w^2 var / (sum w)^2.  Taps outside the image are skipped (the sums renormalise). */
void ora_atrous_5x5(int W, int H, int iter, const double* cv_in, const double* gbuf,
                    const double* rough, double* cv_out, const ora_config* cf) {
    double* grad = (double*)malloc(sizeof(double) * 2 * (size_t)W * H);
    ora_depth_gradient(W, H, gbuf, grad);
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long p = (long)y * W + x;
            if (iter >= pass_budget(rough, p, cf)) {
                for (int c = 0; c < 4; ++c) cv_out[4 * p + c] = cv_in[4 * p + c];
                continue;
            }
            int step = 1 << (iter + start_level(rough, p, cf));
            const double* cp = cv_in + 4 * p;
            double lp = ora_luma(cp);
            double den_l = cf->sigma_l * sqrt(var_prefilter(W, H, cv_in, x, y)) + cf->eps;
            double sw = 0.0, sc[3] = {0.0, 0.0, 0.0}, sv = 0.0;
            for (int k = -2; k <= 2; ++k)
                for (int j = -2; j <= 2; ++j) {
                    int qx = x + j * step, qy = y + k * step;
                    if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                    long q = (long)qy * W + qx;
                    const double* cq = cv_in + 4 * q;
                    double w = B3[j + 2] * B3[k + 2] *
                               w_depth(gbuf[4 * p + 3], gbuf[4 * q + 3], grad + 2 * p,
                                       (double)(j * step), (double)(k * step), cf) *
                               w_normal(gbuf + 4 * p, gbuf + 4 * q, cf) *
                               w_luma(lp, ora_luma(cq), den_l);
                    sw += w;
                    for (int c = 0; c < 3; ++c) sc[c] += w * cq[c];
                    sv += w * w * cq[3];
                }
            for (int c = 0; c < 3; ++c) cv_out[4 * p + c] = sc[c] / sw;
            cv_out[4 * p + 3] = sv / (sw * sw);
        }
    free(grad);
}

/* Separable iteration (Sec. 3.3): the 5x5 kernel split into a horizontal and a vertical 5-tap
 * pass (5 + 5 neighbour visits).  The variance is updated only in the second (vertical) pass:
 * the horizontal pass filters the colour and passes the variance through; the vertical pass
 * filters the horizontal result's colour and its (unchanged) variance.  Both passes use the
 * same edge functions as the 5x5 kernel with the offset along their own axis, and the
 * luminance guide of both is the prefiltered variance of the iteration's input. */
void ora_atrous_separable(int W, int H, int iter, const double* cv_in, const double* gbuf,
                          const double* rough, double* cv_out, const ora_config* cf) {
    size_t n = (size_t)W * H;
    double* grad = (double*)malloc(sizeof(double) * 2 * n);
    double* mid = (double*)malloc(sizeof(double) * 4 * n);
    ora_depth_gradient(W, H, gbuf, grad);
    for (int pass = 0; pass < 2; ++pass) {
        const double* in = pass == 0 ? cv_in : mid;
        double* out = pass == 0 ? mid : cv_out;
#pragma omp parallel for schedule(dynamic, 4)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                long p = (long)y * W + x;
                if (iter >= pass_budget(rough, p, cf)) {
                    for (int c = 0; c < 4; ++c) out[4 * p + c] = in[4 * p + c];
                    continue;
                }
                int step = 1 << (iter + start_level(rough, p, cf));
                const double* cp = in + 4 * p;
                double lp = ora_luma(cp);
                double den_l = cf->sigma_l * sqrt(var_prefilter(W, H, in, x, y)) + cf->eps;
                double sw = 0.0, sc[3] = {0.0, 0.0, 0.0}, sv = 0.0;
                for (int j = -2; j <= 2; ++j) {
                    int dx = pass == 0 ? j * step : 0, dy = pass == 0 ? 0 : j * step;
                    int qx = x + dx, qy = y + dy;
                    if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                    long q = (long)qy * W + qx;
                    const double* cq = in + 4 * q;
                    double w = B3[j + 2] *
                               w_depth(gbuf[4 * p + 3], gbuf[4 * q + 3], grad + 2 * p, (double)dx,
                                       (double)dy, cf) *
                               w_normal(gbuf + 4 * p, gbuf + 4 * q, cf) *
                               w_luma(lp, ora_luma(cq), den_l);
                    sw += w;
                    for (int c = 0; c < 3; ++c) sc[c] += w * cq[c];
                    sv += w * w * cq[3];
                }
                for (int c = 0; c < 3; ++c) out[4 * p + c] = sc[c] / sw;
                out[4 * p + 3] = pass == 0 ? cp[3] : sv / (sw * sw);
            }
    }
    free(mid);
    free(grad);
}

void ora_atrous(int W, int H, int iter, const double* cv_in, const double* gbuf,
                const double* rough, double* cv_out, const ora_config* cf) {
    if (cf->separable) ora_atrous_separable(W, H, iter, cv_in, gbuf, rough, cv_out, cf);
    else ora_atrous_5x5(W, H, iter, cv_in, gbuf, rough, cv_out, cf);
}

/* --------------------------------------------- Sec. 2, Sec. 3.1: variance colour clamp */

/* Mean m and population standard deviation s, per RGB channel, of the current (tone-mapped)
 * colour over the 3x3 neighbourhood (in-image pixels only).  The box the history is expected
 * to lie in is m +- gamma s (Sec. 3.1). */
static void box_stats(int W, int H, const double* cur, int x, int y, double* m, double* s) {
    double v[3] = {0, 0, 0};
    int cnt = 0;
    m[0] = m[1] = m[2] = 0.0;
    for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
            int xx = x + a, yy = y + b;
            if (xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
            for (int c = 0; c < 3; ++c) m[c] += cur[3 * ((long)yy * W + xx) + c];
            ++cnt;
        }
    for (int c = 0; c < 3; ++c) m[c] /= cnt;
    for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
            int xx = x + a, yy = y + b;
            if (xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
            for (int c = 0; c < 3; ++c) {
                double d = cur[3 * ((long)yy * W + xx) + c] - m[c];
                v[c] += d * d;
            }
        }
    for (int c = 0; c < 3; ++c) s[c] = sqrt(v[c] / cnt);
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* History rectification of the history colour h (in place) against the box of centre m and
 * half-extents e = gamma s (Sec. 3.1, Fig. 3).
 *  clamping: each channel limited to [m - e, m + e];
 *  clipping: h moved toward the centre along the segment from m to h until it lies in the box,
 *            h' = m + (h - m) / t with t = max_c |h_c - m_c| / e_c when t > 1 (a channel with
 *            h_c = m_c does not constrain; one with e_c = 0 and h_c != m_c gives t = inf,
 *            i.e. h' = m); h is unchanged when it is inside the box. */
static void rectify(const ora_config* cf, const double* m, const double* s, double* h) {
    double e[3];
    for (int c = 0; c < 3; ++c) e[c] = cf->clamp_gamma * s[c];
    if (cf->rectify_mode == 0) {
        for (int c = 0; c < 3; ++c) h[c] = clampd(h[c], m[c] - e[c], m[c] + e[c]);
        return;
    }
    double t = 0.0;
    for (int c = 0; c < 3; ++c) {
        double d = h[c] - m[c];
        if (d == 0.0) continue;
        double r = e[c] > 0.0 ? fabs(d) / e[c] : INFINITY;
        if (r > t) t = r;
    }
    if (t > 1.0)
        for (int c = 0; c < 3; ++c) h[c] = isinf(t) ? m[c] : m[c] + (h[c] - m[c]) / t;
}

/* Stand-alone rectification stage: clamps (or clips, per rectify_mode) a given history colour
 * image against the 3x3 box of the current tone-mapped colour image. */
void ora_clamp(int W, int H, const double* cur, const double* hist, double* out,
               const ora_config* cf) {
#pragma omp parallel for
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long p = (long)y * W + x;
            double m[3], sd[3], h[3];
            box_stats(W, H, cur, x, y, m, sd);
            for (int c = 0; c < 3; ++c) h[c] = hist[3 * p + c];
            rectify(cf, m, sd, h);
            for (int c = 0; c < 3; ++c) out[3 * p + c] = h[c];
        }
}

/* ------------------------------------------ Sec. 2, Sec. 3 step 4: backward reprojection */

/* Backward reprojection of the previous frame's history to pixel p (the paper names the
 * technique but prints no formula; this is the SVGF form):
 *  - previous position (continuous, pixel-centre convention) q = p + 0.5 - mv(p);
 *  - bilinear footprint: base b = floor(q - 0.5), fraction f = q - 0.5 - b, taps b + {0,1}^2
 *    with weights (1-fx or fx)(1-fy or fy);
 *  - a tap is valid when it is inside the image, a previous frame exists, its previous depth
 *    agrees (|z_prev - z_p| <= depth_rel_tol * z_p) and its previous normal agrees
 *    (|n_p - n_prev|^2 <= 2 (1 - normal_cos_tol), i.e. cos angle >= normal_cos_tol for unit
 *    normals);
 *  - history colour and moments are the valid taps' bilinear average (weights renormalised);
 *    the previous history length is the largest among valid taps with non-zero weight;
 *  - if the valid weight sum is below disocclusion_weight the pixel is disoccluded (n_prev=0).
 * `margin` (optional) receives, per pixel, the smallest relative distance of any of these
 * threshold decisions to its threshold, so that a comparison against a lower-precision
 * implementation can tell which pixels sit on a decision. */
typedef struct {
    int valid;          /* history usable */
    double rgb[3];      /* reprojected history colour */
    double mu1, mu2;    /* reprojected moments */
    double n_prev;      /* previous history length */
    double margin;      /* smallest relative decision margin */
} reproj_result;

static void reproject_pixel(int W, int H, int x, int y, const double* gbuf,
                            const double* prev_gbuf, const double* motion, const double* hist_rgb,
                            const double* hist_mom, int has_history, const ora_config* cf,
                            reproj_result* r) {
    long p = (long)y * W + x;
    r->valid = 0;
    r->rgb[0] = r->rgb[1] = r->rgb[2] = 0.0;
    r->mu1 = r->mu2 = r->n_prev = 0.0;
    r->margin = INFINITY;
    if (!has_history || !prev_gbuf) return;
    double qx = x + 0.5 - motion[2 * p + 0], qy = y + 0.5 - motion[2 * p + 1];
    double bx = floor(qx - 0.5), by = floor(qy - 0.5);
    double fx = qx - 0.5 - bx, fy = qy - 0.5 - by;
    const double* gp = gbuf + 4 * p;
    double zp = gp[3];
    double ztol = cf->depth_rel_tol * zp;
    double ntol = 2.0 * (1.0 - cf->normal_cos_tol);
    double sw = 0.0, nmax = 0.0;
    for (int j = 0; j <= 1; ++j)
        for (int i = 0; i <= 1; ++i) {
            double w = (i ? fx : 1.0 - fx) * (j ? fy : 1.0 - fy);
            if (w <= 0.0) continue;
            double tx = bx + i, ty = by + j;
            if (tx < 0 || ty < 0 || tx >= W || ty >= H) continue;
            long t = (long)ty * W + (long)tx;
            const double* gt = prev_gbuf + 4 * t;
            double dz = fabs(gt[3] - zp);
            double dnx = gp[0] - gt[0], dny = gp[1] - gt[1], dnz = gp[2] - gt[2];
            double dn2 = dnx * dnx + dny * dny + dnz * dnz;
            double mz = fabs(ztol - dz) / (ztol > 0 ? ztol : 1.0);
            double mn = fabs(ntol - dn2) / ntol;
            if (mz < r->margin) r->margin = mz;
            if (mn < r->margin) r->margin = mn;
            if (!(dz <= ztol && dn2 <= ntol)) continue;
            sw += w;
            for (int c = 0; c < 3; ++c) r->rgb[c] += w * hist_rgb[3 * t + c];
            r->mu1 += w * hist_mom[3 * t + 0];
            r->mu2 += w * hist_mom[3 * t + 1];
            if (hist_mom[3 * t + 2] > nmax) nmax = hist_mom[3 * t + 2];
        }
    if (sw > 0.0) {
        double md = fabs(sw - cf->disocclusion_weight) / cf->disocclusion_weight;
        if (md < r->margin) r->margin = md;
    }
    if (sw < cf->disocclusion_weight) {
        r->rgb[0] = r->rgb[1] = r->rgb[2] = 0.0;
        r->mu1 = r->mu2 = r->n_prev = 0.0;
        return;
    }
    for (int c = 0; c < 3; ++c) r->rgb[c] /= sw;
    r->mu1 /= sw;
    r->mu2 /= sw;
    r->n_prev = nmax;
    r->valid = 1;
}

/* Stand-alone reprojection (for stage tests): history colour (3), moments (3: mu1, mu2,
 * n_prev) and a validity flag per pixel. */
void ora_reproject(int W, int H, const double* gbuf, const double* prev_gbuf,
                   const double* motion, const double* hist_rgb, const double* hist_mom,
                   int has_history, double* out_rgb, double* out_mom, double* out_valid,
                   double* margin, const ora_config* cf) {
#pragma omp parallel for
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long p = (long)y * W + x;
            reproj_result r;
            reproject_pixel(W, H, x, y, gbuf, prev_gbuf, motion, hist_rgb, hist_mom, has_history,
                            cf, &r);
            for (int c = 0; c < 3; ++c) out_rgb[3 * p + c] = r.rgb[c];
            out_mom[3 * p + 0] = r.mu1;
            out_mom[3 * p + 1] = r.mu2;
            out_mom[3 * p + 2] = r.n_prev;
            out_valid[p] = r.valid;
            if (margin) margin[p] = r.margin;
        }
}

/* ---------------------------------- Sec. 2, Sec. 3 step 4: accumulation and variance */

/* Spatial variance for short histories (n < min_temporal_frames): the moments of the
 * (2r+1)^2 neighbourhood averaged with depth and normal edge weights (unit-step offsets, no
 * luminance term), var = max(0, mu2 - mu1^2).  Paper silent; this is the SVGF convention. */
static double spatial_variance(int W, int H, int x, int y, const double* mom, const double* gbuf,
                               const double* grad, const ora_config* cf) {
    long p = (long)y * W + x;
    int R = cf->spatial_var_radius;
    double sw = 0.0, s1 = 0.0, s2 = 0.0;
    for (int b = -R; b <= R; ++b)
        for (int a = -R; a <= R; ++a) {
            int qx = x + a, qy = y + b;
            if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
            long q = (long)qy * W + qx;
            double w = w_depth(gbuf[4 * p + 3], gbuf[4 * q + 3], grad + 2 * p, a, b, cf) *
                       w_normal(gbuf + 4 * p, gbuf + 4 * q, cf);
            sw += w;
            s1 += w * mom[3 * q + 0];
            s2 += w * mom[3 * q + 1];
        }
    s1 /= sw;
    s2 /= sw;
    double v = s2 - s1 * s1;
    return v > 0.0 ? v : 0.0;
}

/* Temporal stage of one frame: tone map, reproject, clamp the history colour, accumulate
 * colour and moments, estimate variance.
 *   n      = min(n_prev + 1, max_history) with valid history, else 1
 *   a      = max(alpha, 1/n)          c   = (1 - a) hist + a c'
 *   a_m    = max(alpha_moments, 1/n)  mu_k = (1 - a_m) mu_k_prev + a_m l(c')^k, k = 1, 2
 *   var    = max(0, mu2 - mu1^2) if n >= min_temporal_frames, else the spatial estimate.
 * Output cv = (c, var) and moments (mu1, mu2, n). */
void ora_temporal(int W, int H, const double* noisy, const double* gbuf, const double* prev_gbuf,
                  const double* motion, const double* hist_rgb, const double* hist_mom,
                  int has_history, double* cv_out, double* mom_out, double* margin,
                  const ora_config* cf) {
    size_t n = (size_t)W * H;
    double* cur = (double*)malloc(sizeof(double) * 3 * n);
    double* grad = (double*)malloc(sizeof(double) * 2 * n);
    if (cf->tonemap) ora_tonemap((long)n, noisy, cur, cf);
    else memcpy(cur, noisy, sizeof(double) * 3 * n);
    ora_depth_gradient(W, H, gbuf, grad);
#pragma omp parallel for
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long p = (long)y * W + x;
            reproj_result r;
            reproject_pixel(W, H, x, y, gbuf, prev_gbuf, motion, hist_rgb, hist_mom, has_history,
                            cf, &r);
            const double* c = cur + 3 * p;
            double l = ora_luma(c);
            double hist[3] = {r.rgb[0], r.rgb[1], r.rgb[2]};
            double nn = 1.0, mu1p = 0.0, mu2p = 0.0;
            if (r.valid) {
                if (cf->clamp_enable) {
                    double m[3], sd[3];
                    box_stats(W, H, cur, x, y, m, sd);
                    rectify(cf, m, sd, hist);
                }
                nn = r.n_prev + 1.0;
                if (nn > cf->max_history) nn = cf->max_history;
                mu1p = r.mu1;
                mu2p = r.mu2;
            }
            double a = 1.0 / nn > cf->alpha ? 1.0 / nn : cf->alpha;
            double am = 1.0 / nn > cf->alpha_moments ? 1.0 / nn : cf->alpha_moments;
            for (int k = 0; k < 3; ++k) cv_out[4 * p + k] = (1.0 - a) * hist[k] + a * c[k];
            mom_out[3 * p + 0] = (1.0 - am) * mu1p + am * l;
            mom_out[3 * p + 1] = (1.0 - am) * mu2p + am * l * l;
            mom_out[3 * p + 2] = nn;
            if (margin) margin[p] = r.margin;
        }
#pragma omp parallel for
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long p = (long)y * W + x;
            double v;
            if (mom_out[3 * p + 2] >= cf->min_temporal_frames) {
                v = mom_out[3 * p + 1] - mom_out[3 * p + 0] * mom_out[3 * p + 0];
                if (v < 0.0) v = 0.0;
            } else {
                v = spatial_variance(W, H, x, y, mom_out, gbuf, grad, cf);
            }
            cv_out[4 * p + 3] = v;
        }
    free(grad);
    free(cur);
}

/* ------------------------------------------------------------- one whole frame */

/* Full frame: temporal stage, then atrous_iters a-trous iterations (5x5 or separable) with the
 * adaptive start, the output of pass `history_from_pass` (or the accumulated colour when it
 * is -1 or there are no iterations) becoming the next frame's colour history, then the
 * inverse tone map.  State in: hist_rgb (3), hist_mom (3) of the previous frame, has_history.
 * State out: hist_rgb_next (3), hist_mom_next (3).  Output rgb_out (4): RGB, final variance. */
void ora_denoise_frame(int W, int H, const double* noisy, const double* gbuf,
                       const double* prev_gbuf, const double* motion, const double* rough,
                       const double* hist_rgb, const double* hist_mom, int has_history,
                       double* hist_rgb_next, double* hist_mom_next, double* rgb_out,
                       double* margin, const ora_config* cf) {
    size_t n = (size_t)W * H;
    double* a = (double*)malloc(sizeof(double) * 4 * n);
    double* b = (double*)malloc(sizeof(double) * 4 * n);
    ora_temporal(W, H, noisy, gbuf, prev_gbuf, motion, hist_rgb, hist_mom, has_history, a,
                 hist_mom_next, margin, cf);
    int hp = cf->atrous_iters > 0 ? cf->history_from_pass : -1;
    if (hp < 0 || hp >= cf->atrous_iters)
        for (size_t p = 0; p < n; ++p)
            for (int c = 0; c < 3; ++c) hist_rgb_next[3 * p + c] = a[4 * p + c];
    for (int i = 0; i < cf->atrous_iters; ++i) {
        ora_atrous(W, H, i, a, gbuf, rough, b, cf);
        double* t = a; a = b; b = t;
        if (i == hp)
            for (size_t p = 0; p < n; ++p)
                for (int c = 0; c < 3; ++c) hist_rgb_next[3 * p + c] = a[4 * p + c];
    }
    double* rgb = (double*)malloc(sizeof(double) * 3 * n);
    for (size_t p = 0; p < n; ++p)
        for (int c = 0; c < 3; ++c) rgb[3 * p + c] = a[4 * p + c];
    if (cf->tonemap) ora_inverse_tonemap((long)n, rgb, rgb, cf);
    for (size_t p = 0; p < n; ++p) {
        for (int c = 0; c < 3; ++c) rgb_out[4 * p + c] = rgb[3 * p + c];
        rgb_out[4 * p + 3] = a[4 * p + 3];
    }
    free(rgb);
    free(b);
    free(a);
}

/* ================================================================================ learned part
 *
 * Kernel-predicting network standing in for a-trous iterations 2-5 (i.e. passes 1..4 after pass
 * 0).  Not in the paper: this is the learned extension of the denoiser, stated here plainly:
 *   input    x0 [B][H][W][10]: features of the pass-0 output (tone-mapped colour 3, sqrt of the
 *            variance 1, log2 depth 1, octahedral normal 2, albedo 3);
 *   layers   z_l = b_l + sum_{tap, ci} W_l[co][tap][ci] x_l[p + off(tap)][ci], 3x3 taps
 *            tap = (dy + 1) * 3 + (dx + 1), zero padding; x_{l+1} = max(0, z_l) for l < 3;
 *            channels 10 -> 32 -> 32 -> 32 -> 25; z_3 are the logits;
 *   kernel   K_i = softmax_i(z_3), i = (ky + 2) * 5 + (kx + 2) over the 5x5 offsets o_i = (kx, ky);
 *   apply    c1(p) = sum_i K_i c0(p + o_i) / sum_{i in image} K_i     (dilation 1)
 *            c2(p) = sum_i K_i c1(p + 4 o_i) / sum_{i in image} K_i   (dilation 4, same K)
 *   loss     mean over pixels and RGB of (c2 - target)^2.
 * Parameters are one flat array: for l = 0..3, W_l [co][9][ci] then b_l [co].
 * Pins: finite differences of ora_kpn_loss against ora_kpn_grad; a one-hot centre kernel is the
 * identity.
 *
 * Rounding mode (quant = 1, the *_q entry points): the same network with BF16 operands where a
 * tensor-core implementation keeps them in BF16 -- the weights W_l (not the biases), every
 * activation x_{l+1} = bf16(max(0, z_l)), the logits' gradient dz_3 and every data gradient
 * dz_{l-1} = bf16([z_{l-1} > 0] dx_l) -- with all sums still in FP64.  A BF16 value is the FP32
 * rounding of the exact value rounded to the nearest BF16, ties to even (an FP32 accumulator
 * rounded to BF16).  Features are taken as given (the caller passes BF16 values). */

/* FP32 rounding of v, then the nearest BF16 (ties to even), returned as a double. */
static double bf16_round(double v) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

void ora_bf16_round(long n, const double* in, double* out) {
    for (long i = 0; i < n; ++i) out[i] = bf16_round(in[i]);
}

static const int KPN_CIN[4] = {10, 32, 32, 32};
static const int KPN_COUT[4] = {32, 32, 32, 25};

int ora_kpn_param_count(void) {
    int n = 0;
    for (int l = 0; l < 4; ++l) n += KPN_COUT[l] * 9 * KPN_CIN[l] + KPN_COUT[l];
    return n;
}

static const double* kpn_w(const double* prm, int l) {
    const double* p = prm;
    for (int k = 0; k < l; ++k) p += KPN_COUT[k] * 9 * KPN_CIN[k] + KPN_COUT[k];
    return p;
}
static double* kpn_wm(double* prm, int l) { return (double*)kpn_w(prm, l); }

/* The parameters as the network uses them: a copy with the weights rounded to BF16 when quant is
 * set (the biases stay as given). */
static double* kpn_params_used(const double* prm, int quant) {
    int n = ora_kpn_param_count();
    double* q = (double*)malloc(sizeof(double) * n);
    memcpy(q, prm, sizeof(double) * n);
    if (quant)
        for (int l = 0; l < 4; ++l) {
            double* w = kpn_wm(q, l);
            for (long i = 0; i < (long)KPN_COUT[l] * 9 * KPN_CIN[l]; ++i) w[i] = bf16_round(w[i]);
        }
    return q;
}

/* One 3x3 convolution layer: out [B][H][W][co] = b + sum W x (zero padding). */
static void kpn_conv(int B, int H, int W, const double* x, int ci_n, const double* w,
                     const double* b, int co_n, double* z) {
#pragma omp parallel for collapse(2)
    for (int n = 0; n < B; ++n)
        for (int y = 0; y < H; ++y)
            for (int xx = 0; xx < W; ++xx)
                for (int co = 0; co < co_n; ++co) {
                    double s = b[co];
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int qy = y + dy, qx = xx + dx;
                            if (qy < 0 || qx < 0 || qy >= H || qx >= W) continue;
                            const double* xq = x + (((long)n * H + qy) * W + qx) * ci_n;
                            const double* wk = w + ((long)co * 9 + (dy + 1) * 3 + (dx + 1)) * ci_n;
                            for (int ci = 0; ci < ci_n; ++ci) s += wk[ci] * xq[ci];
                        }
                    z[(((long)n * H + y) * W + xx) * co_n + co] = s;
                }
}

/* Softmax of the 25 logits and the two kernel applications.  K [B][H][W][25], c1, c2 [..][3]. */
static void kpn_apply(int B, int H, int W, const double* logits, const double* c0, double* K,
                      double* c1, double* c2) {
    long np = (long)B * H * W;
    for (long p = 0; p < np; ++p) {
        const double* l = logits + p * 25;
        double m = l[0];
        for (int i = 1; i < 25; ++i) m = l[i] > m ? l[i] : m;
        double s = 0.0;
        for (int i = 0; i < 25; ++i) s += exp(l[i] - m);
        for (int i = 0; i < 25; ++i) K[p * 25 + i] = exp(l[i] - m) / s;
    }
    for (int pass = 0; pass < 2; ++pass) {
        const double* src = pass == 0 ? c0 : c1;
        double* dst = pass == 0 ? c1 : c2;
        int d = pass == 0 ? 1 : 4;
#pragma omp parallel for collapse(2)
        for (int n = 0; n < B; ++n)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    long p = ((long)n * H + y) * W + x;
                    double acc[3] = {0, 0, 0}, sk = 0.0;
                    for (int ky = -2; ky <= 2; ++ky)
                        for (int kx = -2; kx <= 2; ++kx) {
                            int qy = y + d * ky, qx = x + d * kx;
                            if (qy < 0 || qx < 0 || qy >= H || qx >= W) continue;
                            double k = K[p * 25 + (ky + 2) * 5 + (kx + 2)];
                            long q = ((long)n * H + qy) * W + qx;
                            for (int c = 0; c < 3; ++c) acc[c] += k * src[q * 3 + c];
                            sk += k;
                        }
                    for (int c = 0; c < 3; ++c) dst[p * 3 + c] = acc[c] / sk;
                }
    }
}

/* Forward pass: writes the predicted kernels K (optional), c1 (optional) and c2. */
void ora_kpn_forward_q(int B, int H, int W, const double* feat, const double* c0,
                       const double* prm_in, double* K_out, double* c1_out, double* c2_out,
                       int quant) {
    long np = (long)B * H * W;
    double* prm = kpn_params_used(prm_in, quant);
    double* a = (double*)malloc(sizeof(double) * np * 32);
    double* b = (double*)malloc(sizeof(double) * np * 32);
    double* K = K_out ? K_out : (double*)malloc(sizeof(double) * np * 25);
    double* c1 = c1_out ? c1_out : (double*)malloc(sizeof(double) * np * 3);
    const double* x = feat;
    for (int l = 0; l < 4; ++l) {
        const double* w = kpn_w(prm, l);
        const double* bias = w + KPN_COUT[l] * 9 * KPN_CIN[l];
        double* z = (l & 1) ? b : a;
        kpn_conv(B, H, W, x, KPN_CIN[l], w, bias, KPN_COUT[l], z);
        if (l < 3)
            for (long i = 0; i < np * KPN_COUT[l]; ++i) {
                z[i] = z[i] > 0.0 ? z[i] : 0.0;
                if (quant) z[i] = bf16_round(z[i]);
            }
        x = z;
    }
    kpn_apply(B, H, W, x, c0, K, c1, c2_out);
    if (!K_out) free(K);
    if (!c1_out) free(c1);
    free(b);
    free(a);
    free(prm);
}

void ora_kpn_forward(int B, int H, int W, const double* feat, const double* c0,
                     const double* prm, double* K_out, double* c1_out, double* c2_out) {
    ora_kpn_forward_q(B, H, W, feat, c0, prm, K_out, c1_out, c2_out, 0);
}

double ora_kpn_loss(int B, int H, int W, const double* feat, const double* c0,
                    const double* target, const double* prm) {
    long np = (long)B * H * W;
    double* c2 = (double*)malloc(sizeof(double) * np * 3);
    ora_kpn_forward(B, H, W, feat, c0, prm, NULL, NULL, c2);
    double s = 0.0;
    for (long i = 0; i < np * 3; ++i) s += (c2[i] - target[i]) * (c2[i] - target[i]);
    free(c2);
    return s / (double)(np * 3);
}

/* Loss and its gradient with respect to every parameter (flat, same layout). */
double ora_kpn_grad_q(int B, int H, int W, const double* feat, const double* c0,
                      const double* target, const double* prm_in, double* grad, int quant) {
    long np = (long)B * H * W;
    double* prm = kpn_params_used(prm_in, quant);
    int nparam = ora_kpn_param_count();
    /* forward, keeping every layer's input and pre-activation */
    double* xs[5];
    double* zs[4];
    xs[0] = (double*)feat;
    for (int l = 0; l < 4; ++l) {
        zs[l] = (double*)malloc(sizeof(double) * np * KPN_COUT[l]);
        const double* w = kpn_w(prm, l);
        kpn_conv(B, H, W, xs[l], KPN_CIN[l], w, w + KPN_COUT[l] * 9 * KPN_CIN[l], KPN_COUT[l], zs[l]);
        if (l < 3) {
            xs[l + 1] = (double*)malloc(sizeof(double) * np * KPN_COUT[l]);
            for (long i = 0; i < np * KPN_COUT[l]; ++i) {
                xs[l + 1][i] = zs[l][i] > 0.0 ? zs[l][i] : 0.0;
                if (quant) xs[l + 1][i] = bf16_round(xs[l + 1][i]);
            }
        }
    }
    double* K = (double*)malloc(sizeof(double) * np * 25);
    double* c1 = (double*)malloc(sizeof(double) * np * 3);
    double* c2 = (double*)malloc(sizeof(double) * np * 3);
    kpn_apply(B, H, W, zs[3], c0, K, c1, c2);
    double loss = 0.0;
    double* g2 = (double*)malloc(sizeof(double) * np * 3);   /* dL/dc2 */
    for (long i = 0; i < np * 3; ++i) {
        double d = c2[i] - target[i];
        loss += d * d;
        g2[i] = 2.0 * d / (double)(np * 3);
    }
    loss /= (double)(np * 3);
    double* gK = (double*)calloc((size_t)np * 25, sizeof(double));
    double* g1 = (double*)calloc((size_t)np * 3, sizeof(double));  /* dL/dc1 */
    /* apply 2 (dilation 4): c2 = sum K c1(q) / S -> dK and dc1 */
    for (int n = 0; n < B; ++n)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                long p = ((long)n * H + y) * W + x;
                double S = 0.0;
                for (int ky = -2; ky <= 2; ++ky)
                    for (int kx = -2; kx <= 2; ++kx) {
                        int qy = y + 4 * ky, qx = x + 4 * kx;
                        if (qy < 0 || qx < 0 || qy >= H || qx >= W) continue;
                        S += K[p * 25 + (ky + 2) * 5 + (kx + 2)];
                    }
                for (int ky = -2; ky <= 2; ++ky)
                    for (int kx = -2; kx <= 2; ++kx) {
                        int qy = y + 4 * ky, qx = x + 4 * kx;
                        if (qy < 0 || qx < 0 || qy >= H || qx >= W) continue;
                        long q = ((long)n * H + qy) * W + qx;
                        int i = (ky + 2) * 5 + (kx + 2);
                        for (int c = 0; c < 3; ++c) {
                            gK[p * 25 + i] += g2[p * 3 + c] * (c1[q * 3 + c] - c2[p * 3 + c]) / S;
                            g1[q * 3 + c] += g2[p * 3 + c] * K[p * 25 + i] / S;
                        }
                    }
            }
    /* apply 1 (dilation 1): c1 = sum K c0(q) / S -> dK (c0 is an input) */
    for (int n = 0; n < B; ++n)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                long p = ((long)n * H + y) * W + x;
                double S = 0.0;
                for (int ky = -2; ky <= 2; ++ky)
                    for (int kx = -2; kx <= 2; ++kx) {
                        int qy = y + ky, qx = x + kx;
                        if (qy < 0 || qx < 0 || qy >= H || qx >= W) continue;
                        S += K[p * 25 + (ky + 2) * 5 + (kx + 2)];
                    }
                for (int ky = -2; ky <= 2; ++ky)
                    for (int kx = -2; kx <= 2; ++kx) {
                        int qy = y + ky, qx = x + kx;
                        if (qy < 0 || qx < 0 || qy >= H || qx >= W) continue;
                        long q = ((long)n * H + qy) * W + qx;
                        int i = (ky + 2) * 5 + (kx + 2);
                        for (int c = 0; c < 3; ++c)
                            gK[p * 25 + i] += g1[p * 3 + c] * (c0[q * 3 + c] - c1[p * 3 + c]) / S;
                    }
            }
    /* softmax: dz_j = K_j (gK_j - sum_i K_i gK_i) */
    double* gz = (double*)malloc(sizeof(double) * np * 32);
    for (long p = 0; p < np; ++p) {
        double s = 0.0;
        for (int i = 0; i < 25; ++i) s += K[p * 25 + i] * gK[p * 25 + i];
        for (int i = 0; i < 25; ++i) {
            gz[p * 25 + i] = K[p * 25 + i] * (gK[p * 25 + i] - s);
            if (quant) gz[p * 25 + i] = bf16_round(gz[p * 25 + i]);
        }
    }
    /* layers, last to first: dW, db, and dx -> dz of the layer below through the ReLU */
    memset(grad, 0, sizeof(double) * nparam);
    for (int l = 3; l >= 0; --l) {
        int ci_n = KPN_CIN[l], co_n = KPN_COUT[l];
        double* gw = kpn_wm(grad, l);
        double* gb = gw + co_n * 9 * ci_n;
        const double* w = kpn_w(prm, l);
        const double* x = xs[l];
        for (int n = 0; n < B; ++n)
            for (int y = 0; y < H; ++y)
                for (int xx = 0; xx < W; ++xx) {
                    long p = ((long)n * H + y) * W + xx;
                    for (int co = 0; co < co_n; ++co) {
                        double g = gz[p * co_n + co];
                        gb[co] += g;
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                int qy = y + dy, qx = xx + dx;
                                if (qy < 0 || qx < 0 || qy >= H || qx >= W) continue;
                                long q = ((long)n * H + qy) * W + qx;
                                double* gwk = gw + ((long)co * 9 + (dy + 1) * 3 + (dx + 1)) * ci_n;
                                for (int ci = 0; ci < ci_n; ++ci) gwk[ci] += g * x[q * ci_n + ci];
                            }
                    }
                }
        if (l == 0) break;
        double* gx = (double*)calloc((size_t)np * ci_n, sizeof(double));
        for (int n = 0; n < B; ++n)
            for (int y = 0; y < H; ++y)
                for (int xx = 0; xx < W; ++xx) {
                    long p = ((long)n * H + y) * W + xx;
                    for (int co = 0; co < co_n; ++co) {
                        double g = gz[p * co_n + co];
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                int qy = y + dy, qx = xx + dx;
                                if (qy < 0 || qx < 0 || qy >= H || qx >= W) continue;
                                long q = ((long)n * H + qy) * W + qx;
                                const double* wk = w + ((long)co * 9 + (dy + 1) * 3 + (dx + 1)) * ci_n;
                                for (int ci = 0; ci < ci_n; ++ci) gx[q * ci_n + ci] += g * wk[ci];
                            }
                    }
                }
        /* through the ReLU of layer l-1: its input to layer l is max(0, z_{l-1}) */
        free(gz);
        gz = (double*)malloc(sizeof(double) * np * ci_n);
        for (long i = 0; i < np * ci_n; ++i) {
            gz[i] = zs[l - 1][i] > 0.0 ? gx[i] : 0.0;
            if (quant) gz[i] = bf16_round(gz[i]);
        }
        free(gx);
    }
    free(gz);
    free(g1);
    free(gK);
    free(g2);
    free(c2);
    free(c1);
    free(K);
    for (int l = 0; l < 4; ++l) free(zs[l]);
    for (int l = 1; l < 4; ++l) free(xs[l]);
    free(prm);
    return loss;
}

double ora_kpn_grad(int B, int H, int W, const double* feat, const double* c0,
                    const double* target, const double* prm, double* grad) {
    return ora_kpn_grad_q(B, H, W, feat, c0, target, prm, grad, 0);
}

/* Octahedral encoding of a unit normal: p = n.xy / (|x| + |y| + |z|), folded for z < 0 as
 * (1 - |p.y|) sign(p.x), (1 - |p.x|) sign(p.y), with sign(0) = +1. */
static void oct_encode(const double* n, double* o) {
    double s = fabs(n[0]) + fabs(n[1]) + fabs(n[2]);
    double x = n[0] / s, y = n[1] / s;
    if (n[2] < 0.0) {
        double tx = (1.0 - fabs(y)) * (x >= 0.0 ? 1.0 : -1.0);
        double ty = (1.0 - fabs(x)) * (y >= 0.0 ? 1.0 : -1.0);
        x = tx;
        y = ty;
    }
    o[0] = x;
    o[1] = y;
}

/* Network input features of one frame from the pass-0 output cv [H][W][4] (tone-mapped colour,
 * variance), the G-buffer and the albedo [H][W][3]: feat [H][W][10] = colour (3),
 * sqrt(max(0, var)) (1), log2(z) (1), octahedral normal (2), albedo (3). */
void ora_kpn_features(int W, int H, const double* cv, const double* gbuf, const double* albedo,
                      double* feat) {
    for (long p = 0; p < (long)W * H; ++p) {
        double* f = feat + p * 10;
        for (int c = 0; c < 3; ++c) f[c] = cv[4 * p + c];
        f[3] = sqrt(cv[4 * p + 3] > 0.0 ? cv[4 * p + 3] : 0.0);
        f[4] = log2(gbuf[4 * p + 3] > 1e-20 ? gbuf[4 * p + 3] : 1e-20);
        oct_encode(gbuf + 4 * p, f + 5);
        for (int c = 0; c < 3; ++c) f[7 + c] = albedo[3 * p + c];
    }
}

/* One 3x3 convolution layer (exposed for its pin). */
void ora_kpn_conv(int B, int H, int W, const double* x, int ci_n, const double* w,
                  const double* b, int co_n, double* z) {
    kpn_conv(B, H, W, x, ci_n, w, b, co_n, z);
}
