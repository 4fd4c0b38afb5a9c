/*
 * svgf_oracle.c -- plain, slow FP64 CPU statement of the spatiotemporal variance-guided
 * denoiser of "Hybrid-Rendering Techniques in GPU" (Granja & Pereira, 2021): Reinhard tone
 * mapping (Sec. 3.4), temporal accumulation with backward reprojection and moment/variance
 * estimation (Sec. 2, Sec. 3 step 4), history rectification by variance colour clamping
 * (Sec. 3.1), the adaptive start of the blur (Sec. 3.2), the edge-avoiding a-trous wavelet
 * passes with depth/normal/luminance-variance edge stopping (Sec. 2, Fig. 1, Sec. 3 step 5),
 * the separable variant (Sec. 3.3) and the inverse tone map (Sec. 3.4).
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
 * Pins (what fixes each function independently of this file) are listed in the test suite;
 * the composition of all stages over a frame sequence (ora_denoise_frame) is "parity
 * unpinned" beyond the per-stage pins: the paper prints no worked example.
 */
#include <float.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
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
 * colour over the 3x3 neighbourhood (in-image pixels only); the history colour is clamped to
 * [m - gamma s, m + gamma s]. */
static void clamp_box(int W, int H, const double* cur, int x, int y, double gamma, double* lo,
                      double* hi) {
    double m[3] = {0, 0, 0}, v[3] = {0, 0, 0};
    int cnt = 0;
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
    for (int c = 0; c < 3; ++c) {
        double s = sqrt(v[c] / cnt);
        lo[c] = m[c] - gamma * s;
        hi[c] = m[c] + gamma * s;
    }
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Stand-alone clamp stage: clamps a given history colour image against the 3x3 box of the
 * current tone-mapped colour image. */
void ora_clamp(int W, int H, const double* cur, const double* hist, double* out,
               const ora_config* cf) {
#pragma omp parallel for
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long p = (long)y * W + x;
            double lo[3], hi[3];
            clamp_box(W, H, cur, x, y, cf->clamp_gamma, lo, hi);
            for (int c = 0; c < 3; ++c) out[3 * p + c] = clampd(hist[3 * p + c], lo[c], hi[c]);
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
                    double lo[3], hi[3];
                    clamp_box(W, H, cur, x, y, cf->clamp_gamma, lo, hi);
                    for (int k = 0; k < 3; ++k) hist[k] = clampd(hist[k], lo[k], hi[k]);
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
