// Per-pixel CUDA kernels (sm_103a) of the variance-guided denoiser.
//
//   k_temporal          Sec. 3.4 forward map, Sec. 2 / Sec. 3 step 4 backward reprojection,
//                       Sec. 3.1 variance colour clamp, accumulation of colour and moments,
//                       temporal variance; flags tiles that hold short histories.
//   k_spatial_variance  Sec. 2: 7x7 depth/normal-weighted moment variance for n < 4
//                       (only tiles flagged by k_temporal do work).
//   k_atrous<MODE>      Sec. 2 Fig. 1 / Sec. 3 step 5 edge-avoiding a-trous iteration, 5x5
//                       (MODE 0) or the Sec. 3.3 separable horizontal (1) / vertical (2) pass,
//                       with the Sec. 3.2 adaptive start and, on the last pass, the Sec. 3.4
//                       inverse map fused into the store.
//   k_inverse, k_clamp  stand-alone Sec. 3.4 inverse and Sec. 3.1 clamp stages.
//
// One thread per pixel, 32x8 pixels per block: a warp covers 32 consecutive pixels of a row so
// every tap load of a warp is one contiguous 512-byte (float4) span.
//
// Accuracy notes (FP32 against the FP64 definition):
//  - the bilinear fraction of the reprojected position is taken from -mv alone (the pixel index
//    is an integer), so it does not lose the bits a large x would cost;
//  - the clamp's standard deviation is computed two-pass from the nine values in registers;
//  - the normal weight is (1 - t)^sigma_n with t = |n_p - n_q|^2 / 2 evaluated through
//    log1p(-t): t is formed from differences of nearby normals, which are exact or nearly so,
//    instead of 1 - n_p.n_q whose rounding sigma_n = 128 would amplify.
#include <math.h>

#include "svgf_internal.h"

namespace svgf {
namespace {

__device__ __forceinline__ float luma(float r, float g, float b) {
    return 0.2126f * r + 0.7152f * g + 0.0722f * b;
}

__device__ __forceinline__ float3 tonemap(const Params& P, float3 c) {
    if (!P.tonemap) return c;
    float d = 1.0f + luma(c.x, c.y, c.z) * P.luma_k;
    return make_float3(c.x / d, c.y / d, c.z / d);
}

__device__ __forceinline__ float3 inverse_tonemap(const Params& P, float3 c) {
    if (!P.tonemap) return c;
    float l = luma(c.x, c.y, c.z);
    float f;
    if (P.inverse_mode == 1) {
        f = (1.0f + l) * P.inv_weight;
    } else {
        float d = 1.0f - P.luma_k * l;
        d = d < 1e-6f ? 1e-6f : d;
        f = 1.0f / d;
    }
    return make_float3(c.x * f, c.y * f, c.z * f);
}

__device__ __forceinline__ float3 load_rgb(const float* __restrict__ p, long i) {
    return make_float3(__ldg(p + 3 * i), __ldg(p + 3 * i + 1), __ldg(p + 3 * i + 2));
}

// Central-difference depth gradient, one-sided at the borders, 0 along an axis of extent 1.
__device__ __forceinline__ float2 depth_grad(const float4* __restrict__ g, int x, int y, int W,
                                             int H) {
    float gx, gy;
    long row = (long)y * W;
    if (W == 1) gx = 0.f;
    else if (x == 0) gx = __ldg(&g[row + 1].w) - __ldg(&g[row].w);
    else if (x == W - 1) gx = __ldg(&g[row + W - 1].w) - __ldg(&g[row + W - 2].w);
    else gx = 0.5f * (__ldg(&g[row + x + 1].w) - __ldg(&g[row + x - 1].w));
    if (H == 1) gy = 0.f;
    else if (y == 0) gy = __ldg(&g[(long)W + x].w) - __ldg(&g[x].w);
    else if (y == H - 1) gy = __ldg(&g[(long)(H - 1) * W + x].w) - __ldg(&g[(long)(H - 2) * W + x].w);
    else gy = 0.5f * (__ldg(&g[(long)(y + 1) * W + x].w) - __ldg(&g[(long)(y - 1) * W + x].w));
    return make_float2(gx, gy);
}

// Natural log of the normal weight max(0, 1 - |a - b|^2 / 2)^sigma_n (-inf when it is 0).
__device__ __forceinline__ float log_w_normal(float4 a, float4 b, float sigma_n) {
    float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    float t = 0.5f * fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (!(t < 1.0f)) return -INFINITY;
    return sigma_n * log1pf(-t);
}

// Depth term of the log weight: |z_q - z_p| / (sigma_z |grad . offset| + eps).
__device__ __forceinline__ float depth_term(float zp, float zq, float2 gr, float dx, float dy,
                                            float sigma_z, float eps) {
    float den = fmaf(sigma_z, fabsf(fmaf(gr.x, dx, gr.y * dy)), eps);
    return __fdividef(fabsf(zq - zp), den);
}

__device__ __forceinline__ int start_level(const Params& P, const float* __restrict__ rough, long p) {
    if (!P.adaptive_start || rough == nullptr) return 0;
    return __ldg(rough + p) > P.rough_thr ? 1 : 0;
}

// [1 2 1] x [1 2 1] / 16 blur of the variance channel at (x, y), in-image taps renormalised.
__device__ __forceinline__ float var_prefilter(const float4* __restrict__ cv, int x, int y, int W,
                                               int H) {
    float s = 0.f, ws = 0.f;
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
        int yy = y + b;
        if (yy < 0 || yy >= H) continue;
#pragma unroll
        for (int a = -1; a <= 1; ++a) {
            int xx = x + a;
            if (xx < 0 || xx >= W) continue;
            float k = (a == 0 ? 0.5f : 0.25f) * (b == 0 ? 0.5f : 0.25f);
            s = fmaf(k, __ldg(&cv[(long)yy * W + xx].w), s);
            ws += k;
        }
    }
    return s / ws;
}

__device__ __forceinline__ float b3(int j) {  // j in -2..2
    return j == 0 ? 0.375f : ((j == 1 || j == -1) ? 0.25f : 0.0625f);
}

// ------------------------------------------------------------------------- temporal stage

__global__ void __launch_bounds__(TILE_X* TILE_Y)
k_temporal(Params P, const float* __restrict__ noisy, const float4* __restrict__ gbuf,
           const float4* __restrict__ prev_gbuf, const float2* __restrict__ mv,
           const float4* __restrict__ hist_prev, const float4* __restrict__ mom_prev,
           int has_history, float4* __restrict__ cv_out, float4* __restrict__ mom_out,
           float4* __restrict__ hist_accum_out, int* __restrict__ tile_flags) {
    const int W = P.W, H = P.H;
    const int x = blockIdx.x * TILE_X + threadIdx.x;
    const int y = blockIdx.y * TILE_Y + threadIdx.y;
    const bool inside = x < W && y < H;
    int short_history = 0;
    if (inside) {
        const long p = (long)y * W + x;
        const float3 c = tonemap(P, load_rgb(noisy, p));
        const float4 g = __ldg(&gbuf[p]);
        const float2 m = __ldg(&mv[p]);

        bool valid = false;
        float3 hist = make_float3(0.f, 0.f, 0.f);
        float mu1p = 0.f, Sp = 0.f, nprev = 0.f;
        if (has_history && prev_gbuf != nullptr && fabsf(m.x) < 1e7f && fabsf(m.y) < 1e7f) {
            // previous position p + 0.5 - mv; footprint base floor(x - mv), fraction frac(-mv)
            const float ux = -m.x, uy = -m.y;
            const float flx = floorf(ux), fly = floorf(uy);
            const float fx = ux - flx, fy = uy - fly;
            const int bx = x + (int)flx, by = y + (int)fly;
            const float ztol = P.depth_rel_tol * g.w;
            // up to four contributing taps, kept in registers for the two-pass moment blend
            float tw[4], tm1[4], tS[4];
            float sw = 0.f, nmax = 0.f;
            float3 hs = make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j <= 1; ++j)
#pragma unroll
                for (int i = 0; i <= 1; ++i) {
                    const int k = 2 * j + i;
                    tw[k] = 0.f;
                    tm1[k] = 0.f;
                    tS[k] = 0.f;
                    const float w = (i ? fx : 1.0f - fx) * (j ? fy : 1.0f - fy);
                    if (!(w > 0.f)) continue;
                    const int tx = bx + i, ty = by + j;
                    if (tx < 0 || ty < 0 || tx >= W || ty >= H) continue;
                    const long t = (long)ty * W + tx;
                    const float4 gp = __ldg(&prev_gbuf[t]);
                    const float dz = fabsf(gp.w - g.w);
                    const float ax = g.x - gp.x, ay = g.y - gp.y, az = g.z - gp.z;
                    const float dn2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
                    if (!(dz <= ztol && dn2 <= P.normal_tol2)) continue;
                    const float4 hh = __ldg(&hist_prev[t]);
                    const float4 mm = __ldg(&mom_prev[t]);
                    tw[k] = w;
                    tm1[k] = mm.x;
                    tS[k] = mm.y;
                    sw += w;
                    hs.x = fmaf(w, hh.x, hs.x);
                    hs.y = fmaf(w, hh.y, hs.y);
                    hs.z = fmaf(w, hh.z, hs.z);
                    nmax = fmaxf(nmax, mm.z);
                }
            if (sw >= P.disocc_w) {
                valid = true;
                hist = make_float3(hs.x / sw, hs.y / sw, hs.z / sw);
                // blended moments in central form: mean of mu1, and E[S] + Var[mu1] over taps
                float m1 = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) m1 = fmaf(tw[k], tm1[k], m1);
                m1 /= sw;
                float sS = 0.f, sd = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float d = tm1[k] - m1;
                    sS = fmaf(tw[k], tS[k], sS);
                    sd = fmaf(tw[k] * d, d, sd);
                }
                mu1p = m1;
                Sp = (sS + sd) / sw;
                nprev = nmax;
            }
        }

        if (valid && P.clamp_enable) {
            // 3x3 box of the current tone-mapped colour: mean and population std-dev, two-pass
            float3 v[9];
            int cnt = 0;
            float3 s = make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int b = -1; b <= 1; ++b)
#pragma unroll
                for (int a = -1; a <= 1; ++a) {
                    const int xx = x + a, yy = y + b;
                    if (xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
                    const float3 q = tonemap(P, load_rgb(noisy, (long)yy * W + xx));
                    v[cnt++] = q;
                    s.x += q.x; s.y += q.y; s.z += q.z;
                }
            const float fc = (float)cnt;
            const float3 mean = make_float3(s.x / fc, s.y / fc, s.z / fc);
            float3 ss = make_float3(0.f, 0.f, 0.f);
            for (int k = 0; k < cnt; ++k) {
                const float dx = v[k].x - mean.x, dy = v[k].y - mean.y, dz = v[k].z - mean.z;
                ss.x = fmaf(dx, dx, ss.x);
                ss.y = fmaf(dy, dy, ss.y);
                ss.z = fmaf(dz, dz, ss.z);
            }
            const float sx = sqrtf(ss.x / fc), sy = sqrtf(ss.y / fc), sz = sqrtf(ss.z / fc);
            hist.x = fminf(fmaxf(hist.x, mean.x - P.gamma * sx), mean.x + P.gamma * sx);
            hist.y = fminf(fmaxf(hist.y, mean.y - P.gamma * sy), mean.y + P.gamma * sy);
            hist.z = fminf(fmaxf(hist.z, mean.z - P.gamma * sz), mean.z + P.gamma * sz);
        }

        const float nn = valid ? fminf(nprev + 1.0f, P.max_history) : 1.0f;
        const float inv_n = 1.0f / nn;
        const float a = fmaxf(P.alpha, inv_n);
        const float am = fmaxf(P.alpha_m, inv_n);
        float3 ci;
        if (valid) {
            ci = make_float3(fmaf(a, c.x - hist.x, hist.x), fmaf(a, c.y - hist.y, hist.y),
                             fmaf(a, c.z - hist.z, hist.z));
        } else {
            ci = c;
        }
        // Moments in central form (mu1, S = mu2 - mu1^2).  The exponential update of
        // (mu1, mu2) by l is, exactly, mu1' = mu1 + a d and S' = (1 - a)(S + a d^2), d = l - mu1;
        // it keeps S free of the cancellation that mu2 - mu1^2 suffers in FP32.
        const float l = luma(c.x, c.y, c.z);
        float mu1, S;
        if (valid) {
            const float d = l - mu1p;
            mu1 = fmaf(am, d, mu1p);
            S = (1.0f - am) * fmaf(am * d, d, Sp);
        } else {
            mu1 = l;
            S = 0.f;
        }
        float var = 0.f;
        if (nn >= P.min_temporal) {
            var = fmaxf(0.f, S);
        } else {
            short_history = 1;
        }
        cv_out[p] = make_float4(ci.x, ci.y, ci.z, var);
        mom_out[p] = make_float4(mu1, S, nn, 0.f);
        if (hist_accum_out) hist_accum_out[p] = make_float4(ci.x, ci.y, ci.z, 0.f);
    }
    const int any_short = __syncthreads_or(short_history);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        tile_flags[blockIdx.y * gridDim.x + blockIdx.x] = any_short;
}

__global__ void __launch_bounds__(TILE_X* TILE_Y)
k_spatial_variance(Params P, const float4* __restrict__ gbuf, const float4* __restrict__ mom,
                   const int* __restrict__ tile_flags, float4* __restrict__ cv) {
    if (tile_flags[blockIdx.y * gridDim.x + blockIdx.x] == 0) return;
    const int W = P.W, H = P.H;
    const int x = blockIdx.x * TILE_X + threadIdx.x;
    const int y = blockIdx.y * TILE_Y + threadIdx.y;
    if (x >= W || y >= H) return;
    const long p = (long)y * W + x;
    if (__ldg(&mom[p].z) >= P.min_temporal) return;
    const float4 g = __ldg(&gbuf[p]);
    const float2 gr = depth_grad(gbuf, x, y, W, H);
    const int R = P.var_radius;
    // E_w[mu2] - E_w[mu1]^2 = E_w[S] + Var_w[mu1]; Var_w[mu1] is taken about the centre's mu1
    const float c1 = __ldg(&mom[p].x);
    float sw = 0.f, sS = 0.f, s1 = 0.f, s2 = 0.f;
    for (int b = -R; b <= R; ++b) {
        const int qy = y + b;
        if (qy < 0 || qy >= H) continue;
        for (int a = -R; a <= R; ++a) {
            const int qx = x + a;
            if (qx < 0 || qx >= W) continue;
            const long q = (long)qy * W + qx;
            const float4 gq = __ldg(&gbuf[q]);
            const float e = log_w_normal(g, gq, P.sigma_n) -
                            depth_term(g.w, gq.w, gr, (float)a, (float)b, P.sigma_z, P.eps);
            const float w = expf(e);
            const float4 mq = __ldg(&mom[q]);
            const float d = mq.x - c1;
            sw += w;
            sS = fmaf(w, mq.y, sS);
            s1 = fmaf(w, d, s1);
            s2 = fmaf(w * d, d, s2);
        }
    }
    const float m1 = s1 / sw;
    cv[p].w = fmaxf(0.f, sS / sw + (s2 / sw - m1 * m1));
}

// ------------------------------------------------------------------------- a-trous

template <int MODE>
__global__ void __launch_bounds__(TILE_X* TILE_Y)
k_atrous(Params P, int iter, const float4* __restrict__ cv_in, const float4* __restrict__ gbuf,
         const float* __restrict__ rough, float4* __restrict__ cv_out,
         float4* __restrict__ hist_out, float4* __restrict__ rgb_out) {
    const int W = P.W, H = P.H;
    const int x = blockIdx.x * TILE_X + threadIdx.x;
    const int y = blockIdx.y * TILE_Y + threadIdx.y;
    if (x >= W || y >= H) return;
    const long p = (long)y * W + x;
    const int step = 1 << (iter + start_level(P, rough, p));
    const float4 g = __ldg(&gbuf[p]);
    const float2 gr = depth_grad(gbuf, x, y, W, H);
    const float4 cp = __ldg(&cv_in[p]);
    const float lp = luma(cp.x, cp.y, cp.z);
    const float inv_dl = 1.0f / fmaf(P.sigma_l, sqrtf(var_prefilter(cv_in, x, y, W, H)), P.eps);

    float sw = 0.f, sr = 0.f, sg = 0.f, sb = 0.f, sv = 0.f;
    constexpr int KY0 = MODE == 1 ? 0 : -2, KY1 = MODE == 1 ? 0 : 2;
    constexpr int KX0 = MODE == 2 ? 0 : -2, KX1 = MODE == 2 ? 0 : 2;
#pragma unroll
    for (int k = KY0; k <= KY1; ++k) {
        const int qy = y + k * step;
        if (qy < 0 || qy >= H) continue;
#pragma unroll
        for (int j = KX0; j <= KX1; ++j) {
            const int qx = x + j * step;
            if (qx < 0 || qx >= W) continue;
            const long q = (long)qy * W + qx;
            const float4 cq = __ldg(&cv_in[q]);
            const float4 gq = __ldg(&gbuf[q]);
            const float e = log_w_normal(g, gq, P.sigma_n) -
                            depth_term(g.w, gq.w, gr, (float)(j * step), (float)(k * step),
                                       P.sigma_z, P.eps) -
                            fabsf(luma(cq.x, cq.y, cq.z) - lp) * inv_dl;
            const float h = MODE == 0 ? b3(j) * b3(k) : (MODE == 1 ? b3(j) : b3(k));
            const float w = h * expf(e);
            sw += w;
            sr = fmaf(w, cq.x, sr);
            sg = fmaf(w, cq.y, sg);
            sb = fmaf(w, cq.z, sb);
            sv = fmaf(w * w, cq.w, sv);
        }
    }
    float3 out = make_float3(sr / sw, sg / sw, sb / sw);
    const float var = MODE == 1 ? cp.w : sv / (sw * sw);
    if (hist_out) hist_out[p] = make_float4(out.x, out.y, out.z, 0.f);
    if (rgb_out) {
        const float3 o = inverse_tonemap(P, out);
        rgb_out[p] = make_float4(o.x, o.y, o.z, var);
    } else {
        cv_out[p] = make_float4(out.x, out.y, out.z, var);
    }
}

__global__ void k_inverse(Params P, const float4* __restrict__ cv_in, float4* rgb_out, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x) {
        const float4 c = cv_in[i];
        const float3 o = inverse_tonemap(P, make_float3(c.x, c.y, c.z));
        rgb_out[i] = make_float4(o.x, o.y, o.z, c.w);
    }
}

__global__ void __launch_bounds__(TILE_X* TILE_Y)
k_clamp(Params P, const float* __restrict__ noisy, const float4* __restrict__ hist_in,
        float4* __restrict__ hist_out) {
    const int W = P.W, H = P.H;
    const int x = blockIdx.x * TILE_X + threadIdx.x;
    const int y = blockIdx.y * TILE_Y + threadIdx.y;
    if (x >= W || y >= H) return;
    const long p = (long)y * W + x;
    float3 v[9];
    int cnt = 0;
    float3 s = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int b = -1; b <= 1; ++b)
#pragma unroll
        for (int a = -1; a <= 1; ++a) {
            const int xx = x + a, yy = y + b;
            if (xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
            const float3 q = tonemap(P, load_rgb(noisy, (long)yy * W + xx));
            v[cnt++] = q;
            s.x += q.x; s.y += q.y; s.z += q.z;
        }
    const float fc = (float)cnt;
    const float3 mean = make_float3(s.x / fc, s.y / fc, s.z / fc);
    float3 ss = make_float3(0.f, 0.f, 0.f);
    for (int k = 0; k < cnt; ++k) {
        const float dx = v[k].x - mean.x, dy = v[k].y - mean.y, dz = v[k].z - mean.z;
        ss.x = fmaf(dx, dx, ss.x);
        ss.y = fmaf(dy, dy, ss.y);
        ss.z = fmaf(dz, dz, ss.z);
    }
    const float sx = sqrtf(ss.x / fc), sy = sqrtf(ss.y / fc), sz = sqrtf(ss.z / fc);
    const float4 h = hist_in[p];
    hist_out[p] = make_float4(fminf(fmaxf(h.x, mean.x - P.gamma * sx), mean.x + P.gamma * sx),
                              fminf(fmaxf(h.y, mean.y - P.gamma * sy), mean.y + P.gamma * sy),
                              fminf(fmaxf(h.z, mean.z - P.gamma * sz), mean.z + P.gamma * sz), h.w);
}

}  // namespace

cudaError_t launch_temporal(const Params& P, const float* noisy, const float4* gbuf,
                            const float4* prev_gbuf, const float2* mv, const float4* hist_prev,
                            const float4* mom_prev, int has_history, float4* cv_out,
                            float4* mom_out, float4* hist_accum_out, int* tile_flags,
                            cudaStream_t s) {
    k_temporal<<<tile_grid(P.W, P.H), dim3(TILE_X, TILE_Y), 0, s>>>(
        P, noisy, gbuf, prev_gbuf, mv, hist_prev, mom_prev, has_history, cv_out, mom_out,
        hist_accum_out, tile_flags);
    return cudaGetLastError();
}

cudaError_t launch_spatial_variance(const Params& P, const float4* gbuf, const float4* mom,
                                    const int* tile_flags, float4* cv, cudaStream_t s) {
    k_spatial_variance<<<tile_grid(P.W, P.H), dim3(TILE_X, TILE_Y), 0, s>>>(P, gbuf, mom,
                                                                            tile_flags, cv);
    return cudaGetLastError();
}

cudaError_t launch_atrous(const Params& P, int mode, int iter, const float4* cv_in,
                          const float4* gbuf, const float* rough, float4* cv_out,
                          float4* hist_out, float4* rgb_out, cudaStream_t s) {
    const dim3 grid = tile_grid(P.W, P.H), block(TILE_X, TILE_Y);
    switch (mode) {
        case 0: k_atrous<0><<<grid, block, 0, s>>>(P, iter, cv_in, gbuf, rough, cv_out, hist_out, rgb_out); break;
        case 1: k_atrous<1><<<grid, block, 0, s>>>(P, iter, cv_in, gbuf, rough, cv_out, hist_out, rgb_out); break;
        default: k_atrous<2><<<grid, block, 0, s>>>(P, iter, cv_in, gbuf, rough, cv_out, hist_out, rgb_out); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_inverse(const Params& P, const float4* cv_in, float4* rgb_out, cudaStream_t s) {
    const long n = (long)P.W * P.H;
    const int threads = 256;
    long blocks = (n + threads - 1) / threads;
    if (blocks > 152L * 16) blocks = 152L * 16;
    k_inverse<<<(unsigned)blocks, threads, 0, s>>>(P, cv_in, rgb_out, n);
    return cudaGetLastError();
}

cudaError_t launch_clamp(const Params& P, const float* noisy, const float4* hist_in,
                         float4* hist_out, cudaStream_t s) {
    k_clamp<<<tile_grid(P.W, P.H), dim3(TILE_X, TILE_Y), 0, s>>>(P, noisy, hist_in, hist_out);
    return cudaGetLastError();
}

}  // namespace svgf
