// Device code shared by the single-frame kernels (svgf_kernels.cu) and the batched persistent
// kernels (svgf_batch.cu): helpers, the storage policies of the workspace images, and one function
// per stage that processes one tile of one image:
//
//   temporal_tile          Sec. 3.4 forward map, Sec. 2 / Sec. 3 step 4 backward reprojection,
//                          Sec. 3.1 variance colour clamp, accumulation of colour and moments,
//                          temporal variance; flags tiles that hold short histories.
//   spatial_variance_tile  Sec. 2: 7x7 depth/normal-weighted moment variance for n < 4.
//   atrous_tile<MODE>      Sec. 2 Fig. 1 / Sec. 3 step 5 edge-avoiding a-trous iteration, 5x5
//                          (MODE 0) or the Sec. 3.3 separable horizontal (1) / vertical (2) pass,
//                          with the Sec. 3.2 adaptive start and, on the last pass, the Sec. 3.4
//                          inverse map fused into the store.
//
// One thread per pixel; a warp covers 32 consecutive pixels of a row so every tap load of a warp
// is one contiguous span.
//
// Accuracy notes (FP32 against the FP64 definition):
//  - the bilinear fraction of the reprojected position is taken from -mv alone (the pixel index
//    is an integer), so it does not lose the bits a large x would cost;
//  - the clamp's standard deviation is computed two-pass from the window in shared memory;
//  - moments are kept in central form (mu1, S = mu2 - mu1^2) with the exact exponential update
//    of S, so the variance never comes from a cancelling difference of FP32 second moments;
//  - the normal weight is (1 - t)^sigma_n with t = |n_p - n_q|^2 / 2: t is formed from differences
//    of nearby normals, which are exact or nearly so, instead of 1 - n_p.n_q whose rounding
//    sigma_n = 128 would amplify, and log2(1 - t) comes from a series near t = 0.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "svgf_internal.h"

namespace svgf {
namespace dev {


// Rec. 709 luma, Reinhard forward and inverse maps (Sec. 3.4).  Written as explicit fused
// multiply-adds: every kernel that evaluates them then rounds identically (the compiler may not
// contract a plain a * b + c the same way in two kernels).
__device__ __forceinline__ float luma(float r, float g, float b) {
    return fmaf(0.0722f, b, fmaf(0.7152f, g, 0.2126f * r));
}

__device__ __forceinline__ float3 tonemap(const Params& P, float3 c) {
    if (!P.tonemap) return c;
    const float r = 1.0f / fmaf(luma(c.x, c.y, c.z), P.luma_k, 1.0f);
    return make_float3(c.x * r, c.y * r, c.z * r);
}

__device__ __forceinline__ float3 inverse_tonemap(const Params& P, float3 c) {
    if (!P.tonemap) return c;
    float l = luma(c.x, c.y, c.z);
    float f;
    if (P.inverse_mode == 1) {
        f = (1.0f + l) * P.inv_weight;
    } else {
        float d = fmaf(-P.luma_k, l, 1.0f);
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

// depth_grad for a pixel with all four neighbours in the image (same arithmetic, no branches).
__device__ __forceinline__ float2 depth_grad_interior(const float4* __restrict__ gp, int W) {
    return make_float2(0.5f * (__ldg(&gp[1].w) - __ldg(&gp[-1].w)),
                       0.5f * (__ldg(&gp[W].w) - __ldg(&gp[-W].w)));
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
template <class S>
__device__ __forceinline__ float var_prefilter(const typename S::Rec* __restrict__ cv, int x, int y,
                                               int W, int H) {
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
            s = fmaf(k, S::ld_var(cv, yy * W + xx), s);
            ws += k;
        }
    }
    return s / ws;
}

// var_prefilter for a pixel with its 3x3 neighbourhood in the image: the nine weights sum to 1
// exactly, so the same sum in the same order gives the same value.
template <class S>
__device__ __forceinline__ float var_prefilter_interior(const typename S::Rec* __restrict__ cp, int W) {
    float s = 0.f;
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
#pragma unroll
        for (int a = -1; a <= 1; ++a) {
            const float k = (a == 0 ? 0.5f : 0.25f) * (b == 0 ? 0.5f : 0.25f);
            s = fmaf(k, S::ld_var(cp + b * W, a), s);
        }
    }
    return s;
}

// ------------------------------------------------------------------------- storage policies
//
// Workspace images: colour + variance (cv: r, g, b, var), colour history (hist: r, g, b, -) and
// moments (mom: mu1, S = mu2 - mu1^2, n, -).  StoreF32 keeps each pixel as a float4.  Store16<BF>
// packs each into 8 bytes: colour and mu1 as FP16 (BF = false) or BF16 (BF = true); the
// variance-type fields (var, S) always as BF16, whose 8-bit exponent keeps the small variances of
// the late a-trous passes that FP16 would flush to subnormals or zero; n as an exact 16-bit
// integer.  All arithmetic stays FP32: values are widened on load and rounded on store.
struct StoreF32 {
    using Rec = float4;
    __device__ static float4 ld_cv(const Rec* b, int i) { return __ldg(b + i); }
    __device__ static float ld_var(const Rec* b, int i) { return __ldg(&b[i].w); }
    __device__ static void st_cv(Rec* b, int i, float4 v) { b[i] = v; }
    __device__ static void st_var(Rec* b, int i, float v) { b[i].w = v; }
    __device__ static float4 ld_hist(const Rec* b, int i) { return __ldg(b + i); }
    __device__ static void st_hist(Rec* b, int i, float3 c) { b[i] = make_float4(c.x, c.y, c.z, 0.f); }
    __device__ static float4 ld_mom(const Rec* b, int i) { return __ldg(b + i); }
    __device__ static float ld_n(const Rec* b, int i) { return __ldg(&b[i].z); }
    __device__ static void st_mom(Rec* b, int i, float mu1, float S, float n) {
        b[i] = make_float4(mu1, S, n, 0.f);
    }
    __device__ static float4 round_cv(float4 v) { return v; }
};

template <bool BF>
struct Store16 {
    using Rec = uint2;
    __device__ static unsigned enc_c(float x) {
        return BF ? (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(x))
                  : (unsigned)__half_as_ushort(__float2half_rn(x));
    }
    __device__ static float dec_c(unsigned u) {
        return BF ? __uint_as_float(u << 16) : __half2float(__ushort_as_half((unsigned short)u));
    }
    __device__ static unsigned enc_v(float x) {
        return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(x));
    }
    __device__ static float dec_v(unsigned u) { return __uint_as_float(u << 16); }
    __device__ static float4 ld_cv(const Rec* b, int i) {
        const uint2 u = __ldg(b + i);
        return make_float4(dec_c(u.x & 0xffffu), dec_c(u.x >> 16), dec_c(u.y & 0xffffu), dec_v(u.y >> 16));
    }
    __device__ static float ld_var(const Rec* b, int i) {
        return dec_v(__ldg(reinterpret_cast<const unsigned short*>(b) + 4 * i + 3));
    }
    __device__ static void st_cv(Rec* b, int i, float4 v) {
        b[i] = make_uint2(enc_c(v.x) | (enc_c(v.y) << 16), enc_c(v.z) | (enc_v(v.w) << 16));
    }
    __device__ static void st_var(Rec* b, int i, float v) {
        reinterpret_cast<unsigned short*>(b)[4 * i + 3] = (unsigned short)enc_v(v);
    }
    __device__ static float4 ld_hist(const Rec* b, int i) {
        const uint2 u = __ldg(b + i);
        return make_float4(dec_c(u.x & 0xffffu), dec_c(u.x >> 16), dec_c(u.y & 0xffffu), 0.f);
    }
    __device__ static void st_hist(Rec* b, int i, float3 c) {
        b[i] = make_uint2(enc_c(c.x) | (enc_c(c.y) << 16), enc_c(c.z));
    }
    __device__ static float4 ld_mom(const Rec* b, int i) {
        const uint2 u = __ldg(b + i);
        return make_float4(dec_c(u.x & 0xffffu), dec_v(u.x >> 16), (float)(u.y & 0xffffu), 0.f);
    }
    __device__ static float ld_n(const Rec* b, int i) {
        return (float)__ldg(reinterpret_cast<const unsigned short*>(b) + 4 * i + 2);
    }
    __device__ static void st_mom(Rec* b, int i, float mu1, float S, float n) {
        b[i] = make_uint2(enc_c(mu1) | (enc_v(S) << 16), (unsigned)n);
    }
    // The value a cv record would hold after a store and a load.
    __device__ static float4 round_cv(float4 v) {
        return make_float4(dec_c(enc_c(v.x)), dec_c(enc_c(v.y)), dec_c(enc_c(v.z)), dec_v(enc_v(v.w)));
    }
};

// ------------------------------------------------------------------------- temporal stage

// History rectification of h against the 3x3 box of centre m and half-extents e = gamma sigma
// (Sec. 3.1, Fig. 3).  mode 0 (clamping): each channel limited to [m - e, m + e].  mode 1
// (clipping): h moved toward m along the line from m until it lies in the box:
// h' = m + (h - m) / t, t = max_c |h_c - m_c| / e_c, when t > 1; a channel with h_c = m_c
// does not constrain, one with e_c = 0 and h_c != m_c gives t = inf, i.e. h' = m.
__device__ __forceinline__ float3 rectify(int mode, float3 h, const float* m, const float* e) {
    if (mode == 0)
        return make_float3(fminf(fmaxf(h.x, m[0] - e[0]), m[0] + e[0]),
                           fminf(fmaxf(h.y, m[1] - e[1]), m[1] + e[1]),
                           fminf(fmaxf(h.z, m[2] - e[2]), m[2] + e[2]));
    const float d[3] = {h.x - m[0], h.y - m[1], h.z - m[2]};
    float t = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (d[c] == 0.f) continue;
        const float r = e[c] > 0.f ? fabsf(d[c]) / e[c] : INFINITY;
        t = fmaxf(t, r);
    }
    if (!(t > 1.0f)) return h;
    if (isinf(t)) return make_float3(m[0], m[1], m[2]);
    return make_float3(m[0] + d[0] / t, m[1] + d[1] / t, m[2] + d[2] / t);
}

// Shared-memory tile of the temporal stage: the tone-mapped colour of a TILE_X x TILE_Y tile with
// a one-pixel halo, one plane per channel.
struct TemporalSmem {
    float c[3][TILE_Y + 2][TILE_X + 2];
};

// Resident blocks per SM the temporal kernels' register budget is set for: 3 (up to 85
// registers) keeps the twelve reprojection gathers in flight across the tile fill without
// spilling; 4 (64 registers) spilled and measured 20 % slower at 4K.
constexpr int kTemporalBlocksPerSM = 3;

// The temporal stage for the TILE_X x TILE_Y tile at (x0, y0) of a W x H image, by a block of
// TILE_X x TILE_Y threads.  *flag receives whether any pixel of the tile has a short history.
// Contains block-wide barriers: every thread of the block must call it.
template <class S>
__device__ __forceinline__ void temporal_tile(
    const Params& P, int W, int H, int x0, int y0, int* flag, const float* __restrict__ noisy,
    const float4* __restrict__ gbuf, const float4* __restrict__ prev_gbuf,
    const float2* __restrict__ mv, const typename S::Rec* __restrict__ hist_prev,
    const typename S::Rec* __restrict__ mom_prev, int has_history,
    typename S::Rec* __restrict__ cv_out, typename S::Rec* __restrict__ mom_out,
    typename S::Rec* __restrict__ hist_accum_out, TemporalSmem& sm) {
    const int x = x0 + threadIdx.x;
    const int y = y0 + threadIdx.y;
    const bool inside = x < W && y < H;
    // Loads in dependency order, each group issued before the previous one is consumed: the
    // pixel's own G-buffer record and motion vector, the noisy colour of the tile fill, then
    // (once the motion vector is in) the reprojection taps, whose latency thereby overlaps the
    // tile fill and its barrier.
    const long p0 = inside ? (long)y * W + x : 0;
    const float4 g = __ldg(&gbuf[p0]);
    const float2 m = __ldg(&mv[p0]);
    // The tile's tone-mapped colour with a one-pixel halo: each noisy pixel is read and mapped
    // once per block, and the 3x3 clamp window is read from shared memory.
    constexpr int SX = TILE_X + 2, SY = TILE_Y + 2;
    constexpr int kFill = (SX * SY + TILE_X * TILE_Y - 1) / (TILE_X * TILE_Y);
    float(&s_c)[3][SY][SX] = sm.c;
    const int tid = threadIdx.y * TILE_X + threadIdx.x;
    float3 fv[kFill];
#pragma unroll
    for (int r = 0; r < kFill; ++r) {
        const int i = tid + r * TILE_X * TILE_Y;
        const int ly = i / SX, lx = i - ly * SX;
        const int gx = x0 + lx - 1, gy = y0 + ly - 1;
        fv[r] = make_float3(0.f, 0.f, 0.f);
        if (i < SX * SY && gx >= 0 && gy >= 0 && gx < W && gy < H) fv[r] = load_rgb(noisy, (long)gy * W + gx);
    }

    // reprojection footprint: previous position p + 0.5 - mv, base floor(x - mv), fraction
    // frac(-mv); up to four taps, every in-image tap's loads issued at once
    const bool reproject = inside && has_history && prev_gbuf != nullptr && fabsf(m.x) < 1e7f &&
                           fabsf(m.y) < 1e7f;
    float4 tg[4], th[4], tmm[4];
    float twb[4];
    {
        const float ux = -m.x, uy = -m.y;
        const float flx = floorf(ux), fly = floorf(uy);
        const float fx = ux - flx, fy = uy - fly;
        const int bx = x + (int)flx, by = y + (int)fly;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = k & 1, j = k >> 1;
            const int tx = bx + i, ty = by + j;
            twb[k] = (i ? fx : 1.0f - fx) * (j ? fy : 1.0f - fy);
            const bool in = reproject && tx >= 0 && ty >= 0 && tx < W && ty < H && twb[k] > 0.f;
            if (!in) twb[k] = 0.f;
            const int t = in ? ty * W + tx : 0;
            tg[k] = in ? __ldg(&prev_gbuf[t]) : make_float4(0.f, 0.f, 0.f, 0.f);
            th[k] = in ? S::ld_hist(hist_prev, t) : make_float4(0.f, 0.f, 0.f, 0.f);
            tmm[k] = in ? S::ld_mom(mom_prev, t) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }

#pragma unroll
    for (int r = 0; r < kFill; ++r) {
        const int i = tid + r * TILE_X * TILE_Y;
        if (i < SX * SY) {
            const int ly = i / SX, lx = i - ly * SX;
            const int gx = x0 + lx - 1, gy = y0 + ly - 1;
            float3 v = make_float3(0.f, 0.f, 0.f);
            if (gx >= 0 && gy >= 0 && gx < W && gy < H) v = tonemap(P, fv[r]);
            s_c[0][ly][lx] = v.x;
            s_c[1][ly][lx] = v.y;
            s_c[2][ly][lx] = v.z;
        }
    }
    __syncthreads();
    int short_history = 0;
    if (inside) {
        const long p = (long)y * W + x;
        const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
        const float3 c = make_float3(s_c[0][ty][tx], s_c[1][ty][tx], s_c[2][ty][tx]);

        bool valid = false;
        float3 hist = make_float3(0.f, 0.f, 0.f);
        float mu1p = 0.f, Sp = 0.f, nprev = 0.f;
        if (reproject) {
            const float ztol = P.depth_rel_tol * g.w;
            // the contributing taps, kept in registers for the two-pass moment blend
            float tw[4], tm1[4], tS[4];
            float sw = 0.f, nmax = 0.f;
            float3 hs = make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                tw[k] = 0.f;
                tm1[k] = 0.f;
                tS[k] = 0.f;
                const float w = twb[k];
                if (!(w > 0.f)) continue;
                const float4 gp = tg[k];
                const float dz = fabsf(gp.w - g.w);
                const float ax = g.x - gp.x, ay = g.y - gp.y, az = g.z - gp.z;
                const float dn2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
                if (!(dz <= ztol && dn2 <= P.normal_tol2)) continue;
                tw[k] = w;
                tm1[k] = tmm[k].x;
                tS[k] = tmm[k].y;
                sw += w;
                hs.x = fmaf(w, th[k].x, hs.x);
                hs.y = fmaf(w, th[k].y, hs.y);
                hs.z = fmaf(w, th[k].z, hs.z);
                nmax = fmaxf(nmax, tmm[k].z);
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

        if (valid && P.clamp_enable && x > 0 && y > 0 && x + 1 < W && y + 1 < H) {
            // 3x3 box of the current tone-mapped colour, all nine inside: mean and population
            // std-dev, two-pass (the same sums in the same order as the border form below)
            float m[3], sd[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float sum = 0.f;
#pragma unroll
                for (int b = -1; b <= 1; ++b)
#pragma unroll
                    for (int a = -1; a <= 1; ++a) sum += s_c[ch][ty + b][tx + a];
                const float mean = sum * (1.0f / 9.0f);
                float ss = 0.f;
#pragma unroll
                for (int b = -1; b <= 1; ++b)
#pragma unroll
                    for (int a = -1; a <= 1; ++a) {
                        const float d = s_c[ch][ty + b][tx + a] - mean;
                        ss = fmaf(d, d, ss);
                    }
                m[ch] = mean;
                sd[ch] = P.gamma * sqrtf(ss * (1.0f / 9.0f));
            }
            hist = rectify(P.rectify_mode, hist, m, sd);
        } else if (valid && P.clamp_enable) {
            // 3x3 box of the current tone-mapped colour: mean and population std-dev, two-pass
            const bool xl = x > 0, xr = x + 1 < W, yu = y > 0, yd = y + 1 < H;
            const int cnt = (1 + xl + xr) * (1 + yu + yd);
            const float inv_c = 1.0f / (float)cnt;
            float m[3], sd[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float sum = 0.f;
#pragma unroll
                for (int b = -1; b <= 1; ++b)
#pragma unroll
                    for (int a = -1; a <= 1; ++a) {
                        const bool ok = (a < 0 ? xl : a > 0 ? xr : true) && (b < 0 ? yu : b > 0 ? yd : true);
                        if (ok) sum += s_c[ch][ty + b][tx + a];
                    }
                const float mean = sum * inv_c;
                float ss = 0.f;
#pragma unroll
                for (int b = -1; b <= 1; ++b)
#pragma unroll
                    for (int a = -1; a <= 1; ++a) {
                        const bool ok = (a < 0 ? xl : a > 0 ? xr : true) && (b < 0 ? yu : b > 0 ? yd : true);
                        const float d = s_c[ch][ty + b][tx + a] - mean;
                        if (ok) ss = fmaf(d, d, ss);
                    }
                m[ch] = mean;
                sd[ch] = P.gamma * sqrtf(ss * inv_c);
            }
            hist = rectify(P.rectify_mode, hist, m, sd);
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
        float mu1, Sv;
        if (valid) {
            const float d = l - mu1p;
            mu1 = fmaf(am, d, mu1p);
            Sv = (1.0f - am) * fmaf(am * d, d, Sp);
        } else {
            mu1 = l;
            Sv = 0.f;
        }
        float var = 0.f;
        if (nn >= P.min_temporal) {
            var = fmaxf(0.f, Sv);
        } else {
            short_history = 1;
        }
        S::st_cv(cv_out, (int)p, make_float4(ci.x, ci.y, ci.z, var));
        S::st_mom(mom_out, (int)p, mu1, Sv, nn);
        if (hist_accum_out) S::st_hist(hist_accum_out, (int)p, ci);
    }
    const int any_short = __syncthreads_or(short_history);
    if (threadIdx.x == 0 && threadIdx.y == 0) *flag = any_short;
}

// Largest spatial-variance radius (the configuration's range) and the window one tile reads:
// the tile with a margin of the radius on every side.
constexpr int kVarRadiusMax = 7;
constexpr int kVarWindowPx = (TILE_X + 2 * kVarRadiusMax) * (TILE_Y + 2 * kVarRadiusMax);
struct SpatialSmem {
    float4 g[kVarWindowPx];   // G-buffer (normal, depth)
    float2 m[kVarWindowPx];   // first two components of the moment record
};

// The spatial variance of the pixels with a short history in the tile at (x0, y0) (a tile the
// temporal stage flagged).  The block first copies the tile's window of G-buffer and moments to
// shared memory (every load of the window in flight at once), then each short-history pixel
// sums its (2R + 1)^2 taps from there, in the same order as a direct read.  Called by every
// thread of the block (two barriers).  RC > 0 gives the radius as a constant (the loops are
// unrolled); RC = 0 reads it from P.
template <class S, int RC>
__device__ __forceinline__ void spatial_variance_tile_r(const Params& P, int W, int H, int x0,
                                                        int y0, const float4* __restrict__ gbuf,
                                                        const typename S::Rec* __restrict__ mom,
                                                        typename S::Rec* __restrict__ cv,
                                                        SpatialSmem& sm) {
    const int R = RC > 0 ? RC : P.var_radius;
    const int HW = TILE_X + 2 * R, HH = TILE_Y + 2 * R;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, p = y * W + x;
    const bool work = x < W && y < H && S::ld_n(mom, p) < P.min_temporal;
    for (int i = threadIdx.y * TILE_X + threadIdx.x; i < HW * HH; i += TILE_X * TILE_Y) {
        const int yy = i / HW, xx = i - yy * HW;
        const int gx = x0 - R + xx, gy = y0 - R + yy;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const int q = gy * W + gx;
            sm.g[i] = __ldg(&gbuf[q]);
            const float4 mq = S::ld_mom(mom, q);
            sm.m[i] = make_float2(mq.x, mq.y);
        }
    }
    __syncthreads();
    if (work) {
        const int c = (threadIdx.y + R) * HW + threadIdx.x + R;
        const float4 g = sm.g[c];
        const float2 gr = depth_grad(gbuf, x, y, W, H);
        // E_w[mu2] - E_w[mu1]^2 = E_w[S] + Var_w[mu1].  Var_w[mu1] by West's weighted incremental
        // update (running weighted mean and sum of squared deviations), which involves no
        // difference of large sums and so keeps its FP32 accuracy for wide windows
        float sw = 0.f, sS = 0.f, mean = 0.f, m2 = 0.f;
#pragma unroll
        for (int b = -R; b <= R; ++b) {
            const int qy = y + b;
            if (qy < 0 || qy >= H) continue;
#pragma unroll
            for (int a = -R; a <= R; ++a) {
                const int qx = x + a;
                if (qx < 0 || qx >= W) continue;
                const int q = c + b * HW + a;
                const float4 gq = sm.g[q];
                const float e = log_w_normal(g, gq, P.sigma_n) -
                                depth_term(g.w, gq.w, gr, (float)a, (float)b, P.sigma_z, P.eps);
                const float w = expf(e);
                if (!(w > 0.f)) continue;   // a zero weight changes nothing (and would give 0/0 first)
                const float2 mq = sm.m[q];
                const float t = sw + w;
                const float d = mq.x - mean;
                const float r = __fdividef(d * w, t);
                m2 = fmaf(sw * d, r, m2);
                mean += r;
                sw = t;
                sS = fmaf(w, mq.y, sS);
            }
        }
        S::st_var(cv, p, fmaxf(0.f, sS / sw + m2 / sw));
    }
    __syncthreads();   // the window is rewritten by the block's next tile
}

template <class S>
__device__ __forceinline__ void spatial_variance_tile(const Params& P, int W, int H, int x0,
                                                      int y0, const float4* __restrict__ gbuf,
                                                      const typename S::Rec* __restrict__ mom,
                                                      typename S::Rec* __restrict__ cv,
                                                      SpatialSmem& sm) {
    if (P.var_radius == 3) spatial_variance_tile_r<S, 3>(P, W, H, x0, y0, gbuf, mom, cv, sm);
    else spatial_variance_tile_r<S, 0>(P, W, H, x0, y0, gbuf, mom, cv, sm);
}

// ------------------------------------------------------------------------- a-trous
//
// The weight of tap q is w = h_jk * 2^E with E, in log2 units,
//   E = sigma_n log2(1 - t)  -  log2e |z_q - z_p| / (sigma_z |grad z_p . (p - q)| + eps)
//                            -  log2e |l_q - l_p| / (sigma_l sqrt(g(var)_p) + eps),
// t = |n_p - n_q|^2 / 2, so one ex2 per tap gives the product of the three edge functions.
//  - sigma_n log2(1 - t): the series -log2e (t + t^2/2 + t^3/3 + t^4/4) for t < 1/16, lg2 of
//    1 - t above, -inf for t >= 1.  The series' truncation error in the exponent is about
//    sigma_n t^5 / 5, so the weight's absolute error (relative to the centre tap) is at most
//    max_t sigma_n t^5/5 exp(-sigma_n t) = 625/sigma_n^4 e^-5 (1.6e-8 at sigma_n = 128; 2e-7 at
//    sigma_n = 1, reached at t = 1/16).  Above 1/16 the weight is below 2^(-0.093 sigma_n) and
//    lg2's absolute error (2^-22) is harmless;
//  - the depth denominator depends on the tap only through |j A + k B|, the same for the taps
//    (j, k) and (-j, -k): one reciprocal serves both;
//  - log2e is folded into the per-pixel constants.
// Blocks whose tile lies at least two maximal steps inside the image take a path without
// bounds checks (block-uniform branch).

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// Per-launch constants of the tap weight, in log2 units.  With t2 = |n_p - n_q|^2 the normal
// weight is (1 - t2/2)^sigma_n, and sigma_n log2(1 - t2/2) = sum_m c_m t2^m with
// c_m = -sigma_n log2e / (m 2^m); the host computes c_1..c_4 into Params (as the launch
// parameters they cost the 5x5 pass no registers).
struct TapConsts {
    float c1, c2, c3, c4;
    float sigma_n;
};
__device__ __forceinline__ TapConsts tap_consts(const Params& P) {
    return {P.tc1, P.tc2, P.tc3, P.tc4, P.sigma_n};
}

// Normal edge-stopping weights this sharp or sharper take the series alone (NM = 2 below).
constexpr float kSeriesOnlySigma = 64.0f;

// log2 h + sigma_n log2(1 - t2/2) (-inf when the normal weight is 0).  Below t2 = 1/8 the
// degree-4 series keeps the relative accuracy that lg2.approx loses near 1.  NM = 0 branches to
// the lg2 form above; NM = 1 evaluates both forms and selects one (fewer control instructions,
// more arithmetic: faster for the two-tap separable passes, slower for the 24-tap 5x5 pass,
// where the lg2 form is rarely taken).  NM = 2, for sigma_n >= kSeriesOnlySigma, takes the
// series everywhere: its terms are all negative, so beyond t2 = 1/8 the weight it gives stays
// below exp(-sigma_n t2 / 2) and, like the exact weight, vanishes; the largest absolute error
// of the weight over t2 in [0, 4] is 2.2e-7 at sigma_n = 64 and 1.5e-8 at 128 (at t2 = 0.15
// and 0.08).
template <int NM>
__device__ __forceinline__ float normal_log2w(float t2, const TapConsts& T, float log2h) {
    if (NM == 2) return fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, T.c4, T.c3), T.c2), T.c1), log2h);
    if (NM == 1) {
        const float series = fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, T.c4, T.c3), T.c2), T.c1), log2h);
        const float direct = fmaf(T.sigma_n, lg2_approx(fmaf(t2, -0.5f, 1.0f)), log2h);
        return t2 < 0.125f ? series : (t2 < 2.0f ? direct : -INFINITY);
    }
    if (t2 < 0.125f) return fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, T.c4, T.c3), T.c2), T.c1), log2h);
    return t2 < 2.0f ? fmaf(T.sigma_n, lg2_approx(fmaf(t2, -0.5f, 1.0f)), log2h) : -INFINITY;
}

// Tap pairs (j, k) with (-j, -k) as the partner: k > 0, or k == 0 and j > 0.
template <int MODE>
struct TapPairs;
template <>
struct TapPairs<0> {
    static constexpr int N = 12;
    __device__ static constexpr int j(int i) { return i < 2 ? i + 1 : ((i - 2) % 5) - 2; }
    __device__ static constexpr int k(int i) { return i < 2 ? 0 : (i < 7 ? 1 : 2); }
};
template <>
struct TapPairs<1> {
    static constexpr int N = 2;
    __device__ static constexpr int j(int i) { return i + 1; }
    __device__ static constexpr int k(int) { return 0; }
};
template <>
struct TapPairs<2> {
    static constexpr int N = 2;
    __device__ static constexpr int j(int) { return 0; }
    __device__ static constexpr int k(int i) { return i + 1; }
};

// log2 of the B3 taps 3/8, 1/4, 1/16
__device__ __forceinline__ constexpr float log2_b3(int j) {
    return j == 0 ? -1.4150374992788438f : ((j == 1 || j == -1) ? -2.0f : -4.0f);
}

struct AtrousAcc {
    float sw, sr, sg, sb, sv;
};

// One tap q of pixel p: cq, gq point at q's records.  The B3 weight h enters the exponent as
// log2 h, so w = 2^(log2 h + log2 w_n + log2 w_z + log2 w_l) is one ex2.
template <class S, int NM>
__device__ __forceinline__ void atrous_tap(const typename S::Rec* __restrict__ cq_ptr,
                                           const float4* __restrict__ gq_ptr, float log2h,
                                           float rden, const float4& g, float lp, float inv_dl2,
                                           const TapConsts& T, AtrousAcc& a) {
    const float4 cq = S::ld_cv(cq_ptr, 0);
    const float4 gq = __ldg(gq_ptr);
    const float ax = g.x - gq.x, ay = g.y - gq.y, az = g.z - gq.z;
    const float t2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
    float e = normal_log2w<NM>(t2, T, log2h);
    e = fmaf(-fabsf(gq.w - g.w), rden, e);
    // the series-only form also folds -lp into the luminance's multiply-add chain
    const float dl = NM == 2 ? fmaf(0.0722f, cq.z, fmaf(0.7152f, cq.y, fmaf(0.2126f, cq.x, -lp)))
                             : luma(cq.x, cq.y, cq.z) - lp;
    e = fmaf(-fabsf(dl), inv_dl2, e);
    const float w = ex2_approx(e);
    a.sw += w;
    a.sr = fmaf(w, cq.x, a.sr);
    a.sg = fmaf(w, cq.y, a.sg);
    a.sb = fmaf(w, cq.z, a.sb);
    a.sv = fmaf(w * w, cq.w, a.sv);
}

// Output of one a-trous pass at pixel p: colour (and the history copy of it), or, for the last
// pass, the inverse tone-mapped FP32 colour with the variance.
template <class S>
__device__ __forceinline__ void atrous_store(const Params& P, int p, float4 v,
                                             typename S::Rec* __restrict__ cv_out,
                                             typename S::Rec* __restrict__ hist_out,
                                             float4* __restrict__ rgb_out) {
    if (hist_out) S::st_hist(hist_out, p, make_float3(v.x, v.y, v.z));
    if (rgb_out) {
        // the fused inverse map sees the colour at the storage precision, as the stage path does
        const float4 r = S::round_cv(v);
        const float3 o = inverse_tonemap(P, make_float3(r.x, r.y, r.z));
        rgb_out[p] = make_float4(o.x, o.y, o.z, r.w);
    } else {
        S::st_cv(cv_out, p, v);
    }
}

// Number of a-trous passes pixel p takes part in (Sec. 3.5): roughness <= t0 -> n0,
// <= t1 -> n1, otherwise all.
__device__ __forceinline__ int pass_budget(const Params& P, const float* __restrict__ rough, int p) {
    if (!P.iter_budget || rough == nullptr) return P.iter_all;
    const float r = __ldg(rough + p);
    return r <= P.iter_t0 ? P.iter_n0 : (r <= P.iter_t1 ? P.iter_n1 : P.iter_all);
}

// One pixel of one a-trous iteration at dilation `step`.  CHECK = false requires the whole 5x5
// footprint, the 3x3 prefilter and the gradient neighbours inside the image.  NS: the normal
// term by the series alone (sigma_n >= kSeriesOnlySigma).
template <int MODE, class S, bool CHECK, bool NS>
__device__ __forceinline__ void atrous_pixel(const Params& P, int W, int H, int step, int x, int y,
                                             const typename S::Rec* __restrict__ cv_in,
                                             const float4* __restrict__ gbuf,
                                             typename S::Rec* __restrict__ cv_out,
                                             typename S::Rec* __restrict__ hist_out,
                                             float4* __restrict__ rgb_out) {
    using Rec = typename S::Rec;
    const int p = y * W + x;
    const Rec* __restrict__ cvp = cv_in + p;
    const float4* __restrict__ gp = gbuf + p;
    const float4 g = __ldg(gp);
    const float2 gr = CHECK ? depth_grad(gbuf, x, y, W, H) : depth_grad_interior(gp, W);
    const float4 cp = S::ld_cv(cvp, 0);
    const float lp = luma(cp.x, cp.y, cp.z);
    const float vf = CHECK ? var_prefilter<S>(cv_in, x, y, W, H) : var_prefilter_interior<S>(cvp, W);
    // log2e / (sigma_l sqrt(g(var)) + eps): only scales an exponent, so the approximate square
    // root and reciprocal (a few ulp) are enough
    const float inv_dl2 = kLog2e * rcp_approx(fmaf(P.sigma_l, sqrt_approx(vf), P.eps));
    // |grad . offset| * sigma_z * ln2 = |j A + k B|; eps * ln2 keeps E in log2 units
    const float A = kLn2 * P.sigma_z * gr.x * (float)step;
    const float B = kLn2 * P.sigma_z * gr.y * (float)step;
    const float eps2 = kLn2 * P.eps;
    const TapConsts T = tap_consts(P);

    const float h0 = MODE == 0 ? 0.375f * 0.375f : 0.375f;
    AtrousAcc a = {h0, h0 * cp.x, h0 * cp.y, h0 * cp.z, h0 * h0 * cp.w};
#pragma unroll
    for (int i = 0; i < TapPairs<MODE>::N; ++i) {
        const int j = TapPairs<MODE>::j(i), k = TapPairs<MODE>::k(i);
        const float rden = rcp_approx(fabsf(fmaf((float)j, A, (float)k * B)) + eps2);
        const float log2h = MODE == 0 ? log2_b3(j) + log2_b3(k) : (MODE == 1 ? log2_b3(j) : log2_b3(k));
#pragma unroll
        for (int sgn = 1; sgn >= -1; sgn -= 2) {
            const int dx = sgn * j * step, dy = sgn * k * step;
            if (CHECK) {
                const int qx = x + dx, qy = y + dy;
                if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
            }
            atrous_tap<S, NS ? 2 : (MODE != 0 ? 1 : 0)>((cvp + dy * W) + dx, (gp + dy * W) + dx, log2h,
                                                        rden, g, lp, inv_dl2, T, a);
        }
    }
    const float inv = 1.0f / a.sw;
    atrous_store<S>(P, p, make_float4(a.sr * inv, a.sg * inv, a.sb * inv,
                                      MODE == 1 ? cp.w : a.sv * (inv * inv)),
                    cv_out, hist_out, rgb_out);
}


// One a-trous iteration for a tile of TX columns from x0 and TY rows y0, y0 + ys, ...,
// y0 + (TY - 1) ys of a W x H image, by a block of TX x TY threads.  With ys = the pass's step
// the vertical taps of one row are the rows of the others (adaptive-start pixels, at twice the
// step, stay on the same lattice), so a block touches TY + 4 tap rows instead of 5 TY.  Tiles
// lying two maximal steps (plus the gradient/prefilter pixel) inside the image take the path
// without bounds checks; the branch is uniform over the block.  NS as for atrous_pixel.  MASK:
// only the pixels whose 32x32 tile is set in `need` (need_tx tiles a row) are computed; the rest
// of cv_out keeps what it held.
template <int MODE, class S, int TX, int TY, bool NS, bool MASK = false>
__device__ __forceinline__ void atrous_tile(const Params& P, int W, int H, int iter, int x0, int y0,
                                            int ys, const typename S::Rec* __restrict__ cv_in,
                                            const float4* __restrict__ gbuf,
                                            const float* __restrict__ rough,
                                            typename S::Rec* __restrict__ cv_out,
                                            typename S::Rec* __restrict__ hist_out,
                                            float4* __restrict__ rgb_out,
                                            const unsigned char* __restrict__ need = nullptr,
                                            int need_tx = 0) {
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y * ys;
    if (MASK && (x >= W || y >= H || !need[(y >> 5) * need_tx + (x >> 5)])) return;
    const int reach = 2 << (iter + (P.adaptive_start && rough != nullptr ? 1 : 0));
    const int rx = MODE == 2 ? 1 : reach, ry = MODE == 1 ? 1 : reach;
    const bool interior = x0 - rx >= 1 && x0 + TX - 1 + rx < W - 1 && y0 - ry >= 1 &&
                          y0 + (TY - 1) * ys + ry < H - 1;
    if (P.iter_budget && x < W && y < H && iter >= pass_budget(P, rough, y * W + x)) {
        // past its pass budget: the pixel keeps its input (its neighbours still read it)
        const int p = y * W + x;
        atrous_store<S>(P, p, S::ld_cv(cv_in, p), cv_out, hist_out, rgb_out);
        return;
    }
    if (interior) {
        const int lvl = iter + start_level(P, rough, y * W + x);
        if (MODE == 0) {
            // the 24-tap pass with the step as a constant: each case inlines its own copy, so
            // every tap address is a row pointer plus an immediate (measured faster; the
            // two-tap separable passes gain nothing from it)
            switch (lvl) {
#define SVGF_ATROUS_AT(L)                                                                         \
    case L:                                                                                       \
        atrous_pixel<MODE, S, false, NS>(P, W, H, 1 << L, x, y, cv_in, gbuf, cv_out, hist_out, rgb_out); \
        return;
                SVGF_ATROUS_AT(0)
                SVGF_ATROUS_AT(1)
                SVGF_ATROUS_AT(2)
                SVGF_ATROUS_AT(3)
                SVGF_ATROUS_AT(4)
                SVGF_ATROUS_AT(5)
#undef SVGF_ATROUS_AT
                default: break;
            }
        }
        atrous_pixel<MODE, S, false, NS>(P, W, H, 1 << lvl, x, y, cv_in, gbuf, cv_out, hist_out, rgb_out);
    } else if (x < W && y < H) {
        atrous_pixel<MODE, S, true, NS>(P, W, H, 1 << (iter + start_level(P, rough, y * W + x)), x, y,
                                    cv_in, gbuf, cv_out, hist_out, rgb_out);
    }
}

}  // namespace dev
}  // namespace svgf
