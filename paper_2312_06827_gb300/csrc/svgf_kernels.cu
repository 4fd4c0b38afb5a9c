// Single-frame CUDA kernels (sm_103a) of the variance-guided denoiser: one block per tile.
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
//   k_state_*           temporal state to and from the FP32 exchange layout.
//
// The per-tile stage bodies live in svgf_device.cuh, shared with the batched kernels.
#include "svgf_device.cuh"

namespace svgf {
namespace {
using namespace dev;

template <class S>
__global__ void __launch_bounds__(TILE_X* TILE_Y, kTemporalBlocksPerSM)
k_temporal(Params P, const float* __restrict__ noisy, const float4* __restrict__ gbuf,
           const float4* __restrict__ prev_gbuf, const float2* __restrict__ mv,
           const typename S::Rec* __restrict__ hist_prev, const typename S::Rec* __restrict__ mom_prev,
           int has_history, typename S::Rec* __restrict__ cv_out, typename S::Rec* __restrict__ mom_out,
           typename S::Rec* __restrict__ hist_accum_out, int* __restrict__ tile_flags) {
    __shared__ TemporalSmem sm;
    temporal_tile<S>(P, P.W, P.H, blockIdx.x * TILE_X, blockIdx.y * TILE_Y,
                     &tile_flags[blockIdx.y * gridDim.x + blockIdx.x], noisy, gbuf, prev_gbuf, mv,
                     hist_prev, mom_prev, has_history, cv_out, mom_out, hist_accum_out, sm);
}

// Resident blocks per SM of the spatial-variance grid (32 registers a thread).
constexpr int kSpatialBlocksPerSM = 5;

// A resident grid walks the tiles t = blockIdx.x + k gridDim.x: the block reads the flags of
// TILE_X * TILE_Y such tiles at once (one per thread), gathers the set ones in a shared bit mask
// and runs the tile kernel on each.  In a steady-state frame few tiles are flagged, and the rest
// then cost one load each rather than a block launch.
template <class S>
__global__ void __launch_bounds__(TILE_X* TILE_Y, kSpatialBlocksPerSM)
k_spatial_variance(Params P, const float4* __restrict__ gbuf, const typename S::Rec* __restrict__ mom,
                   const int* __restrict__ tile_flags, int n_tiles, int tiles_x,
                   typename S::Rec* __restrict__ cv) {
    constexpr int kThreads = TILE_X * TILE_Y;
    __shared__ unsigned mask[kThreads / 32];
    __shared__ SpatialSmem sm;
    const int tid = threadIdx.y * TILE_X + threadIdx.x;
    for (int k0 = 0; (long)k0 * gridDim.x + blockIdx.x < n_tiles; k0 += kThreads) {
        const long t = (long)(k0 + tid) * gridDim.x + blockIdx.x;
        const unsigned b = __ballot_sync(~0u, t < n_tiles && tile_flags[t] != 0);
        if ((tid & 31) == 0) mask[tid >> 5] = b;
        __syncthreads();
        for (int w = 0; w < kThreads / 32; ++w) {
            for (unsigned m = mask[w]; m != 0; m &= m - 1) {
                const int tt = (k0 + w * 32 + __ffs(m) - 1) * gridDim.x + blockIdx.x;
                const int by = tt / tiles_x, bx = tt - by * tiles_x;
                spatial_variance_tile<S>(P, P.W, P.H, bx * TILE_X, by * TILE_Y, gbuf, mom, cv, sm);
            }
        }
        __syncthreads();   // the mask is rewritten by the next group
    }
}

// Resident blocks per SM the register budget is set for: the 24-tap 5x5 pass needs more than 40
// registers to keep its loads in flight without spilling (5 blocks: up to 48); the two-tap
// separable passes fit in 40 (6 blocks).
template <int MODE>
__host__ __device__ constexpr int atrous_min_blocks() { return MODE == 0 ? 5 : 6; }

// Tile of the single-frame 5x5 kernel (the separable passes keep TILE_X x TILE_Y): 64 x 4 measured
// marginally faster than 32 x 8, 128 x 2, 64 x 8 and 128 x 4 (303 against 305-336 us a 4K pass).
#ifndef SVGF_A5_TX
#define SVGF_A5_TX 64
#endif
#ifndef SVGF_A5_TY
#define SVGF_A5_TY 4
#endif
#ifndef SVGF_A5_MINB
#define SVGF_A5_MINB 5
#endif
template <int MODE>
__host__ __device__ constexpr int atrous_tx() { return MODE == 0 ? SVGF_A5_TX : TILE_X; }
template <int MODE>
__host__ __device__ constexpr int atrous_ty() { return MODE == 0 ? SVGF_A5_TY : TILE_Y; }
template <int MODE>
__host__ __device__ constexpr int atrous_minb() { return MODE == 0 ? SVGF_A5_MINB * 256 / (SVGF_A5_TX * SVGF_A5_TY) : atrous_min_blocks<MODE>(); }

template <int MODE, class S, bool NS>
__global__ void __launch_bounds__(atrous_tx<MODE>() * atrous_ty<MODE>(), atrous_minb<MODE>())
k_atrous(Params P, int iter, const typename S::Rec* __restrict__ cv_in,
         const float4* __restrict__ gbuf, const float* __restrict__ rough,
         typename S::Rec* __restrict__ cv_out, typename S::Rec* __restrict__ hist_out,
         float4* __restrict__ rgb_out) {
    constexpr int TX = atrous_tx<MODE>(), TY = atrous_ty<MODE>();
    const int ys = atrous_row_spacing(MODE, iter), Y = blockIdx.y / ys;
    const int y0 = Y * TY * ys + (blockIdx.y - Y * ys);
    atrous_tile<MODE, S, TX, TY, NS>(P, P.W, P.H, iter, blockIdx.x * TX, y0, ys, cv_in,
                                     gbuf, rough, cv_out, hist_out, rgb_out);
}

// k_atrous restricted to the 32x32 tiles set in `need` (the region a later pass reads).
template <int MODE, class S, bool NS>
__global__ void __launch_bounds__(atrous_tx<MODE>() * atrous_ty<MODE>(), atrous_minb<MODE>())
k_atrous_need(Params P, int iter, const typename S::Rec* __restrict__ cv_in,
              const float4* __restrict__ gbuf, const float* __restrict__ rough,
              typename S::Rec* __restrict__ cv_out, typename S::Rec* __restrict__ hist_out,
              float4* __restrict__ rgb_out, const unsigned char* __restrict__ need, int need_tx) {
    constexpr int TX = atrous_tx<MODE>(), TY = atrous_ty<MODE>();
    const int ys = atrous_row_spacing(MODE, iter), Y = blockIdx.y / ys;
    const int y0 = Y * TY * ys + (blockIdx.y - Y * ys);
    atrous_tile<MODE, S, TX, TY, NS, true>(P, P.W, P.H, iter, blockIdx.x * TX, y0, ys, cv_in, gbuf,
                                           rough, cv_out, hist_out, rgb_out, need, need_tx);
}

template <class S>
__global__ void k_inverse(Params P, const typename S::Rec* __restrict__ cv_in, float4* rgb_out,
                          int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 c = S::ld_cv(cv_in, i);
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
    const float m[3] = {mean.x, mean.y, mean.z};
    const float e[3] = {P.gamma * sqrtf(ss.x / fc), P.gamma * sqrtf(ss.y / fc), P.gamma * sqrtf(ss.z / fc)};
    const float4 h = hist_in[p];
    const float3 r = rectify(P.rectify_mode, make_float3(h.x, h.y, h.z), m, e);
    hist_out[p] = make_float4(r.x, r.y, r.z, h.w);
}

// Temporal state to / from the float4 exchange layout (history r, g, b, 0; moments mu1, S, n, 0).
template <class S>
__global__ void k_state_export(const typename S::Rec* __restrict__ hist,
                               const typename S::Rec* __restrict__ mom, float4* hist_out,
                               float4* mom_out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        hist_out[i] = S::ld_hist(hist, i);
        mom_out[i] = S::ld_mom(mom, i);
    }
}

template <class S>
__global__ void k_state_import(const float4* __restrict__ hist_in, const float4* __restrict__ mom_in,
                               typename S::Rec* hist, typename S::Rec* mom, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 h = hist_in[i], m = mom_in[i];
        S::st_hist(hist, i, make_float3(h.x, h.y, h.z));
        S::st_mom(mom, i, m.x, m.y, fminf(fmaxf(rintf(m.z), 0.f), 65535.f));
    }
}

}  // namespace

cudaError_t launch_temporal(int prec, const Params& P, const float* noisy, const float4* gbuf,
                            const float4* prev_gbuf, const float2* mv, const void* hist_prev,
                            const void* mom_prev, int has_history, void* cv_out, void* mom_out,
                            void* hist_accum_out, int* tile_flags, cudaStream_t s) {
    const dim3 grid = tile_grid(P.W, P.H), block(TILE_X, TILE_Y);
#define SVGF_TEMPORAL(ST)                                                                         \
    k_temporal<ST><<<grid, block, 0, s>>>(                                                        \
        P, noisy, gbuf, prev_gbuf, mv, (const ST::Rec*)hist_prev, (const ST::Rec*)mom_prev,       \
        has_history, (ST::Rec*)cv_out, (ST::Rec*)mom_out, (ST::Rec*)hist_accum_out, tile_flags)
    switch (prec) {
        case 0: SVGF_TEMPORAL(StoreF32); break;
        case 1: SVGF_TEMPORAL(Store16<false>); break;
        default: SVGF_TEMPORAL(Store16<true>); break;
    }
#undef SVGF_TEMPORAL
    return cudaGetLastError();
}

cudaError_t launch_spatial_variance(int prec, const Params& P, const float4* gbuf, const void* mom,
                                    const int* tile_flags, void* cv, cudaStream_t s) {
    const dim3 tiles = tile_grid(P.W, P.H), block(TILE_X, TILE_Y);
    const int n_tiles = (int)(tiles.x * tiles.y);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int grid = n_tiles < sms * kSpatialBlocksPerSM ? n_tiles : sms * kSpatialBlocksPerSM;
    // Block b takes tiles b, b + grid, ...: with grid and the tile row length coprime, a column of
    // flagged tiles (the image edge a camera pan uncovers) lands on as many blocks as it has
    // tiles instead of on grid / gcd of them, where they would run one after another.
    auto gcd = [](int a, int b) {
        while (b) {
            const int r = a % b;
            a = b;
            b = r;
        }
        return a;
    };
    while (grid > 1 && gcd(grid, (int)tiles.x) != 1) --grid;
#define SVGF_SPATIAL(ST)                                                                        \
    k_spatial_variance<ST><<<grid, block, 0, s>>>(P, gbuf, (const ST::Rec*)mom, tile_flags, n_tiles, \
                                                   (int)tiles.x, (ST::Rec*)cv)
    switch (prec) {
        case 0: SVGF_SPATIAL(StoreF32); break;
        case 1: SVGF_SPATIAL(Store16<false>); break;
        default: SVGF_SPATIAL(Store16<true>); break;
    }
#undef SVGF_SPATIAL
    return cudaGetLastError();
}

template <class ST>
static void atrous_dispatch(int mode, const Params& P, int iter, const void* cv_in,
                            const float4* gbuf, const float* rough, void* cv_out, void* hist_out,
                            float4* rgb_out, const unsigned char* need, int need_tx, cudaStream_t s) {
    const int tx = mode == 0 ? SVGF_A5_TX : TILE_X, ty = mode == 0 ? SVGF_A5_TY : TILE_Y;
    const int ys = atrous_row_spacing(mode, iter), rows = ty * ys;
    const dim3 grid((unsigned)((P.W + tx - 1) / tx), (unsigned)(((P.H + rows - 1) / rows) * ys)), block(tx, ty);
    const typename ST::Rec* in = (const typename ST::Rec*)cv_in;
    typename ST::Rec* out = (typename ST::Rec*)cv_out;
    typename ST::Rec* hist = (typename ST::Rec*)hist_out;
    // the 24-tap pass takes the series-only normal term for sharp normal weights
    // (sigma_n >= kSeriesOnlySigma); the two-tap separable passes keep the select form
#define SVGF_AT(M, NS)                                                                                 \
    if (need)                                                                                          \
        k_atrous_need<M, ST, NS><<<grid, block, 0, s>>>(P, iter, in, gbuf, rough, out, hist, rgb_out, need, need_tx); \
    else                                                                                               \
        k_atrous<M, ST, NS><<<grid, block, 0, s>>>(P, iter, in, gbuf, rough, out, hist, rgb_out)
    switch (mode) {
        case 0:
            if (P.sigma_n >= kSeriesOnlySigma) {
                SVGF_AT(0, true);
            } else {
                SVGF_AT(0, false);
            }
            break;
        case 1: SVGF_AT(1, false); break;
        default: SVGF_AT(2, false); break;
    }
#undef SVGF_AT
}

cudaError_t launch_atrous(int prec, const Params& P, int mode, int iter, const void* cv_in,
                          const float4* gbuf, const float* rough, void* cv_out, void* hist_out,
                          float4* rgb_out, cudaStream_t s, const unsigned char* need, int need_tx) {
    switch (prec) {
        case 0: atrous_dispatch<StoreF32>(mode, P, iter, cv_in, gbuf, rough, cv_out, hist_out, rgb_out, need, need_tx, s); break;
        case 1: atrous_dispatch<Store16<false>>(mode, P, iter, cv_in, gbuf, rough, cv_out, hist_out, rgb_out, need, need_tx, s); break;
        default: atrous_dispatch<Store16<true>>(mode, P, iter, cv_in, gbuf, rough, cv_out, hist_out, rgb_out, need, need_tx, s); break;
    }
    return cudaGetLastError();
}

static unsigned flat_blocks(long n) {
    long blocks = (n + 255) / 256;
    return (unsigned)(blocks > 152L * 16 ? 152L * 16 : (blocks < 1 ? 1 : blocks));
}

cudaError_t launch_inverse(int prec, const Params& P, const void* cv_in, float4* rgb_out,
                           cudaStream_t s) {
    const int n = P.W * P.H;
    switch (prec) {
        case 0: k_inverse<StoreF32><<<flat_blocks(n), 256, 0, s>>>(P, (const float4*)cv_in, rgb_out, n); break;
        case 1: k_inverse<Store16<false>><<<flat_blocks(n), 256, 0, s>>>(P, (const uint2*)cv_in, rgb_out, n); break;
        default: k_inverse<Store16<true>><<<flat_blocks(n), 256, 0, s>>>(P, (const uint2*)cv_in, rgb_out, n); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_state_export(int prec, int n, const void* hist, const void* mom,
                                float4* hist_out, float4* mom_out, cudaStream_t s) {
    switch (prec) {
        case 0: k_state_export<StoreF32><<<flat_blocks(n), 256, 0, s>>>((const float4*)hist, (const float4*)mom, hist_out, mom_out, n); break;
        case 1: k_state_export<Store16<false>><<<flat_blocks(n), 256, 0, s>>>((const uint2*)hist, (const uint2*)mom, hist_out, mom_out, n); break;
        default: k_state_export<Store16<true>><<<flat_blocks(n), 256, 0, s>>>((const uint2*)hist, (const uint2*)mom, hist_out, mom_out, n); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_state_import(int prec, int n, const float4* hist_in, const float4* mom_in,
                                void* hist, void* mom, cudaStream_t s) {
    switch (prec) {
        case 0: k_state_import<StoreF32><<<flat_blocks(n), 256, 0, s>>>(hist_in, mom_in, (float4*)hist, (float4*)mom, n); break;
        case 1: k_state_import<Store16<false>><<<flat_blocks(n), 256, 0, s>>>(hist_in, mom_in, (uint2*)hist, (uint2*)mom, n); break;
        default: k_state_import<Store16<true>><<<flat_blocks(n), 256, 0, s>>>(hist_in, mom_in, (uint2*)hist, (uint2*)mom, n); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_clamp(const Params& P, const float* noisy, const float4* hist_in,
                         float4* hist_out, cudaStream_t s) {
    k_clamp<<<tile_grid(P.W, P.H), dim3(TILE_X, TILE_Y), 0, s>>>(P, noisy, hist_in, hist_out);
    return cudaGetLastError();
}

}  // namespace svgf
