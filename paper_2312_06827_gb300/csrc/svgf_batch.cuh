// Batched persistent kernels: one launch per stage covers the tiles of many streams' frames of
// uneven sizes (the batched form of the denoiser).  The per-stream descriptors travel by value in
// the kernel parameters, so the batch needs no device memory of its own; each block walks the
// global tile list with a grid stride (or, launched with one block per tile, takes one tile) and
// runs the same per-tile stage bodies as the single-frame kernels (svgf_device.cuh), so a batched
// frame is bit-identical to the same frames denoised one by one.  Grid strides need no work
// queue and no waits.
//
// Parameters.  A stream's Params read through a run-time stream index are loads from the
// parameter bank into registers, where the single-frame kernels take them as constant-bank
// operands; in the 24-tap pass that pressure spilled.  When every stream of a launch has the same
// Params apart from its size (the common case: one channel's configuration), the host sets
// `uniform` and the kernels (UP = true) read the launch-wide copy at a fixed offset instead.
//
// This header is compiled once per storage precision (svgf_batch_<prec>.cu), which keeps each
// translation unit's instantiations few and lets them build in parallel.
#pragma once

#include "svgf_device.cuh"

namespace svgf {
namespace batch {
using namespace dev;

// Stream owning global tile t: the last descriptor whose tile_base is <= t (binary search over
// the sorted bases; uniform across the block).
template <class A>
__device__ __forceinline__ int stream_of(const A& a, int t) {
    int lo = 0, hi = a.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.s[mid].tile_base <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class S, bool UP>
__global__ void __launch_bounds__(TILE_X* TILE_Y, kTemporalBlocksPerSM)
kb_temporal(const __grid_constant__ BatchTemporalArgs A) {
    __shared__ TemporalSmem sm;
    for (int t = blockIdx.x; t < A.total; t += gridDim.x) {
        const BTemporal& d = A.s[stream_of(A, t)];
        const int lt = t - d.tile_base, by = lt / d.tiles_x, bx = lt - by * d.tiles_x;
        using R = typename S::Rec;
        temporal_tile<S>(UP ? A.P : d.P, d.W, d.H, bx * TILE_X, by * TILE_Y, d.flags + lt, d.noisy,
                         d.gbuf, d.prev_gbuf, d.mv, (const R*)d.hist_prev, (const R*)d.mom_prev,
                         d.has_history, (R*)d.cv_out, (R*)d.mom_out, (R*)d.hist_accum, sm);
    }
}

template <class S, bool UP>
__global__ void __launch_bounds__(TILE_X* TILE_Y)
kb_spatial_variance(const __grid_constant__ BatchSpatialArgs A) {
    // the flags of TILE_X * TILE_Y of the block's tiles are read at once, one per thread, and the
    // set ones collected in a shared bit mask (as in the single-frame kernel)
    constexpr int kThreads = TILE_X * TILE_Y;
    __shared__ unsigned mask[kThreads / 32];
    __shared__ SpatialSmem sm;
    const int tid = threadIdx.y * TILE_X + threadIdx.x;
    for (int k0 = 0; (long)k0 * gridDim.x + blockIdx.x < A.total; k0 += kThreads) {
        const long t = (long)(k0 + tid) * gridDim.x + blockIdx.x;
        bool f = false;
        if (t < A.total) {
            const BSpatial& d = A.s[stream_of(A, (int)t)];
            f = d.flags[t - d.tile_base] != 0;
        }
        const unsigned b = __ballot_sync(~0u, f);
        if ((tid & 31) == 0) mask[tid >> 5] = b;
        __syncthreads();
        for (int w = 0; w < kThreads / 32; ++w) {
            for (unsigned m = mask[w]; m != 0; m &= m - 1) {
                const int tt = (k0 + w * 32 + __ffs(m) - 1) * gridDim.x + blockIdx.x;
                const BSpatial& d = A.s[stream_of(A, tt)];
                const int lt = tt - d.tile_base, by = lt / d.tiles_x, bx = lt - by * d.tiles_x;
                using R = typename S::Rec;
                spatial_variance_tile<S>(UP ? A.P : d.P, d.W, d.H, bx * TILE_X, by * TILE_Y, d.gbuf,
                                         (const R*)d.mom, (R*)d.cv, sm);
            }
        }
        __syncthreads();
    }
}

// NSM: the 5x5 pass's normal-term form, fixed on the host so that the kernel holds one form
// (0: the series with the log2 fallback, 1: the series alone, as the single-frame 5x5 launch
// takes it for sigma_n >= kSeriesOnlySigma, 2: chosen per stream, for launches whose streams
// differ).  PERSIST: a grid-stride walk over the tiles; otherwise one block per tile.
// Resident threads per SM the register budget is set for, as in the single-frame kernels: 1280
// for the 24-tap pass (48 registers), 1536 for the two-tap separable passes (40).
#ifndef SVGF_BATCH_A5_THREADS
#define SVGF_BATCH_A5_THREADS 1280
#endif
template <int MODE>
constexpr int batch_threads_per_sm() { return MODE == 0 ? SVGF_BATCH_A5_THREADS : 1536; }

template <int MODE, class S, int TX, int TY, int NSM, bool UP, bool PERSIST>
__global__ void __launch_bounds__(TX* TY, batch_threads_per_sm<MODE>() / (TX * TY))
kb_atrous(const __grid_constant__ BatchAtrousArgs A) {
    for (int t = blockIdx.x; t < A.total; t += gridDim.x) {
        const BAtrous& d = A.s[stream_of(A, t)];
        const Params& P = UP ? A.P : d.P;
        const int lt = t - d.tile_base, by = lt / d.tiles_x, bx = lt - by * d.tiles_x;
        const int ys = atrous_row_spacing(MODE, A.iter), Y = by / ys;
        using R = typename S::Rec;
        const int ty0 = Y * TY * ys + (by - Y * ys);
        if (MODE == 0 && (NSM == 1 || (NSM == 2 && P.sigma_n >= kSeriesOnlySigma)))
            atrous_tile<MODE, S, TX, TY, true>(P, d.W, d.H, A.iter, bx * TX, ty0, ys, (const R*)d.cv_in,
                                               d.gbuf, d.rough, (R*)d.cv_out, (R*)d.hist_out, d.rgb_out);
        else
            atrous_tile<MODE, S, TX, TY, false>(P, d.W, d.H, A.iter, bx * TX, ty0, ys, (const R*)d.cv_in,
                                                d.gbuf, d.rough, (R*)d.cv_out, (R*)d.hist_out, d.rgb_out);
        if (!PERSIST) break;
    }
}

// ---- launchers of one storage precision --------------------------------------------------------

template <class S>
cudaError_t temporal(const BatchTemporalArgs& a, int grid, cudaStream_t s) {
    const dim3 block(TILE_X, TILE_Y);
    if (a.uniform) kb_temporal<S, true><<<grid, block, 0, s>>>(a);
    else kb_temporal<S, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <class S>
cudaError_t spatial(const BatchSpatialArgs& a, int grid, cudaStream_t s) {
    const dim3 block(TILE_X, TILE_Y);
    if (a.uniform) kb_spatial_variance<S, true><<<grid, block, 0, s>>>(a);
    else kb_spatial_variance<S, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

// The kernel a launch takes: its form (NSM, UP) follows from the descriptors; `per` from the grid.
template <int M, class S, int TX, int TY, bool PER>
struct AtrousKernels {
    using K = void (*)(const BatchAtrousArgs);
    static K pick(int form) {
        if constexpr (M != 0) {
            return form == 2 ? kb_atrous<M, S, TX, TY, 0, false, PER> : kb_atrous<M, S, TX, TY, 0, true, PER>;
        } else {
            switch (form) {
                case 0: return kb_atrous<M, S, TX, TY, 0, true, PER>;
                case 1: return kb_atrous<M, S, TX, TY, 1, true, PER>;
                default: return kb_atrous<M, S, TX, TY, 2, false, PER>;
            }
        }
    }
};

template <int M, class S, bool PER>
typename AtrousKernels<M, S, 32, 8, PER>::K atrous_kernel_shape(int shape, int form) {
    switch (shape) {
        case 0: return AtrousKernels<M, S, 32, 8, PER>::pick(form);
        case 1: return AtrousKernels<M, S, 32, 4, PER>::pick(form);
        case 2: return AtrousKernels<M, S, 16, 16, PER>::pick(form);
        default: return AtrousKernels<M, S, 64, 4, PER>::pick(form);
    }
}

// form: 0 uniform Params with the log2 fallback, 1 uniform with the series alone, 2 per-stream
// Params (the 5x5 pass then picks the normal term per stream).
template <class S>
typename AtrousKernels<0, S, 32, 8, false>::K atrous_kernel(int mode, int shape, int form, bool per) {
    switch (mode) {
        case 0: return per ? atrous_kernel_shape<0, S, true>(shape, form) : atrous_kernel_shape<0, S, false>(shape, form);
        case 1: return per ? atrous_kernel_shape<1, S, true>(shape, form) : atrous_kernel_shape<1, S, false>(shape, form);
        default: return per ? atrous_kernel_shape<2, S, true>(shape, form) : atrous_kernel_shape<2, S, false>(shape, form);
    }
}

inline int atrous_form(const BatchAtrousArgs& a) {
    if (!a.uniform) return 2;
    return series_only_normal(a.P.sigma_n) ? 1 : 0;
}

template <class S>
cudaError_t atrous(int mode, int shape, const BatchAtrousArgs& a, int grid, cudaStream_t s) {
    int tx, ty;
    atrous_shape(shape, &tx, &ty);
    const auto k = atrous_kernel<S>(mode, shape, atrous_form(a), grid < a.total);
    k<<<grid, dim3(tx, ty), 0, s>>>(a);
    return cudaGetLastError();
}

template <class S>
int atrous_occupancy(int mode, int shape, int form) {
    int tx, ty, n = 0;
    atrous_shape(shape, &tx, &ty);
    const auto k = atrous_kernel<S>(mode, shape, form, true);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, tx * ty, 0) != cudaSuccess) return 0;
    return n;
}

}  // namespace batch
}  // namespace svgf

// One storage precision's launchers, defined in its translation unit.
#define SVGF_BATCH_DEFINE(SUFFIX, S)                                                                 \
    namespace svgf {                                                                                 \
    cudaError_t launch_batch_temporal_##SUFFIX(const BatchTemporalArgs& a, int grid, cudaStream_t s) { \
        return batch::temporal<S>(a, grid, s);                                                       \
    }                                                                                                \
    cudaError_t launch_batch_spatial_##SUFFIX(const BatchSpatialArgs& a, int grid, cudaStream_t s) {  \
        return batch::spatial<S>(a, grid, s);                                                        \
    }                                                                                                \
    cudaError_t launch_batch_atrous_##SUFFIX(int mode, int shape, const BatchAtrousArgs& a, int grid, \
                                             cudaStream_t s) {                                       \
        return batch::atrous<S>(mode, shape, a, grid, s);                                            \
    }                                                                                                \
    int batch_atrous_occupancy_##SUFFIX(int mode, int shape, int form) {                             \
        return batch::atrous_occupancy<S>(mode, shape, form);                                        \
    }                                                                                                \
    }
