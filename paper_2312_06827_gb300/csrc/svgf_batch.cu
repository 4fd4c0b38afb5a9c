// Batched persistent kernels: one launch per stage covers the tiles of many streams' frames of
// uneven sizes (the batched form of the denoiser).  The per-stream descriptors travel by value in
// the kernel parameters, so the batch needs no device memory of its own; each block walks the
// global tile list with a grid stride (or, launched with one block per tile, takes one tile) and
// runs the same per-tile stage bodies as the single-frame kernels (svgf_device.cuh), so a batched
// frame is bit-identical to the same frames denoised one by one.  Grid strides need no work
// queue and no waits.
#include "svgf_device.cuh"

namespace svgf {
namespace {
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

template <class S>
__global__ void __launch_bounds__(TILE_X* TILE_Y)
kb_temporal(const __grid_constant__ BatchTemporalArgs A) {
    __shared__ TemporalSmem sm;
    for (int t = blockIdx.x; t < A.total; t += gridDim.x) {
        const BTemporal& d = A.s[stream_of(A, t)];
        const int lt = t - d.tile_base, by = lt / d.tiles_x, bx = lt - by * d.tiles_x;
        using R = typename S::Rec;
        temporal_tile<S>(d.P, d.W, d.H, bx * TILE_X, by * TILE_Y, d.flags + lt, d.noisy, d.gbuf,
                         d.prev_gbuf, d.mv, (const R*)d.hist_prev, (const R*)d.mom_prev,
                         d.has_history, (R*)d.cv_out, (R*)d.mom_out, (R*)d.hist_accum, sm);
    }
}

template <class S>
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
                spatial_variance_tile<S>(d.P, d.W, d.H, bx * TILE_X, by * TILE_Y, d.gbuf,
                                         (const R*)d.mom, (R*)d.cv, sm);
            }
        }
        __syncthreads();
    }
}

template <int MODE, class S, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, 1280 / (TX * TY))
kb_atrous(const __grid_constant__ BatchAtrousArgs A) {
    for (int t = blockIdx.x; t < A.total; t += gridDim.x) {
        const BAtrous& d = A.s[stream_of(A, t)];
        const int lt = t - d.tile_base, by = lt / d.tiles_x, bx = lt - by * d.tiles_x;
        const int ys = atrous_row_spacing(MODE, A.iter), Y = by / ys;
        using R = typename S::Rec;
        const int ty0 = Y * TY * ys + (by - Y * ys);
        // each stream's own choice of the normal term's form (as its single-frame launch makes
        // it: the series alone in the 5x5 pass for sigma_n >= kSeriesOnlySigma)
        if (MODE == 0 && d.P.sigma_n >= kSeriesOnlySigma)
            atrous_tile<MODE, S, TX, TY, true>(d.P, d.W, d.H, A.iter, bx * TX, ty0, ys, (const R*)d.cv_in,
                                               d.gbuf, d.rough, (R*)d.cv_out, (R*)d.hist_out, d.rgb_out);
        else
            atrous_tile<MODE, S, TX, TY, false>(d.P, d.W, d.H, A.iter, bx * TX, ty0, ys, (const R*)d.cv_in,
                                                d.gbuf, d.rough, (R*)d.cv_out, (R*)d.hist_out, d.rgb_out);
    }
}

template <class S>
void atrous_modes(int mode, int shape, const BatchAtrousArgs& a, int grid, cudaStream_t s) {
#define SVGF_KB(M, X, Y) kb_atrous<M, S, X, Y><<<grid, dim3(X, Y), 0, s>>>(a)
#define SVGF_SHAPES(M)                          \
    switch (shape) {                            \
        case 0: SVGF_KB(M, 32, 8); break;       \
        case 1: SVGF_KB(M, 32, 4); break;       \
        case 2: SVGF_KB(M, 16, 16); break;      \
        default: SVGF_KB(M, 64, 4); break;      \
    }
    switch (mode) {
        case 0: SVGF_SHAPES(0); break;
        case 1: SVGF_SHAPES(1); break;
        default: SVGF_SHAPES(2); break;
    }
#undef SVGF_SHAPES
#undef SVGF_KB
}

}  // namespace

cudaError_t launch_batch_temporal(int prec, const BatchTemporalArgs& a, int grid, cudaStream_t s) {
    const dim3 block(TILE_X, TILE_Y);
    switch (prec) {
        case 0: kb_temporal<StoreF32><<<grid, block, 0, s>>>(a); break;
        case 1: kb_temporal<Store16<false>><<<grid, block, 0, s>>>(a); break;
        default: kb_temporal<Store16<true>><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_spatial(int prec, const BatchSpatialArgs& a, int grid, cudaStream_t s) {
    const dim3 block(TILE_X, TILE_Y);
    switch (prec) {
        case 0: kb_spatial_variance<StoreF32><<<grid, block, 0, s>>>(a); break;
        case 1: kb_spatial_variance<Store16<false>><<<grid, block, 0, s>>>(a); break;
        default: kb_spatial_variance<Store16<true>><<<grid, block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <class S>
int occupancy_of(int mode, int shape) {
    int n = 0;
    auto q = [&](auto kernel, int threads) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0);
    };
#define SVGF_OCC(M)                                                  \
    switch (shape) {                                                 \
        case 0: q(kb_atrous<M, S, 32, 8>, 256); break;               \
        case 1: q(kb_atrous<M, S, 32, 4>, 128); break;               \
        case 2: q(kb_atrous<M, S, 16, 16>, 256); break;              \
        default: q(kb_atrous<M, S, 64, 4>, 256); break;              \
    }
    switch (mode) {
        case 0: SVGF_OCC(0); break;
        case 1: SVGF_OCC(1); break;
        default: SVGF_OCC(2); break;
    }
#undef SVGF_OCC
    return n;
}

int batch_atrous_occupancy(int prec, int mode, int shape) {
    switch (prec) {
        case 0: return occupancy_of<StoreF32>(mode, shape);
        case 1: return occupancy_of<Store16<false>>(mode, shape);
        default: return occupancy_of<Store16<true>>(mode, shape);
    }
}

cudaError_t launch_batch_atrous(int prec, int mode, int shape, const BatchAtrousArgs& a, int grid,
                                cudaStream_t s) {
    switch (prec) {
        case 0: atrous_modes<StoreF32>(mode, shape, a, grid, s); break;
        case 1: atrous_modes<Store16<false>>(mode, shape, a, grid, s); break;
        default: atrous_modes<Store16<true>>(mode, shape, a, grid, s); break;
    }
    return cudaGetLastError();
}

}  // namespace svgf
