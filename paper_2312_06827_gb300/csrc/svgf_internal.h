// Internal declarations shared by the host API (svgf_api.cu) and the kernels (svgf_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace svgf {

// Kernel-side copy of the configuration (derived values precomputed on the host).
struct Params {
    int W, H;
    float alpha, alpha_m, gamma;
    float sigma_z, sigma_n, sigma_l;
    int clamp_enable, adaptive_start;
    float rough_thr;
    int tonemap;
    float luma_k, inv_weight;
    int inverse_mode;
    float depth_rel_tol;
    float normal_tol2;     // 2 (1 - normal_cos_tol): bound on |n_p - n_prev|^2
    float disocc_w;
    float max_history;
    float min_temporal;
    int var_radius;
    float eps;
    int rectify_mode;      // 0 clamp, 1 clip (Sec. 3.1)
    int iter_budget;       // roughness-adapted pass budget on/off (Sec. 3.5)
    float iter_t0, iter_t1;
    int iter_n0, iter_n1, iter_all;
    // coefficients of the degree-4 series of sigma_n log2(1 - t2/2) in t2 (the a-trous normal
    // term): c/2, c/8, c/24, c/64 with c = -sigma_n log2(e), each rounded to FP32
    float tc1, tc2, tc3, tc4;
};

// Thread-block tile of the per-pixel kernels: 32 x 8 pixels, one warp per row segment.
constexpr int TILE_X = 32;
constexpr int TILE_Y = 8;

inline dim3 tile_grid(int W, int H) {
    return dim3((unsigned)((W + TILE_X - 1) / TILE_X), (unsigned)((H + TILE_Y - 1) / TILE_Y));
}

// Row spacing of the a-trous tiles of pass `iter` (mode 0 = 5x5, 1 = horizontal, 2 = vertical):
// the pass's step, capped at 16; 1 for the horizontal pass, whose taps share the row.  Tile row
// index by = Y ys + r covers rows Y TILE_Y ys + r + i ys, i < TILE_Y.
__host__ __device__ inline int atrous_row_spacing(int mode, int iter) {
    return mode == 1 ? 1 : (iter >= 4 ? 16 : 1 << iter);
}
inline dim3 atrous_grid(int mode, int iter, int W, int H) {
    const int ys = atrous_row_spacing(mode, iter), rows = TILE_Y * ys;
    return dim3((unsigned)((W + TILE_X - 1) / TILE_X), (unsigned)(((H + rows - 1) / rows) * ys));
}

// Bytes per pixel of a workspace image (colour + variance, colour history, moments) in each
// storage precision (svgf_config.precision): float4, or an 8-byte 16-bit record.
inline size_t image_bytes_per_px(int prec) { return prec == 0 ? 16 : 8; }

// Launchers: each enqueues one kernel on `s` and returns the launch error.  `prec` selects the
// storage of the workspace images (0 FP32, 1 FP16, 2 BF16); their pointers are untyped.
cudaError_t launch_temporal(int prec, const Params& P, const float* noisy, const float4* gbuf,
                            const float4* prev_gbuf, const float2* mv, const void* hist_prev,
                            const void* mom_prev, int has_history, void* cv_out, void* mom_out,
                            void* hist_accum_out, int* tile_flags, cudaStream_t s);
cudaError_t launch_spatial_variance(int prec, const Params& P, const float4* gbuf, const void* mom,
                                    const int* tile_flags, void* cv, cudaStream_t s);
// mode: 0 = 5x5, 1 = horizontal pass, 2 = vertical pass.
// rgb_out != nullptr: fused inverse tone map, FP32 output to rgb_out instead of cv_out.
// need != nullptr: only the pixels of the 32x32 tiles set in need (need_tx tiles a row) are
// computed.
cudaError_t launch_atrous(int prec, const Params& P, int mode, int iter, const void* cv_in,
                          const float4* gbuf, const float* rough, void* cv_out, void* hist_out,
                          float4* rgb_out, cudaStream_t s, const unsigned char* need = nullptr,
                          int need_tx = 0);
cudaError_t launch_inverse(int prec, const Params& P, const void* cv_in, float4* rgb_out,
                           cudaStream_t s);
cudaError_t launch_clamp(const Params& P, const float* noisy, const float4* hist_in,
                         float4* hist_out, cudaStream_t s);
cudaError_t launch_state_export(int prec, int n, const void* hist, const void* mom,
                                float4* hist_out, float4* mom_out, cudaStream_t s);
cudaError_t launch_state_import(int prec, int n, const float4* hist_in, const float4* mom_in,
                                void* hist, void* mom, cudaStream_t s);

// ---- batched frames: descriptors passed by value in the kernel parameters -------------------
// One persistent launch per stage covers the tiles of up to kMaxBatch images; a block walks the
// tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...; tile t belongs to the last stream whose
// tile_base is <= t.  Each stream carries its own Params, so the streams of one launch may be
// different channels (tone mapping, thresholds, rectification, ...) as long as they share the
// storage precision, the spatial mode and the pass count.  The argument structs stay under the
// 32 KB kernel-parameter limit (static_asserts below).
constexpr int kMaxBatch = 64;

struct BTemporal {
    Params P;
    const float* noisy;
    const float4* gbuf;
    const float4* prev_gbuf;
    const float2* mv;
    const void* hist_prev;
    const void* mom_prev;
    void* cv_out;
    void* mom_out;
    void* hist_accum;
    int* flags;
    int W, H, tiles_x, tile_base, has_history;
};
struct BatchTemporalArgs {
    int n, total;
    int uniform;   // every stream has P's values apart from W, H: the kernels read P
    Params P;
    BTemporal s[kMaxBatch];
};

struct BSpatial {
    Params P;
    const float4* gbuf;
    const void* mom;
    const int* flags;
    void* cv;
    int W, H, tiles_x, tile_base;
};
struct BatchSpatialArgs {
    int n, total;
    int uniform;   // every stream has P's values apart from W, H: the kernels read P
    Params P;
    BSpatial s[kMaxBatch];
};

struct BAtrous {
    Params P;
    const void* cv_in;
    const float4* gbuf;
    const float* rough;
    void* cv_out;
    void* hist_out;
    float4* rgb_out;
    int W, H, tiles_x, tile_base;
};
struct BatchAtrousArgs {
    int n, total, iter;
    int uniform;   // every stream has P's values apart from W, H: the kernels read P
    Params P;
    BAtrous s[kMaxBatch];
};
static_assert(sizeof(BatchTemporalArgs) <= 32764, "kernel parameter limit");
static_assert(sizeof(BatchSpatialArgs) <= 32764, "kernel parameter limit");
static_assert(sizeof(BatchAtrousArgs) <= 32764, "kernel parameter limit");

// Tile shapes the batched a-trous kernel is compiled for (the autotuner picks one).
constexpr int kAtrousShapes = 4;
inline void atrous_shape(int shape, int* tx, int* ty) {
    static const int X[kAtrousShapes] = {32, 32, 16, 64}, Y[kAtrousShapes] = {8, 4, 16, 4};
    *tx = X[shape];
    *ty = Y[shape];
}

cudaError_t launch_batch_temporal(int prec, const BatchTemporalArgs& a, int grid, cudaStream_t s);
cudaError_t launch_batch_spatial(int prec, const BatchSpatialArgs& a, int grid, cudaStream_t s);
// mode: 0 = 5x5, 1 = horizontal, 2 = vertical; shape: index into atrous_shape.
cudaError_t launch_batch_atrous(int prec, int mode, int shape, const BatchAtrousArgs& a, int grid,
                                cudaStream_t s);
// Resident blocks per SM of the batched a-trous kernel (for persistent grid sizes); form: 0 and 1
// launch-wide Params with the 5x5 normal term's log2 fallback or series alone, 2 per-stream Params.
int batch_atrous_occupancy(int prec, int mode, int shape, int form);
// Whether the 5x5 pass takes the normal term by the series alone at this sigma_n.
bool series_only_normal(float sigma_n);
// Whether two streams' Params agree apart from the image size (one launch-wide copy serves both).
bool same_params_but_size(const Params& a, const Params& b);

}  // namespace svgf
