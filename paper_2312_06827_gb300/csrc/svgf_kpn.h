// Internal declarations of the learned part (svgf_kpn.cu kernels, used by svgf_api.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "svgf_internal.h"

namespace svgf {
namespace kpn {

// Layer shapes: 3x3 convolutions 10 -> 32 -> 32 -> 32 -> 25; the conv kernels see 16 input
// channels in layer 0 (features padded) and 32 output channels in layer 3 (logits padded).
__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? 10 : 32; }
__host__ __device__ constexpr int cout_of(int l) { return l == 3 ? 25 : 32; }
__host__ __device__ constexpr int cin_pad_of(int l) { return l == 0 ? 16 : 32; }
__host__ __device__ constexpr int layer_params(int l) { return cout_of(l) * 9 * cin_of(l) + cout_of(l); }
__host__ __device__ constexpr int param_offset(int l) {
    return l == 0 ? 0 : param_offset(l - 1) + layer_params(l - 1);
}
constexpr int kParamCount = param_offset(4);

// Bit of the device error word raised by a bounded tensor-core wait that gave up.
constexpr int kErrWaitGaveUp = 2;


// BF16 weight copies used by the conv kernels (see k_prep_weights) and FP32 biases.
struct WeightPtrs {
    __nv_bfloat16* fwd[4];     // [9][32][cin_pad]
    __nv_bfloat16* dgrad[4];   // [9][32][32], layers 1..3
    float* bias[4];            // [32]
};

cudaError_t prep_weights(const float* prm, const WeightPtrs& w, cudaStream_t s);
// dgrad = false: layer forward (layers 0..2: + bias, ReLU, BF16; layer 3: + bias and the softmax,
// the kernels K as 25 FP32 planes [25][B*H*W]).  dgrad = true: data gradient of layer `layer` (1..3) masked by
// (mask > 0), BF16.
// layer = 4: layer 3 with the softmax written as FP16, pixel-major, 64 B per pixel ([p][32], 25
// used; read by apply_h).
// On the tcgen05 tensor cores; a wait that gives up sets kErrWaitGaveUp in *err (a device int).
cudaError_t conv(int layer, bool dgrad, const __nv_bfloat16* in, const WeightPtrs& w,
                 const __nv_bfloat16* mask, void* out, int B, int H, int W, int sm_count,
                 cudaStream_t s, int* err);
// The four layers in one tcgen05 kernel: features [B][H][W][16] in, the softmax weights out as
// conv layer 4 writes them (FP16, pixel-major, 64 B per pixel), bit for bit; the activations
// stay in shared memory.  Waits as in conv.
cudaError_t net_forward(const __nv_bfloat16* feats, const WeightPtrs& w, void* Kh, int B, int H, int W,
                        int sm_count, cudaStream_t s, int* err);
// The network as two tcgen05 kernels of two layers each: features -> layers 0-1 -> mid
// [B][H][W][32] BF16 (the layer-1 activation) -> layers 2-3 -> the softmax weights as conv layer
// 4 writes them, bit for bit.  Waits as in conv.
cudaError_t net_pairs(const __nv_bfloat16* feats, const WeightPtrs& w, __nv_bfloat16* mid, void* Kh, int B, int H,
                      int W, int sm_count, cudaStream_t s, int* err);
// Self-test of the bounded wait: one block waits, with the convolution's wait, on a barrier
// phase that nothing completes, gives up after `tries` polls and raises kErrWaitGaveUp in *err
// the way a convolution block does.  Nothing else is touched.
cudaError_t wait_expiry_probe(int tries, int* err, cudaStream_t s);
// Adds the layer's weight and bias gradients into grad_flat (flat parameter layout).
cudaError_t wgrad(int layer, const __nv_bfloat16* X, const __nv_bfloat16* dZ, float* grad_flat,
                  int B, int H, int W, int sm_count, cudaStream_t s);
// c_out = K-weighted mean of c_in at the given dilation (K planar [25][B*H*W]); with rgb_out, the
// inverse tone map is fused and rgb_out.w = var_src.w.
cudaError_t apply(const float* K, const float4* c_in, float4* c_out, int B, int H, int W,
                  int dilation, const Params& P, float4* rgb_out, const float4* var_src, cudaStream_t s);
// apply with the FP16 pixel-major kernels of conv layer 4.
cudaError_t apply_h(const void* Kh, const float4* c_in, float4* c_out, int B, int H, int W,
                    int dilation, const Params& P, float4* rgb_out, const float4* var_src, cudaStream_t s);
cudaError_t backward_apply(const float* K, const float4* c0, const float4* c1, const float4* c2,
                           const float4* T, float* gK, float4* u, __nv_bfloat16* dz, float* loss_sum,
                           int B, int H, int W, cudaStream_t s);
cudaError_t adam(float* prm, const float* grad, float* m, float* v, float lr, float b1, float b2,
                 float eps, float bc1, float bc2, cudaStream_t s);
cudaError_t features(int prec, const void* cv, const float4* gbuf, const float* albedo,
                     __nv_bfloat16* feat, float4* c0, int npx, cudaStream_t s);
// Fallback: per 32x32 tile, flag = (standard deviation of the luminance of c0.xyz over the tile
// > thr), counted into *count.
cudaError_t tile_flags(const float4* c0, int H, int W, float thr, unsigned char* flags, int* count,
                       cudaStream_t s);
// out = in dilated by r tiles (square neighbourhood) on a tiles_x x tiles_y grid.
cudaError_t tile_dilate(const unsigned char* in, unsigned char* out, int tiles_x, int tiles_y, int r,
                        cudaStream_t s);
cudaError_t tile_select(const float4* plain, const unsigned char* flags, float4* rgb_out, int H, int W,
                        cudaStream_t s);
// *loss_out = *sum / (3 n)
cudaError_t loss_finish(const float* sum, float* loss_out, long n, cudaStream_t s);

}  // namespace kpn
}  // namespace svgf
