// Batched kernels with FP32 storage of the workspace images (see svgf_batch.cuh).
#include "svgf_batch.cuh"

SVGF_BATCH_DEFINE(f32, dev::StoreF32)
