// Batched kernels with BF16 storage of the workspace images (see svgf_batch.cuh).
#include "svgf_batch.cuh"

SVGF_BATCH_DEFINE(bf16, dev::Store16<true>)
