// Batched kernels with FP16 storage of the workspace images (see svgf_batch.cuh).
#include "svgf_batch.cuh"

SVGF_BATCH_DEFINE(f16, dev::Store16<false>)
