// Host side of the batched form: the storage-precision dispatch of the batched launchers (their
// kernels are in svgf_batch.cuh, compiled once per precision in svgf_batch_<prec>.cu) and the
// launch-wide parameter test.
#include <string.h>

#include "svgf_device.cuh"

namespace svgf {

cudaError_t launch_batch_temporal_f32(const BatchTemporalArgs& a, int grid, cudaStream_t s);
cudaError_t launch_batch_temporal_f16(const BatchTemporalArgs& a, int grid, cudaStream_t s);
cudaError_t launch_batch_temporal_bf16(const BatchTemporalArgs& a, int grid, cudaStream_t s);
cudaError_t launch_batch_spatial_f32(const BatchSpatialArgs& a, int grid, cudaStream_t s);
cudaError_t launch_batch_spatial_f16(const BatchSpatialArgs& a, int grid, cudaStream_t s);
cudaError_t launch_batch_spatial_bf16(const BatchSpatialArgs& a, int grid, cudaStream_t s);
cudaError_t launch_batch_atrous_f32(int mode, int shape, const BatchAtrousArgs& a, int grid, cudaStream_t s);
cudaError_t launch_batch_atrous_f16(int mode, int shape, const BatchAtrousArgs& a, int grid, cudaStream_t s);
cudaError_t launch_batch_atrous_bf16(int mode, int shape, const BatchAtrousArgs& a, int grid, cudaStream_t s);
int batch_atrous_occupancy_f32(int mode, int shape, int form);
int batch_atrous_occupancy_f16(int mode, int shape, int form);
int batch_atrous_occupancy_bf16(int mode, int shape, int form);

bool series_only_normal(float sigma_n) { return sigma_n >= dev::kSeriesOnlySigma; }

bool same_params_but_size(const Params& a, const Params& b) {
    Params x = a, y = b;
    x.W = x.H = y.W = y.H = 0;
    return memcmp(&x, &y, sizeof(Params)) == 0;
}

cudaError_t launch_batch_temporal(int prec, const BatchTemporalArgs& a, int grid, cudaStream_t s) {
    switch (prec) {
        case 0: return launch_batch_temporal_f32(a, grid, s);
        case 1: return launch_batch_temporal_f16(a, grid, s);
        default: return launch_batch_temporal_bf16(a, grid, s);
    }
}

cudaError_t launch_batch_spatial(int prec, const BatchSpatialArgs& a, int grid, cudaStream_t s) {
    switch (prec) {
        case 0: return launch_batch_spatial_f32(a, grid, s);
        case 1: return launch_batch_spatial_f16(a, grid, s);
        default: return launch_batch_spatial_bf16(a, grid, s);
    }
}

cudaError_t launch_batch_atrous(int prec, int mode, int shape, const BatchAtrousArgs& a, int grid,
                                cudaStream_t s) {
    switch (prec) {
        case 0: return launch_batch_atrous_f32(mode, shape, a, grid, s);
        case 1: return launch_batch_atrous_f16(mode, shape, a, grid, s);
        default: return launch_batch_atrous_bf16(mode, shape, a, grid, s);
    }
}

int batch_atrous_occupancy(int prec, int mode, int shape, int form) {
    switch (prec) {
        case 0: return batch_atrous_occupancy_f32(mode, shape, form);
        case 1: return batch_atrous_occupancy_f16(mode, shape, form);
        default: return batch_atrous_occupancy_bf16(mode, shape, form);
    }
}

}  // namespace svgf
