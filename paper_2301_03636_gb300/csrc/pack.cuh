// Parameter packing launchers (pack.cu).
#pragma once
#include "common.cuh"

namespace adv {
cudaError_t launch_repack(const ModelLayout& L, uint8_t* P, cudaStream_t s);
cudaError_t launch_set_params(const ModelLayout& L, uint8_t* P, const float* params, const double* mu,
                              const double* sigma, cudaStream_t s);
cudaError_t launch_copy_f32(const float* src, float* dst, int64_t n, cudaStream_t s);
// FP8 activation scales from the FP32 inputs of every hidden layer on a
// calibration sample (acts[l]: n x widths[l] floats).
cudaError_t launch_fp8_calibrate(const ModelLayout& L, uint8_t* P, const float* const* acts, int64_t n,
                                 cudaStream_t s);
}  // namespace adv
