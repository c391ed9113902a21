// dg_mlp.h -- host interface between the C ABI and the indicator kernels.
#pragma once
#include <cuda_runtime.h>

#include "dg_common.cuh"

namespace dg {
namespace mlp {
int n_params(int order);
// tab64: the degree's FP64 table (its max_S |phi_l| row is read)
cudaError_t features_for(int k, const double* y, const Geo& g, const double* tab64, void* X, cudaStream_t s);
cudaError_t gate_for(int k, const double* y, const Geo& g, const double* tab64, const int* list_in,
                     const unsigned* count_in, const float* P, float logit_thr, int* list_out, unsigned* count_out,
                     unsigned long long* queued_total, cudaStream_t s);
}  // namespace mlp
}  // namespace dg
