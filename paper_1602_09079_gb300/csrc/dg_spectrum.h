// dg_spectrum.h -- velocity power spectrum of the state (arXiv:1602.09079,
// Sect. 3.3): the state polynomial's velocity sampled on sub^3 points per
// cell, a 3D real-to-complex FFT per component (cuFFT), shell sums of the
// power. Called by the C ABI (dg_api.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace dg {
namespace spec {

// bins: floor(sqrt(3) M / 2) + 2 for the M = n * sub points per axis
int n_bins(int M);

// A context's cuFFT plan of the last transform size it used (the plan owns
// no work area: the caller's buffer is attached on every call); made on the
// first call for a size, kept until the size changes or release().
struct PlanCache {
  int handle = 0;  // cufftHandle
  int M = 0;       // points per axis of the cached plan, 0: none
  size_t ws = 0;   // its work-area bytes
};
void release(PlanCache* cache);

// device bytes the caller provides: bins, one real M^3 grid, one complex
// half-spectrum and cuFFT's work area; 0 if cuFFT cannot plan the size
size_t work_bytes(int M, PlanCache* cache);

// E(bin) = sum over wave vectors with round(|n|) = bin of |v_hat(n)|^2 / M^6,
// summed over the three velocity components (sum over bins = mean |v|^2 over
// the sample points). y: state [5][N][nc] of a cubic mesh of n^3 cells,
// degree k. bins_out: host array of n_bins(M) doubles (the call synchronises
// the stream). *cufft_status: 0, a cufftResult, or -1 if bytes is too small.
cudaError_t velocity_spectrum(int k, const double* y, int n, int sub, void* work, size_t bytes, double* bins_out,
                              cudaStream_t s, int* cufft_status, PlanCache* cache);

// density PDF: counts of ln(rho) at the sub^3 sub-cell centres of every cell
// in nb equal bins of [lo, hi), plus counts[0] (below lo, or rho not
// positive/finite) and counts[nb + 1] (at or above hi). counts_dev: device
// array of nb + 2 entries (cleared here); counts_host receives them
// (synchronises the stream).
cudaError_t density_pdf(int k, const double* y, int n, int sub, double lo, double hi, int nb,
                        unsigned long long* counts_dev, long long* counts_host, cudaStream_t s);

}  // namespace spec
}  // namespace dg
