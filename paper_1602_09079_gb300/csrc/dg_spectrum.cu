// dg_spectrum.cu -- velocity power spectrum (arXiv:1602.09079, Sect. 3.3):
// E_w(k) is the shell average of |w_hat(k)|^2 scaled so that its integral
// over k equals the mean square of w. Here the velocity of the state
// polynomial is sampled at sub^3 points per cell (cell-centred sub-cells),
// each component is transformed by a 3D real-to-complex FFT (cuFFT, on a
// caller-provided work area), and the power of every wave vector n is added
// to the shell round(|n|).
#include "dg_spectrum.h"

#include <cufft.h>

#include <cmath>

#include "dg_common.cuh"

namespace dg {
namespace spec {
namespace {

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// sqrt(2u+1) P_u(x) by the three-term recurrence
__device__ __forceinline__ double scaled_legendre(int u, double x) {
  double pm = 1.0, p = x;
  if (u == 0) return 1.0;
  for (int j = 2; j <= u; ++j) {
    const double pn = ((2 * j - 1) * x * p - (j - 1) * pm) / j;
    pm = p;
    p = pn;
  }
  return sqrt(2.0 * u + 1.0) * p;
}

// out[(Z * M + Y) * M + X] = m_comp / rho of the state polynomial at the
// centre of sub-cell (X % sub, Y % sub, Z % sub) of cell (X, Y, Z) / sub
__global__ void sample_kernel(const double* __restrict__ y, int k, int n, int sub, int comp, double* __restrict__ out) {
  const int N = nmodes(k), M = n * sub;
  const long long total = (long long)M * M * M, nc = (long long)n * n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(e % M), Y = (int)((e / M) % M), Z = (int)(e / ((long long)M * M));
    const long long cell = ((long long)(Z / sub) * n + Y / sub) * n + X / sub;
    const double xi[3] = {-1.0 + (2.0 * (X % sub) + 1.0) / sub, -1.0 + (2.0 * (Y % sub) + 1.0) / sub,
                          -1.0 + (2.0 * (Z % sub) + 1.0) / sub};
    double P[3][4];
    for (int a = 0; a < 3; ++a)
      for (int u = 0; u <= k; ++u) P[a][u] = scaled_legendre(u, xi[a]);
    double rho = 0.0, m = 0.0;
    for (int l = 0; l < N; ++l) {
      int u, v, w;
      mode_uvw(l, u, v, w);
      const double phi = P[0][u] * P[1][v] * P[2][w];
      rho += y[(size_t)l * nc + cell] * phi;
      m += y[(size_t)((1 + comp) * N + l) * nc + cell] * phi;
    }
    out[e] = m / rho;
  }
}

// shell sums of the half spectrum [M][M][M/2 + 1]: each element stands for
// itself and (unless its last index is 0 or M/2) its conjugate partner
__global__ void bin_kernel(const double2* __restrict__ sp, int M, int nb, double* __restrict__ bins) {
  extern __shared__ double sh[];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0.0;
  __syncthreads();
  const int H = M / 2 + 1;
  const long long total = (long long)M * M * H;
  const double norm = 1.0 / ((double)M * M * M) / ((double)M * M * M);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % H), b = (int)((e / H) % M), a = (int)(e / ((long long)H * M));
    const int kx = c, ky = b <= M / 2 ? b : b - M, kz = a <= M / 2 ? a : a - M;
    const double kk = sqrt((double)kx * kx + (double)ky * ky + (double)kz * kz);
    const int bin = (int)floor(kk + 0.5);
    const double w = (c == 0 || (M % 2 == 0 && c == M / 2)) ? 1.0 : 2.0;
    const double2 z = sp[e];
    if (bin < nb) atomicAdd(&sh[bin], w * (z.x * z.x + z.y * z.y) * norm);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (sh[b] != 0.0) atomicAdd(&bins[b], sh[b]);
}

// cuFFT plan of an M^3 D2Z transform with a caller-owned work area
cufftResult make_plan(int M, cufftHandle* plan, size_t* ws) {
  cufftResult r = cufftCreate(plan);
  if (r != CUFFT_SUCCESS) return r;
  r = cufftSetAutoAllocation(*plan, 0);
  if (r == CUFFT_SUCCESS) r = cufftMakePlan3d(*plan, M, M, M, CUFFT_D2Z, ws);
  if (r != CUFFT_SUCCESS) cufftDestroy(*plan);
  return r;
}

// histogram of ln(rho) of the state polynomial at the sub-cell centres:
// counts[0] below lo (and non-positive or non-finite densities),
// counts[1 + j] for floor((ln rho - lo) / (hi - lo) * nb) = j, counts[nb + 1]
// at or above hi; integer counts (order-independent)
__global__ void density_hist_kernel(const double* __restrict__ y, int k, int n, int sub, double lo, double hi, int nb,
                                    unsigned long long* __restrict__ counts) {
  extern __shared__ unsigned int shc[];
  for (int b = threadIdx.x; b < nb + 2; b += blockDim.x) shc[b] = 0u;
  __syncthreads();
  const int N = nmodes(k), M = n * sub;
  const long long total = (long long)M * M * M, nc = (long long)n * n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(e % M), Y = (int)((e / M) % M), Z = (int)(e / ((long long)M * M));
    const long long cell = ((long long)(Z / sub) * n + Y / sub) * n + X / sub;
    const double xi[3] = {-1.0 + (2.0 * (X % sub) + 1.0) / sub, -1.0 + (2.0 * (Y % sub) + 1.0) / sub,
                          -1.0 + (2.0 * (Z % sub) + 1.0) / sub};
    double P[3][4];
    for (int a = 0; a < 3; ++a)
      for (int u = 0; u <= k; ++u) P[a][u] = scaled_legendre(u, xi[a]);
    double rho = 0.0;
    for (int l = 0; l < N; ++l) {
      int u, v, w;
      mode_uvw(l, u, v, w);
      rho += y[(size_t)l * nc + cell] * (P[0][u] * P[1][v] * P[2][w]);
    }
    int b = 0;
    if (rho > 0.0 && isfinite(rho)) {
      const double sv = log(rho);
      if (sv >= hi) {
        b = nb + 1;
      } else if (sv >= lo) {
        const int j = (int)floor((sv - lo) / (hi - lo) * nb);
        b = 1 + (j < nb ? j : nb - 1);
      }
    }
    atomicAdd(&shc[b], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb + 2; b += blockDim.x)
    if (shc[b]) atomicAdd(&counts[b], (unsigned long long)shc[b]);
}

}  // namespace

cudaError_t density_pdf(int k, const double* y, int n, int sub, double lo, double hi, int nb,
                        unsigned long long* counts_dev, long long* counts_host, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counts_dev, 0, sizeof(unsigned long long) * (nb + 2), s);
  if (e != cudaSuccess) return e;
  density_hist_kernel<<<1024, 256, sizeof(unsigned int) * (nb + 2), s>>>(y, k, n, sub, lo, hi, nb, counts_dev);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = cudaMemcpyAsync(counts_host, counts_dev, sizeof(unsigned long long) * (nb + 2), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

int n_bins(int M) { return (int)std::floor(std::sqrt(3.0) * M / 2.0) + 2; }

void release(PlanCache* cache) {
  if (cache->M) cufftDestroy((cufftHandle)cache->handle);
  cache->M = 0;
  cache->ws = 0;
}

// the cached plan for M points per axis, made if the cache holds another
// size or none
static cufftResult cached_plan(int M, PlanCache* cache) {
  if (cache->M == M) return CUFFT_SUCCESS;
  release(cache);
  cufftHandle plan;
  size_t ws = 0;
  const cufftResult r = make_plan(M, &plan, &ws);
  if (r != CUFFT_SUCCESS) return r;
  cache->handle = (int)plan;
  cache->M = M;
  cache->ws = ws;
  return CUFFT_SUCCESS;
}

size_t work_bytes(int M, PlanCache* cache) {
  if (cached_plan(M, cache) != CUFFT_SUCCESS) return 0;
  const size_t ws = cache->ws;
  const size_t M3 = (size_t)M * M * M, half = (size_t)M * M * (M / 2 + 1);
  return align256(sizeof(double) * n_bins(M)) + align256(sizeof(double) * M3) + align256(sizeof(double2) * half) +
         align256(ws);
}

cudaError_t velocity_spectrum(int k, const double* y, int n, int sub, void* work, size_t bytes, double* bins_out,
                              cudaStream_t s, int* cufft_status, PlanCache* cache) {
  *cufft_status = 0;
  const int M = n * sub, nb = n_bins(M);
  const size_t M3 = (size_t)M * M * M, half = (size_t)M * M * (M / 2 + 1);
  cufftResult r = cached_plan(M, cache);
  if (r != CUFFT_SUCCESS) {
    *cufft_status = (int)r;
    return cudaSuccess;
  }
  const cufftHandle plan = (cufftHandle)cache->handle;
  const size_t ws = cache->ws;
  unsigned char* p = static_cast<unsigned char*>(work);
  double* bins = reinterpret_cast<double*>(p);
  double* real = reinterpret_cast<double*>(p + align256(sizeof(double) * nb));
  double2* cplx = reinterpret_cast<double2*>(reinterpret_cast<unsigned char*>(real) + align256(sizeof(double) * M3));
  void* area = reinterpret_cast<unsigned char*>(cplx) + align256(sizeof(double2) * half);
  if (static_cast<unsigned char*>(area) + ws > p + bytes) {
    *cufft_status = -1;
    return cudaSuccess;
  }
  cudaError_t e = cudaSuccess;
  if ((r = cufftSetWorkArea(plan, area)) == CUFFT_SUCCESS) r = cufftSetStream(plan, s);
  if (r == CUFFT_SUCCESS) e = cudaMemsetAsync(bins, 0, sizeof(double) * nb, s);
  for (int comp = 0; comp < 3 && r == CUFFT_SUCCESS && e == cudaSuccess; ++comp) {
    sample_kernel<<<2048, 256, 0, s>>>(y, k, n, sub, comp, real);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((r = cufftExecD2Z(plan, real, reinterpret_cast<cufftDoubleComplex*>(cplx))) != CUFFT_SUCCESS) break;
    bin_kernel<<<1024, 256, sizeof(double) * nb, s>>>(cplx, M, nb, bins);
    e = cudaGetLastError();
  }
  if (r == CUFFT_SUCCESS && e == cudaSuccess)
    e = cudaMemcpyAsync(bins_out, bins, sizeof(double) * nb, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (r != CUFFT_SUCCESS) *cufft_status = (int)r;
  return e;
}

}  // namespace spec
}  // namespace dg
