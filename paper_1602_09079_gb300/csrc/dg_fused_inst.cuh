// dg_fused_inst.cuh -- instantiates the fused FP32-mixed stage kernel and its
// launcher for one polynomial degree DG_K (included by dg_f<K>.cu).
#pragma once
#include "dg_fused.cuh"
#include "dg_launch.h"

#include <algorithm>

#ifndef DG_K
#error "define DG_K before including dg_fused_inst.cuh"
#endif

namespace dg {
namespace {

constexpr int FK = DG_K;
using FC = FusedCfg<FK>;

template <bool FORCE, int FLUX>
cudaError_t set_smem() {
  return cudaFuncSetAttribute(fused_f32_kernel<FK, FORCE, FLUX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)FC::smem());
}

cudaError_t fz_upload(const double* h64) {
  using TB = Tab<FK>;
  using FT = FzTab<FK>;
  constexpr int KQ = (FK + 1) * (FK + 1), N = nmodes(FK);
  float t[FzTab<3>::SIZE] = {};
  for (int j = 0; j < KQ; ++j) {
    t[FT::P + j] = (float)h64[TB::P1 + j];
    t[FT::PW + j] = (float)h64[TB::P1W + j];
    t[FT::DW + j] = (float)h64[TB::D1W + j];
  }
  for (int e = 0; e <= FK; ++e) {
    t[FT::EM + e] = (float)h64[TB::FEND + e];
    t[FT::EP + e] = (float)h64[TB::FEND + FK + 1 + e];
  }
  for (int l = 0; l < N; ++l) {
    t[FT::LM + l] = (float)h64[TB::LMAX + l];
    t[FT::LMV + l] = (float)h64[TB::LMAXV + l];
  }
  cudaError_t e = cudaMemcpyToSymbol(c_fz, t, sizeof(float) * FT::SIZE);
  if (e != cudaSuccess) return e;
  cudaError_t r[4] = {set_smem<false, 0>(), set_smem<true, 0>(), set_smem<false, 1>(), set_smem<true, 1>()};
  for (cudaError_t x : r)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

// planes per z segment: the candidate with the fewest plane iterations per
// SM over the waves of the grid (two tiles per SM on 152 SMs)
int choose_lz(const Geo& g, long long columns) {
  const long long slots = 152LL * FC::MINB;
  int best = 4;
  long long best_cost = -1;
  for (int lz : {4, 8, 16, 32, 64}) {
    const long long segs = (g.nz + lz - 1) / lz;
    const long long waves = (columns * segs + slots - 1) / slots;
    const long long cost = waves * (std::min(lz, g.nz) + 2);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = lz;
    }
  }
  return best;
}

cudaError_t fz_run(bool force, int flux, const Geo& g, FusedArgs& a, cudaStream_t s) {
  a.nbx = (g.nx + FC::BX - 1) / FC::BX;
  a.nby = (g.ny + FC::BY - 1) / FC::BY;
  const long long columns = (long long)a.nbx * a.nby;
  a.lz = choose_lz(g, columns);
  a.eps_r = (float)g.eps_rho;
  a.eps_p = (float)g.eps_p;
  const long long grid = columns * ((g.nz + a.lz - 1) / a.lz);
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned nb = (unsigned)grid;
  if (flux == 1) {
    if (force) fused_f32_kernel<FK, true, 1><<<nb, FC::THREADS, FC::smem(), s>>>(g, a);
    else fused_f32_kernel<FK, false, 1><<<nb, FC::THREADS, FC::smem(), s>>>(g, a);
  } else {
    if (force) fused_f32_kernel<FK, true, 0><<<nb, FC::THREADS, FC::smem(), s>>>(g, a);
    else fused_f32_kernel<FK, false, 0><<<nb, FC::THREADS, FC::smem(), s>>>(g, a);
  }
  return cudaGetLastError();
}

}  // namespace

#define DG_FPASTE2(a, b) a##b
#define DG_FPASTE(a, b) DG_FPASTE2(a, b)
FusedLaunchers DG_FPASTE(fused_launchers_k, DG_K)() {
  FusedLaunchers L;
  L.k = FK;
  L.upload = fz_upload;
  L.run = fz_run;
  return L;
}

}  // namespace dg
