// dg_inst.cuh -- instantiates the kernels and launchers for one polynomial
// degree DG_K (included by dg_k<K>.cu with DG_K defined).
#pragma once
#include <cmath>

#include "dg_kernels.cuh"
#include "dg_launch.h"

#ifndef DG_K
#error "define DG_K before including dg_inst.cuh"
#endif

namespace dg {
namespace {

constexpr int KK = DG_K;
using TB = Tab<KK>;

// Degree-KK basis/quadrature tables in device memory, FP64 and FP32 copies.
// Every device that loads the library holds its own copy; the host keeps
// each device's symbol address.
__device__ double g_tab64[TAB_STRIDE];
__device__ float g_tab32[TAB_STRIDE];
constexpr int kMaxDev = 64;
const double* h_tab64[kMaxDev] = {};
const float* h_tab32[kMaxDev] = {};

inline int cur_dev() {
  int d = 0;
  cudaGetDevice(&d);
  return d < kMaxDev ? d : 0;
}

template <typename T>
const T* tab_ptr();
template <>
const double* tab_ptr<double>() { return h_tab64[cur_dev()]; }
template <>
const float* tab_ptr<float>() { return h_tab32[cur_dev()]; }

inline unsigned grid1(long long n, int per) { return (unsigned)((n + per - 1) / per); }

// FP32 degrees 0-2: tiled register kernels; sum factorisation pays from
// degree 2 on (fewer multiply-adds than the dense quadrature)
constexpr bool kRegF32 = KK <= 2;
constexpr bool kSumFact = KK >= 2;

template <typename T, int MODE, bool FORCE>
cudaError_t set_volume_smem() {
  if constexpr (kSumFact && sizeof(T) == 8)
    return cudaFuncSetAttribute(volume_sf_kernel<KK, T, MODE, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)VolSF<KK, T>::smem());
  else if constexpr (kSumFact)
    return cudaFuncSetAttribute(volume_sfb_kernel<KK, T, MODE, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)VolSF<KK, T>::smem());
  else
    return cudaFuncSetAttribute(volume_kernel<KK, T, MODE, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)VolCfg<KK, T>::smem(FORCE));
}


template <int MODE, bool FORCE>
cudaError_t set_f32_smem_fw() {
  return cudaFuncSetAttribute(volume_f32_kernel<KK, MODE, FORCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)VolF32<KK>::smem(FORCE));
}

cudaError_t upload(const double* h64, const float* h32) {
  cudaError_t e = cudaMemcpyToSymbol(g_tab64, h64, sizeof(double) * TB::SIZE);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(g_tab32, h32, sizeof(float) * TB::SIZE);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_tab32, h32, sizeof(float) * TB::SIZE)) != cudaSuccess) return e;
  {
    constexpr int KQ = (KK + 1) * (KK + 1), NSF = 3 * KQ + 2 * (KK + 1);
    double f64[3 * 16 + 8];
    float f32[3 * 16 + 8];
    for (int i = 0; i < KQ; ++i) {
      f64[i] = h64[TB::P1 + i];
      f64[KQ + i] = h64[TB::P1W + i];
      f64[2 * KQ + i] = h64[TB::D1W + i];
    }
    for (int i = 0; i < 2 * (KK + 1); ++i) f64[3 * KQ + i] = h64[TB::FEND + i];
    for (int i = 0; i < NSF; ++i) f32[i] = (float)f64[i];
    if ((e = cudaMemcpyToSymbol(c_sf64, f64, sizeof(double) * NSF)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_sf32, f32, sizeof(float) * NSF)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(face_sf64_kernel<KK, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)FaceSF64<KK>::smem())) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(face_sf64_kernel<KK, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)FaceSF64<KK>::smem())) != cudaSuccess)
      return e;
  }
  void* p = nullptr;
  const int dev = cur_dev();
  if ((e = cudaGetSymbolAddress(&p, g_tab64)) != cudaSuccess) return e;
  h_tab64[dev] = static_cast<const double*>(p);
  if ((e = cudaGetSymbolAddress(&p, g_tab32)) != cudaSuccess) return e;
  h_tab32[dev] = static_cast<const float*>(p);
  cudaError_t r = cudaFuncSetAttribute(limit_list_kernel<KK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)ListLim<KK>::smem());
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(limit_screen_list_kernel<KK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ListLim<KK>::smem());
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(energy_reset_sf_kernel<KK, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ResetSF<KK, float>::smem());
  if (r == cudaSuccess)
    r = cudaFuncSetAttribute(energy_reset_sf_kernel<KK, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ResetSF<KK, double>::smem());
  if constexpr (kRegF32) {
    cudaError_t f[4] = {set_f32_smem_fw<MODE_RHS, false>(), set_f32_smem_fw<MODE_RHS, true>(),
                        set_f32_smem_fw<MODE_STAGE, false>(), set_f32_smem_fw<MODE_STAGE, true>()};
    for (cudaError_t x : f)
      if (x != cudaSuccess) r = x;
  }
  cudaError_t s[8] = {set_volume_smem<double, MODE_RHS, false>(),  set_volume_smem<double, MODE_RHS, true>(),
                      set_volume_smem<double, MODE_STAGE, false>(), set_volume_smem<double, MODE_STAGE, true>(),
                      set_volume_smem<float, MODE_RHS, false>(),   set_volume_smem<float, MODE_RHS, true>(),
                      set_volume_smem<float, MODE_STAGE, false>(),  set_volume_smem<float, MODE_STAGE, true>()};
  for (cudaError_t x : s)
    if (x != cudaSuccess) r = x;
  return r;
}

template <int FLUX>
cudaError_t face64(const double* y, void* fh, const Geo& g, Ctrl* ctrl, cudaStream_t s) {
  using CF = FaceSF64<KK>;
  face_sf64_kernel<KK, FLUX><<<grid1(g.nc, 32), CF::THREADS, CF::smem(), s>>>(y, static_cast<double*>(fh), g, ctrl);
  return cudaGetLastError();
}

// FP32 path: the face kernel (constant-bank tables) reads the FP32 shadow at
// every degree; the volume kernel is the tiled register kernel for degrees
// <= 2 and the sum-factorised shared-memory kernel for degree 3.

template <int FLUX>
cudaError_t face_f(int prec, const double* y, const float* yf, void* fh, const Geo& g, Ctrl* ctrl, cudaStream_t s) {
  if (prec) {  // FP32 path: sum-factorised traces of the FP32 shadow
    face_flux_f32_kernel<KK, FLUX><<<grid1(g.nc, 32), 96, 0, s>>>(yf, static_cast<float*>(fh), g, ctrl);
    return cudaGetLastError();
  }
  return face64<FLUX>(y, fh, g, ctrl, s);
}

cudaError_t face(int prec, int flux, const double* y, const float* yf, void* fh, const Geo& g, Ctrl* ctrl,
                 cudaStream_t s) {
  return flux == 1 ? face_f<1>(prec, y, yf, fh, g, ctrl, s) : face_f<0>(prec, y, yf, fh, g, ctrl, s);
}

template <int MODE, bool FORCE>
cudaError_t vol_f32(const float* yf, const void* fh, const void* field, const Geo& g, StageArgs st, double* R,
                    Ctrl* ctrl, cudaStream_t s) {
  using CF = VolF32<KK>;
  volume_f32_kernel<KK, MODE, FORCE><<<grid1(g.nc, CF::C), CF::THREADS, CF::smem(FORCE), s>>>(
      yf, static_cast<const float*>(fh), static_cast<const float*>(field), tab_ptr<double>(), g, st, R, ctrl);
  return cudaGetLastError();
}

template <typename T, int MODE, bool FORCE>
cudaError_t vol_t(const double* y, const float* yf, const void* fh, const void* field, const Geo& g, StageArgs st,
                  double* R, Ctrl* ctrl, cudaStream_t s) {
  if constexpr (kSumFact && sizeof(T) == 8) {
    using CF = VolSF<KK, T>;
    volume_sf_kernel<KK, T, MODE, FORCE><<<grid1(g.nc, CF::C), kThreads, CF::smem(), s>>>(
        y, yf, static_cast<const T*>(fh), static_cast<const T*>(field), tab_ptr<T>(), tab_ptr<double>(), g, st, R,
        ctrl);
  } else if constexpr (kSumFact) {
    using CF = VolSF<KK, T>;
    volume_sfb_kernel<KK, T, MODE, FORCE><<<grid1(g.nc, CF::C), kThreads, CF::smem(), s>>>(
        y, yf, static_cast<const T*>(fh), static_cast<const T*>(field), tab_ptr<T>(), tab_ptr<double>(), g, st, R,
        ctrl);
  } else {
    using CF = VolCfg<KK, T>;
    volume_kernel<KK, T, MODE, FORCE><<<grid1(g.nc, CF::C), kThreads, CF::smem(FORCE), s>>>(
        y, static_cast<const T*>(fh), static_cast<const T*>(field), tab_ptr<T>(), tab_ptr<double>(), g, st, R, ctrl);
  }
  return cudaGetLastError();
}

cudaError_t volume_rhs(int prec, bool force, const double* y, const float* yf, const void* fh, const void* field,
                       const Geo& g, double* R, Ctrl* ctrl, cudaStream_t s) {
  StageArgs st{};
  if constexpr (kRegF32) {
    if (prec)
      return force ? vol_f32<MODE_RHS, true>(yf, fh, field, g, st, R, ctrl, s)
                   : vol_f32<MODE_RHS, false>(yf, fh, field, g, st, R, ctrl, s);
  }
  if (prec)
    return force ? vol_t<float, MODE_RHS, true>(y, yf, fh, field, g, st, R, ctrl, s)
                 : vol_t<float, MODE_RHS, false>(y, yf, fh, field, g, st, R, ctrl, s);
  return force ? vol_t<double, MODE_RHS, true>(y, yf, fh, field, g, st, R, ctrl, s)
               : vol_t<double, MODE_RHS, false>(y, yf, fh, field, g, st, R, ctrl, s);
}

cudaError_t volume_stage(int prec, bool force, const void* fh, const void* field, const Geo& g, const double* ys,
                         const double* y0, double* out, double a0, double b0, double dt, int* list, float* yf,
                         Ctrl* ctrl, cudaStream_t s) {
  StageArgs st{ys, y0, out, a0, b0, dt, list, yf};
  if constexpr (kRegF32) {
    if (prec)
      return force ? vol_f32<MODE_STAGE, true>(yf, fh, field, g, st, nullptr, ctrl, s)
                   : vol_f32<MODE_STAGE, false>(yf, fh, field, g, st, nullptr, ctrl, s);
  }
  if (prec)
    return force ? vol_t<float, MODE_STAGE, true>(ys, yf, fh, field, g, st, nullptr, ctrl, s)
                 : vol_t<float, MODE_STAGE, false>(ys, yf, fh, field, g, st, nullptr, ctrl, s);
  return force ? vol_t<double, MODE_STAGE, true>(ys, yf, fh, field, g, st, nullptr, ctrl, s)
               : vol_t<double, MODE_STAGE, false>(ys, yf, fh, field, g, st, nullptr, ctrl, s);
}

cudaError_t limit_list(double* y, const int* list, const unsigned* count, const Geo& g, Ctrl* ctrl, int count_queued,
                       float* yf, const double* y0, float* d, int* deep, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&ctrl->n_deep, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  using LL = ListLim<KK>;
  limit_screen_list_kernel<KK><<<152 * LL::MINB, LL::THREADS, LL::smem(), s>>>(
      y, list, count, tab_ptr<double>(), tab_ptr<float>(), g, ctrl, count_queued, deep);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  limit_list_kernel<KK><<<152 * LL::MINB, LL::THREADS, LL::smem(), s>>>(y, deep, &ctrl->n_deep, tab_ptr<double>(), g,
                                                                       ctrl, yf, y0, d);
  return cudaGetLastError();
}

cudaError_t screen(const double* y, uint8_t* scr, const Geo& g, cudaStream_t s) {
  screen_kernel<KK><<<grid1(g.nc, kThreads), kThreads, 0, s>>>(y, scr, tab_ptr<double>(), g);
  return cudaGetLastError();
}

cudaError_t limit(double* y, int8_t* flags, const Geo& g, Ctrl* ctrl, cudaStream_t s) {
  limit_kernel<KK><<<grid1(g.nc, kThreads), kThreads, 0, s>>>(y, flags, tab_ptr<double>(), g, ctrl, tab_ptr<float>());
  return cudaGetLastError();
}

cudaError_t cfl(const double* y, const Geo& g, Ctrl* ctrl, cudaStream_t s) {
  cfl_kernel<KK><<<grid1(g.nc, kCflThreads), kCflThreads, 0, s>>>(y, g, ctrl);
  return cudaGetLastError();
}

template <typename T>
cudaError_t reset_t(double* y, const Geo& g, double c2g, double inv_rho0, double* part, int* n_part, int* list,
                    Ctrl* ctrl, float* yf, cudaStream_t s) {
  using RS = ResetSF<KK, T>;
  unsigned nb = grid1(g.nc, RS::C);
  *n_part = (int)nb;
  ResetConsts<T> rc;
  rc.c2g = (T)c2g;
  rc.inv_rho0 = (T)inv_rho0;
  rc.gm1 = (T)(g.gamma - 1.0);
  rc.two_thirds = std::fabs(g.gamma - 1.0 - 2.0 / 3.0) < 1e-15 ? 1 : 0;
  energy_reset_sf_kernel<KK, T><<<nb, RS::THREADS, RS::smem(), s>>>(y, tab_ptr<T>(), g, rc, part, list, ctrl, yf);
  return cudaGetLastError();
}

cudaError_t diagnostics(int prec, const double* y, const void* field, int force, const Geo& g, double* part, int nb,
                        cudaStream_t s) {
  if (prec)
    diag_partial_kernel<KK, float><<<nb, 256, 0, s>>>(y, static_cast<const float*>(field), tab_ptr<double>(), g,
                                                      force, part);
  else
    diag_partial_kernel<KK, double><<<nb, 256, 0, s>>>(y, static_cast<const double*>(field), tab_ptr<double>(), g,
                                                       force, part);
  return cudaGetLastError();
}

cudaError_t energy_reset(int prec, double* y, const Geo& g, double c2g, double inv_rho0, double* part, int* n_part,
                         int* list, Ctrl* ctrl, float* yf, cudaStream_t s) {
  return prec ? reset_t<float>(y, g, c2g, inv_rho0, part, n_part, list, ctrl, yf, s)
              : reset_t<double>(y, g, c2g, inv_rho0, part, n_part, list, ctrl, yf, s);
}

cudaError_t project(const double* f, double* y, const Geo& g, long long first, long long count, cudaStream_t s) {
  project_kernel<KK><<<grid1(5 * count, kThreads), kThreads, 0, s>>>(f, y, tab_ptr<double>(), g, first, count);
  return cudaGetLastError();
}

template <typename T>
cudaError_t field_t(void* field, const double* modes, int n, const Geo& g, const double* L, cudaStream_t s) {
  dim3 grid(grid1(g.nc, kThreads), TB::Q3);
  forcing_field_kernel<KK, T><<<grid, kThreads, 0, s>>>(static_cast<T*>(field), modes, n, tab_ptr<double>(), g, L[0], L[1],
                                                       L[2]);
  return cudaGetLastError();
}

cudaError_t forcing_field(int prec, void* field, const double* modes, int n, const Geo& g, const double* L,
                          cudaStream_t s) {
  return prec ? field_t<float>(field, modes, n, g, L, s) : field_t<double>(field, modes, n, g, L, s);
}

}  // namespace

#define DG_PASTE2(a, b) a##b
#define DG_PASTE(a, b) DG_PASTE2(a, b)
Launchers DG_PASTE(launchers_k, DG_K)() {
  Launchers L;
  L.k = KK;
  L.upload = upload;
  L.f32_shadow = true;
  L.face = face;
  L.volume_rhs = volume_rhs;
  L.volume_stage = volume_stage;
  L.limit = limit;
  L.limit_list = limit_list;
  L.screen = screen;
  L.cfl = cfl;
  L.energy_reset = energy_reset;
  L.diagnostics = diagnostics;
  L.project = project;
  L.forcing_field = forcing_field;
  L.tab64 = tab_ptr<double>;
  L.table_size = TB::SIZE;
  return L;
}

}  // namespace dg
