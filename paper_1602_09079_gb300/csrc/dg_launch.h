// dg_launch.h -- host-side launch interface between the C ABI (dg_api.cu)
// and the per-degree kernel translation units (dg_k0.cu .. dg_k3.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_common.cuh"

namespace dg {

struct StageArgs;

struct Launchers {
  int k;
  // copy the degree's tables (FP64 and FP32 copies) to the current device
  cudaError_t (*upload)(const double* h64, const float* h32);
  // true when the FP32 path reads an FP32 shadow of the state (yf) instead
  // of the FP64 state
  bool f32_shadow;
  // one numerical flux per face point (flux 0: HLLC, 1: exact Riemann
  // solver; a failed exact iteration sets ERRB_NEWTON in ctrl->err); fh
  // holds T = double (prec 0) or float (prec 1)
  cudaError_t (*face)(int prec, int flux, const double* y, const float* yf, void* fh, const Geo& g, Ctrl* ctrl,
                      cudaStream_t s);
  // R(y) written in FP64, state layout
  cudaError_t (*volume_rhs)(int prec, bool force, const double* y, const float* yf, const void* fh,
                            const void* field, const Geo& g, double* R, Ctrl* ctrl, cudaStream_t s);
  // SSP-RK3 stage combination + limiter screen: cells failing the screen are
  // queued in list / ctrl->n_flag (ctrl->n_flag must be 0 on entry)
  cudaError_t (*volume_stage)(int prec, bool force, const void* fh, const void* field, const Geo& g,
                              const double* ys, const double* y0, double* out, double a0, double b0,
                              double dt, int* list, float* yf, Ctrl* ctrl, cudaStream_t s);
  // full limiter on the *count cells of list (count_queued: also add them
  // to the screen-failure total, i.e. no indicator filtered the list); yf
  // (nullable): FP32 shadow updated for the cells the limiter changes; d
  // (nullable): the fused stage kernels' FP32 increment y - y0 of the step,
  // recomputed for the cells the limiter changes; deep: scratch list of
  // g.nc entries (not list) for the cells that need the FP64 point
  // evaluations (ctrl->n_deep)
  cudaError_t (*limit_list)(double* y, const int* list, const unsigned* count, const Geo& g, Ctrl* ctrl,
                            int count_queued, float* yf, const double* y0, float* d, int* deep, cudaStream_t s);
  // screen[c] = 1 if cell c fails the limiter screen
  cudaError_t (*screen)(const double* y, uint8_t* screen, const Geo& g, cudaStream_t s);
  cudaError_t (*limit)(double* y, int8_t* flags, const Geo& g, Ctrl* ctrl, cudaStream_t s);
  cudaError_t (*cfl)(const double* y, const Geo& g, Ctrl* ctrl, cudaStream_t s);
  // returns the number of partial sums written to part; cells failing the
  // limiter screen afterwards are queued in list / ctrl->n_flag (0 on entry)
  cudaError_t (*energy_reset)(int prec, double* y, const Geo& g, double c2g, double inv_rho0, double* part,
                              int* n_part, int* list, Ctrl* ctrl, float* yf, cudaStream_t s);
  // projection of the cells first .. first + count - 1
  cudaError_t (*project)(const double* f, double* y, const Geo& g, long long first, long long count, cudaStream_t s);
  cudaError_t (*forcing_field)(int prec, void* field, const double* modes, int n_modes, const Geo& g,
                               const double* L, cudaStream_t s);
  // per-block partial sums of the turbulence diagnostics into part[3 * nb]
  // (field: the cached driving field in the precision prec selects, or
  // ignored when force == 0)
  cudaError_t (*diagnostics)(int prec, const double* y, const void* field, int force, const Geo& g, double* part,
                             int nb, cudaStream_t s);
  // the degree's FP64 table on the current device
  const double* (*tab64)();
  size_t table_size;
};

// Fused FP32-mixed stage kernel (face fluxes, volume quadrature and stage
// update in one launch per stage; dg_fused.cuh), built for the degrees that
// have one; run == nullptr otherwise.
// Arguments of one fused launch.
struct FusedArgs {
  const double* ys;    // stage input y^(s), state layout
  double* out;         // stage output (must not alias ys: neighbours read ys)
  float* d;            // FP32 increment y^(s) - y^(0): read in stages 2-3, written in 1-2
  float* yf;           // FP32 copy of the output written in stage 3 (nullable)
  double* R;           // stage 0: R(ys), state layout
  const float* field;  // driving field a(x) at the volume points, [3][Q^3][nc]
  int* list;           // cells failing the limiter screen
  Ctrl* ctrl;
  float b0dt, a0;      // delta = b0 dt dw/dt - a0 d
  double b0dt_d, a0_d, b0_d;  // the same in FP64, and b0 (mean density)
  const double* y0;    // y^(0) of the step (stages 2-3; may alias out in stage 3)
  float eps_r, eps_p;  // positivity floors (FP32) for the limiter screen
  int stage;           // 0: R(y); 1, 2, 3: SSP-RK3 stage
  int lz;              // planes per z segment
  int nbx, nby;        // tile columns along x and y
};

struct FusedLaunchers {
  int k;
  // 1D tables of the degree (from its FP64 table, Tab<K> layout) and the
  // kernels' shared-memory attribute, on the current device
  cudaError_t (*upload)(const double* h64);
  // one launch: args.stage 0 computes R(ys), 1-3 one SSP-RK3 stage
  cudaError_t (*run)(bool force, int flux, const Geo& g, FusedArgs& args, cudaStream_t s);
};

FusedLaunchers fused_launchers_k2();
FusedLaunchers fused_launchers_k3();

Launchers launchers_k0();
Launchers launchers_k1();
Launchers launchers_k2();
Launchers launchers_k3();

}  // namespace dg
