// dg_kernels.cuh -- CUDA kernels of the modal DG hot path (arXiv:1602.09079,
// Sect. 2.3-2.5, 3.1-3.2), templated on the polynomial degree K and the
// quadrature type T (double: plain FP64 path; float: mixed path whose RK
// accumulation, limiter and reductions stay FP64).
//
// State layout: y[(i*N + l) * nc + c], rows contiguous over cells (x-fastest),
// so every per-row access of a warp over consecutive cells is coalesced.
//
// One RHS evaluation = a face kernel (one Riemann flux per face point, face
// owned by its upper cell, written once) + a volume kernel (volume
// quadrature, flux projection onto the basis gradients, the two face fluxes
// of each direction projected onto the face traces, and an epilogue: R, or
// the SSP-RK3 stage combination in FP64 followed by the limiter screen of
// the next stage's input).
#pragma once
#include "dg_common.cuh"

namespace dg {

constexpr int kThreads = 256;

enum VolMode { MODE_RHS = 0, MODE_STAGE = 1 };

// Cells per CTA of the volume kernel: the flux staging buffer
// (15 Q^3 values per cell) stays near 128 KB of shared memory.
template <int K, typename T>
struct VolCfg {
  static constexpr int Q3 = (K + 1) * (K + 1) * (K + 1);
  static constexpr int raw = (128 * 1024) / (15 * Q3 * (int)sizeof(T));
  static constexpr int C = raw >= 128 ? 128 : raw >= 64 ? 64 : raw >= 32 ? 32 : 16;
  static constexpr int N = nmodes(K);
  static constexpr size_t smem(bool force) {
    return sizeof(T) * (size_t)(5 * N * C)            // sW: stage input
           + sizeof(T) * (size_t)(15 * Q3 * C)        // sF: volume fluxes
           + (force ? sizeof(T) * (size_t)(4 * Q3 * C) : 0)  // sS: source
           + sizeof(double) * (size_t)(5 * N * C);    // sY: FP64 stage output
  }
};

struct StageArgs {
  const double* ys;  // stage input y^(s)
  const double* y0;  // y^(0) of the step
  double* out;       // stage output (may alias ys or y0; cells are CTA-private)
  double a0, b0, dt; // out = a0 y0 + b0 (ys - dt R(ys))
  int* list;         // cells whose limiter screen failed
  float* yf;         // FP32 shadow of the stage state (FP32 path): read for
                     // this CTA's cells, then overwritten with the output
};

__device__ __forceinline__ void cell_xyz(long long c, const Geo& g, int& ix, int& iy, int& iz) {
  int cc = (int)c;
  ix = cc % g.nx;
  int r = cc / g.nx;
  iy = r % g.ny;
  iz = r / g.ny;
}

__device__ __forceinline__ long long neighbour(const Geo& g, int ix, int iy, int iz, int d, int s) {
  if (d == 0) ix = (ix + s + g.nx) % g.nx;
  else if (d == 1) iy = (iy + s + g.ny) % g.ny;
  else iz = (iz + s + g.nz) % g.nz;
  return ((long long)iz * g.ny + iy) * g.nx + ix;
}

// ------------------------------------------------------------ face fluxes
// Face (d, c) joins the lower cell c - e_d (left state, its high face) and
// cell c (right state, its low face), fh[((d*5 + i)*Q2 + p)*nc + c]; the
// kernels (face_sf64_kernel, face_flux_f32_kernel) follow the FP32 section.

// Screen of the positivity limiter from a cell's FP64 means and the sums
// sabs_i = sum_{l>=1} |w_il| max_S |phi_l| (same test and margins as
// limit_cell): true when the cell provably needs no limiting.
template <int K>
__device__ __forceinline__ bool limiter_screen(const double* mean, const double* sabs, bool finite, double gamma,
                                               double eps_r, double eps_p) {
  if (!finite) return false;
  const double gm1 = gamma - 1.0;
  const double r = mean[0];
  const double pbar = gm1 * (mean[4] - 0.5 * (mean[1] * mean[1] + mean[2] * mean[2] + mean[3] * mean[3]) / r);
  if (!(r >= eps_r) || !(pbar >= eps_p)) return false;
  if (nmodes(K) == 1) return true;
  const double rlo = r - sabs[0];
  if (!(rlo >= eps_r + 1e-13 * (fabs(r) + sabs[0]))) return false;
  const double elo = mean[4] - sabs[4];
  double kin = 0.0;
#pragma unroll
  for (int a = 1; a <= 3; ++a) {
    const double mh = fabs(mean[a]) + sabs[a];
    kin += mh * mh;
  }
  kin *= 0.5 / rlo;
  const double plo = gm1 * (elo - kin);
  return plo >= eps_p + 1e-13 * gm1 * (fabs(mean[4]) + sabs[4] + kin);
}

// --------------------------------------------------------------- volume
template <int K, typename T, int MODE, bool FORCE>
__global__ void __launch_bounds__(kThreads) volume_kernel(const double* __restrict__ yin, const T* __restrict__ fh,
                                                          const T* __restrict__ field, const T* __restrict__ tab,
                                                          const double* __restrict__ tab64, Geo g, StageArgs st,
                                                          double* __restrict__ R, Ctrl* ctrl) {
  using TB = Tab<K>;
  using CF = VolCfg<K, T>;
  constexpr int N = TB::N, Q2 = TB::Q2, Q3 = TB::Q3, C = CF::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sY = reinterpret_cast<double*>(smem_raw);
  T* sW = reinterpret_cast<T*>(sY + 5 * N * C);
  T* sF = sW + 5 * N * C;
  T* sS = sF + 15 * Q3 * C;
  const long long nc = g.nc;
  const long long c0 = (long long)blockIdx.x * C;
  const int tid = threadIdx.x;
  const double* ysrc = (MODE == MODE_STAGE) ? st.ys : yin;

  // phase 1: stage input -> shared (converted to T), coalesced rows
  for (int it = tid; it < 5 * N * C; it += kThreads) {
    const int c = it % C, r = it / C;
    const long long cell = c0 + c;
    sW[r * C + c] = cell < nc ? (T)ysrc[(size_t)r * nc + cell] : T(0);
  }
  __syncthreads();

  // phase 2: values at the volume Gauss points, Euler fluxes, source
  const T gm1 = (T)(g.gamma - 1.0);
  const T idx0 = (T)g.inv_dx[0], idx1 = (T)g.inv_dx[1], idx2 = (T)g.inv_dx[2];
  for (int it = tid; it < Q3 * C; it += kThreads) {
    const int c = it % C, q = it / C;
    const long long cell = c0 + c;
    if (cell >= nc) continue;
    const T* ph = tab + TB::VPHI + q * N;
    T U[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      T a = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) a += sW[(i * N + l) * C + c] * __ldg(ph + l);
      U[i] = a;
    }
    const T ir = T(1) / U[0];
    const T v[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const T p = gm1 * (U[4] - T(0.5) * U[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
    const T idx[3] = {idx0, idx1, idx2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T F[5];
      euler_flux<T>(d, U, v, p, F);
#pragma unroll
      for (int i = 0; i < 5; ++i) sF[((d * 5 + i) * Q3 + q) * C + c] = F[i] * idx[d];
    }
    if (FORCE) {
      T a[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) a[d] = __ldg(field + ((size_t)d * Q3 + q) * nc + cell);
      sS[(0 * Q3 + q) * C + c] = U[0] * a[0];
      sS[(1 * Q3 + q) * C + c] = U[0] * a[1];
      sS[(2 * Q3 + q) * C + c] = U[0] * a[2];
      sS[(3 * Q3 + q) * C + c] = U[1] * a[0] + U[2] * a[1] + U[3] * a[2];
    }
  }
  __syncthreads();

  // phase 3: projection onto the basis (volume, source, faces): dw/dt
  for (int it = tid; it < 5 * C; it += kThreads) {
    const int c = it % C, i = it / C;
    const long long cell = c0 + c;
    if (cell >= nc) continue;
    T acc[N];
#pragma unroll
    for (int l = 0; l < N; ++l) acc[l] = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      for (int q = 0; q < Q3; ++q) {
        const T f = sF[((d * 5 + i) * Q3 + q) * C + c];
        const T* dp = tab + TB::VDPHI + (d * Q3 + q) * N;
#pragma unroll
        for (int l = 0; l < N; ++l) acc[l] += f * __ldg(dp + l);
      }
    }
    if (FORCE && i > 0) {
      for (int q = 0; q < Q3; ++q) {
        const T s = sS[((i - 1) * Q3 + q) * C + c];
        const T* pw = tab + TB::VPHIW + q * N;
#pragma unroll
        for (int l = 0; l < N; ++l) acc[l] += s * __ldg(pw + l);
      }
    }
    int ix, iy, iz;
    cell_xyz(cell, g, ix, iy, iz);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long long cu = neighbour(g, ix, iy, iz, d, +1);
      const T idx = (T)g.inv_dx[d];
      for (int p = 0; p < Q2; ++p) {
        const size_t base = ((size_t)(d * 5 + i) * Q2 + p) * nc;
        const T fm = __ldg(fh + base + cell) * idx;  // low face of this cell
        const T fp = __ldg(fh + base + cu) * idx;    // high face (owned by the upper cell)
        const T* wl = tab + TB::FPHIW + ((d * 2 + 0) * Q2 + p) * N;
        const T* wh = tab + TB::FPHIW + ((d * 2 + 1) * Q2 + p) * N;
#pragma unroll
        for (int l = 0; l < N; ++l) acc[l] += fm * __ldg(wl + l) - fp * __ldg(wh + l);
      }
    }
    if (MODE == MODE_RHS) {
#pragma unroll
      for (int l = 0; l < N; ++l) R[(size_t)(i * N + l) * nc + cell] = -(double)acc[l];
    } else {
#pragma unroll
      for (int l = 0; l < N; ++l) {
        const size_t a = (size_t)(i * N + l) * nc + cell;
        sY[(i * N + l) * C + c] = st.a0 * st.y0[a] + st.b0 * (st.ys[a] + st.dt * (double)acc[l]);
      }
    }
  }
  if (MODE == MODE_RHS) return;
  __syncthreads();

  // phase 4: limiter screen of the next stage's input (FP64); cells that
  // fail it are queued for the full limiter
  for (int it = tid; it < 5 * N * C; it += kThreads) {
    const int c = it % C, r = it / C;
    const long long cell = c0 + c;
    if (cell < nc) st.out[(size_t)r * nc + cell] = sY[r * C + c];
  }
  if (tid < C) {
    const long long cell = c0 + tid;
    if (cell < nc) {
      double m[5], a[5];
      bool fin = true;
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        m[i] = sY[(i * N) * C + tid];
        double sa = 0.0;
        for (int l = 1; l < N; ++l) sa += fabs(sY[(i * N + l) * C + tid]) * __ldg(tab64 + (g.lim_vol ? TB::LMAXV : TB::LMAX) + l);
        a[i] = sa;
        for (int l = 0; l < N; ++l) fin &= isfinite(sY[(i * N + l) * C + tid]);
      }
      if (!limiter_screen<K>(m, a, fin, g.gamma, g.eps_rho, g.eps_p)) {
        const unsigned slot = atomicAdd(&ctrl->n_flag, 1u);
        st.list[slot] = (int)cell;
      }
    }
  }
}

// ============================================================ FP32 path

// FP32 copy of this degree's tables in constant memory: with the point and
// mode loops unrolled, every table value is a compile-time offset into the
// constant bank and becomes an FMA operand (no load instruction).
namespace {
__constant__ float c_tab32[Tab<3>::SIZE];
// 1D tables of the sum-factorised kernels for this translation unit's
// degree (KQ = (k+1)^2): Pt_u(x_a) at [u*Q + a], Pt_u(x_a) w_a at KQ + [u*Q + a],
// Pt_u'(x_a) w_a at 2 KQ + [u*Q + a], Pt_e(-1) at 3 KQ + e, Pt_e(+1) at
// 3 KQ + (k+1) + e. With unrolled loops every entry is a constant-bank operand.
__constant__ float c_sf32[3 * 16 + 8];
__constant__ double c_sf64[3 * 16 + 8];
}

template <typename T>
__device__ __forceinline__ T sfc(int i);
template <>
__device__ __forceinline__ float sfc<float>(int i) { return c_sf32[i]; }
template <>
__device__ __forceinline__ double sfc<double>(int i) { return c_sf64[i]; }

// Face fluxes, FP32 (from the FP32 shadow of the state): tiles of 32
// consecutive cells, warp d computes the low
// face in direction d of each cell (left state = the lower neighbour's high
// face, right state = the cell's own low face). Traces are sum-factorised:
// the coefficients are first contracted with Pt_e(+-1) along the normal into
// the tangential coefficients E[i][(a,b)], which then give the values at all
// Q^2 face points through the tangential products (constant tables).
template <int K, int D, int FLUX>
__device__ __forceinline__ unsigned face_f32_dir(const float* __restrict__ yf, float* __restrict__ fh, const Geo& g,
                                                 long long c, int ix, int iy, int iz) {
  using TB = Tab<K>;
  constexpr int N = TB::N, Q2 = TB::Q2, T = TB::T;
  const long long nc = g.nc;
  const long long cl = neighbour(g, ix, iy, iz, D, -1);
  float EL[5 * T], ER[5 * T];
#pragma unroll
  for (int j = 0; j < 5 * T; ++j) {
    EL[j] = 0.f;
    ER[j] = 0.f;
  }
  // exponents along (normal, tangential 1, tangential 2) -> (u, v, w)
#pragma unroll
  for (int a = 0, j = 0; a <= K; ++a)
#pragma unroll
    for (int b = 0; a + b <= K; ++b, ++j)
#pragma unroll
      for (int e = 0; e + a + b <= K; ++e) {
        const int m = D == 0 ? mode_index(e, a, b) : (D == 1 ? mode_index(a, e, b) : mode_index(a, b, e));
        const float pl = c_tab32[TB::FEND + (K + 1) + e];  // lower cell: its high face, xi_d = +1
        const float pr = c_tab32[TB::FEND + e];            // own cell: its low face, xi_d = -1
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          EL[i * T + j] += __ldg(yf + (size_t)(i * N + m) * nc + cl) * pl;
          ER[i * T + j] += __ldg(yf + (size_t)(i * N + m) * nc + c) * pr;
        }
      }
  const float gamma = (float)g.gamma;
  unsigned err = 0;
#pragma unroll 1
  for (int p = 0; p < Q2; ++p) {
    float UL[5], UR[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      float aL = 0.f, aR = 0.f;
#pragma unroll
      for (int j = 0; j < T; ++j) {
        const float t2 = c_tab32[TB::F2D + p * T + j];
        aL += EL[i * T + j] * t2;
        aR += ER[i * T + j] * t2;
      }
      UL[i] = aL;
      UR[i] = aR;
    }
    float F[5];
    err |= riemann_flux<FLUX, float>(D, UL, UR, gamma, F);
#pragma unroll
    for (int i = 0; i < 5; ++i) fh[((size_t)(D * 5 + i) * Q2 + p) * nc + c] = F[i];
  }
  return err;
}

// Face fluxes, FP64, sum-factorised traces: tile of 32 cells, warp d = face
// direction (the low face of each cell). Both cells' coefficients are
// contracted along the normal with Pt_e(+-1) into the tangential
// coefficients E[i][(a,b)]; then, per tangential Gauss row t2,
// H[i][a] = sum_b E[i][(a,b)] Pt_b(t2) and per point U_i = sum_a H[i][a]
// Pt_a(t1) (E and H in shared memory, one column per thread): 5 (Q T + Q^2 (k+1))
// multiply-adds per side instead of 5 N Q^2.
template <int K>
struct FaceSF64 {
  static constexpr int TP = (K + 1) * (K + 2) / 2;
  static constexpr int THREADS = 96;
  // per thread: E of both sides (2 x 5 x TP) and H of both sides (2 x 5 x (K+1))
  static constexpr size_t smem() { return sizeof(double) * 2 * 5 * (TP + K + 1) * THREADS; }
};

template <int K, int D, int FLUX>
__device__ __forceinline__ unsigned face_sf64_dir(const double* __restrict__ y, double* __restrict__ fh,
                                                  const Geo& g, long long c, int ix, int iy, int iz, double* sE) {
  constexpr int N = nmodes(K), Q = K + 1, KP = K + 1, Q2 = Q * Q, TP = FaceSF64<K>::TP;
  constexpr int TH = FaceSF64<K>::THREADS, FE = 3 * KP * Q;
  const long long nc = g.nc;
  const long long cl = neighbour(g, ix, iy, iz, D, -1);
  double* eL = sE + threadIdx.x;                  // [i][pair] column of this thread
  double* eR = sE + 5 * TP * TH + threadIdx.x;
#pragma unroll
  for (int j = 0; j < 5 * TP; ++j) {
    eL[j * TH] = 0.0;
    eR[j * TH] = 0.0;
  }
  // one mode at a time (few live registers): its exponent along the normal
  // selects Pt_e(+-1), the tangential pair selects the E entry
#pragma unroll 1
  for (int m = 0; m < N; ++m) {
    int u, v, w;
    mode_uvw(m, u, v, w);
    const int e = D == 0 ? u : (D == 1 ? v : w);
    const int j = pair_index(K, D == 0 ? v : u, D == 2 ? v : w);
    const double pl = c_sf64[FE + KP + e];  // lower cell, xi_d = +1
    const double pr = c_sf64[FE + e];       // own cell, xi_d = -1
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      eL[(i * TP + j) * TH] += __ldg(y + (size_t)(i * N + m) * nc + cl) * pl;
      eR[(i * TP + j) * TH] += __ldg(y + (size_t)(i * N + m) * nc + c) * pr;
    }
  }
  const double gamma = g.gamma;
  unsigned err = 0;
  double* hLp = sE + 2 * 5 * TP * TH + threadIdx.x;  // [i][a] column of this thread
  double* hRp = hLp + 5 * KP * TH;
#pragma unroll 1
  for (int t2 = 0; t2 < Q; ++t2) {
#pragma unroll 1
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int a = 0; a <= K; ++a) {
        double sl = 0.0, sr = 0.0;
#pragma unroll
        for (int b = 0; a + b <= K; ++b) {
          const double pb = c_sf64[b * Q + t2];
          const int j = pair_index(K, a, b);
          sl += eL[(i * TP + j) * TH] * pb;
          sr += eR[(i * TP + j) * TH] * pb;
        }
        hLp[(i * KP + a) * TH] = sl;
        hRp[(i * KP + a) * TH] = sr;
      }
#pragma unroll 1
    for (int t1 = 0; t1 < Q; ++t1) {
      double UL[5], UR[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        double ul = 0.0, ur = 0.0;
#pragma unroll
        for (int a = 0; a <= K; ++a) {
          const double pa = c_sf64[a * Q + t1];
          ul += hLp[(i * KP + a) * TH] * pa;
          ur += hRp[(i * KP + a) * TH] * pa;
        }
        UL[i] = ul;
        UR[i] = ur;
      }
      double F[5];
      err |= riemann_flux<FLUX, double>(D, UL, UR, gamma, F);
      const int p = t1 + Q * t2;
#pragma unroll
      for (int i = 0; i < 5; ++i) fh[((size_t)(D * 5 + i) * Q2 + p) * nc + c] = F[i];
    }
  }
  return err;
}

template <int K, int FLUX>
__global__ void __launch_bounds__(FaceSF64<K>::THREADS) face_sf64_kernel(const double* __restrict__ y,
                                                                         double* __restrict__ fh, Geo g, Ctrl* ctrl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sE = reinterpret_cast<double*>(smem_raw);
  const long long c = (long long)blockIdx.x * 32 + (threadIdx.x & 31);
  if (c >= g.nc) return;  // no block-wide barrier below
  const int d = threadIdx.x >> 5;  // warp-uniform direction
  int ix, iy, iz;
  cell_xyz(c, g, ix, iy, iz);
  unsigned e;
  if (d == 0) e = face_sf64_dir<K, 0, FLUX>(y, fh, g, c, ix, iy, iz, sE);
  else if (d == 1) e = face_sf64_dir<K, 1, FLUX>(y, fh, g, c, ix, iy, iz, sE);
  else e = face_sf64_dir<K, 2, FLUX>(y, fh, g, c, ix, iy, iz, sE);
  if (e) atomicOr(&ctrl->err, e);
}

// CTAs per SM the face kernel's register budget is sized for (measured at
// degree 2, 128^3: 4 CTAs 0.82 ms, 6 CTAs 0.92 ms, 8 CTAs 1.06 ms)
template <int K>
struct FaceF32 {
  static constexpr int MINB = 4;
};

template <int K, int FLUX>
__global__ void __launch_bounds__(96, FaceF32<K>::MINB) face_flux_f32_kernel(const float* __restrict__ yf, float* __restrict__ fh,
                                                              Geo g, Ctrl* ctrl) {
  const long long c = (long long)blockIdx.x * 32 + (threadIdx.x & 31);
  if (c >= g.nc) return;
  const int d = threadIdx.x >> 5;  // warp-uniform direction
  int ix, iy, iz;
  cell_xyz(c, g, ix, iy, iz);
  unsigned e;
  if (d == 0) e = face_f32_dir<K, 0, FLUX>(yf, fh, g, c, ix, iy, iz);
  else if (d == 1) e = face_f32_dir<K, 1, FLUX>(yf, fh, g, c, ix, iy, iz);
  else e = face_f32_dir<K, 2, FLUX>(yf, fh, g, c, ix, iy, iz);
  if (e) atomicOr(&ctrl->err, e);
}

// Volume quadrature, FP32, tiled in two phases over a tile of C cells:
//  A) one warp per group of PG volume points (warp-uniform group, so the
//     point loop unrolls against compile-time constant-table offsets): the
//     cell's coefficients in registers, values at the points, Euler fluxes
//     (and the driving source) to shared memory;
//  B) one warp per conserved variable: the N accumulators of one (cell,
//     variable) in registers, the flux projection onto the basis gradients,
//     the source projection and the six face fluxes projected onto the face
//     traces, every table value a constant-bank operand; then R, or the FP64
//     SSP-RK3 stage combination and the limiter screen (cells failing it are
//     queued for the full limiter).
template <int K>
struct VolF32 {
  static constexpr int Q3 = (K + 1) * (K + 1) * (K + 1);
  static constexpr int N = nmodes(K);
  static constexpr int C = K >= 2 ? 32 : 64;  // cells per tile (a multiple of 32)
  static constexpr int NW = K >= 2 ? 3 : (K == 1 ? 2 : 1);  // warps of phase A (point subgroups)
  static constexpr int NCH = K >= 2 ? 3 : 1;                // point chunks (phase A/B rounds)
  static constexpr int PC = Q3 / NCH;                       // points per chunk
  static constexpr int PW = PC / NW;                        // points per phase-A warp and chunk
  static constexpr int THREADS = 5 * C;
  // CTAs per SM the register budget is sized for (degree 2: 56 registers,
  // no spills; 7 CTAs also fill the shared memory). Measured at 128^3,
  // degree 2: 5 CTAs 3.49 ms, 6 3.13, 7 3.00, 8 3.12
  static constexpr int MINB = K >= 2 ? 7 : 3;
  static constexpr size_t smem(bool force) {
    return sizeof(float) * (size_t)(5 * N * C + 15 * PC * C + (force ? 4 * PC * C : 0)) +
           sizeof(double) * (size_t)(10 * C);
  }
  static_assert(K > 2 || (Q3 % NCH == 0 && PC % NW == 0), "point chunks");
};

// phase A of one chunk for one warp: points q = CH*PC + W*PW + j
template <int K, int CH, int W, bool FORCE>
__device__ __forceinline__ void vol_f32_points(const float* sW, float* sF, float* sS, const float* __restrict__ field,
                                               int c, long long cell, long long nc, float gm1, const float* idx) {
  using TB = Tab<K>;
  using CF = VolF32<K>;
  constexpr int N = TB::N, Q3 = TB::Q3, C = CF::C, PC = CF::PC, PW = CF::PW;
  // one point at a time: the coefficients are re-read from shared memory
  // for each point, so no more than the point's five values stay live (the
  // kernel then fits its register budget without spilling)
#pragma unroll
  for (int j = 0; j < PW; ++j) {
    const int ql = W * PW + j;  // point within the chunk
    const int q = CH * PC + ql;
    float U[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) a += sW[(i * N + l) * C + c] * c_tab32[TB::VPHI + q * N + l];
      U[i] = a;
    }
    const float ir = 1.f / U[0];
    const float v[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const float p = gm1 * (U[4] - 0.5f * U[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float F[5];
      euler_flux<float>(d, U, v, p, F);
#pragma unroll
      for (int i = 0; i < 5; ++i) sF[((d * 5 + i) * PC + ql) * C + c] = F[i] * idx[d];
    }
    if (FORCE) {
      float a[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) a[d] = __ldg(field + ((size_t)d * Q3 + q) * nc + cell);
      sS[(0 * PC + ql) * C + c] = U[0] * a[0];
      sS[(1 * PC + ql) * C + c] = U[0] * a[1];
      sS[(2 * PC + ql) * C + c] = U[0] * a[2];
      sS[(3 * PC + ql) * C + c] = U[1] * a[0] + U[2] * a[1] + U[3] * a[2];
    }
    // without the driving-field loads the scheduler hoists the next points'
    // shared loads over this one and spills (ptxas: 836 B per thread); a
    // compiler memory barrier keeps one point live at a time
    if (!FORCE) asm volatile("" ::: "memory");
  }
}

// phase B of one chunk: accumulate the projections of its points
template <int K, int CH, bool FORCE>
__device__ __forceinline__ void vol_f32_project(const float* sF, const float* sS, int c, int i, float (&acc)[nmodes(K)]) {
  using TB = Tab<K>;
  using CF = VolF32<K>;
  constexpr int N = TB::N, Q3 = TB::Q3, C = CF::C, PC = CF::PC;
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int ql = 0; ql < PC; ++ql) {
      const int q = CH * PC + ql;
      const float f = sF[((d * 5 + i) * PC + ql) * C + c];
#pragma unroll
      for (int l = 0; l < N; ++l) acc[l] += f * c_tab32[TB::VDPHI + (d * Q3 + q) * N + l];
    }
  if (FORCE && i > 0) {
#pragma unroll
    for (int ql = 0; ql < PC; ++ql) {
      const int q = CH * PC + ql;
      const float sv = sS[((i - 1) * PC + ql) * C + c];
#pragma unroll
      for (int l = 0; l < N; ++l) acc[l] += sv * c_tab32[TB::VPHIW + q * N + l];
    }
  }
}

template <int K, int CH, bool FORCE>
__device__ __forceinline__ void vol_f32_chunk(const float* sW, float* sF, float* sS, const float* __restrict__ field,
                                              long long c0, long long nc, float gm1, const float* idx,
                                              float (&acc)[nmodes(K)]) {
  using CF = VolF32<K>;
  constexpr int C = CF::C;
  const int tid = threadIdx.x;
  {
    const int c = tid % C, wg = tid / C;  // warp-uniform phase-A role
    const long long cell = c0 + c;
    const long long cellc = cell < nc ? cell : nc - 1;  // ragged tail: in-bounds field reads
    if (wg == 0) vol_f32_points<K, CH, 0, FORCE>(sW, sF, sS, field, c, cellc, nc, gm1, idx);
    if (CF::NW > 1 && wg == 1) vol_f32_points<K, CH, (CF::NW > 1 ? 1 : 0), FORCE>(sW, sF, sS, field, c, cellc, nc, gm1, idx);
    if (CF::NW > 2 && wg == 2) vol_f32_points<K, CH, (CF::NW > 2 ? 2 : 0), FORCE>(sW, sF, sS, field, c, cellc, nc, gm1, idx);
  }
  __syncthreads();
  vol_f32_project<K, CH, FORCE>(sF, sS, tid % C, tid / C, acc);
  __syncthreads();
}

// Volume quadrature, FP32, over a tile of C cells in NCH chunks of points:
//  A) NW warps, each on a fixed subgroup of the chunk's points (warp-uniform,
//     so the point loop unrolls against compile-time constant-table offsets):
//     the cell's coefficients, values at the points, Euler fluxes (and the
//     driving source) to shared memory;
//  B) one warp per conserved variable: the N accumulators of one (cell,
//     variable) in registers, projection onto the basis gradients (and the
//     source onto the basis), every table value a constant-bank operand.
// After the last chunk, the six face fluxes are projected onto the face
// traces; then R, or the FP64 SSP-RK3 stage combination and the limiter
// screen (cells failing it are queued for the full limiter).
template <int K, int MODE, bool FORCE>
__global__ void __launch_bounds__(VolF32<K>::THREADS, VolF32<K>::MINB) volume_f32_kernel(
    const float* yfin, const float* __restrict__ fh, const float* __restrict__ field,
    const double* __restrict__ tab64, Geo g, StageArgs st, double* __restrict__ R, Ctrl* ctrl) {
  using TB = Tab<K>;
  using CF = VolF32<K>;
  constexpr int N = TB::N, Q2 = TB::Q2, C = CF::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sM = reinterpret_cast<double*>(smem_raw);  // [5][C] stage means
  double* sA = sM + 5 * C;                            // [5][C] sum |w_l| max|phi_l|
  float* sW = reinterpret_cast<float*>(sA + 5 * C);   // [5N][C]
  float* sF = sW + 5 * N * C;                         // [15][PC][C]
  float* sS = sF + 15 * CF::PC * C;                   // [4][PC][C]
  const long long nc = g.nc;
  const long long c0 = (long long)blockIdx.x * C;
  const int tid = threadIdx.x;
  const float* ysrc = (MODE == MODE_STAGE) ? st.yf : yfin;
  for (int it = tid; it < 5 * N * C; it += CF::THREADS) {
    const int c = it % C, r = it / C;
    const long long cell = c0 + c;
    sW[r * C + c] = cell < nc ? ysrc[(size_t)r * nc + cell] : (r == 0 ? 1.f : 0.f);
  }
  __syncthreads();
  const float idx[3] = {(float)g.inv_dx[0], (float)g.inv_dx[1], (float)g.inv_dx[2]};
  const float gm1 = (float)(g.gamma - 1.0);
  float acc[N];
#pragma unroll
  for (int l = 0; l < N; ++l) acc[l] = 0.f;
  vol_f32_chunk<K, 0, FORCE>(sW, sF, sS, field, c0, nc, gm1, idx, acc);
  if (CF::NCH > 1) vol_f32_chunk<K, (CF::NCH > 1 ? 1 : 0), FORCE>(sW, sF, sS, field, c0, nc, gm1, idx, acc);
  if (CF::NCH > 2) vol_f32_chunk<K, (CF::NCH > 2 ? 2 : 0), FORCE>(sW, sF, sS, field, c0, nc, gm1, idx, acc);
  const int c = tid % C, i = tid / C;  // i: conserved variable, warp-uniform
  const long long cell = c0 + c;
  const bool live = cell < nc;
  if (live) {
    int ix, iy, iz;
    cell_xyz(cell, g, ix, iy, iz);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const long long cu = neighbour(g, ix, iy, iz, d, +1);
#pragma unroll
      for (int p = 0; p < Q2; ++p) {
        const size_t base = ((size_t)(d * 5 + i) * Q2 + p) * nc;
        const float fm = __ldg(fh + base + cell) * idx[d];
        const float fp = __ldg(fh + base + cu) * idx[d];
#pragma unroll
        for (int l = 0; l < N; ++l)
          acc[l] += fm * c_tab32[TB::FPHIW + ((d * 2 + 0) * Q2 + p) * N + l] -
                    fp * c_tab32[TB::FPHIW + ((d * 2 + 1) * Q2 + p) * N + l];
      }
    }
  }
  if (MODE == MODE_RHS) {
    if (live) {
#pragma unroll
      for (int l = 0; l < N; ++l) R[(size_t)(i * N + l) * nc + cell] = -f32_to_f64(acc[l]);
    }
    return;
  }
  double mean = 0.0;
  float sabsf = 0.f;
  bool finite = true;
  // first stage (a0 = 0, b0 = 1): out = y_s + dt dw/dt exactly, without
  // reading y_0
  const bool first = st.a0 == 0.0 && st.b0 == 1.0;
  if (live) {
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const size_t a = (size_t)(i * N + l) * nc + cell;
      const double inc = __ldcg(st.ys + a) + st.dt * f32_to_f64(acc[l]);
      const double v = first ? inc : st.a0 * __ldcg(st.y0 + a) + st.b0 * inc;
      st.out[a] = v;
      const float vf = f64_to_f32(v);
      st.yf[a] = vf;
      finite &= finite64(v);
      if (l == 0) mean = v;
      else sabsf += fabsf(vf) * (g.lim_vol ? c_tab32[TB::LMAXV + l] : c_tab32[TB::LMAX + l]);
    }
  }
  // the screen's excursion sums are taken in FP32 from the rounded values
  // (relative error below 1e-6); a relative margin of 1e-5 keeps the test a
  // sufficient one
  const double sabs = (double)sabsf * (1.0 + 1e-5);
  sM[i * C + c] = finite ? mean : __longlong_as_double(0x7ff8000000000000LL);  // NaN marks non-finite
  sA[i * C + c] = sabs;
  __syncthreads();
  if (tid < C && live) {
    double m[5], a[5];
    bool fin = true;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      m[j] = sM[j * C + tid];
      a[j] = sA[j * C + tid];
      fin &= isfinite(m[j]);
    }
    if (!limiter_screen<K>(m, a, fin, g.gamma, g.eps_rho, g.eps_p)) {
      const unsigned slot = atomicAdd(&ctrl->n_flag, 1u);
      st.list[slot] = (int)cell;
    }
  }
}

// Full positivity limiter on the cells queued by a stage kernel (list of
// *count cells), in two passes, one thread per cell. The first
// (limit_screen_list_kernel) runs limit_cell's sufficient tests, the modal
// bounds and then the FP32 point screen; the cells that fail both go to a
// second list (*n_deep), which the second pass (limit_list_kernel) limits
// with the FP64 point evaluations. A cell's FP64 points run in one thread on the FP64
// pipe, so compacting these cells keeps its warps full (in the first pass
// one troubled cell among 32 would hold up the FP64 pipe for the whole
// warp). Each thread copies its cell's 5N coefficients to shared memory once
// and works on them there: the tests and the point evaluations read every
// coefficient several times (once per point), and from global memory the
// scattered cells of a warp would pull a 128-byte line per coefficient and
// thread through L1 again at every read. Limited cells are written back.
template <int K>
struct ListLim {
  static constexpr int N = nmodes(K);
  static constexpr int THREADS = 128;
  static constexpr int MINB = K >= 3 ? 2 : 4;  // 5 N doubles per thread: 100 KB per block at degree 3
  static constexpr size_t smem() { return (size_t)5 * N * THREADS * sizeof(double); }
};

template <int K>
__global__ void __launch_bounds__(ListLim<K>::THREADS, ListLim<K>::MINB)
    limit_screen_list_kernel(const double* __restrict__ y, const int* __restrict__ list, const unsigned* count,
                             const double* __restrict__ tab64, const float* __restrict__ tab32, Geo g, Ctrl* ctrl,
                             int count_queued, int* __restrict__ deep) {
  constexpr int N = nmodes(K), LT = ListLim<K>::THREADS;
  extern __shared__ __align__(16) double ws[];
  const unsigned n = *count;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(&ctrl->n_full_total, (unsigned long long)n);
    if (count_queued) atomicAdd(&ctrl->n_queued_total, (unsigned long long)n);
  }
  unsigned e = 0;
  double* w = ws + threadIdx.x;  // this thread's column, stride LT
  for (unsigned i = blockIdx.x * LT + threadIdx.x; i < n; i += gridDim.x * LT) {
    const int cell = list[i];
    for (int r = 0; r < 5 * N; ++r) w[r * LT] = y[(size_t)r * g.nc + cell];
    double mean[5], sabs[5];
    bool rho_safe, p_safe, none;
    if (limit_prelude<K>(w, LT, tab64, g.gamma, g.eps_rho, g.eps_p, &e, g.lim_vol, tab32, mean, sabs, &rho_safe,
                         &p_safe, &none) &&
        !none)
      deep[atomicAdd(&ctrl->n_deep, 1u)] = cell;
  }
  if (e) atomicOr(&ctrl->err, e);
}

template <int K>
__global__ void __launch_bounds__(ListLim<K>::THREADS, ListLim<K>::MINB)
    limit_list_kernel(double* __restrict__ y, const int* __restrict__ list, const unsigned* count,
                      const double* __restrict__ tab64, Geo g, Ctrl* ctrl, float* __restrict__ yf,
                      const double* __restrict__ y0, float* __restrict__ dinc) {
  constexpr int N = nmodes(K), LT = ListLim<K>::THREADS;
  extern __shared__ __align__(16) double ws[];
  const unsigned n = *count;
  unsigned e = 0;
  double* w = ws + threadIdx.x;  // this thread's column, stride LT
  for (unsigned i = blockIdx.x * LT + threadIdx.x; i < n; i += gridDim.x * LT) {
    const long long cell = list[i];
    const long long nc = g.nc;
    for (int r = 0; r < 5 * N; ++r) w[r * LT] = y[(size_t)r * nc + cell];
    if (limit_cell<K>(w, LT, tab64, g.gamma, g.eps_rho, g.eps_p, &e, g.lim_vol)) {
      for (int r = 0; r < 5 * N; ++r) {
        const double v = w[r * LT];
        y[(size_t)r * nc + cell] = v;
        if (yf) yf[(size_t)r * nc + cell] = (float)v;
        if (dinc) dinc[(size_t)r * nc + cell] = (float)(v - y0[(size_t)r * nc + cell]);
      }
    }
  }
  if (e) atomicOr(&ctrl->err, e);
}


// screen[c] = 1 when cell c fails the limiter screen (capture of training data)
template <int K>
__global__ void __launch_bounds__(kThreads) screen_kernel(const double* __restrict__ y, uint8_t* __restrict__ screen,
                                                          const double* __restrict__ tab64, Geo g) {
  constexpr int N = nmodes(K);
  const long long cell = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (cell >= g.nc) return;
  double m[5], a[5];
  bool fin = true;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    m[i] = y[(size_t)(i * N) * g.nc + cell];
    double sa = 0.0;
    for (int l = 1; l < N; ++l) {
      const double v = y[(size_t)(i * N + l) * g.nc + cell];
      sa += fabs(v) * __ldg(tab64 + (g.lim_vol ? Tab<K>::LMAXV : Tab<K>::LMAX) + l);
      fin &= isfinite(v);
    }
    fin &= isfinite(m[i]);
    a[i] = sa;
  }
  screen[cell] = limiter_screen<K>(m, a, fin, g.gamma, g.eps_rho, g.eps_p) ? 0 : 1;
}

// ============================================== sum-factorised volume kernel
// FP64 path (and the FP32 path of degree 3): the tensor-product structure of
// the complete-degree basis turns each contraction over the Q^3 points into
// three one-dimensional ones (sum factorisation), every stage a cooperative
// pass of the block over (cell, index) items in shared memory:
//  values   A1[u,v][c] = sum_w w_uvw P_w(c); A2[u][b,c] = sum_v A1[u,v][c] P_v(b);
//           U[a,b,c] = sum_u A2[u][b,c] P_u(a)
//  fluxes   G_d = F_d(U) / (4 dx_d) at every point (and S/8 for the source)
//  project  H_d[u][b,c] = sum_a G_d X_d(u,a); J[u,v][c] = sum_b H_0 Pw + H_1 Dw;
//           I2[u,v][c] = sum_b H_2 Pw; dw_uvw = sum_c J Pw(w,c) + I2 Dw(w,c)
//           (X_0 = Dw, X_1 = X_2 = Pw; Pw = P w_a, Dw = P' w_a)
//  faces    Mt[a][t2] = sum_t1 Fhat Pw(a,t1); M[a,b] = +-sum_t2 Mt Pw(b,t2)/(4 dx_d);
//           expanded along the normal by Pt_e(-1) (low face) or Pt_e(+1) (high).
// Multiply-adds per cell and variable at degree 2: 165 for the values, 465
// for the projection, 55 per face (dense quadrature: 270, 810, 90).
template <int K, typename T>
struct VolSF {
  static constexpr int Q = K + 1, KP = K + 1, Q2 = Q * Q, Q3 = Q * Q * Q, N = nmodes(K), TP = (K + 1) * (K + 2) / 2;
  static constexpr int mx(int a, int b) { return a > b ? a : b; }
  static constexpr int MT0 = 14 * TP * Q;  // offset of the face moments Mt in buffer 2
  // buffer 1: A1, U, H, M; buffer 2: A2, fluxes, (J, I2, SI | Mt)
  static constexpr int BUF1 = mx(mx(5 * TP * Q, 5 * Q3), mx(19 * KP * Q2, 30 * TP));
  static constexpr int BUF2 = mx(mx(5 * KP * Q2, 19 * Q3), MT0 + 30 * KP * Q);
  static constexpr int C = sizeof(T) == 8 ? (K >= 3 ? 4 : 8) : 8;
  static constexpr size_t smem() {
    return (size_t)C * (8 * (5 * N + 10) + sizeof(T) * (BUF1 + BUF2));
  }
};

template <int K>
__device__ __forceinline__ void pair_uv(int j, int& u, int& v) {
  u = 0;
  while (j > K - u) {
    j -= K - u + 1;
    ++u;
  }
  v = j;
}


// Cooperative form (FP64): one output per (cell, index) item, inner loops
// over the exact triangular ranges, so no FP64 multiply-add is issued for an
// absent mode (the FP64 pipe is the bound).
template <int K, typename T, int MODE, bool FORCE>
__global__ void __launch_bounds__(kThreads) volume_sf_kernel(const double* __restrict__ yin,
                                                             const float* __restrict__ yf32, const T* __restrict__ fh,
                                                             const T* __restrict__ field, const T* __restrict__ tab,
                                                             const double* __restrict__ tab64, Geo g, StageArgs st,
                                                             double* __restrict__ R, Ctrl* ctrl) {
  using TB = Tab<K>;
  using CF = VolSF<K, T>;
  constexpr int N = TB::N, Q = CF::Q, Q2 = CF::Q2, Q3 = CF::Q3, TP = CF::TP, C = CF::C, KP = K + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sV = reinterpret_cast<double*>(smem_raw);  // stage output (FP64)
  double* sM = sV + 5 * N * C;
  double* sA = sM + 5 * C;
  T* sW = reinterpret_cast<T*>(sV);  // stage input (T), read only by the first pass
  T* b1 = reinterpret_cast<T*>(sA + 5 * C);
  T* b2 = b1 + CF::BUF1 * C;
  const long long nc = g.nc;
  const long long c0 = (long long)blockIdx.x * C;
  const int tid = threadIdx.x;
  const T* P1 = tab + TB::P1;
  const T* P1W = tab + TB::P1W;
  const T* D1W = tab + TB::D1W;
  // stage input: FP64 state (T = double) or its FP32 shadow (T = float)
  const double* ysrc = (MODE == MODE_STAGE) ? st.ys : yin;
  const float* yfsrc = (MODE == MODE_STAGE) ? st.yf : yf32;
  for (int it = tid; it < 5 * N * C; it += kThreads) {
    const int c = it % C, r = it / C;
    const long long cell = c0 + c;
    T v = r == 0 ? T(1) : T(0);
    if (cell < nc) {
      if constexpr (sizeof(T) == 4) v = yfsrc[(size_t)r * nc + cell];
      else v = ysrc[(size_t)r * nc + cell];
    }
    sW[r * C + c] = v;
  }
  __syncthreads();
  // A1[i][pair(u,v)][qc] -> b1
  for (int it = tid; it < 5 * TP * Q * C; it += kThreads) {
    const int c = it % C, r = it / C, qc = r % Q, j = (r / Q) % TP, i = r / (Q * TP);
    int u, v;
    pair_uv<K>(j, u, v);
    T a = T(0);
    for (int w = 0; w <= K - u - v; ++w) a += sW[(i * N + mode_index(u, v, w)) * C + c] * __ldg(P1 + w * Q + qc);
    b1[it] = a;
  }
  __syncthreads();
  // A2[i][u][qb + Q qc] -> b2
  for (int it = tid; it < 5 * KP * Q2 * C; it += kThreads) {
    const int c = it % C, r = it / C, bc = r % Q2, u = (r / Q2) % KP, i = r / (Q2 * KP);
    const int qb = bc % Q, qc = bc / Q;
    T a = T(0);
    for (int v = 0; v <= K - u; ++v) a += b1[((i * TP + pair_index(K, u, v)) * Q + qc) * C + c] * __ldg(P1 + v * Q + qb);
    b2[it] = a;
  }
  __syncthreads();
  // U[i][qa + Q qb + Q2 qc] -> b1
  for (int it = tid; it < 5 * Q3 * C; it += kThreads) {
    const int c = it % C, r = it / C, q = r % Q3, i = r / Q3;
    const int qa = q % Q, bc = q / Q;
    T a = T(0);
#pragma unroll
    for (int u = 0; u <= K; ++u) a += b2[((i * KP + u) * Q2 + bc) * C + c] * __ldg(P1 + u * Q + qa);
    b1[it] = a;
  }
  __syncthreads();
  // fluxes G[d*5+i][q] = F_d / (4 dx_d), source S[i-1][q] = S / 8 -> b2
  const T gm1 = (T)(g.gamma - 1.0);
  for (int it = tid; it < Q3 * C; it += kThreads) {
    const int c = it % C, q = it / C;
    T U[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) U[i] = b1[(i * Q3 + q) * C + c];
    const T ir = T(1) / U[0];
    const T v[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const T p = gm1 * (U[4] - T(0.5) * U[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T F[5];
      euler_flux<T>(d, U, v, p, F);
      const T sc = (T)(0.25 * g.inv_dx[d]);
#pragma unroll
      for (int i = 0; i < 5; ++i) b2[((d * 5 + i) * Q3 + q) * C + c] = F[i] * sc;
    }
    if (FORCE) {
      const long long cell = c0 + c < nc ? c0 + c : nc - 1;  // ragged tail: in-bounds reads
      T a[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) a[d] = __ldg(field + ((size_t)d * Q3 + q) * nc + cell);
      const T e8 = T(0.125);
      b2[((15 + 0) * Q3 + q) * C + c] = U[0] * a[0] * e8;
      b2[((15 + 1) * Q3 + q) * C + c] = U[0] * a[1] * e8;
      b2[((15 + 2) * Q3 + q) * C + c] = U[0] * a[2] * e8;
      b2[((15 + 3) * Q3 + q) * C + c] = (U[1] * a[0] + U[2] * a[1] + U[3] * a[2]) * e8;
    }
  }
  __syncthreads();
  // H[comp][u][qb + Q qc] = sum_a G[comp][qa,qb,qc] X(u,qa) -> b1
  constexpr int NCP = FORCE ? 19 : 15;
  for (int it = tid; it < NCP * KP * Q2 * C; it += kThreads) {
    const int c = it % C, r = it / C, bc = r % Q2, u = (r / Q2) % KP, comp = r / (Q2 * KP);
    const T* X = (comp < 5) ? D1W : P1W;
    T a = T(0);
#pragma unroll
    for (int qa = 0; qa < Q; ++qa) a += b2[(comp * Q3 + qa + Q * bc) * C + c] * __ldg(X + u * Q + qa);
    b1[it] = a;
  }
  __syncthreads();
  // rows 0..4: J_i = sum_b H_{0,i} Pw + H_{1,i} Dw; rows 5..9: I2_i = sum_b H_{2,i} Pw;
  // rows 10..13: SI = sum_b SH Pw -> b2[row][pair][qc]. Face moments
  // Mt[d*2+side][i][a][t2] = sum_t1 Fhat Pw(a, t1) -> b2 + MT0
  constexpr int NR = FORCE ? 14 : 10;
  constexpr int NJ = NR * TP * Q * C;
  for (int it = tid; it < NJ + 30 * Q * C; it += kThreads) {
    if (it < NJ) {
      const int c = it % C, r = it / C, qc = r % Q, j = (r / Q) % TP, row = r / (Q * TP);
      int u, v;
      pair_uv<K>(j, u, v);
      T a = T(0);
      if (row < 5) {
        const T* h0 = b1 + ((row * KP + u) * Q2) * C;
        const T* h1 = b1 + (((5 + row) * KP + u) * Q2) * C;
#pragma unroll
        for (int qb = 0; qb < Q; ++qb)
          a += h0[(qb + Q * qc) * C + c] * __ldg(P1W + v * Q + qb) + h1[(qb + Q * qc) * C + c] * __ldg(D1W + v * Q + qb);
      } else {
        const int comp = row < 10 ? 10 + (row - 5) : 15 + (row - 10);
        const T* h = b1 + ((comp * KP + u) * Q2) * C;
#pragma unroll
        for (int qb = 0; qb < Q; ++qb) a += h[(qb + Q * qc) * C + c] * __ldg(P1W + v * Q + qb);
      }
      b2[it] = a;
    } else {
      const int jt = it - NJ;
      const int c = jt % C, r = jt / C, t2 = r % Q, i = (r / Q) % 5, ds = r / (5 * Q);
      const int d = ds >> 1, side = ds & 1;
      const long long cell = c0 + c;
      T m[KP];
#pragma unroll
      for (int a = 0; a <= K; ++a) m[a] = T(0);
      if (cell < nc) {
        long long fc = cell;  // low face: this cell's; high face: the upper cell's
        if (side) {
          int ix, iy, iz;
          cell_xyz(cell, g, ix, iy, iz);
          fc = neighbour(g, ix, iy, iz, d, +1);
        }
        const T* fp = fh + ((size_t)(d * 5 + i) * Q2 + Q * t2) * nc + fc;
#pragma unroll
        for (int t1 = 0; t1 < Q; ++t1) {
          const T f = __ldg(fp + (size_t)t1 * nc);
#pragma unroll
          for (int a = 0; a <= K; ++a) m[a] += f * __ldg(P1W + a * Q + t1);
        }
      }
#pragma unroll
      for (int a = 0; a <= K; ++a) b2[CF::MT0 * C + (((ds * 5 + i) * KP + a) * Q + t2) * C + c] = m[a];
    }
  }
  __syncthreads();
  // M[d*2+side][i][pair(a,b)] = +-(1/(4 dx_d)) sum_t2 Mt[a][t2] Pw(b, t2) -> b1
  for (int it = tid; it < 30 * TP * C; it += kThreads) {
    const int c = it % C, r = it / C, j = r % TP, i = (r / TP) % 5, ds = r / (5 * TP);
    const int d = ds >> 1, side = ds & 1;
    int a, b;
    pair_uv<K>(j, a, b);
    const T* mt = b2 + CF::MT0 * C + (((ds * 5 + i) * KP + a) * Q) * C + c;
    T m = T(0);
#pragma unroll
    for (int t2 = 0; t2 < Q; ++t2) m += mt[t2 * C] * __ldg(P1W + b * Q + t2);
    const T sc = (T)(0.25 * g.inv_dx[d]);
    b1[it] = side == 0 ? m * sc : -(m * sc);
  }
  __syncthreads();
  // dw/dt per (cell, variable, mode): volume + source + six faces
  for (int it = tid; it < 5 * N * C; it += kThreads) {
    const int c = it % C, r = it / C, l = r % N, i = r / N;
    const long long cell = c0 + c;
    int u, v, w;
    mode_uvw(l, u, v, w);
    const int j = pair_index(K, u, v);
    const T* jr = b2 + ((i * TP + j) * Q) * C + c;
    const T* ir2 = b2 + (((5 + i) * TP + j) * Q) * C + c;
    T a = T(0);
#pragma unroll
    for (int qc = 0; qc < Q; ++qc) a += jr[qc * C] * __ldg(P1W + w * Q + qc) + ir2[qc * C] * __ldg(D1W + w * Q + qc);
    if (FORCE && i > 0) {
      const T* sr = b2 + (((10 + i - 1) * TP + j) * Q) * C + c;
#pragma unroll
      for (int qc = 0; qc < Q; ++qc) a += sr[qc * C] * __ldg(P1W + w * Q + qc);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int e = d == 0 ? u : (d == 1 ? v : w);
      const int pa = d == 0 ? v : u, pb = d == 2 ? v : w;
      const int jf = pair_index(K, pa, pb);
#pragma unroll
      for (int side = 0; side < 2; ++side)
        a += b1[(((d * 2 + side) * 5 + i) * TP + jf) * C + c] * __ldg(tab + TB::FEND + side * KP + e);
    }
    if (cell < nc) {
      const size_t at = (size_t)r * nc + cell;
      if (MODE == MODE_RHS) {
        R[at] = -(double)a;
      } else {
        const double vv = st.a0 * st.y0[at] + st.b0 * (st.ys[at] + st.dt * (double)a);
        st.out[at] = vv;
        if constexpr (sizeof(T) == 4) st.yf[at] = (float)vv;
        sV[r * C + c] = vv;
      }
    }
  }
  if (MODE == MODE_RHS) return;
  __syncthreads();
  // limiter screen of the next stage's input (FP64); cells that fail it are
  // queued for the full limiter
  for (int it = tid; it < 5 * C; it += kThreads) {
    const int c = it % C, i = it / C;
    if (c0 + c >= nc) continue;
    const double* row = sV + (i * N) * C + c;
    double sa = 0.0;
    bool fin = isfinite(row[0]);
    for (int l = 1; l < N; ++l) {
      sa += fabs(row[l * C]) * __ldg(tab64 + (g.lim_vol ? TB::LMAXV : TB::LMAX) + l);
      fin &= isfinite(row[l * C]);
    }
    sM[it] = fin ? row[0] : __longlong_as_double(0x7ff8000000000000LL);
    sA[it] = sa;
  }
  __syncthreads();
  if (tid < C && c0 + tid < nc) {
    double m[5], a[5];
    bool fin = true;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      m[i] = sM[i * C + tid];
      a[i] = sA[i * C + tid];
      fin &= isfinite(m[i]);
    }
    if (!limiter_screen<K>(m, a, fin, g.gamma, g.eps_rho, g.eps_p)) {
      const unsigned slot = atomicAdd(&ctrl->n_flag, 1u);
      st.list[slot] = (int)(c0 + tid);
    }
  }
}

// Register-blocked form (FP32): an item loads its inputs along the
// contracted index once and produces all outputs along the new index, the
// 1D tables as constant-bank operands. Triangular ranges become predicated
// unrolled loops, which costs nothing where the FP32 pipe is not the bound.
template <int K, typename T, int MODE, bool FORCE>
__global__ void __launch_bounds__(kThreads) volume_sfb_kernel(const double* __restrict__ yin,
                                                             const float* __restrict__ yf32, const T* __restrict__ fh,
                                                             const T* __restrict__ field, const T* __restrict__ tab,
                                                             const double* __restrict__ tab64, Geo g, StageArgs st,
                                                             double* __restrict__ R, Ctrl* ctrl) {
  static_assert(sizeof(T) == 4, "register-blocked form: FP32 path only");
  using TB = Tab<K>;
  using CF = VolSF<K, T>;
  constexpr int N = TB::N, Q = CF::Q, Q2 = CF::Q2, Q3 = CF::Q3, TP = CF::TP, C = CF::C, KP = K + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sV = reinterpret_cast<double*>(smem_raw);  // stage output (FP64)
  double* sM = sV + 5 * N * C;
  double* sA = sM + 5 * C;
  T* sW = reinterpret_cast<T*>(sV);  // stage input (T), read only by the first pass
  T* b1 = reinterpret_cast<T*>(sA + 5 * C);
  T* b2 = b1 + CF::BUF1 * C;
  const long long nc = g.nc;
  const long long c0 = (long long)blockIdx.x * C;
  const int tid = threadIdx.x;
  // stage input: FP64 state (T = double) or its FP32 shadow (T = float)
  const double* ysrc = (MODE == MODE_STAGE) ? st.ys : yin;
  const float* yfsrc = (MODE == MODE_STAGE) ? st.yf : yf32;
  for (int it = tid; it < 5 * N * C; it += kThreads) {
    const int c = it % C, r = it / C;
    const long long cell = c0 + c;
    T v = r == 0 ? T(1) : T(0);
    if (cell < nc) {
      if constexpr (sizeof(T) == 4) v = yfsrc[(size_t)r * nc + cell];
      else v = ysrc[(size_t)r * nc + cell];
    }
    sW[r * C + c] = v;
  }
  __syncthreads();
  // Every pass below is a register-blocked 1D contraction: an item loads
  // its inputs along the contracted index once and produces all outputs
  // along the new index, the 1D table entries being constant-bank operands
  // (loops unrolled over compile-time indices).
  constexpr int OP = 0, OPW = KP * Q, ODW = 2 * KP * Q;  // P, P w, P' w in c_sf*
  // A1[i][pair(u,v)][qc] = sum_w w_i,uvw P_w(qc) -> b1
  for (int it = tid; it < 5 * TP * C; it += kThreads) {
    const int c = it % C, r = it / C, j = r % TP, i = r / TP;
    int u, v;
    pair_uv<K>(j, u, v);
    T acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = T(0);
#pragma unroll
    for (int w = 0; w <= K; ++w)
      if (w <= K - u - v) {
        const T x = sW[(i * N + mode_index(u, v, w)) * C + c];
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q] += x * sfc<T>(OP + w * Q + q);
      }
#pragma unroll
    for (int q = 0; q < Q; ++q) b1[((i * TP + j) * Q + q) * C + c] = acc[q];
  }
  __syncthreads();
  // A2[i][u][qb + Q qc] = sum_v A1[i][pair(u,v)][qc] P_v(qb) -> b2
  for (int it = tid; it < 5 * KP * Q * C; it += kThreads) {
    const int c = it % C, r = it / C, qc = r % Q, u = (r / Q) % KP, i = r / (Q * KP);
    T acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = T(0);
#pragma unroll
    for (int v = 0; v <= K; ++v)
      if (v <= K - u) {
        const T x = b1[((i * TP + pair_index(K, u, v)) * Q + qc) * C + c];
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q] += x * sfc<T>(OP + v * Q + q);
      }
#pragma unroll
    for (int q = 0; q < Q; ++q) b2[((i * KP + u) * Q2 + q + Q * qc) * C + c] = acc[q];
  }
  __syncthreads();
  // U[i][qa + Q bc] = sum_u A2[i][u][bc] P_u(qa) -> b1
  for (int it = tid; it < 5 * Q2 * C; it += kThreads) {
    const int c = it % C, r = it / C, bc = r % Q2, i = r / Q2;
    T acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = T(0);
#pragma unroll
    for (int u = 0; u <= K; ++u) {
      const T x = b2[((i * KP + u) * Q2 + bc) * C + c];
#pragma unroll
      for (int q = 0; q < Q; ++q) acc[q] += x * sfc<T>(OP + u * Q + q);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) b1[(i * Q3 + q + Q * bc) * C + c] = acc[q];
  }
  __syncthreads();
  // fluxes G[d*5+i][q] = F_d / (4 dx_d), source S[i-1][q] = S / 8 -> b2
  const T gm1 = (T)(g.gamma - 1.0);
  for (int it = tid; it < Q3 * C; it += kThreads) {
    const int c = it % C, q = it / C;
    T U[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) U[i] = b1[(i * Q3 + q) * C + c];
    const T ir = T(1) / U[0];
    const T v[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const T p = gm1 * (U[4] - T(0.5) * U[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T F[5];
      euler_flux<T>(d, U, v, p, F);
      const T sc = (T)(0.25 * g.inv_dx[d]);
#pragma unroll
      for (int i = 0; i < 5; ++i) b2[((d * 5 + i) * Q3 + q) * C + c] = F[i] * sc;
    }
    if (FORCE) {
      const long long cell = c0 + c < nc ? c0 + c : nc - 1;  // ragged tail: in-bounds reads
      T a[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) a[d] = __ldg(field + ((size_t)d * Q3 + q) * nc + cell);
      const T e8 = T(0.125);
      b2[((15 + 0) * Q3 + q) * C + c] = U[0] * a[0] * e8;
      b2[((15 + 1) * Q3 + q) * C + c] = U[0] * a[1] * e8;
      b2[((15 + 2) * Q3 + q) * C + c] = U[0] * a[2] * e8;
      b2[((15 + 3) * Q3 + q) * C + c] = (U[1] * a[0] + U[2] * a[1] + U[3] * a[2]) * e8;
    }
  }
  __syncthreads();
  // H[comp][u][bc] = sum_qa G[comp][qa + Q bc] X(u, qa), X = P' w for the
  // x-fluxes (comp < 5), P w otherwise -> b1
  constexpr int NCP = FORCE ? 19 : 15;
  for (int it = tid; it < NCP * Q2 * C; it += kThreads) {
    const int c = it % C, r = it / C, bc = r % Q2, comp = r / Q2;
    T gq[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) gq[q] = b2[(comp * Q3 + q + Q * bc) * C + c];
    if (comp < 5) {
#pragma unroll
      for (int u = 0; u <= K; ++u) {
        T a = T(0);
#pragma unroll
        for (int q = 0; q < Q; ++q) a += gq[q] * sfc<T>(ODW + u * Q + q);
        b1[((comp * KP + u) * Q2 + bc) * C + c] = a;
      }
    } else {
#pragma unroll
      for (int u = 0; u <= K; ++u) {
        T a = T(0);
#pragma unroll
        for (int q = 0; q < Q; ++q) a += gq[q] * sfc<T>(OPW + u * Q + q);
        b1[((comp * KP + u) * Q2 + bc) * C + c] = a;
      }
    }
  }
  __syncthreads();
  // rows 0..4: J_i[pair(u,v)][qc] = sum_b H_{0,i}[u][b,qc] Pw(v,b) + H_{1,i} Dw(v,b);
  // rows 5..9: I2_i = sum_b H_{2,i} Pw; rows 10..13: SI = sum_b SH Pw -> b2.
  // Face moments Mt[d*2+side][i][a][t2] = sum_t1 Fhat Pw(a, t1) -> b2 + MT0
  constexpr int NR = FORCE ? 14 : 10;
  constexpr int NJ = NR * KP * Q * C;
  for (int it = tid; it < NJ + 30 * Q * C; it += kThreads) {
    if (it < NJ) {
      const int c = it % C, r = it / C, qc = r % Q, u = (r / Q) % KP, row = r / (Q * KP);
      const int comp = row < 5 ? row : (row < 10 ? 10 + (row - 5) : 15 + (row - 10));
      T h0[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) h0[q] = b1[((comp * KP + u) * Q2 + q + Q * qc) * C + c];
      if (row < 5) {
        T h1[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) h1[q] = b1[(((5 + row) * KP + u) * Q2 + q + Q * qc) * C + c];
#pragma unroll
        for (int v = 0; v <= K; ++v)
          if (v <= K - u) {
            T a = T(0);
#pragma unroll
            for (int q = 0; q < Q; ++q) a += h0[q] * sfc<T>(OPW + v * Q + q) + h1[q] * sfc<T>(ODW + v * Q + q);
            b2[((row * TP + pair_index(K, u, v)) * Q + qc) * C + c] = a;
          }
      } else {
#pragma unroll
        for (int v = 0; v <= K; ++v)
          if (v <= K - u) {
            T a = T(0);
#pragma unroll
            for (int q = 0; q < Q; ++q) a += h0[q] * sfc<T>(OPW + v * Q + q);
            b2[((row * TP + pair_index(K, u, v)) * Q + qc) * C + c] = a;
          }
      }
    } else {
      const int jt = it - NJ;
      const int c = jt % C, r = jt / C, t2 = r % Q, i = (r / Q) % 5, ds = r / (5 * Q);
      const int d = ds >> 1, side = ds & 1;
      const long long cell = c0 + c;
      T m[KP];
#pragma unroll
      for (int a = 0; a <= K; ++a) m[a] = T(0);
      if (cell < nc) {
        long long fc = cell;  // low face: this cell's; high face: the upper cell's
        if (side) {
          int ix, iy, iz;
          cell_xyz(cell, g, ix, iy, iz);
          fc = neighbour(g, ix, iy, iz, d, +1);
        }
        const T* fp = fh + ((size_t)(d * 5 + i) * Q2 + Q * t2) * nc + fc;
#pragma unroll
        for (int t1 = 0; t1 < Q; ++t1) {
          const T f = __ldg(fp + (size_t)t1 * nc);
#pragma unroll
          for (int a = 0; a <= K; ++a) m[a] += f * sfc<T>(OPW + a * Q + t1);
        }
      }
#pragma unroll
      for (int a = 0; a <= K; ++a) b2[CF::MT0 * C + (((ds * 5 + i) * KP + a) * Q + t2) * C + c] = m[a];
    }
  }
  __syncthreads();
  // M[d*2+side][i][pair(a,b)] = +-(1/(4 dx_d)) sum_t2 Mt[a][t2] Pw(b, t2) -> b1
  for (int it = tid; it < 30 * KP * C; it += kThreads) {
    const int c = it % C, r = it / C, a = r % KP, i = (r / KP) % 5, ds = r / (5 * KP);
    const int d = ds >> 1, side = ds & 1;
    T mt[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) mt[q] = b2[CF::MT0 * C + (((ds * 5 + i) * KP + a) * Q + q) * C + c];
    const T sc = side == 0 ? (T)(0.25 * g.inv_dx[d]) : (T)(-0.25 * g.inv_dx[d]);
#pragma unroll
    for (int b = 0; b <= K; ++b)
      if (b <= K - a) {
        T m = T(0);
#pragma unroll
        for (int q = 0; q < Q; ++q) m += mt[q] * sfc<T>(OPW + b * Q + q);
        b1[((ds * 5 + i) * TP + pair_index(K, a, b)) * C + c] = m * sc;
      }
  }
  __syncthreads();
  // dw/dt per (cell, variable, (u,v)) for all w: volume + source + six faces
  for (int it = tid; it < 5 * TP * C; it += kThreads) {
    const int c = it % C, r = it / C, j = r % TP, i = r / TP;
    const long long cell = c0 + c;
    int u, v;
    pair_uv<K>(j, u, v);
    T jr[Q], i2[Q], sr[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      jr[q] = b2[((i * TP + j) * Q + q) * C + c];
      i2[q] = b2[(((5 + i) * TP + j) * Q + q) * C + c];
      sr[q] = (FORCE && i > 0) ? b2[(((10 + i - 1) * TP + j) * Q + q) * C + c] : T(0);
    }
    const T* Mi = b1 + (i * TP) * C + c;  // M[ds][i][pair] at Mi[(ds*5*TP + pair) * C]
#pragma unroll
    for (int w = 0; w <= K; ++w)
      if (w <= K - u - v) {
        T a = T(0);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          a += jr[q] * sfc<T>(OPW + w * Q + q) + i2[q] * sfc<T>(ODW + w * Q + q);
          if (FORCE) a += sr[q] * sfc<T>(OPW + w * Q + q);
        }
        // faces: along x the normal exponent is u and the tangential pair
        // (v, w); along y v and (u, w); along z w and (u, v)
        const int jx = pair_index(K, v, w), jy = pair_index(K, u, w);
        a += Mi[((0 * 5) * TP + jx) * C] * __ldg(tab + TB::FEND + u) +
             Mi[((1 * 5) * TP + jx) * C] * __ldg(tab + TB::FEND + KP + u);
        a += Mi[((2 * 5) * TP + jy) * C] * __ldg(tab + TB::FEND + v) +
             Mi[((3 * 5) * TP + jy) * C] * __ldg(tab + TB::FEND + KP + v);
        a += Mi[((4 * 5) * TP + j) * C] * sfc<T>(3 * KP * Q + w) +
             Mi[((5 * 5) * TP + j) * C] * sfc<T>(3 * KP * Q + KP + w);
        if (cell < nc) {
          const int l = mode_index(u, v, w);
          const size_t at = (size_t)(i * N + l) * nc + cell;
          if (MODE == MODE_RHS) {
            R[at] = -f32_to_f64(a);
          } else {
            const double inc = st.ys[at] + st.dt * f32_to_f64(a);
            const double vv = (st.a0 == 0.0 && st.b0 == 1.0) ? inc : st.a0 * st.y0[at] + st.b0 * inc;
            st.out[at] = vv;
            st.yf[at] = f64_to_f32(vv);
            sV[(i * N + l) * C + c] = vv;
          }
        }
      }
  }
  if (MODE == MODE_RHS) return;
  __syncthreads();
  // limiter screen of the next stage's input (FP64); cells that fail it are
  // queued for the full limiter
  for (int it = tid; it < 5 * C; it += kThreads) {
    const int c = it % C, i = it / C;
    if (c0 + c >= nc) continue;
    const double* row = sV + (i * N) * C + c;
    double sa = 0.0;
    bool fin = isfinite(row[0]);
    for (int l = 1; l < N; ++l) {
      sa += fabs(row[l * C]) * __ldg(tab64 + (g.lim_vol ? TB::LMAXV : TB::LMAX) + l);
      fin &= isfinite(row[l * C]);
    }
    sM[it] = fin ? row[0] : __longlong_as_double(0x7ff8000000000000LL);
    sA[it] = sa;
  }
  __syncthreads();
  if (tid < C && c0 + tid < nc) {
    double m[5], a[5];
    bool fin = true;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      m[i] = sM[i * C + tid];
      a[i] = sA[i * C + tid];
      fin &= isfinite(m[i]);
    }
    if (!limiter_screen<K>(m, a, fin, g.gamma, g.eps_rho, g.eps_p)) {
      const unsigned slot = atomicAdd(&ctrl->n_flag, 1u);
      st.list[slot] = (int)(c0 + tid);
    }
  }
}

// ------------------------------------------------------ standalone limiter
template <int K>
__global__ void __launch_bounds__(kThreads) limit_kernel(double* __restrict__ y, int8_t* __restrict__ flags,
                                                         const double* __restrict__ tab64, Geo g, Ctrl* ctrl,
                                                         const float* __restrict__ tab32) {
  __shared__ unsigned s_err;
  __shared__ unsigned s_cnt;
  if (threadIdx.x == 0) {
    s_err = 0u;
    s_cnt = 0u;
  }
  __syncthreads();
  const long long cell = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (cell < g.nc) {
    unsigned e = 0;
    int f = limit_cell<K>(y + cell, g.nc, tab64, g.gamma, g.eps_rho, g.eps_p, &e, g.lim_vol, tab32);
    if (flags) flags[cell] = (int8_t)f;
    if (f) atomicAdd(&s_cnt, 1u);
    if (e) atomicOr(&s_err, e);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_err) atomicOr(&ctrl->err, s_err);
    if (s_cnt) atomicAdd(&ctrl->n_limited, (unsigned long long)s_cnt);
  }
}

// ------------------------------------------------------------ CFL (max s)
// s_K = sum_a (|v_a| + c) / dx_a from the cell means; the result is the FP64
// maximum over cells, bit for bit what the plain FP64 loop gives, but the
// FP64 division and square root (the FP64 pipe is about 1/64 of the FP32
// rate) run for a few cells per block only. One cell per thread: s in FP32
// first (means converted on the integer pipe, correctly rounded reciprocal
// and square root), then the block's FP32 maximum over the trusted cells; the cells
// within a relative 1e-3 of it and the untrusted ones (means not finite or
// not clearly positive, pressure from a cancellation E - kin with kin above
// 0.99 E) are evaluated in FP64, and the FP64 maximum of those is the
// block's maximum. A trusted cell's FP32 s is within a relative 1e-4 of its
// FP64 s (a few roundings, the pressure's amplified at most 199x by the
// cancellation, halved by the square root), so the cell holding the
// block's FP64 maximum is always among the re-evaluated ones. Blocks combine
// by one atomicMax on the bit pattern of the non-negative double. Blocks of
// 1024 cells: a block's re-evaluations (usually the one cell that holds its
// maximum) occupy the FP64 pipe for a whole warp, so fewer, larger blocks.
constexpr int kCflThreads = 1024;

template <int K>
__global__ void __launch_bounds__(kCflThreads) cfl_kernel(const double* __restrict__ y, Geo g, Ctrl* ctrl) {
  constexpr int N = nmodes(K);
  const long long nc = g.nc;
  const long long c = (long long)blockIdx.x * kCflThreads + threadIdx.x;
  double r = 1.0, m1 = 0.0, m2 = 0.0, m3 = 0.0, E = 0.0;
  float sf = 0.f;
  bool trusted = false;
  if (c < nc) {
    r = y[c];
    m1 = y[(size_t)N * nc + c];
    m2 = y[(size_t)2 * N * nc + c];
    m3 = y[(size_t)3 * N * nc + c];
    E = y[(size_t)4 * N * nc + c];
    const float rf = f64_to_f32(r), m1f = f64_to_f32(m1), m2f = f64_to_f32(m2), m3f = f64_to_f32(m3);
    const float Ef = f64_to_f32(E);
    const float irf = __frcp_rn(rf);
    const float kin = 0.5f * (m1f * m1f + m2f * m2f + m3f * m3f) * irf;
    const float prf = f64_to_f32(g.gamma - 1.0) * (Ef - kin);
    const float csf = sqrtf(f64_to_f32(g.gamma) * prf * irf);
    sf = (fabsf(m1f) * irf + csf) * f64_to_f32(g.inv_dx[0]) + (fabsf(m2f) * irf + csf) * f64_to_f32(g.inv_dx[1]) +
         (fabsf(m3f) * irf + csf) * f64_to_f32(g.inv_dx[2]);
    trusted = rf >= 1e-30f && rf <= 1e30f && Ef <= 1e30f && kin <= 0.99f * Ef && prf >= 1e-30f && sf <= 3e38f;
  }
  __shared__ float s_wf[kCflThreads / 32];
  __shared__ double s_w[kCflThreads / 32];
  __shared__ unsigned s_err;
  float mf = trusted ? sf : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mf = fmaxf(mf, __shfl_xor_sync(0xffffffffu, mf, o));
  if (threadIdx.x == 0) s_err = 0u;
  if ((threadIdx.x & 31) == 0) s_wf[threadIdx.x >> 5] = mf;
  __syncthreads();
  mf = s_wf[0];
#pragma unroll
  for (int w = 1; w < kCflThreads / 32; ++w) mf = fmaxf(mf, s_wf[w]);
  double smax = 0.0;
  unsigned e = 0;
  if (c < nc && (!trusted || sf >= mf * (1.f - 1e-3f))) {
    const double ir = 1.0 / r;
    const double pr = (g.gamma - 1.0) * (E - 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) * ir);
    if (!(r > 0.0) || !(pr > 0.0)) {
      e = (isfinite(r) && isfinite(pr)) ? ERRB_POSITIVITY : ERRB_NONFINITE;
    } else {
      const double cs = sqrt(g.gamma * pr * ir);
      smax = (fabs(m1) * ir + cs) * g.inv_dx[0] + (fabs(m2) * ir + cs) * g.inv_dx[1] +
             (fabs(m3) * ir + cs) * g.inv_dx[2];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = smax;
  if (e) atomicOr(&s_err, e);
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kCflThreads / 32 ? s_w[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) {
      atomicMax(&ctrl->cfl_max_bits, (unsigned long long)__double_as_longlong(v));
      if (s_err) atomicOr(&ctrl->err, s_err);
    }
  }
}

// ------------------------------------------------------- energy reset
// Sect. 3.2: at every volume point rho eps = c^2/(gamma-1) rho (rho/rho0)^(gamma-1),
// E_q = 1/2 |m_q|^2 / rho_q + rho_q eps_q, energy modes re-projected (one
// thread per (cell, mode)); only the energy rows are written back. Cells
// that then fail the limiter screen are queued (list / ctrl->n_flag) for the
// full limiter. part[blockIdx.x] receives the block's sum of
// (e_before - e_after), e = E - |m|^2 / (2 rho) from the means.
// Constants of the energy reset in the kernel's arithmetic type, prepared
// on the host (the FP32 kernel then does no per-thread FP64 set-up work).
template <typename T>
struct ResetConsts {
  T c2g, inv_rho0, gm1;  // c^2/(gamma-1), 1/rho0, gamma-1
  int two_thirds;        // gamma - 1 within 1e-15 of 2/3
};

// Energy reset with sum-factorised point values and projection (the same
// sums as a dense evaluation, reordered): one thread per (cell, variable)
// for rho and the momenta loads the variable's N coefficients once and
// evaluates them at the Q^3 Gauss points along z, then y, then x (the 1D
// tables of the sum-factorised kernels), writing rows of Q^3 values per cell
// to shared memory with 16-byte stores; one thread per (cell, point) forms
// E_q; the projection of E contracts x first (one (cell, qz, qy) per
// thread), then y and z per mode. Rows are padded to a multiple of 16 bytes
// whose stride spreads the 8 rows of a quarter warp over all 32 banks. The
// screen sums of rho and the momenta come from the coefficients the value
// threads hold; those of E from the new modes.
template <int K, typename T>
struct ResetSF {
  static constexpr int C = 32;  // cells per block: one warp per variable
  static constexpr int THREADS = 4 * C;
  static constexpr int Q = K + 1, Q3 = Q * Q * Q, N = nmodes(K);
  static constexpr int V = 16 / (int)sizeof(T);  // elements per 16-byte access
  // row length: at least Q^3, a multiple of V, and (in 4-byte words) an odd
  // multiple of 4 modulo 32 apart from row to row
  static constexpr int ROWW = ((Q3 * (int)sizeof(T) / 4 + 3) / 4) * 4;  // words, multiple of 4
  static constexpr int ROW = ((ROWW / 4) % 2 == 1 ? ROWW : ROWW + 4) * 4 / (int)sizeof(T);
  // dynamic shared memory: point values [4][C][ROW] and E [C][ROW]
  static constexpr size_t smem() { return (size_t)5 * C * ROW * sizeof(T); }
};

template <int K, typename T>
__global__ void __launch_bounds__(ResetSF<K, T>::THREADS) energy_reset_sf_kernel(
    double* __restrict__ y, const T* __restrict__ tab, Geo g, ResetConsts<T> rc, double* __restrict__ part,
    int* __restrict__ list, Ctrl* ctrl, float* __restrict__ yf) {
  using RS = ResetSF<K, T>;
  using TB = Tab<K>;
  constexpr int C = RS::C, Q = RS::Q, Q3 = RS::Q3, N = RS::N, ROW = RS::ROW, V = RS::V;
  struct alignas(16) Vec {
    T v[V];
  };
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);  // [variable][cell][point]
  T* sE = sU + 4 * C * ROW;                // [cell][point]
  __shared__ double sEn[N * C];                // new energy modes [mode][cell]
  __shared__ double sM[5 * C];                 // means (old energy mean in row 4)
  __shared__ double sA[5 * C];                 // sum_l |w_il| max |phi_l|
  __shared__ int sFin[5 * C];
  const long long nc = g.nc;
  const long long c0 = (long long)blockIdx.x * C;
  const int tid = threadIdx.x;
  const bool from_shadow = sizeof(T) == 4 && yf != nullptr;
  // ------------------------------------------------ point values of rho, m
  {
    const int i = tid / C, c = tid % C;  // warp = variable
    const long long cell = c0 + c;
    const bool in = cell < nc;
    T w[N];
    double mean = in ? y[(size_t)(i * N) * nc + cell] : (i == 0 ? 1.0 : 0.0);
    if constexpr (sizeof(T) == 4) w[0] = f64_to_f32(mean);
    else w[0] = mean;
#pragma unroll
    for (int l = 1; l < N; ++l) {
      if (!in) w[l] = T(0);
      else if (from_shadow) w[l] = (T)yf[(size_t)(i * N + l) * nc + cell];
      else w[l] = (T)y[(size_t)(i * N + l) * nc + cell];
    }
    sM[i * C + c] = mean;
    if (tid < C) sM[4 * C + c] = in ? y[(size_t)(4 * N) * nc + cell] : 0.0;
    // screen sums of this variable from the coefficients held (FP32: of the
    // rounded coefficients, widened by a relative 1e-5, still an upper bound)
    {
      T sa = T(0);
      bool fin = true;
#pragma unroll
      for (int l = 1; l < N; ++l) {
        T lm;
        if constexpr (sizeof(T) == 4) lm = g.lim_vol ? c_tab32[TB::LMAXV + l] : c_tab32[TB::LMAX + l];
        else lm = __ldg(tab + (g.lim_vol ? TB::LMAXV : TB::LMAX) + l);
        sa += fabs(w[l]) * lm;
        fin &= isfinite(w[l]);
      }
      sA[i * C + c] = in ? (sizeof(T) == 4 ? (double)sa * (1.0 + 1e-5) : (double)sa) : 0.0;
      sFin[i * C + c] = in ? (int)fin : 1;
    }
    // values at q = qx + Q (qy + Q qz): contract z, then y, then x with
    // Pt_u(x_a) (sfc<T>(u Q + a))
    T vals[Q3];
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) {
      T A1[(K + 1) * (K + 2) / 2];
#pragma unroll
      for (int u = 0, j = 0; u <= K; ++u)
#pragma unroll
        for (int v = 0; u + v <= K; ++v, ++j) {
          T s = T(0);
#pragma unroll
          for (int ww = 0; u + v + ww <= K; ++ww) s += w[mode_index(u, v, ww)] * sfc<T>(ww * Q + qz);
          A1[j] = s;
        }
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) {
        T A2[K + 1];
#pragma unroll
        for (int u = 0, j = 0; u <= K; ++u) {
          T s = T(0);
#pragma unroll
          for (int v = 0; u + v <= K; ++v, ++j) s += A1[j] * sfc<T>(v * Q + qy);
          A2[u] = s;
        }
#pragma unroll
        for (int qx = 0; qx < Q; ++qx) {
          T s = T(0);
#pragma unroll
          for (int u = 0; u <= K; ++u) s += A2[u] * sfc<T>(u * Q + qx);
          vals[qx + Q * (qy + Q * qz)] = s;
        }
      }
    }
    Vec* out = reinterpret_cast<Vec*>(sU + (i * C + c) * ROW);
#pragma unroll
    for (int k = 0; k < ROW / V; ++k) {
      Vec t;
#pragma unroll
      for (int e = 0; e < V; ++e) t.v[e] = k * V + e < Q3 ? vals[k * V + e] : T(0);
      out[k] = t;
    }
  }
  __syncthreads();
  // --------------------------------------------------- E at the points
  const T gm1 = rc.gm1;
  const bool two_thirds = rc.two_thirds != 0;
  const T tc2g = rc.c2g, tir0 = rc.inv_rho0;
  for (int it = tid; it < Q3 * C; it += RS::THREADS) {
    const int c = it / Q3, q = it - c * Q3;  // consecutive threads: consecutive points of a cell
    const T r = sU[(0 * C + c) * ROW + q];
    const T m1 = sU[(1 * C + c) * ROW + q], m2 = sU[(2 * C + c) * ROW + q], m3 = sU[(3 * C + c) * ROW + q];
    // gamma = 5/3 (gamma - 1 within 1e-15 of 2/3): x^(2/3) as cbrt(x)^2
    const T x = r * tir0;
    T xg;
    if (two_thirds) {
      const T cx = cbrt(x);
      xg = cx * cx;
    } else {
      xg = pow(x, gm1);
    }
    sE[c * ROW + q] = T(0.5) * (m1 * m1 + m2 * m2 + m3 * m3) / r + r * (tc2g * xg);
  }
  __syncthreads();
  // --------------------------------------------------- projection of E
  // sum-factorised: G[(qz, qy)][u] = sum_qx E Pt_u(x_qx) w_qx (one (cell,
  // qz, qy) per thread, into the dead point-value rows), then every mode
  // (u, v, w) as sum_qz Pt_w w_qz sum_qy Pt_v w_qy G[(qz, qy)][u] (one
  // (cell, mode) per thread); Pt w from the 1D tables (sfc<T>(KQ + u Q + a))
  constexpr int KQ = (K + 1) * Q, GROW = Q * Q * (K + 1);
  T* sG = sU;  // [cell][(qz Q + qy) (K + 1) + u]
  for (int it = tid; it < Q * Q * C; it += RS::THREADS) {
    const int c = it / (Q * Q), r = it - c * (Q * Q);  // r = qz Q + qy
    const T* e = sE + c * ROW + r * Q;
    T ev[Q];
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) ev[qx] = e[qx];
#pragma unroll
    for (int u = 0; u <= K; ++u) {
      T s = T(0);
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) s += ev[qx] * sfc<T>(KQ + u * Q + qx);
      sG[c * GROW + r * (K + 1) + u] = s;
    }
  }
  __syncthreads();
  for (int it = tid; it < N * C; it += RS::THREADS) {
    const int l = it / C, c = it - l * C;  // a warp: one mode of 32 cells
    int u, v, ww;
    mode_uvw(l, u, v, ww);
    T pv[Q], pz[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      pv[q] = sfc<T>(KQ + v * Q + q);
      pz[q] = sfc<T>(KQ + ww * Q + q);
    }
    const T* gc = sG + c * GROW + u;
    T acc = T(0);
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) {
      T h = T(0);
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) h += gc[(qz * Q + qy) * (K + 1)] * pv[qy];
      acc += h * pz[qz];
    }
    acc *= T(0.125);  // the reference cell's volume 8: w_l = 1/8 sum_q E phi_l w_q
    if constexpr (sizeof(T) == 4) sEn[l * C + c] = f32_to_f64(acc);
    else sEn[l * C + c] = acc;
  }
  __syncthreads();
  // ------------------------------- screen of the reset state, dissipation
  double diss = 0.0;
  if (tid < C && c0 + tid < nc) {
    const int c = tid;
    const long long cell = c0 + c;
    double ae = 0.0;
    bool fin = isfinite(sEn[c]);
    if constexpr (sizeof(T) == 4) {
      float sf = 0.f;
#pragma unroll
      for (int l = 1; l < N; ++l) {
        const float v = f64_to_f32(sEn[l * C + c]);
        sf += fabsf(v) * (g.lim_vol ? c_tab32[TB::LMAXV + l] : c_tab32[TB::LMAX + l]);
        fin &= isfinite(v);
      }
      ae = (double)sf * (1.0 + 1e-5);
    } else {
#pragma unroll
      for (int l = 1; l < N; ++l) {
        const double v = sEn[l * C + c];
        ae += fabs(v) * __ldg(tab + (g.lim_vol ? TB::LMAXV : TB::LMAX) + l);
        fin &= isfinite(v);
      }
    }
    const double r = sM[c], m1 = sM[C + c], m2 = sM[2 * C + c], m3 = sM[3 * C + c];
    const double kin = 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) / r;
    diss = (sM[4 * C + c] - kin) - (sEn[c] - kin);
    double m[5] = {r, m1, m2, m3, sEn[c]}, a[5];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = sA[i * C + c];
      fin &= sFin[i * C + c] != 0;
    }
    a[4] = ae;
    if (!limiter_screen<K>(m, a, fin, g.gamma, g.eps_rho, g.eps_p)) {
      const unsigned slot = atomicAdd(&ctrl->n_flag, 1u);
      list[slot] = (int)cell;
    }
  }
  // block sum of the dissipation: the C = 32 cells are warp 0's (fixed
  // shuffle order: deterministic)
  if (tid < 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) diss += __shfl_xor_sync(0xffffffffu, diss, o);
    if (tid == 0) part[blockIdx.x] = diss;
  }
  for (int it = tid; it < N * C; it += RS::THREADS) {
    const int l = it / C, c = it - l * C;
    const long long cell = c0 + c;
    if (cell < nc) {
      y[(size_t)(4 * N + l) * nc + cell] = sEn[l * C + c];
      if (yf) yf[(size_t)(4 * N + l) * nc + cell] = f64_to_f32(sEn[l * C + c]);
    }
  }
}

// ------------------------------------------------------------- projection
// w_l = 1/8 sum_q f(x_q) phi_l(xi_q) omega_q (Sect. 2.3), f canonical
// [nc][5][Q^3]. One thread per (cell, variable).
// Cells first .. first + count - 1; f holds their point values only.
template <int K>
__global__ void __launch_bounds__(kThreads) project_kernel(const double* __restrict__ f, double* __restrict__ y,
                                                           const double* __restrict__ tab64, Geo g, long long first,
                                                           long long count) {
  using TB = Tab<K>;
  constexpr int N = TB::N, Q3 = TB::Q3;
  const long long nc = g.nc;
  const long long it = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (it >= 5 * count) return;
  const long long local = it % count;
  const long long cell = first + local;
  const int i = (int)(it / count);
  double acc[N];
#pragma unroll
  for (int l = 0; l < N; ++l) acc[l] = 0.0;
  for (int q = 0; q < Q3; ++q) {
    const double v = f[((size_t)local * 5 + i) * Q3 + q];
    const double* pw = tab64 + TB::VPHIW + q * N;
#pragma unroll
    for (int l = 0; l < N; ++l) acc[l] += v * __ldg(pw + l);
  }
#pragma unroll
  for (int l = 0; l < N; ++l) y[(size_t)(i * N + l) * nc + cell] = acc[l];
}

// --------------------------------------------------------- forcing field
// a(x_q) = sum_j Re a_j cos(k_j.x) - Im a_j sin(k_j.x), k_j = 2 pi n_j / L
// (Sect. 3.1), cached at every volume point: field[(d*Q3 + q)*nc + c].
// modes: [n][9] = n_x, n_y, n_z (as doubles), Re a (3), Im a (3).
// Turbulence diagnostics (Sect. 4.1 rms Mach number, Sect. 4.2 injected
// energy): per-block partial sums, in a fixed order, of the per-cell
// (|m|/rho / c)^2 and |m|^2/(2 rho) of the cell means and, with forcing, the
// injected power density sum_q (m . a)(xi_q) omega_q / 8 (the state
// polynomial's momentum at the volume Gauss points times the cached driving
// field). part[j * gridDim.x + b], j = 0, 1, 2.
template <int K, typename T>
__global__ void __launch_bounds__(256) diag_partial_kernel(const double* __restrict__ y, const T* __restrict__ field,
                                                           const double* __restrict__ tab64, Geo g, int force,
                                                           double* __restrict__ part) {
  using TB = Tab<K>;
  constexpr int N = TB::N, Q3 = TB::Q3;
  __shared__ double s[3][256];
  const long long nc = g.nc;
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long c = (long long)blockIdx.x * 256 + threadIdx.x; c < nc; c += (long long)gridDim.x * 256) {
    const double rho = y[c], E = y[(size_t)4 * N * nc + c];
    double m[3], mm = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      m[d] = y[(size_t)(1 + d) * N * nc + c];
      mm += m[d] * m[d];
    }
    const double pr = (g.gamma - 1.0) * (E - 0.5 * mm / rho);
    acc[0] += (mm / (rho * rho)) / (g.gamma * pr / rho);
    acc[1] += 0.5 * mm / rho;
    if (force) {
      double w[3][N];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int l = 0; l < N; ++l) w[d][l] = y[(size_t)((1 + d) * N + l) * nc + c];
      double pw = 0.0;
      for (int q = 0; q < Q3; ++q) {
        const double* ph = tab64 + TB::VPHIW + q * N;  // phi_l omega_q / 8
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          double md = 0.0;
#pragma unroll
          for (int l = 0; l < N; ++l) md += w[d][l] * __ldg(ph + l);
          pw += md * (double)field[((size_t)d * Q3 + q) * nc + c];
        }
      }
      acc[2] += pw;
    }
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) s[j][threadIdx.x] = acc[j];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int j = 0; j < 3; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) part[threadIdx.x * gridDim.x + blockIdx.x] = s[threadIdx.x][0];
}

template <int K, typename T>
__global__ void __launch_bounds__(kThreads) forcing_field_kernel(T* __restrict__ field, const double* __restrict__ modes,
                                                                 int n_modes, const double* __restrict__ tab64, Geo g,
                                                                 double L0, double L1, double L2) {
  using TB = Tab<K>;
  constexpr int Q = TB::Q, Q3 = TB::Q3;
  const long long nc = g.nc;
  const long long cell = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (cell >= nc) return;
  const int q = blockIdx.y;
  const int a = q % Q, b = (q / Q) % Q, cz = q / (Q * Q);
  int ix, iy, iz;
  cell_xyz(cell, g, ix, iy, iz);
  const double* gx = tab64 + TB::GX;
  const double x = (ix + 0.5) * g.dx[0] + 0.5 * g.dx[0] * gx[a];
  const double yy = (iy + 0.5) * g.dx[1] + 0.5 * g.dx[1] * gx[b];
  const double z = (iz + 0.5) * g.dx[2] + 0.5 * g.dx[2] * gx[cz];
  const double tp = 6.283185307179586476925286766559;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < n_modes; ++j) {
    const double* m = modes + 9 * j;
    const double ph = tp * (m[0] * x / L0 + m[1] * yy / L1 + m[2] * z / L2);
    double s, c;
    sincos(ph, &s, &c);
#pragma unroll
    for (int d = 0; d < 3; ++d) acc[d] += m[3 + d] * c - m[6 + d] * s;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) field[((size_t)d * Q3 + q) * nc + cell] = (T)acc[d];
}

}  // namespace dg
