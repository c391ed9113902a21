// dg_kernels.cuh -- CUDA kernels of the modal DG hot path (arXiv:1602.09079,
// Sect. 2.3-2.5, 3.1-3.2), templated on the polynomial degree K and the
// quadrature type T (double: plain FP64 path; float: mixed path whose RK
// accumulation, limiter and reductions stay FP64).
//
// State layout: y[(i*N + l) * nc + c], rows contiguous over cells (x-fastest),
// so every per-row access of a warp over consecutive cells is coalesced.
//
// One RHS evaluation = face_flux_kernel (one HLLC flux per face point, face
// owned by its upper cell, written once) + volume_kernel (volume quadrature,
// flux projection onto the basis gradients, the two face fluxes of each
// direction projected onto the face traces, and an epilogue: R, or the
// SSP-RK3 stage combination in FP64 followed by the positivity limiter of
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
// grid: x over cells, y = face point p in [0, Q^2), z = direction d.
// Face (d, c) joins the lower cell c - e_d (left state, its high face) and
// cell c (right state, its low face). fh[((d*5 + i)*Q2 + p)*nc + c].
template <int K, typename T>
__global__ void __launch_bounds__(kThreads) face_flux_kernel(const double* __restrict__ y, T* __restrict__ fh,
                                                             const T* __restrict__ tab, Geo g) {
  using TB = Tab<K>;
  constexpr int N = TB::N, Q2 = TB::Q2;
  const long long nc = g.nc;
  const long long c = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (c >= nc) return;
  const int p = blockIdx.y, d = blockIdx.z;
  int ix, iy, iz;
  cell_xyz(c, g, ix, iy, iz);
  const long long cl = neighbour(g, ix, iy, iz, d, -1);
  const T* phL = tab + TB::FPHI + ((d * 2 + 1) * Q2 + p) * N;
  const T* phR = tab + TB::FPHI + ((d * 2 + 0) * Q2 + p) * N;
  T UL[5], UR[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    T aL = T(0), aR = T(0);
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const size_t row = (size_t)(i * N + l) * nc;
      aL += (T)__ldg(y + row + cl) * __ldg(phL + l);
      aR += (T)__ldg(y + row + c) * __ldg(phR + l);
    }
    UL[i] = aL;
    UR[i] = aR;
  }
  T F[5];
  hllc_flux<T>(d, UL, UR, (T)g.gamma, F);
#pragma unroll
  for (int i = 0; i < 5; ++i) fh[((size_t)(d * 5 + i) * Q2 + p) * nc + c] = F[i];
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
  __shared__ unsigned s_err;

  const long long nc = g.nc;
  const long long c0 = (long long)blockIdx.x * C;
  const int tid = threadIdx.x;
  if (tid == 0) s_err = 0u;
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

  // phase 4: positivity limiter of the next stage's input (FP64)
  if (tid < C) {
    const long long cell = c0 + tid;
    if (cell < nc) {
      unsigned e = 0;
      limit_cell<K>(sY + tid, C, tab64, g.gamma, g.eps_rho, g.eps_p, &e);
      if (e) atomicOr(&s_err, e);
    }
  }
  __syncthreads();
  for (int it = tid; it < 5 * N * C; it += kThreads) {
    const int c = it % C, r = it / C;
    const long long cell = c0 + c;
    if (cell < nc) st.out[(size_t)r * nc + cell] = sY[r * C + c];
  }
  if (tid == 0 && s_err) atomicOr(&ctrl->err, s_err);
}

// ------------------------------------------------------ standalone limiter
template <int K>
__global__ void __launch_bounds__(kThreads) limit_kernel(double* __restrict__ y, int8_t* __restrict__ flags,
                                                         const double* __restrict__ tab64, Geo g, Ctrl* ctrl) {
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
    int f = limit_cell<K>(y + cell, g.nc, tab64, g.gamma, g.eps_rho, g.eps_p, &e);
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
// s_K = sum_a (|v_a| + c) / dx_a from the cell means; max over cells by a
// warp-shuffle / shared-memory / one-atomic-per-block reduction on the bit
// pattern of the non-negative double.
template <int K>
__global__ void __launch_bounds__(kThreads) cfl_kernel(const double* __restrict__ y, Geo g, Ctrl* ctrl) {
  constexpr int N = nmodes(K);
  const long long nc = g.nc;
  double smax = 0.0;
  unsigned e = 0;
  for (long long c = (long long)blockIdx.x * kThreads + threadIdx.x; c < nc; c += (long long)gridDim.x * kThreads) {
    const double r = y[c];
    const double m1 = y[(size_t)N * nc + c], m2 = y[(size_t)2 * N * nc + c], m3 = y[(size_t)3 * N * nc + c];
    const double E = y[(size_t)4 * N * nc + c];
    const double pr = (g.gamma - 1.0) * (E - 0.5 * (m1 * m1 + m2 * m2 + m3 * m3) / r);
    if (!(r > 0.0) || !(pr > 0.0)) {
      e |= (isfinite(r) && isfinite(pr)) ? ERRB_POSITIVITY : ERRB_NONFINITE;
      continue;
    }
    const double cs = sqrt(g.gamma * pr / r);
    const double s = (fabs(m1 / r) + cs) / g.dx[0] + (fabs(m2 / r) + cs) / g.dx[1] + (fabs(m3 / r) + cs) / g.dx[2];
    smax = fmax(smax, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  __shared__ double s_w[kThreads / 32];
  __shared__ unsigned s_err;
  if (threadIdx.x == 0) s_err = 0u;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = smax;
  if (e) atomicOr(&s_err, e);
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kThreads / 32 ? s_w[threadIdx.x] : 0.0;
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
// E_q = 1/2 |m_q|^2 / rho_q + rho_q eps_q, energy modes re-projected; then the
// limiter. part[blockIdx.x] receives the block's sum of (e_before - e_after).
template <int K, typename T, int C>
__global__ void __launch_bounds__(kThreads) energy_reset_kernel(double* __restrict__ y, const T* __restrict__ tab,
                                                                const double* __restrict__ tab64, Geo g, double c2g,
                                                                double inv_rho0, double* __restrict__ part,
                                                                Ctrl* ctrl) {
  using TB = Tab<K>;
  constexpr int N = TB::N, Q3 = TB::Q3;
  __shared__ T sW[4 * N * C];
  __shared__ T sE[Q3 * C];
  __shared__ double sY[5 * N * C];
  __shared__ double s_red[kThreads / 32];
  __shared__ unsigned s_err;
  const long long nc = g.nc;
  const long long c0 = (long long)blockIdx.x * C;
  const int tid = threadIdx.x;
  if (tid == 0) s_err = 0u;
  for (int it = tid; it < 5 * N * C; it += kThreads) {
    const int c = it % C, r = it / C;
    const long long cell = c0 + c;
    const double v = cell < nc ? y[(size_t)r * nc + cell] : (r == 0 ? 1.0 : 0.0);
    sY[r * C + c] = v;
    if (r < 4 * N) sW[r * C + c] = (T)v;
  }
  __syncthreads();
  const T gm1 = (T)(g.gamma - 1.0);
  const T tc2g = (T)c2g, tir0 = (T)inv_rho0;
  for (int it = tid; it < Q3 * C; it += kThreads) {
    const int c = it % C, q = it / C;
    const T* ph = tab + TB::VPHI + q * N;
    T U[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T a = T(0);
#pragma unroll
      for (int l = 0; l < N; ++l) a += sW[(i * N + l) * C + c] * __ldg(ph + l);
      U[i] = a;
    }
    const T eps = tc2g * pow(U[0] * tir0, gm1);
    sE[q * C + c] = T(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0] + U[0] * eps;
  }
  __syncthreads();
  double diss = 0.0;
  if (tid < C && c0 + tid < nc) {
    const int c = tid;
    const double before = sY[(4 * N) * C + c] - 0.5 * (sY[N * C + c] * sY[N * C + c] + sY[2 * N * C + c] * sY[2 * N * C + c] +
                                                      sY[3 * N * C + c] * sY[3 * N * C + c]) / sY[c];
    T acc[N];
#pragma unroll
    for (int l = 0; l < N; ++l) acc[l] = T(0);
    for (int q = 0; q < Q3; ++q) {
      const T e = sE[q * C + c];
      const T* pw = tab + TB::VPHIW + q * N;
#pragma unroll
      for (int l = 0; l < N; ++l) acc[l] += e * __ldg(pw + l);
    }
#pragma unroll
    for (int l = 0; l < N; ++l) sY[(4 * N + l) * C + c] = (double)acc[l];
    const double after = sY[(4 * N) * C + c] - 0.5 * (sY[N * C + c] * sY[N * C + c] + sY[2 * N * C + c] * sY[2 * N * C + c] +
                                                     sY[3 * N * C + c] * sY[3 * N * C + c]) / sY[c];
    diss = before - after;
    unsigned e = 0;
    limit_cell<K>(sY + c, C, tab64, g.gamma, g.eps_rho, g.eps_p, &e);
    if (e) atomicOr(&s_err, e);
  }
  // block sum of the dissipation (fixed order: deterministic)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) diss += __shfl_xor_sync(0xffffffffu, diss, o);
  if ((tid & 31) == 0) s_red[tid >> 5] = diss;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += s_red[w];
    part[blockIdx.x] = s;
    if (s_err) atomicOr(&ctrl->err, s_err);
  }
  for (int it = tid; it < 5 * N * C; it += kThreads) {
    const int c = it % C, r = it / C;
    const long long cell = c0 + c;
    if (cell < nc) y[(size_t)r * nc + cell] = sY[r * C + c];
  }
}

// ------------------------------------------------------------- projection
// w_l = 1/8 sum_q f(x_q) phi_l(xi_q) omega_q (Sect. 2.3), f canonical
// [nc][5][Q^3]. One thread per (cell, variable).
template <int K>
__global__ void __launch_bounds__(kThreads) project_kernel(const double* __restrict__ f, double* __restrict__ y,
                                                           const double* __restrict__ tab64, Geo g) {
  using TB = Tab<K>;
  constexpr int N = TB::N, Q3 = TB::Q3;
  const long long nc = g.nc;
  const long long it = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (it >= 5 * nc) return;
  const long long cell = it % nc;
  const int i = (int)(it / nc);
  double acc[N];
#pragma unroll
  for (int l = 0; l < N; ++l) acc[l] = 0.0;
  for (int q = 0; q < Q3; ++q) {
    const double v = f[((size_t)cell * 5 + i) * Q3 + q];
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
