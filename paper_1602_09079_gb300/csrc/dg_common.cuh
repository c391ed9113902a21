// dg_common.cuh -- shared device definitions of the GB300 modal DG solver
// (arXiv:1602.09079, Sect. 2): table layout, ideal-gas physics, HLLC flux,
// positivity limiter, launch geometry.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dg {

// ------------------------------------------------------------- sizes
__host__ __device__ constexpr int nmodes(int k) { return (k + 1) * (k + 2) * (k + 3) / 6; }
__host__ __device__ constexpr int gll_m(int k) { return k <= 1 ? 2 : 3; }
// index of the tangential pair (a, b), a + b <= k, in the order a
// ascending, b ascending
__host__ __device__ constexpr int pair_index(int k, int a, int b) {
  int j = 0;
  for (int ap = 0; ap < a; ++ap) j += k - ap + 1;
  return j + b;
}
// index of mode (u, v, w) in the exchange order (total degree ascending,
// then u descending, then v descending)
__host__ __device__ constexpr int mode_index(int u, int v, int w) {
  const int D = u + v + w;
  int idx = D > 0 ? nmodes(D - 1) : 0;
  for (int up = D; up > u; --up) idx += D - up + 1;
  return idx + (D - u - v);
}

// (u, v, w) of mode l in the canonical order (degree ascending, u then v
// descending).
__device__ __forceinline__ void mode_uvw(int l, int& u, int& v, int& w) {
  int D = 0;
  while (l >= nmodes(D)) ++D;
  int r = l - (D > 0 ? nmodes(D - 1) : 0);
  u = D;
  while (r > D - u) {
    r -= D - u + 1;
    --u;
  }
  v = D - u - r;
  w = D - u - v;
}

// Per-degree basis/quadrature tables (Sect. 2.2-2.5), all values at the
// method's point sets, offsets in elements. Weights are folded in so the
// kernels only multiply and add.
template <int K>
struct Tab {
  static constexpr int Q = K + 1;
  static constexpr int Q2 = Q * Q;
  static constexpr int Q3 = Q * Q * Q;
  static constexpr int N = nmodes(K);
  static constexpr int M = gll_m(K);
  static constexpr int NL = 3 * M * Q2;  // positivity point set S
  // phi_l(xi_q) at volume Gauss points, [Q3][N]
  static constexpr int VPHI = 0;
  // dphi_l/dxi_a (xi_q) * omega_q / 4, [3][Q3][N]
  static constexpr int VDPHI = VPHI + Q3 * N;
  // phi_l(xi_q) * omega_q / 8, [Q3][N]
  static constexpr int VPHIW = VDPHI + 3 * Q3 * N;
  // phi_l at face points of face (a, s), s = 0 low (xi_a = -1) / 1 high, [3][2][Q2][N]
  static constexpr int FPHI = VPHIW + Q3 * N;
  // same times omega_2D / 4, [3][2][Q2][N]
  static constexpr int FPHIW = FPHI + 6 * Q2 * N;
  // phi_l at the limiter points, [NL][N]
  static constexpr int LPHI = FPHIW + 6 * Q2 * N;
  // max over S of |phi_l|, [N]
  static constexpr int LMAX = LPHI + NL * N;
  // tangential products Pt_a(x_t1) Pt_b(x_t2) at the face points, pairs
  // (a, b) with a + b <= K in the order a ascending, b ascending, [Q2][T]
  static constexpr int T = (K + 1) * (K + 2) / 2;
  static constexpr int F2D = LMAX + N;
  // Pt_e(-1) and Pt_e(+1), [2][K+1]
  static constexpr int FEND = F2D + Q2 * T;
  // 1D tables at the Gauss points for sum factorisation, [K+1][Q] each:
  // Pt_u(x_a), Pt_u(x_a) w_a, Pt_u'(x_a) w_a
  static constexpr int P1 = FEND + 2 * (K + 1);
  static constexpr int P1W = P1 + (K + 1) * Q;
  static constexpr int D1W = P1W + (K + 1) * Q;
  // 1D Gauss nodes and weights, [Q] each
  static constexpr int GX = D1W + (K + 1) * Q;
  static constexpr int GW = GX + Q;
  // max over S and the volume Gauss points of |phi_l|, [N]
  static constexpr int LMAXV = GW + Q;
  static constexpr int SIZE = LMAXV + N;
};
constexpr int TAB_STRIDE = 16384;  // >= Tab<3>::SIZE
static_assert(Tab<3>::SIZE <= TAB_STRIDE, "table stride");

// ------------------------------------------------------------ error word
enum : unsigned {
  ERRB_NONFINITE = 1u,
  ERRB_POSITIVITY = 2u,
  ERRB_NEWTON = 4u,
};

// Control block at the start of the scratch buffer.
struct Ctrl {
  unsigned long long cfl_max_bits;  // max over cells of the wave-speed sum (bits of a double >= 0)
  unsigned int err;                 // sticky ERRB_* bits
  unsigned int n_flag;              // cells queued for the full limiter
  unsigned long long n_limited;     // limiter count
  unsigned int n_gate;              // queued cells the indicator passes on
  unsigned int n_deep;              // queued cells the FP32 point screen does not clear
  unsigned long long n_queued_total;  // cells that failed the limiter screen (all stages)
  unsigned long long n_full_total;    // cells that went through the full limiter
  double pad1[2];
};

struct Geo {
  int nx, ny, nz;
  long long nc;  // cells
  double dx[3];
  double inv_dx[3];
  double gamma;
  double eps_rho, eps_p;
  int lim_vol;  // limiter point set: 0 = S, 1 = S and the volume Gauss points
};

// --------------------------------------------------------------- physics
template <typename T>
__device__ __forceinline__ T pressure_of(const T* U, T gm1) {
  T ke = T(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0];
  return gm1 * (U[4] - ke);
}

// Euler flux along direction d from conserved U, given velocity and pressure.
template <typename T>
__device__ __forceinline__ void euler_flux(int d, const T* U, const T* v, T p, T* F) {
  T mn = U[1 + d];
  F[0] = mn;
  F[1] = mn * v[0];
  F[2] = mn * v[1];
  F[3] = mn * v[2];
  F[1 + d] += p;
  F[4] = (U[4] + p) * v[d];
}

// HLLC numerical flux across a face with normal +e_d, left = lower cell
// (Sect. 2.3, the approximate HLLC Riemann solver): Einfeldt wave-speed
// estimates from Roe averages, middle wave and star states from the
// Rankine-Hugoniot conditions across the three waves (Toro's formulation).
// ------------------------------------------- IEEE 754 conversions
// binary32 <-> binary64 from the format definitions (sign, biased exponent,
// fraction) on the integer pipe, for the FP32 path's FP64 stage epilogue:
// GB300 issues the hardware conversions on its FP64 unit, which the FP32
// volume kernel otherwise keeps 45 % busy. Exact for every input: values
// outside the fast range (zeros, subnormals, infinities, NaNs) take the
// hardware conversion. dg_selftest_conversions compares both with the
// hardware.

// binary32 -> binary64: exponent rebias 127 -> 1023, fraction widened
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)x;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// binary64 -> binary32, round to nearest, ties to even: results in the
// binary32 normal range (biased exponents 897..1150) and magnitudes below
// 2^-150 (round to a signed zero) on the integer pipe
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u <= 253u) {
    unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;  // the 29 dropped fraction bits
    f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
  }
  if (e < 873u) return __uint_as_float(hi & 0x80000000u);
  return (float)x;
}

// finite test on the exponent field (integer pipe)
__device__ __forceinline__ bool finite64(double x) {
  return (((unsigned)__double2hiint(x) >> 20) & 0x7ffu) != 0x7ffu;
}

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ void hllc_flux(int d, const T* UL, const T* UR, T gamma, T* F) {
  const T gm1 = gamma - T(1);
  // one reciprocal square root per side gives 1/rho and sqrt(rho)
  const T rL = rsq(UL[0]), rR = rsq(UR[0]);
  const T irL = rL * rL, irR = rR * rR;
  T vL[3] = {UL[1] * irL, UL[2] * irL, UL[3] * irL};
  T vR[3] = {UR[1] * irR, UR[2] * irR, UR[3] * irR};
  T pL = gm1 * (UL[4] - T(0.5) * UL[0] * (vL[0] * vL[0] + vL[1] * vL[1] + vL[2] * vL[2]));
  T pR = gm1 * (UR[4] - T(0.5) * UR[0] * (vR[0] * vR[0] + vR[1] * vR[1] + vR[2] * vR[2]));
  // a face pressure at the positivity floor can round to <= 0 (FP32 traces
  // of an FP64-limited state; FP64 near vacuum when gamma - 1 is small): the
  // sound speed is then 0, the limit p -> 0+
  const T cL = sqrt(fmax(gamma * pL * irL, T(0)));
  const T cR = sqrt(fmax(gamma * pR * irR, T(0)));
  const T sL = UL[0] * rL, sR = UR[0] * rR;
  T iss = T(1) / (sL + sR);
  T vt[3], v2 = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    vt[a] = (sL * vL[a] + sR * vR[a]) * iss;
    v2 += vt[a] * vt[a];
  }
  T Ht = (rL * (UL[4] + pL) + rR * (UR[4] + pR)) * iss;
  T c2t = gm1 * (Ht - T(0.5) * v2);
  T ct = c2t > T(0) ? sqrt(c2t) : T(0);
  T uL = vL[d], uR = vR[d];
  T SL = fmin(uL - cL, vt[d] - ct);
  T SR = fmax(uR + cR, vt[d] + ct);
  if (SL >= T(0)) {
    euler_flux(d, UL, vL, pL, F);
    return;
  }
  if (SR <= T(0)) {
    euler_flux(d, UR, vR, pR, F);
    return;
  }
  T aL = UL[0] * (SL - uL), aR = UR[0] * (SR - uR);
  T Ss = (pR - pL + uL * aL - uR * aR) / (aL - aR);
  // both sound speeds 0 in a receding flow: S_L = u_L and S_R = u_R, so
  // aL = aR = 0. Take S* = 0; the flux is then (0, p e_d, 0), the flux at a
  // vacuum interface.
  if (aL - aR == T(0)) Ss = T(0);
  // the side of the contact, selected by value (no pointer into either
  // side's arrays, which would put them in local memory)
  const bool left = Ss >= T(0);
  T U[5], v[3];
#pragma unroll
  for (int i = 0; i < 5; ++i) U[i] = left ? UL[i] : UR[i];
#pragma unroll
  for (int a = 0; a < 3; ++a) v[a] = left ? vL[a] : vR[a];
  T p = left ? pL : pR;
  T S = left ? SL : SR;
  T ak = left ? aL : aR;  // rho_K (S_K - u_K)
  T ir = left ? irL : irR;
  T uk = left ? uL : uR;
  euler_flux(d, U, v, p, F);
  // star state: chi = rho_K (S_K - u_K) / (S_K - S*), and
  // E* = chi (E_K / rho_K + (S* - u_K) (S* + p_K / (rho_K (S_K - u_K))))
  const T isd = T(1) / (S - Ss);
  T chi = ak * isd;
  T Us[5];
  Us[0] = chi;
  Us[1] = chi * v[0];
  Us[2] = chi * v[1];
  Us[3] = chi * v[2];
  Us[1 + d] = chi * Ss;
  Us[4] = chi * (U[4] * ir + (Ss - uk) * Ss) + (Ss - uk) * p * isd;
#pragma unroll
  for (int i = 0; i < 5; ++i) F[i] += S * (Us[i] - U[i]);
}

// ------------------------------------------------- exact Riemann solver
// Godunov flux from the exact solution of the Riemann problem (the exact
// option of Sect. 2.3 next to HLLC): the star pressure p* is the root of
// f_L(p) + f_R(p) + u_R - u_L, where f_K is the velocity jump across the
// wave of side K (shock branch from the Rankine-Hugoniot conditions for
// p > p_K, rarefaction branch from the Riemann invariant for p <= p_K);
// Newton's method from the adaptive starting value (linearised estimate for
// close pressures, else the two-rarefaction or two-shock estimate), at most
// kExactIters steps; the face state is the self-similar solution at x/t = 0.
// Returns ERRB_NEWTON if the iteration did not converge (FP64) or produced a
// non-finite pressure.
constexpr int kExactIters = 50;

template <typename T>
struct ExactSide {
  T rho, u, p, c;
  T A, B;   // shock branch: sqrt(A / (p + B)) (p - p_K)
  T crf;    // rarefaction branch: 2 c_K / (gamma - 1)
  __device__ __forceinline__ void init(T r, T un, T pr, T gamma) {
    // FP32 traces of a state limited in FP64 can round a pressure at the
    // floor to zero or below: clamp it to a tiny positive value
    if constexpr (sizeof(T) == 4) pr = fmaxf(pr, 1e-30f);
    rho = r;
    u = un;
    p = pr;
    c = sqrt(gamma * pr / r);
    A = T(2) / ((gamma + T(1)) * r);
    B = (gamma - T(1)) / (gamma + T(1)) * pr;
    crf = T(2) * c / (gamma - T(1));
  }
  // f_K(ps) and its derivative; z = (gamma - 1) / (2 gamma)
  __device__ __forceinline__ void jump(T ps, T z, T gamma, T& f, T& df) const {
    if (ps > p) {
      const T q = sqrt(A / (ps + B));
      f = (ps - p) * q;
      df = q * (T(1) - T(0.5) * (ps - p) / (ps + B));
    } else {
      const T r = pow(ps / p, z);
      f = crf * (r - T(1));
      df = c * r / (gamma * ps);
    }
  }
};

// state (rho, u, p) inside the rarefaction fan of side K at x/t = 0;
// sgn = +1 for the left fan, -1 for the right one
template <typename T>
__device__ __forceinline__ void fan_at_origin(const ExactSide<T>& k, T sgn, T gamma, T* W) {
  // positive inside the fan; the clamp only absorbs rounding at its edge
  const T cf = fmax(T(2) / (gamma + T(1)) * (k.c + sgn * T(0.5) * (gamma - T(1)) * k.u), T(0));
  const T ratio = cf / k.c;
  W[0] = k.rho * pow(ratio, T(2) / (gamma - T(1)));
  W[1] = sgn * cf;
  W[2] = k.p * pow(ratio, T(2) * gamma / (gamma - T(1)));
}

template <typename T>
__device__ __forceinline__ unsigned exact_flux(int d, const T* UL, const T* UR, T gamma, T* F) {
  const T gm1 = gamma - T(1);
  const T irL = T(1) / UL[0], irR = T(1) / UR[0];
  const T vL[3] = {UL[1] * irL, UL[2] * irL, UL[3] * irL};
  const T vR[3] = {UR[1] * irR, UR[2] * irR, UR[3] * irR};
  ExactSide<T> L, R;
  L.init(UL[0], vL[d], gm1 * (UL[4] - T(0.5) * UL[0] * (vL[0] * vL[0] + vL[1] * vL[1] + vL[2] * vL[2])), gamma);
  R.init(UR[0], vR[d], gm1 * (UR[4] - T(0.5) * UR[0] * (vR[0] * vR[0] + vR[1] * vR[1] + vR[2] * vR[2])), gamma);
  const T du = R.u - L.u;
  const T z = gm1 / (T(2) * gamma);
  T W[3];
  bool left;  // face state on the left of the contact (tangential velocities of L)
  unsigned err = 0;
  if (L.crf + R.crf <= du) {
    // the rarefactions open a vacuum between their tails
    const T tL = L.u + L.crf, tR = R.u - R.crf;
    if (L.u - L.c >= T(0)) {
      W[0] = L.rho; W[1] = L.u; W[2] = L.p; left = true;
    } else if (tL > T(0)) {
      fan_at_origin(L, T(1), gamma, W); left = true;
    } else if (R.u + R.c <= T(0)) {
      W[0] = R.rho; W[1] = R.u; W[2] = R.p; left = false;
    } else if (tR < T(0)) {
      fan_at_origin(R, T(-1), gamma, W); left = false;
    } else {
      W[0] = T(0); W[1] = T(0); W[2] = T(0); left = true;
    }
  } else {
    const T pmin = fmin(L.p, R.p), pmax = fmax(L.p, R.p);
    T ps = T(0.5) * (L.p + R.p) - T(0.125) * du * (L.rho + R.rho) * (L.c + R.c);
    ps = fmax(ps, T(0));
    if (!(pmax <= T(2) * pmin && ps >= pmin && ps <= pmax)) {
      if (ps < pmin) {
        const T num = L.c + R.c - T(0.5) * gm1 * du;
        ps = pow(num / (L.c * pow(L.p, -z) + R.c * pow(R.p, -z)), T(1) / z);
      } else {
        const T gL = sqrt(L.A / (ps + L.B)), gR = sqrt(R.A / (ps + R.B));
        ps = (gL * L.p + gR * R.p - du) / (gL + gR);
      }
    }
    const T tiny = sizeof(T) == 8 ? T(1e-14) * pmin : fmax(T(1e-14) * pmin, T(1e-36));
    const T tol = sizeof(T) == 8 ? T(1e-14) : T(2e-6);
    ps = fmax(ps, tiny);
    bool conv = false;
    const T rtol = sizeof(T) == 8 ? T(1e-15) : T(1e-6);
    for (int it = 0; it < kExactIters && !conv; ++it) {
      T fl, dfl, fr, dfr;
      L.jump(ps, z, gamma, fl, dfl);
      R.jump(ps, z, gamma, fr, dfr);
      const T f = fl + fr + du;
      // residual at the rounding level of its terms (near a vacuum the root
      // is too ill-conditioned for the relative step to reach tol)
      if (fabs(f) <= rtol * (fabs(fl) + fabs(fr) + fabs(du))) {
        conv = true;
        break;
      }
      const T pn = fmax(ps - f / (dfl + dfr), tiny);
      conv = fabs(pn - ps) <= tol * pn;
      ps = pn;
    }
    if (!isfinite(ps) || (sizeof(T) == 8 && !conv)) err = ERRB_NEWTON;
    T fl, dfl, fr, dfr;
    L.jump(ps, z, gamma, fl, dfl);
    R.jump(ps, z, gamma, fr, dfr);
    const T us = T(0.5) * (L.u + R.u) + T(0.5) * (fr - fl);
    left = us >= T(0);
    const ExactSide<T>& K = left ? L : R;
    const T sg = left ? T(1) : T(-1);  // +1: wave moves left of the contact
    const T ratio = ps / K.p;
    if (ps > K.p) {
      // shock speed from the jump conditions
      const T S = K.u - sg * K.c * sqrt((gamma + T(1)) / (T(2) * gamma) * ratio + z);
      if (sg * S >= T(0)) {
        W[0] = K.rho; W[1] = K.u; W[2] = K.p;
      } else {
        const T g6 = gm1 / (gamma + T(1));
        W[0] = K.rho * (ratio + g6) / (g6 * ratio + T(1)); W[1] = us; W[2] = ps;
      }
    } else {
      const T head = K.u - sg * K.c, tail = us - sg * K.c * pow(ratio, z);
      if (sg * head >= T(0)) {
        W[0] = K.rho; W[1] = K.u; W[2] = K.p;
      } else if (sg * tail < T(0)) {
        W[0] = K.rho * pow(ratio, T(1) / gamma); W[1] = us; W[2] = ps;
      } else {
        fan_at_origin(K, sg, gamma, W);
      }
    }
  }
  const T* vt = left ? vL : vR;
  T v[3] = {vt[0], vt[1], vt[2]};
  v[d] = W[1];
  const T mn = W[0] * W[1];
  F[0] = mn;
#pragma unroll
  for (int a = 0; a < 3; ++a) F[1 + a] = mn * v[a];
  F[1 + d] += W[2];
  F[4] = (W[2] / gm1 + T(0.5) * W[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) + W[2]) * W[1];
  return err;
}

// numerical flux selected at compile time: 0 = HLLC, 1 = exact Riemann solver
template <int FLUX, typename T>
__device__ __forceinline__ unsigned riemann_flux(int d, const T* UL, const T* UR, T gamma, T* F) {
  if constexpr (FLUX == 1) {
    return exact_flux<T>(d, UL, UR, gamma, F);
  } else {
    hllc_flux<T>(d, UL, UR, gamma, F);
    return 0u;
  }
}

// --------------------------------------------------------------- limiter
// tau in [0,1] with P(qbar + tau (q - qbar)) = eps: Newton from tau = 1.
// The pressure is concave along the segment, so the iterates decrease
// monotonically; stop when a step is below 1e-15 (50 iterations at most).
__device__ __forceinline__ double positivity_tau(const double* qb, const double* q, double gm1,
                                                 double eps, int* iters) {
  double d[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) d[i] = q[i] - qb[i];
  double tau = 1.0;
  int it = 0;
  while (it < 50) {
    double s0 = qb[0] + tau * d[0];
    double s1 = qb[1] + tau * d[1];
    double s2 = qb[2] + tau * d[2];
    double s3 = qb[3] + tau * d[3];
    double s4 = qb[4] + tau * d[4];
    double m2 = s1 * s1 + s2 * s2 + s3 * s3;
    double ir = 1.0 / s0;
    double f = gm1 * (s4 - 0.5 * m2 * ir) - eps;
    double md = s1 * d[1] + s2 * d[2] + s3 * d[3];
    double fp = gm1 * (d[4] - md * ir + 0.5 * m2 * d[0] * ir * ir);
    double tn = tau - f / fp;
    if (!(tn >= 0.0)) tn = 0.0;
    if (tn > tau) tn = tau;
    double step = tau - tn;
    tau = tn;
    ++it;
    if (step <= 1e-15) break;
  }
  *iters = it;
  return tau;
}

// Second sufficient test of the positivity limiter, for cells whose modal
// bound fails: density and pressure at every point of the limiter's point
// set (S, and the volume Gauss points when vol), evaluated in FP32 from the
// coefficients rounded to FP32 (tab32: the FP32 copy of the degree's table).
// A point value u = sum_l w_l phi_l computed so carries an error of at most
// (N + 3) 2^-24 sum_l |w_l phi_l| <= 2e-6 (|w_0| + sabs_u) for N <= 20
// (rounding of the coefficients, of the table entries and of the N products
// and sums), so e_u = 2e-6 (|mean_u| + sabs_u) bounds it; with these bounds
// the density and the pressure (bounded below through the density's lower
// and the momenta's upper bounds, multiplied through by the density bound)
// must clear the floors with a further 1e-5 relative margin, which covers
// the FP32 rounding of the test itself. True when the cell provably needs
// no limiting (theta1 = theta2 = 1): the FP64 limiter would leave it as it is.
template <int K>
__device__ bool point_screen_f32(const double* w, long long stride, const float* __restrict__ tab32,
                                 const double* mean, const double* sabs, double gamma, double eps_r, double eps_p,
                                 int vol) {
  using TB = Tab<K>;
  constexpr int N = TB::N;
  float wf[5 * N];
#pragma unroll
  for (int j = 0; j < 5 * N; ++j) wf[j] = f64_to_f32(w[j * stride]);
  float e[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) e[i] = f64_to_f32(2e-6 * (fabs(mean[i]) + sabs[i]));
  const float thr_r = f64_to_f32(eps_r * (1.0 + 1e-6) + 1e-5 * (fabs(mean[0]) + sabs[0]));
  const float eps_pf = f64_to_f32(eps_p * (1.0 + 1e-6));
  const float gm1 = f64_to_f32(gamma - 1.0);
  const int npts = TB::NL + (vol ? TB::Q3 : 0);
  for (int s = 0; s < npts; ++s) {
    const float* ph = s < TB::NL ? tab32 + TB::LPHI + s * N : tab32 + TB::VPHI + (s - TB::NL) * N;
    float U[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      float a = 0.f;
#pragma unroll
      for (int l = 0; l < N; ++l) a = fmaf(wf[i * N + l], __ldg(ph + l), a);
      U[i] = a;
    }
    const float rlo = U[0] - e[0];
    if (!(rlo >= thr_r)) return false;
    float k2 = 0.f;
#pragma unroll
    for (int a = 1; a <= 3; ++a) {
      const float mh = fabsf(U[a]) + e[a];
      k2 = fmaf(mh, mh, k2);
    }
    k2 *= 0.5f;
    const float elo = U[4] - e[4];
    const float lhs = gm1 * fmaf(elo, rlo, -k2);
    const float rhs = fmaf(eps_pf, rlo, 1e-5f * gm1 * fmaf(fabsf(U[4]) + e[4], rlo, k2));
    if (!(lhs >= rhs)) return false;
  }
  return true;
}

// The cheap part of the Zhang-Shu limiter of one cell (Sect. 2.5) on its 5N
// FP64 coefficients w[(i*N + l) * stride]: the means (finite, positive:
// otherwise an error bit is ORed into err and false returned), the
// excursion bounds sabs_i = sum_{l>=1} |w_il| max |phi_l| and the modal
// sufficient tests (mean minus sabs with a rounding margin) for the density
// (rho_safe) and the pressure (p_safe; needs rho_safe). When both hold, or
// (tab32 != nullptr) the FP32 point screen (point_screen_f32) holds, the
// limiter provably leaves the cell unchanged and *none is set.
template <int K>
__device__ bool limit_prelude(const double* w, long long stride, const double* __restrict__ tab, double gamma,
                              double eps_r, double eps_p, unsigned* err, int vol, const float* __restrict__ tab32,
                              double* mean, double* sabs, bool* rho_safe, bool* p_safe, bool* none) {
  using TB = Tab<K>;
  constexpr int N = TB::N;
  const double gm1 = gamma - 1.0;
  bool finite = true;
#pragma unroll
  for (int i = 0; i < 5; ++i) mean[i] = w[(i * N) * stride];
  for (int j = 0; j < 5 * N; ++j) finite &= isfinite(w[j * stride]);
  if (!finite) {
    *err |= ERRB_NONFINITE;
    return false;
  }
  const double pbar = gm1 * (mean[4] - 0.5 * (mean[1] * mean[1] + mean[2] * mean[2] + mean[3] * mean[3]) / mean[0]);
  if (!(mean[0] >= eps_r) || !(pbar >= eps_p)) {
    *err |= ERRB_POSITIVITY;
    return false;
  }
  if (N == 1) return false;
  const double* lmax = tab + (vol ? TB::LMAXV : TB::LMAX);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    double s = 0.0;
    for (int l = 1; l < N; ++l) s += fabs(w[(i * N + l) * stride]) * __ldg(lmax + l);
    sabs[i] = s;
  }
  const double rlo = mean[0] - sabs[0];
  *rho_safe = rlo >= eps_r + 1e-13 * (fabs(mean[0]) + sabs[0]);
  *p_safe = false;
  if (*rho_safe) {
    const double elo = mean[4] - sabs[4];
    double kin = 0.0;
#pragma unroll
    for (int a = 1; a <= 3; ++a) {
      const double mh = fabs(mean[a]) + sabs[a];
      kin += mh * mh;
    }
    kin *= 0.5 / rlo;
    *p_safe = gm1 * (elo - kin) >= eps_p + 1e-13 * gm1 * (fabs(mean[4]) + sabs[4] + kin);
  }
  *none = (*rho_safe && *p_safe) ||
          (tab32 && point_screen_f32<K>(w, stride, tab32, mean, sabs, gamma, eps_r, eps_p, vol));
  return true;
}

// Zhang-Shu positivity limiter of one cell (Sect. 2.5) on its 5N FP64
// coefficients w[(i*N + l) * stride]: limit_prelude's sufficient tests skip
// the FP64 point evaluations when the limiter provably leaves the cell as it
// is. Returns flag bits (1: theta1 < 1, 2: theta2 < 1) and ORs errors into
// err.
template <int K>
__device__ int limit_cell(double* w, long long stride, const double* __restrict__ tab, double gamma,
                          double eps_r, double eps_p, unsigned* err, int vol,
                          const float* __restrict__ tab32 = nullptr) {
  using TB = Tab<K>;
  constexpr int N = TB::N;
  const double gm1 = gamma - 1.0;
  double mean[5], sabs[5];
  bool rho_safe, p_safe, none;
  if (!limit_prelude<K>(w, stride, tab, gamma, eps_r, eps_p, err, vol, tab32, mean, sabs, &rho_safe, &p_safe,
                        &none) ||
      none)
    return 0;
  const double* lphi = tab + TB::LPHI;
  const double* vphi = tab + TB::VPHI;
  // the point set: S (TB::NL points), then optionally the volume Gauss points
  const int npts = TB::NL + (vol ? TB::Q3 : 0);
  int flag = 0;
  // density: theta1
  if (!rho_safe) {
    double rmin = mean[0];
    for (int s = 0; s < npts; ++s) {
      const double* ph = s < TB::NL ? lphi + s * N : vphi + (s - TB::NL) * N;
      double r = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) r += w[l * stride] * __ldg(ph + l);
      rmin = fmin(rmin, r);
    }
    if (rmin < eps_r) {
      double th1 = fmin(fabs((mean[0] - eps_r) / (mean[0] - rmin)), 1.0);
      if (th1 < 1.0) {
        for (int l = 1; l < N; ++l) w[l * stride] *= th1;
        flag |= 1;
      }
    }
  }
  // pressure: theta2 (the prelude's modal test p_safe holds only where
  // rho_safe did, i.e. where theta1 left the cell unchanged)
  if (!p_safe) {
    double th2 = 1.0;
    bool newton_fail = false;
    for (int s = 0; s < npts; ++s) {
      const double* ph = s < TB::NL ? lphi + s * N : vphi + (s - TB::NL) * N;
      double U[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int l = 0; l < N; ++l) acc += w[(i * N + l) * stride] * __ldg(ph + l);
        U[i] = acc;
      }
      double p = gm1 * (U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0]);
      if (p < eps_p) {
        int it;
        double tau = positivity_tau(mean, U, gm1, eps_p, &it);
        if (it >= 50) newton_fail = true;
        th2 = fmin(th2, tau);
      }
    }
    if (newton_fail) *err |= ERRB_NEWTON;
    if (th2 < 1.0) {
      for (int i = 0; i < 5; ++i)
        for (int l = 1; l < N; ++l) w[(i * N + l) * stride] *= th2;
      flag |= 2;
    }
  }
  return flag;
}

}  // namespace dg
