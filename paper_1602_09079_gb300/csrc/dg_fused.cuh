// dg_fused.cuh -- one kernel per SSP-RK3 stage of the FP32-mixed path
// (arXiv:1602.09079, Sect. 2.3-2.5): face traces, the numerical flux of every
// face, the surface and volume integrals and the FP64 stage update of a
// column of cells, with no face-flux buffer in global memory.
//
// Tile: a column of BX x BY cells that marches along z through a segment of
// lz planes, one thread per (cell, variable). Per plane:
//  P1  every thread loads its N coefficients (FP64 state, converted to FP32
//      on the integer pipe) and writes the traces of its faces to shared
//      memory in each face's frame; a ring of neighbour cells around the
//      column supplies the traces of the column's outer x and y faces;
//  P2  one numerical flux per face point (x, y faces of the plane, and the
//      z face between the previous plane and this one): the branch-free FP32
//      HLLC of the face frame;
//  P3  the z face between the previous plane and this one completes the
//      previous plane's cells, then
//  P4  finishes them: R, or the stage update y_{s+1} = y_s + delta with
//      delta = b0 dt dw/dt - a0 d (FP32) added in FP64, d = y_s - y_0 the
//      FP32 increment of the step so far (the mean density in the FP64
//      Shu-Osher form from FP64 face sums); each thread's accumulators then
//      restart with this plane's low z face and its x and y faces (every
//      face's flux is projected onto both cells that share it);
//  P5  the limiter screen of those cells (sufficient test in FP32 with a
//      1e-5 relative margin; failing cells are queued for the full FP64
//      limiter);
//  P6  volume integral of this plane in Q slices of constant z: values at
//      the slice's Gauss points, Euler fluxes and the driving source, and
//      their projection onto the basis and its gradients, all sum-factorised.
// Faces on the column's outer sides and at the ends of a z segment are
// computed by both tiles that touch them, from the same inputs by the same
// explicitly rounded operations, so both sides receive bit-identical fluxes.
#pragma once
#include "dg_common.cuh"
#include "dg_launch.h"

namespace dg {

template <int K>
struct FusedCfg {
  static constexpr int Q = K + 1, Q2 = Q * Q, Q3 = Q2 * Q, N = nmodes(K), T = (K + 1) * (K + 2) / 2;
  // plane tile: 8 x 8 cells at degree <= 2; 8 x 4 at degree 3, whose
  // Q^2 = 16 face points per face double the trace storage
  static constexpr int BX = 8, BY = K >= 3 ? 4 : 8, NC = BX * BY;
  static constexpr int THREADS = 5 * NC;  // one (cell, variable) per thread
  // face slots: the low face of every cell of the plane, then the high face
  // of the last cell of every row (x) / column (y); z faces use the first NC
  static constexpr int SX = NC + BY, SY = NC + BX;
  // every direction's traces are laid out with the same slot stride SZ, so
  // that a face point's offset is one index and the variables' offsets are
  // compile-time constants
  static constexpr int SZ = SX > SY ? SX : SY;
  // shared memory, in floats: traces [5][Q2][SZ] left (L) and right (R) of
  // every face; the flux overwrites the right trace
  static constexpr int XL = 0, XR = XL + 5 * Q2 * SZ, YL = XR + 5 * Q2 * SZ, YR = YL + 5 * Q2 * SZ,
                       ZR = YR + 5 * Q2 * SZ, FACE_END = ZR + 5 * Q2 * SZ;
  // volume slice (aliases the face traces, which are dead by then): values
  // [5][Q2][NC], fluxes [3*5][Q2][NC], source [4][Q2][NC]
  static constexpr int VU = 0, VF = VU + 5 * Q2 * NC, VS = VF + 15 * Q2 * NC, VOL_END = VS + 4 * Q2 * NC;
  // high-z traces of the previous plane
  static constexpr int ZL = FACE_END > VOL_END ? FACE_END : VOL_END;
  static constexpr int TOTAL = ZL + 5 * Q2 * SZ;
  // the screen's inputs (means and excursion bounds, [5][NC] each) live in
  // the left y traces, which are dead between the numerical fluxes and the
  // next plane's traces
  static constexpr int SMN = YL, SAB = YL + 5 * NC;
  static_assert(10 * NC <= 5 * Q2 * SZ, "screen buffers fit the left y traces");
  static constexpr size_t smem() { return sizeof(float) * (size_t)TOTAL; }
  static constexpr int MINB = K >= 3 ? 3 : 2;  // CTAs per SM the register budget is sized for
  static constexpr int NFACE = (SX + SY + NC) * Q2;
  // degree 3: the volume slices and the face points stay loops (unrolled,
  // the kernel outgrows the instruction cache: ncu showed instruction-fetch
  // stalls as the largest stall reason; at odd degrees no exact table zero
  // depends on the slice, so nothing is lost to the rolled loop)
  static constexpr int SLICE_UNROLL = K >= 3 ? 1 : Q;
  static constexpr int FACE_UNROLL = K >= 3 ? 1 : 2;
  // degree 2: the plane's driving field is prefetched to L1 before the
  // volume slices (3 Q^3 values per cell; at degree 3 the three CTAs per SM
  // leave too little L1 beside their shared memory)
  static constexpr bool FIELD_L1 = K <= 2;
};

// 1D tables of this translation unit's degree in the constant bank:
// Pt_u(x_a) at P + u*Q + a, Pt_u(x_a) w_a at PW + ..., Pt_u'(x_a) w_a at
// DW + ..., Pt_e(-1) at EM + e, Pt_e(+1) at EP + e, max_S |phi_l| at LM + l
// and the maximum over S and the volume Gauss points at LMV + l.
template <int K>
struct FzTab {
  static constexpr int Q = K + 1, KQ = (K + 1) * Q, N = nmodes(K);
  static constexpr int P = 0, PW = KQ, DW = 2 * KQ, EM = 3 * KQ, EP = EM + K + 1, LM = EP + K + 1, LMV = LM + N,
                       SIZE = LMV + N;
};
namespace {
__constant__ float c_fz[FzTab<3>::SIZE];
}

// Exact zeros of the 1D tables: a Gauss rule with an odd number of points
// has a node at 0, where the odd Legendre polynomials and the derivatives of
// the even ones vanish, and Pt_0' = 0 everywhere. The multiply-adds by them
// are dropped at compile time (the loops are unrolled); for finite operands
// the sums are unchanged, bit for bit.
template <int K>
__host__ __device__ constexpr bool zero_p(int u, int q) {
  return K % 2 == 0 && 2 * q == K && u % 2 == 1;
}
template <int K>
__host__ __device__ constexpr bool zero_d(int u, int q) {
  return u == 0 || (K % 2 == 0 && 2 * q == K && u % 2 == 0);
}

// mode index of the exponents along (normal, tangential 1, tangential 2) of a
// face normal to axis D (tangential axes in ascending order)
template <int D>
__host__ __device__ constexpr int face_mode(int e, int a, int b) {
  return D == 0 ? mode_index(e, a, b) : (D == 1 ? mode_index(a, e, b) : mode_index(a, b, e));
}

// an upper bound of |x| in binary32 from the high word of x (20 fraction
// bits, rounded up: at most 2^-20 above |x|); magnitudes below 2^-126 map to
// 2^-126, huge and non-finite values to infinity
__device__ __forceinline__ float abs_up(double x) {
  unsigned u = (unsigned)__double2hiint(x) & 0x7fffffffu;
  u = min(max(u, 0x38100000u), 0x47efffffu);
  return __uint_as_float(((u - 0x38000000u) << 3) + 8u);
}

// binary64 -> binary32 on the integer pipe (no FP64-unit conversion):
// rounded to nearest on the 29 dropped fraction bits (ties away from zero,
// which differs from ties-to-even only when they are exactly 2^28);
// magnitudes below 2^-126 give a signed zero, magnitudes of 2^128 and above,
// infinities and NaNs a signed infinity (the stage's screen then queues the
// cell and the full limiter reports the non-finite state)
__device__ __forceinline__ float f64_to_f32_q(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned mag = hi & 0x7fffffffu;
  unsigned r = (__funnelshift_l(lo, hi, 3) - 0xC0000000u) + ((lo >> 28) & 1u);
  r = mag < 0x38100000u ? 0u : r;
  r = mag >= 0x47f00000u ? 0x7f800000u : r;
  return __uint_as_float(r | (hi & 0x80000000u));
}

// binary32 -> binary64 on the integer pipe: exact for normal numbers,
// subnormals give a signed zero, infinities and NaNs stay what they are
__device__ __forceinline__ double f32_to_f64_q(float x) {
  const unsigned u = __float_as_uint(x), mag = u & 0x7fffffffu, sg = u & 0x80000000u;
  unsigned hi = sg | ((mag >> 3) + 0x38000000u);
  unsigned lo = u << 29;
  hi = mag >= 0x7f800000u ? (hi | 0x7ff00000u) : hi;
  hi = mag < 0x00800000u ? sg : hi;
  lo = mag < 0x00800000u ? 0u : lo;
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
#ifdef __CUDA_ARCH__
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
#else
  (void)p;
#endif
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
#ifdef __CUDA_ARCH__
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
#else
  (void)p;
#endif
}

// approximate reciprocal and reciprocal square root (one MUFU operation
// each, subnormals flushed to zero: relative error of a few ulp)
__device__ __forceinline__ float rcp_fast(float x) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return 1.f / x;
#endif
}
__device__ __forceinline__ float rsqrt_fast(float x) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#else
  return 1.f / std::sqrt(x);
#endif
}
// sqrt(max(x, 0)): 0 for x <= 0, the limit of a sound speed at p -> 0+
__device__ __forceinline__ float sqrt_fast(float x) { return x > 0.f ? x * rsqrt_fast(x) : 0.f; }

// Every operation of the face flux is an explicit, separately rounded IEEE
// operation (or an fmaf, or one MUFU approximation): the compiler may
// neither contract nor reorder them, so a face whose flux two tiles
// compute (column sides, segment ends) gets the same bits in both, whatever
// the instruction schedule of each inlined copy.
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }

// Euler flux along x of the conserved state U (velocity v, pressure p)
__device__ __forceinline__ void euler_flux_x(const float* U, const float* v, float p, float* F) {
  const float mn = U[1];
  F[0] = mn;
  F[1] = fmaf(mn, v[0], p);
  F[2] = fm(mn, v[1]);
  F[3] = fm(mn, v[2]);
  F[4] = fm(fa(U[4], p), v[0]);
}

// HLLC flux across a face with normal +x in the face's frame (Sect. 2.3),
// the same algorithm as hllc_flux (Einfeldt wave speeds from Roe averages,
// Toro's star states, sound speed 0 at pressures <= 0, S* = 0 for a receding
// vacuum interface) with the FP32 path's fast reciprocal and square root,
// written without branches: both sides' fluxes and the star correction of
// the side of the contact are formed and the wave pattern selects one
// (an operand that is not selected may be non-finite without effect)
__device__ __forceinline__ void hllc_x_fast(const float* UL, const float* UR, float gamma, float* F) {
  const float gm1 = fs(gamma, 1.f);
  const float rL = rsqrt_fast(UL[0]), rR = rsqrt_fast(UR[0]);
  const float irL = fm(rL, rL), irR = fm(rR, rR);
  const float vL[3] = {fm(UL[1], irL), fm(UL[2], irL), fm(UL[3], irL)};
  const float vR[3] = {fm(UR[1], irR), fm(UR[2], irR), fm(UR[3], irR)};
  const float kL = fmaf(vL[0], vL[0], fmaf(vL[1], vL[1], fm(vL[2], vL[2])));
  const float kR = fmaf(vR[0], vR[0], fmaf(vR[1], vR[1], fm(vR[2], vR[2])));
  const float pL = fm(gm1, fs(UL[4], fm(fm(0.5f, UL[0]), kL)));
  const float pR = fm(gm1, fs(UR[4], fm(fm(0.5f, UR[0]), kR)));
  const float cL = sqrt_fast(fm(fm(gamma, pL), irL)), cR = sqrt_fast(fm(fm(gamma, pR), irR));
  const float sL = fm(UL[0], rL), sR = fm(UR[0], rR);
  const float iss = rcp_fast(fa(sL, sR));
  float vt[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) vt[a] = fm(fmaf(sL, vL[a], fm(sR, vR[a])), iss);
  const float v2 = fmaf(vt[0], vt[0], fmaf(vt[1], vt[1], fm(vt[2], vt[2])));
  const float Ht = fm(fmaf(rL, fa(UL[4], pL), fm(rR, fa(UR[4], pR))), iss);
  const float ct = sqrt_fast(fm(gm1, fs(Ht, fm(0.5f, v2))));
  const float uL = vL[0], uR = vR[0];
  const float SL = fminf(fs(uL, cL), fs(vt[0], ct));
  const float SR = fmaxf(fa(uR, cR), fa(vt[0], ct));
  float FL[5], FR[5];
  euler_flux_x(UL, vL, pL, FL);
  euler_flux_x(UR, vR, pR, FR);
  const float aL = fm(UL[0], fs(SL, uL)), aR = fm(UR[0], fs(SR, uR));
  const float den = fs(aL, aR);
  const float num = fs(fa(fs(pR, pL), fm(uL, aL)), fm(uR, aR));
  const float Ss = den == 0.f ? 0.f : fm(num, rcp_fast(den));
  const bool left = Ss >= 0.f;
  float U[5], FK[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    U[i] = left ? UL[i] : UR[i];
    FK[i] = left ? FL[i] : FR[i];
  }
  const float v1 = left ? vL[1] : vR[1], v2t = left ? vL[2] : vR[2];
  const float p = left ? pL : pR, S = left ? SL : SR, ak = left ? aL : aR, ir = left ? irL : irR;
  const float uk = left ? uL : uR;
  const float isd = rcp_fast(fs(S, Ss));
  const float chi = fm(ak, isd);
  const float dsu = fs(Ss, uk);
  float Us[5];
  Us[0] = chi;
  Us[1] = fm(chi, Ss);
  Us[2] = fm(chi, v1);
  Us[3] = fm(chi, v2t);
  Us[4] = fa(fm(chi, fa(fm(U[4], ir), fm(dsu, Ss))), fm(fm(dsu, p), isd));
  const bool supL = SL >= 0.f, supR = SR <= 0.f;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float fsi = fmaf(S, fs(Us[i], U[i]), FK[i]);
    F[i] = supL ? FL[i] : (supR ? FR[i] : fsi);
  }
}

// numerical flux in the face's frame: HLLC (fast FP32 form) or the exact
// Riemann solver
template <int FLUX>
__device__ __forceinline__ unsigned face_flux_x(const float* UL, const float* UR, float gamma, float* F) {
  if constexpr (FLUX == 1) {
    return exact_flux<float>(0, UL, UR, gamma, F);
  } else {
    hllc_x_fast(UL, UR, gamma, F);
    return 0u;
  }
}

// Values of one conserved variable on face (D, S) (S = 0: xi_D = -1, S = 1:
// xi_D = +1) at its Q^2 Gauss points p = t1 + Q t2, sum-factorised: the
// coefficients contracted along the normal with Pt_e(+-1), then along t2 and
// t1 (Sect. 2.3, the face traces of Eq. dg:eqn:surface_int).
template <int K, int D, int S>
__device__ __forceinline__ void fz_trace(const float (&w)[nmodes(K)], float* dst, int pstride) {
  using TB = FzTab<K>;
  constexpr int Q = K + 1, T = (K + 1) * (K + 2) / 2;
  float E[T];
#pragma unroll
  for (int a = 0, j = 0; a <= K; ++a)
#pragma unroll
    for (int b = 0; a + b <= K; ++b, ++j) {
      float s = 0.f;
#pragma unroll
      for (int e = 0; e + a + b <= K; ++e) s = fmaf(w[face_mode<D>(e, a, b)], c_fz[(S ? TB::EP : TB::EM) + e], s);
      E[j] = s;
    }
#pragma unroll
  for (int t2 = 0; t2 < Q; ++t2) {
    float H[K + 1];
#pragma unroll
    for (int a = 0, j = 0; a <= K; ++a) {
      float s = 0.f;
#pragma unroll
      for (int b = 0; a + b <= K; ++b, ++j)
        if (!zero_p<K>(b, t2)) s = fmaf(E[j], c_fz[TB::P + b * Q + t2], s);
      H[a] = s;
    }
#pragma unroll
    for (int t1 = 0; t1 < Q; ++t1) {
      float s = 0.f;
#pragma unroll
      for (int a = 0; a <= K; ++a)
        if (!zero_p<K>(a, t1)) s = fmaf(H[a], c_fz[TB::P + a * Q + t1], s);
      dst[(t1 + Q * t2) * pstride] = s;
    }
  }
}

// Face moments H[(a,b)] = sum_{t1,t2} F(t1 + Q t2) Pt_a(x_t1) w_t1 Pt_b(x_t2) w_t2
// of a flux (already scaled by 1/(4 dx)) at the face's Gauss points.
template <int K>
__device__ __forceinline__ void fz_moments(const float* src, int pstride, float (&H)[(K + 1) * (K + 2) / 2]) {
  using TB = FzTab<K>;
  constexpr int Q = K + 1, T = (K + 1) * (K + 2) / 2;
#pragma unroll
  for (int j = 0; j < T; ++j) H[j] = 0.f;
#pragma unroll
  for (int t2 = 0; t2 < Q; ++t2) {
    float G[K + 1];
#pragma unroll
    for (int a = 0; a <= K; ++a) G[a] = 0.f;
#pragma unroll
    for (int t1 = 0; t1 < Q; ++t1) {
      const float f = src[(t1 + Q * t2) * pstride];
#pragma unroll
      for (int a = 0; a <= K; ++a)
        if (!zero_p<K>(a, t1)) G[a] = fmaf(f, c_fz[TB::PW + a * Q + t1], G[a]);
    }
#pragma unroll
    for (int a = 0, j = 0; a <= K; ++a)
#pragma unroll
      for (int b = 0; a + b <= K; ++b, ++j)
        if (!zero_p<K>(b, t2)) H[j] = fmaf(G[a], c_fz[TB::PW + b * Q + t2], H[j]);
  }
}

// dw/dt += Pt_e(-1) H_low - Pt_e(+1) H_high for the modes (e, a, b) of a face
// pair normal to D (Eq. dg:eqn:surface_int with the outward normal sign)
template <int K, int D>
__device__ __forceinline__ void fz_apply(const float (&Hl)[(K + 1) * (K + 2) / 2],
                                         const float (&Hh)[(K + 1) * (K + 2) / 2], float (&acc)[nmodes(K)]) {
  using TB = FzTab<K>;
#pragma unroll
  for (int a = 0, j = 0; a <= K; ++a)
#pragma unroll
    for (int b = 0; a + b <= K; ++b, ++j)
#pragma unroll
      for (int e = 0; e + a + b <= K; ++e) {
        const int m = face_mode<D>(e, a, b);
        acc[m] = fmaf(c_fz[TB::EM + e], Hl[j], acc[m]);
        acc[m] = fmaf(-c_fz[TB::EP + e], Hh[j], acc[m]);
      }
}

// position of conserved variable i in the frame of a face normal to axis d:
// (rho, m_n, m_t1, m_t2, E) with t1 < t2 the other two axes. Traces and
// fluxes are stored in this order, so the numerical flux is evaluated with
// a compile-time normal and no reordering.
__device__ __forceinline__ int face_var(int d, int i) {
  if (i == 0 || i == 4) return i;
  const int ax = i - 1, t1 = d == 0 ? 1 : 0;
  return ax == d ? 1 : (ax == t1 ? 2 : 3);
}

// Sufficient limiter screen in FP32 from the cell means m and the excursion
// bounds s_i >= sum_{l>=1} |w_il| max|phi_l|: true when the density and the
// pressure provably stay above the floors at every point of the limiter's
// point set (same bounds as the FP64 screen, multiplied through by the
// density bound, with a 1e-5 relative margin that covers the FP32 rounding
// of the inputs and of the test). NaN inputs fail.
__device__ __forceinline__ bool screen_f32(const float* m, const float* s, float gm1, float er, float ep) {
  const float r = m[0];
  const float rlo = r - s[0];
  if (!(rlo >= er + 1e-5f * (fabsf(r) + s[0]))) return false;
  float k2 = 0.f;
#pragma unroll
  for (int a = 1; a <= 3; ++a) {
    const float mh = fabsf(m[a]) + s[a];
    k2 = fmaf(mh, mh, k2);
  }
  k2 *= 0.5f;
  const float elo = m[4] - s[4];
  const float lhs = gm1 * fmaf(elo, rlo, -k2);
  const float rhs = fmaf(ep, rlo, 1e-5f * gm1 * fmaf(fabsf(m[4]) + s[4], rlo, k2));
  return lhs >= rhs;
}

template <int K, bool FORCE, int FLUX>
__global__ void __launch_bounds__(FusedCfg<K>::THREADS, FusedCfg<K>::MINB) fused_f32_kernel(Geo g, FusedArgs a) {
  using CF = FusedCfg<K>;
  using TB = FzTab<K>;
  constexpr int Q = CF::Q, Q2 = CF::Q2, Q3 = CF::Q3, N = CF::N, T = CF::T;
  constexpr int NC = CF::NC, BX = CF::BX, BY = CF::BY, SX = CF::SX, SY = CF::SY, SZ = CF::SZ;
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x;
  const int i = tid / NC;  // conserved variable (warp-uniform)
  const int c = tid % NC;
  const int cx = c % BX, cy = c / BX;
  int rem = blockIdx.x;
  const int bx = rem % a.nbx;
  rem /= a.nbx;
  const int by = rem % a.nby;
  const int bz = rem / a.nby;
  const int x0 = bx * BX, y0 = by * BY, z0 = bz * a.lz;
  const int vx = min(BX, g.nx - x0), vy = min(BY, g.ny - y0), vz = min(a.lz, g.nz - z0);
  const bool cval = cx < vx && cy < vy;
  const int gx = x0 + cx, gy = y0 + cy;
  const long long nc = g.nc;
  const float gm1 = (float)(g.gamma - 1.0), gam = (float)g.gamma;
  const float scale[3] = {(float)(0.25 * g.inv_dx[0]), (float)(0.25 * g.inv_dx[1]), (float)(0.25 * g.inv_dx[2])};
  // slots of this cell's high x and y faces
  const int hx = cx + 1 < vx ? c + 1 : NC + cy;
  const int hy = cy + 1 < vy ? c + BX : NC + cx;
  unsigned err = 0;
  // 32-bit cell indices (nc < 2^31) and periodic wraps by comparison: no
  // integer division and no 64-bit multiply inside the plane loop
  const int plane = g.nx * g.ny;
  const int cxy = cval ? gy * g.nx + gx : y0 * g.nx + x0;  // in-plane index of this thread's cell
  const size_t rs = (size_t)nc;                            // row stride of the state layout
  const double* ysi = a.ys + (size_t)(i * N) * rs;         // this thread's variable
  // ring items (own planes): one (side, variable, row or column) per thread.
  // 8 x 8 tiles: warps 0-3 take one side each for variables 0-3, warp 4
  // variable 4 of all sides (no divergence between trace variants within
  // warps 0-3); other tiles: side-major order
  int rside, riv, rr;
  if constexpr (BX == 8 && BY == 8) {
    const int rwv = tid >> 5, rlane = tid & 31;
    rside = rwv < 4 ? rwv : rlane >> 3;
    riv = rwv < 4 ? rlane >> 3 : 4;
    rr = rlane & 7;  // row (x sides) or column (y sides)
  } else {
    int t = tid;
    if (t < 10 * BY) {
      rside = t / (5 * BY);
      t -= rside * 5 * BY;
      riv = t / BY;
      rr = t - riv * BY;
    } else {
      t -= 10 * BY;
      rside = 2 + t / (5 * BX);
      t -= (rside - 2) * 5 * BX;
      riv = t / BX;
      rr = t - riv * BX;
    }
  }
  const bool rval = tid < 10 * (BX + BY) && (rside < 2 ? rr < vy : rr < vx);
  int rxy = 0;
  {
    int rx, ry;
    if (rside == 0) { rx = x0 - 1 < 0 ? x0 - 1 + g.nx : x0 - 1; ry = y0 + rr; }
    else if (rside == 1) { rx = x0 + vx >= g.nx ? x0 + vx - g.nx : x0 + vx; ry = y0 + rr; }
    else if (rside == 2) { rx = x0 + rr; ry = y0 - 1 < 0 ? y0 - 1 + g.ny : y0 - 1; }
    else { rx = x0 + rr; ry = y0 + vy >= g.ny ? y0 + vy - g.ny : y0 + vy; }
    if (rval) rxy = ry * g.nx + rx;
  }
  const double* ysr = a.ys + (size_t)((rval ? riv : 0) * N) * rs;
  // this thread's variable (and its ring item's) in each face frame
  const int fvx = face_var(0, i), fvy = face_var(1, i), fvz = face_var(2, i);
  const int rfvx = face_var(0, riv), rfvy = face_var(1, riv);
  const float eps_r = a.eps_r, eps_p = a.eps_p;

  float w[N], acc[N];
#pragma unroll
  for (int l = 0; l < N; ++l) acc[l] = 0.f;
  // the density threads (i = 0) also sum the mean mode's face terms in FP64:
  // each face moment is the same FP32 value in both cells that share the
  // face, so these sums telescope and the FP64 stage update conserves mass
  // to FP64 rounding (the FP32 sums of the other modes round independently
  // in every cell)
  double accm = 0.0;

  for (int pz = -1; pz <= vz; ++pz) {
    int zc = z0 + pz;
    zc = zc < 0 ? zc + g.nz : (zc >= g.nz ? zc - g.nz : zc);
    const bool own = pz >= 0 && pz < vz;
    const int zoff = zc * plane;
    const int zprev = zc == 0 ? (g.nz - 1) * plane : zoff - plane;  // plane pz - 1
    const int znext = zc == g.nz - 1 ? 0 : zoff + plane;            // plane pz + 1
    // ---------------------------------------------------------------- P1
    {
      const double* p = ysi + (zoff + cxy);
#pragma unroll
      for (int l = 0; l < N; ++l, p += rs)
        w[l] = cval ? f64_to_f32_q(__ldg(p)) : ((l == 0 && (i == 0 || i == 4)) ? 1.f : 0.f);
      if (cval) {
        if (pz >= 0) fz_trace<K, 2, 0>(w, sm + CF::ZR + fvz * Q2 * SZ + c, SZ);
        if (own) {
          fz_trace<K, 0, 0>(w, sm + CF::XR + fvx * Q2 * SZ + c, SZ);
          fz_trace<K, 0, 1>(w, sm + CF::XL + fvx * Q2 * SZ + hx, SZ);
          fz_trace<K, 1, 0>(w, sm + CF::YR + fvy * Q2 * SZ + c, SZ);
          fz_trace<K, 1, 1>(w, sm + CF::YL + fvy * Q2 * SZ + hy, SZ);
        }
      }
      // ring of neighbour cells around the column (own planes): warps 0-3
      // take one side each for variables 0-3, warp 4 variable 4 of all sides
      if (own && rval) {
        float wr[N];
        const double* p = ysr + (zoff + rxy);
#pragma unroll
        for (int l = 0; l < N; ++l, p += rs) wr[l] = f64_to_f32_q(__ldg(p));
        if (rside == 0) fz_trace<K, 0, 1>(wr, sm + CF::XL + rfvx * Q2 * SZ + rr * BX, SZ);
        else if (rside == 1) fz_trace<K, 0, 0>(wr, sm + CF::XR + rfvx * Q2 * SZ + NC + rr, SZ);
        else if (rside == 2) fz_trace<K, 1, 1>(wr, sm + CF::YL + rfvy * Q2 * SZ + rr, SZ);
        else fz_trace<K, 1, 0>(wr, sm + CF::YR + rfvy * Q2 * SZ + NC + rr, SZ);
      }
    }
    __syncthreads();
    // ---------------------------------------------------------------- P2
    if (pz >= 0) {
      const int first = own ? 0 : (SX + SY) * Q2;
#pragma unroll (CF::FACE_UNROLL)
      for (int it = first + tid; it < CF::NFACE; it += CF::THREADS) {
        // item -> direction, face slot and point; o = p SZ + slot is the
        // face point's offset in its direction's trace arrays
        int oL, oR, slot, o;
        bool valid;
        float sc;
        if (it < SX * Q2) {
          slot = it % SX;
          o = (it / SX) * SZ + slot;
          oL = CF::XL;
          oR = CF::XR;
          sc = scale[0];
          valid = slot < NC ? ((slot % BX) < vx && (slot / BX) < vy) : slot - NC < vy;
        } else if (it < (SX + SY) * Q2) {
          const int r = it - SX * Q2;
          slot = r % SY;
          o = (r / SY) * SZ + slot;
          oL = CF::YL;
          oR = CF::YR;
          sc = scale[1];
          valid = slot < NC ? ((slot % BX) < vx && (slot / BX) < vy) : slot - NC < vx;
        } else {
          const int r = it - (SX + SY) * Q2;
          slot = r % NC;
          o = (r / NC) * SZ + slot;
          oL = CF::ZL;
          oR = CF::ZR;
          sc = scale[2];
          valid = (slot % BX) < vx && (slot / BX) < vy;
        }
        if (valid) {
          // both traces are stored in the face's frame (normal momentum
          // first, then the two tangential ones in ascending axis order)
          const float* pl = sm + oL + o;
          float* pr = sm + oR + o;
          float UL[5], UR[5], F[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            UL[v] = pl[v * Q2 * SZ];
            UR[v] = pr[v * Q2 * SZ];
          }
          err |= face_flux_x<FLUX>(UL, UR, gam, F);
#pragma unroll
          for (int v = 0; v < 5; ++v) pr[v * Q2 * SZ] = F[v] * sc;
        }
      }
    }
    __syncthreads();
    // ------------------------------------------------------------ P3, P4
    // On entry acc holds the previous plane's dw/dt without its high z
    // face. The z face closes it (P4: R or the stage update), then acc
    // restarts with this plane's low z face and its x and y faces.
    if (cval) {
      float H[T];
      if (pz >= 0) fz_moments<K>(sm + CF::ZR + fvz * Q2 * SZ + c, SZ, H);
      if (pz >= 1) {
#pragma unroll
        for (int aa = 0, j = 0; aa <= K; ++aa)
#pragma unroll
          for (int b = 0; aa + b <= K; ++b, ++j)
#pragma unroll
            for (int e = 0; e + aa + b <= K; ++e) {
              const int m = face_mode<2>(e, aa, b);
              acc[m] = fmaf(-c_fz[TB::EP + e], H[j], acc[m]);
            }
        if (i == 0) accm -= f32_to_f64_q(H[0]);  // Pt_0(+1) = 1
        const size_t o0 = (size_t)(i * N) * rs + (size_t)(zprev + cxy);
        if (a.stage == 0) {
          double* pr = a.R + o0;
#pragma unroll
          for (int l = 0; l < N; ++l, pr += rs) *pr = (l == 0 && i == 0) ? -accm : f32_to_f64_q(-acc[l]);
        } else {
          float sab = 0.f;
          double mean = 0.0;
          size_t o = o0;
#pragma unroll
          for (int l = 0; l < N; ++l, o += rs) {
            const double ysv = __ldg(a.ys + o);
            const float dl = a.stage >= 2 ? a.d[o] : 0.f;
            double v;
            float dnew;
            if (l == 0 && i == 0) {
              // mean density: the Shu-Osher combination in FP64, a0 y_0 +
              // b0 y_s + b0 dt dw/dt, with dw/dt from the FP64 face sum (y_0
              // is read for this one value per cell; in stage 1 y_0 = y_s)
              const double y00 = a.stage >= 2 ? a.y0[o] : ysv;
              v = fma(a.a0_d, y00, fma(a.b0_d, ysv, a.b0dt_d * accm));
              dnew = f64_to_f32_q(v - y00);
            } else {
              const float delta = fmaf(a.b0dt, acc[l], -a.a0 * dl);
              v = ysv + f32_to_f64_q(delta);
              dnew = dl + delta;
            }
            a.out[o] = v;
            if (a.stage <= 2) a.d[o] = dnew;
            else if (a.yf) a.yf[o] = f64_to_f32_q(v);
            if (l == 0) mean = v;
            else sab = fmaf(abs_up(v), c_fz[(g.lim_vol ? TB::LMV : TB::LM) + l], sab);
          }
          sm[CF::SMN + i * NC + c] = f64_to_f32_q(mean);
          sm[CF::SAB + i * NC + c] = sab * (1.f + 1e-5f);
        }
      }
#pragma unroll
      for (int l = 0; l < N; ++l) acc[l] = 0.f;
      if (i == 0) accm = pz >= 0 ? f32_to_f64_q(H[0]) : 0.0;  // Pt_0(-1) = 1
      if (pz >= 0) {
#pragma unroll
        for (int aa = 0, j = 0; aa <= K; ++aa)
#pragma unroll
          for (int b = 0; aa + b <= K; ++b, ++j)
#pragma unroll
            for (int e = 0; e + aa + b <= K; ++e) {
              const int m = face_mode<2>(e, aa, b);
              acc[m] = fmaf(c_fz[TB::EM + e], H[j], acc[m]);
            }
      }
      if (own) {
        float Hl[T], Hh[T];
        // x and y face pairs: a rolled loop at degree 3 (instruction cache),
        // written out at degree 2, where the loop form measured 4 % slower
        // (2.23 vs 2.13 ms per stage at 128^3)
        if constexpr (CF::SLICE_UNROLL == 1) {
#pragma unroll 1
          for (int d = 0; d < 2; ++d) {
            const float* base = sm + (d ? CF::YR + fvy * Q2 * SZ : CF::XR + fvx * Q2 * SZ);
            fz_moments<K>(base + c, SZ, Hl);
            fz_moments<K>(base + (d ? hy : hx), SZ, Hh);
            if (d == 0) fz_apply<K, 0>(Hl, Hh, acc);
            else fz_apply<K, 1>(Hl, Hh, acc);
            if (i == 0) accm += f32_to_f64_q(Hl[0]) - f32_to_f64_q(Hh[0]);
          }
        } else {
          fz_moments<K>(sm + CF::XR + fvx * Q2 * SZ + c, SZ, Hl);
          fz_moments<K>(sm + CF::XR + fvx * Q2 * SZ + hx, SZ, Hh);
          fz_apply<K, 0>(Hl, Hh, acc);
          if (i == 0) accm += f32_to_f64_q(Hl[0]) - f32_to_f64_q(Hh[0]);
          fz_moments<K>(sm + CF::YR + fvy * Q2 * SZ + c, SZ, Hl);
          fz_moments<K>(sm + CF::YR + fvy * Q2 * SZ + hy, SZ, Hh);
          fz_apply<K, 1>(Hl, Hh, acc);
          if (i == 0) accm += f32_to_f64_q(Hl[0]) - f32_to_f64_q(Hh[0]);
        }
      }
      // high-z traces of this plane for the next plane's z faces (the
      // previous ones were consumed in P2)
      if (pz < vz) fz_trace<K, 2, 1>(w, sm + CF::ZL + fvz * Q2 * SZ + c, SZ);
    }
    __syncthreads();
    // ---------------------------------------------------------------- P5
    if (pz >= 1 && a.stage > 0 && tid < NC) {
      const int tx = tid % BX, ty = tid / BX;
      if (tx < vx && ty < vy) {
        float m[5], s[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          m[v] = sm[CF::SMN + v * NC + tid];
          s[v] = sm[CF::SAB + v * NC + tid];
        }
        if (!screen_f32(m, s, gm1, eps_r, eps_p)) {
          const unsigned slot = atomicAdd(&a.ctrl->n_flag, 1u);
          a.list[slot] = zprev + (y0 + ty) * g.nx + x0 + tx;
        }
      }
    }
    // L2 prefetch of what the next plane reads from global memory: its
    // coefficients (own cells and ring) and, for the epilogue of this
    // plane, the increments d
    if (pz < vz) {
      if (cval) {
        const double* p = ysi + (znext + cxy);
#pragma unroll
        for (int l = 0; l < N; ++l, p += rs) prefetch_l2(p);
        if (own && a.stage >= 2) {
          const float* q = a.d + (size_t)(i * N) * rs + (size_t)(zoff + cxy);
#pragma unroll
          for (int l = 0; l < N; ++l, q += rs) prefetch_l2(q);
        }
      }
      if (pz + 1 < vz && rval) {
        const double* p = ysr + (znext + rxy);
#pragma unroll
        for (int l = 0; l < N; ++l, p += rs) prefetch_l2(p);
      }
    }
    // L1 prefetch of this plane's driving field (3 Q^3 rows of the tile's BY
    // rows of 8 values), read by the volume slices below
    if (CF::FIELD_L1 && FORCE && own) {
      for (int it = tid; it < 3 * Q3 * BY; it += CF::THREADS) {
        const int row = it / BY, ty = it - row * BY;
        if (ty < vy) prefetch_l1(a.field + (size_t)row * rs + (size_t)(zoff + (y0 + ty) * g.nx + x0));
      }
    }
    // ---------------------------------------------------------------- P6
    if (own) {
#pragma unroll (CF::SLICE_UNROLL)
      for (int qz = 0; qz < Q; ++qz) {
        // values of variable i at the slice's points
        {
          float A1[T];
#pragma unroll
          for (int u = 0, j = 0; u <= K; ++u)
#pragma unroll
            for (int v = 0; u + v <= K; ++v, ++j) {
              float s = 0.f;
#pragma unroll
              for (int ww = 0; u + v + ww <= K; ++ww)
                if (!zero_p<K>(ww, qz)) s = fmaf(w[mode_index(u, v, ww)], c_fz[TB::P + ww * Q + qz], s);
              A1[j] = s;
            }
#pragma unroll
          for (int qy = 0; qy < Q; ++qy) {
            float A2[K + 1];
#pragma unroll
            for (int u = 0, j = 0; u <= K; ++u) {
              float s = 0.f;
#pragma unroll
              for (int v = 0; u + v <= K; ++v, ++j)
                if (!zero_p<K>(v, qy)) s = fmaf(A1[j], c_fz[TB::P + v * Q + qy], s);
              A2[u] = s;
            }
#pragma unroll
            for (int qx = 0; qx < Q; ++qx) {
              float s = 0.f;
#pragma unroll
              for (int u = 0; u <= K; ++u)
                if (!zero_p<K>(u, qx)) s = fmaf(A2[u], c_fz[TB::P + u * Q + qx], s);
              sm[CF::VU + (i * Q2 + qx + Q * qy) * NC + c] = s;
            }
          }
        }
        __syncthreads();
        // Euler fluxes (and the driving source) at the slice's points:
        // NIT items per thread, their driving-field loads issued first
        {
          constexpr int NIT = (Q2 * NC + CF::THREADS - 1) / CF::THREADS;
          float ac[NIT][3];
#pragma unroll
          for (int k = 0; k < NIT; ++k) {
            const int it = tid + k * CF::THREADS;
            const int cc = it % NC, qs = it / NC;
            const int tx = cc % BX, ty = cc / BX;
#pragma unroll
            for (int dd = 0; dd < 3; ++dd) ac[k][dd] = 0.f;
            if (FORCE && it < Q2 * NC && tx < vx && ty < vy) {
              const float* fp = a.field + (size_t)(qz * Q2 + qs) * rs + (size_t)(zoff + (y0 + ty) * g.nx + x0 + tx);
#pragma unroll
              for (int dd = 0; dd < 3; ++dd, fp += (size_t)Q3 * rs) ac[k][dd] = __ldg(fp);
            }
          }
#pragma unroll
          for (int k = 0; k < NIT; ++k) {
            const int it = tid + k * CF::THREADS;
            if (it < Q2 * NC) {
              const int cc = it % NC, qs = it / NC;
              float U[5];
#pragma unroll
              for (int v = 0; v < 5; ++v) U[v] = sm[CF::VU + (v * Q2 + qs) * NC + cc];
              const float ir = rcp_fast(U[0]);
              const float vel[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
              const float p = gm1 * (U[4] - 0.5f * U[0] * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]));
#pragma unroll
              for (int dd = 0; dd < 3; ++dd) {
                float F[5];
                euler_flux<float>(dd, U, vel, p, F);
#pragma unroll
                for (int v = 0; v < 5; ++v) sm[CF::VF + ((dd * 5 + v) * Q2 + qs) * NC + cc] = F[v] * scale[dd];
              }
              if (FORCE) {
                sm[CF::VS + (0 * Q2 + qs) * NC + cc] = 0.125f * U[0] * ac[k][0];
                sm[CF::VS + (1 * Q2 + qs) * NC + cc] = 0.125f * U[0] * ac[k][1];
                sm[CF::VS + (2 * Q2 + qs) * NC + cc] = 0.125f * U[0] * ac[k][2];
                sm[CF::VS + (3 * Q2 + qs) * NC + cc] = 0.125f * (U[1] * ac[k][0] + U[2] * ac[k][1] + U[3] * ac[k][2]);
              }
            }
          }
        }
        __syncthreads();
        // projection onto the basis gradients (and the basis, for the
        // source) of variable i, sum-factorised along x, then y, then z
        {
          float H1[T], H2[T];
#pragma unroll
          for (int j = 0; j < T; ++j) {
            H1[j] = 0.f;
            H2[j] = 0.f;
          }
          const float* fx = sm + CF::VF + ((0 * 5 + i) * Q2) * NC + c;
          const float* fy = sm + CF::VF + ((1 * 5 + i) * Q2) * NC + c;
          const float* fzp = sm + CF::VF + ((2 * 5 + i) * Q2) * NC + c;
          const float* fs = sm + CF::VS + ((i > 0 ? i - 1 : 0) * Q2) * NC + c;
          const bool src = FORCE && i > 0;
#pragma unroll
          for (int qy = 0; qy < Q; ++qy) {
            float Gx[K + 1], Gy[K + 1], Gz[K + 1];
#pragma unroll
            for (int u = 0; u <= K; ++u) {
              Gx[u] = 0.f;
              Gy[u] = 0.f;
              Gz[u] = 0.f;
            }
#pragma unroll
            for (int qx = 0; qx < Q; ++qx) {
              const int qs = qx + Q * qy;
              const float vx_ = fx[qs * NC], vy_ = fy[qs * NC], vz_ = fzp[qs * NC];
              const float vs_ = src ? fs[qs * NC] : 0.f;
#pragma unroll
              for (int u = 0; u <= K; ++u) {
                if (!zero_d<K>(u, qx)) Gx[u] = fmaf(vx_, c_fz[TB::DW + u * Q + qx], Gx[u]);
                if (!zero_p<K>(u, qx)) {
                  // the source is weighted by Pt w along all three axes, like
                  // the x flux along y and z: it joins the x flux's sums here
                  if (FORCE) Gx[u] = fmaf(vs_, c_fz[TB::PW + u * Q + qx], Gx[u]);
                  Gy[u] = fmaf(vy_, c_fz[TB::PW + u * Q + qx], Gy[u]);
                  Gz[u] = fmaf(vz_, c_fz[TB::PW + u * Q + qx], Gz[u]);
                }
              }
            }
#pragma unroll
            for (int u = 0, j = 0; u <= K; ++u)
#pragma unroll
              for (int v = 0; u + v <= K; ++v, ++j) {
                if (!zero_p<K>(v, qy)) {
                  H1[j] = fmaf(Gx[u], c_fz[TB::PW + v * Q + qy], H1[j]);
                  H2[j] = fmaf(Gz[u], c_fz[TB::PW + v * Q + qy], H2[j]);
                }
                if (!zero_d<K>(v, qy)) H1[j] = fmaf(Gy[u], c_fz[TB::DW + v * Q + qy], H1[j]);
              }
          }
#pragma unroll
          for (int u = 0, j = 0; u <= K; ++u)
#pragma unroll
            for (int v = 0; u + v <= K; ++v, ++j)
#pragma unroll
              for (int ww = 0; u + v + ww <= K; ++ww) {
                const int m = mode_index(u, v, ww);
                if (!zero_p<K>(ww, qz)) acc[m] = fmaf(H1[j], c_fz[TB::PW + ww * Q + qz], acc[m]);
                if (!zero_d<K>(ww, qz)) acc[m] = fmaf(H2[j], c_fz[TB::DW + ww * Q + qz], acc[m]);
              }
        }
      }
    }
    __syncthreads();
  }
  if (err) atomicOr(&a.ctrl->err, err);
}

}  // namespace dg
