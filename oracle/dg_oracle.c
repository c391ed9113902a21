/*
 * dg_oracle.c -- plain FP64 CPU oracle of the TENET modal DG method
 * (Bauer et al., arXiv:1602.09079, Sect. 2 and Sect. 3.1-3.2).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and
 * bench.py's CPU baseline; never by the product path.
 *
 * Written to be checked against the paper by eye: every quadrature sum is the
 * literal sum of the paper's equation, evaluated point by point with the
 * basis evaluated through the Legendre three-term recurrence, no sum
 * factorisation, no fusion; every face flux is evaluated by each of its two
 * cells with the lower-index cell as the left state. OpenMP runs over cells
 * only.
 */
#include "dg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXK 3
#define MAXN 20
#define MAXQ 4

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------- tables */

int orc_nmodes(int k) { return (k + 1) * (k + 2) * (k + 3) / 6; } /* Sect. 2.2 */

/* Mode list: total degree d ascending, u descending, v descending. */
void orc_mode_exponents(int k, int32_t* uvw) {
  int l = 0;
  for (int d = 0; d <= k; ++d)
    for (int u = d; u >= 0; --u)
      for (int v = d - u; v >= 0; --v) {
        uvw[3 * l + 0] = u;
        uvw[3 * l + 1] = v;
        uvw[3 * l + 2] = d - u - v;
        ++l;
      }
}

/* Legendre P_0..P_n and derivatives by the three-term recurrence
 * (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1},  P'_{j+1} = P'_{j-1} + (2j+1) P_j. */
static void legendre(int n, double x, double* P, double* dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (n >= 1) {
    P[1] = x;
    dP[1] = 1.0;
  }
  for (int j = 1; j < n; ++j) {
    P[j + 1] = ((2 * j + 1) * x * P[j] - j * P[j - 1]) / (j + 1);
    dP[j + 1] = dP[j - 1] + (2 * j + 1) * P[j];
  }
}

/* Gauss-Legendre rule with q points on [-1,1] (weights sum to 2):
 * nodes are the roots of P_q found by Newton's method, weights
 * 2 / ((1 - x^2) P_q'(x)^2). Nodes ascending. */
void orc_gauss(int q, double* x, double* w) {
  double P[16], dP[16];
  for (int i = 0; i < q; ++i) {
    double z = -cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      legendre(q, z, P, dP);
      double dz = P[q] / dP[q];
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    legendre(q, z, P, dP);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dP[q] * dP[q]);
  }
}

/* Gauss-Lobatto-Legendre rule with m >= 2 points: the end points and the
 * roots of P'_{m-1}; weights 2 / (m (m-1) P_{m-1}(x)^2). */
void orc_gll(int m, double* x, double* w) {
  double P[16], dP[16];
  int n = m - 1;
  x[0] = -1.0;
  x[m - 1] = 1.0;
  for (int i = 1; i < m - 1; ++i) {
    /* Chebyshev-Gauss-Lobatto initial guess, Newton on P'_n using
     * P''_n = (2x P'_n - n(n+1) P_n)/(1-x^2) */
    double z = -cos(M_PI * i / n);
    for (int it = 0; it < 100; ++it) {
      legendre(n, z, P, dP);
      double d2 = (2.0 * z * dP[n] - n * (n + 1.0) * P[n]) / (1.0 - z * z);
      double dz = dP[n] / d2;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  for (int i = 0; i < m; ++i) {
    legendre(n, x[i], P, dP);
    w[i] = 2.0 / (m * (m - 1.0) * P[n] * P[n]);
  }
}

/* Number of GLL points of the positivity point set: the first GLL weight
 * (weights summing to 2) is 1 for order 2 and 1/3 for orders 3 and 4
 * (Sect. 2.5), i.e. m = 2 for k <= 1 and m = 3 for k = 2, 3. */
int orc_gll_count(int k) { return k <= 1 ? 2 : 3; }

/* phi_l and its xi-gradient at one reference point. */
void orc_basis(int k, const double xi[3], double* phi, double* dphi) {
  double P[3][MAXK + 2], dP[3][MAXK + 2];
  int32_t uvw[3 * MAXN];
  int N = orc_nmodes(k);
  orc_mode_exponents(k, uvw);
  for (int a = 0; a < 3; ++a) {
    legendre(k, xi[a], P[a], dP[a]);
    for (int u = 0; u <= k; ++u) {
      double s = sqrt(2.0 * u + 1.0); /* orthonormal scaling */
      P[a][u] *= s;
      dP[a][u] *= s;
    }
  }
  for (int l = 0; l < N; ++l) {
    int u = uvw[3 * l], v = uvw[3 * l + 1], w = uvw[3 * l + 2];
    phi[l] = P[0][u] * P[1][v] * P[2][w];
    if (dphi) {
      dphi[3 * l + 0] = dP[0][u] * P[1][v] * P[2][w];
      dphi[3 * l + 1] = P[0][u] * dP[1][v] * P[2][w];
      dphi[3 * l + 2] = P[0][u] * P[1][v] * dP[2][w];
    }
  }
}

/* ------------------------------------------------------------ mesh helpers */

static long ncells(const orc_params* p) { return (long)p->n[0] * p->n[1] * p->n[2]; }

static void cell_ijk(const orc_params* p, long c, int ijk[3]) {
  ijk[0] = (int)(c % p->n[0]);
  ijk[1] = (int)((c / p->n[0]) % p->n[1]);
  ijk[2] = (int)(c / ((long)p->n[0] * p->n[1]));
}

static long cell_index(const orc_params* p, const int ijk[3]) {
  int i[3];
  for (int a = 0; a < 3; ++a) i[a] = ((ijk[a] % p->n[a]) + p->n[a]) % p->n[a]; /* periodic */
  return ((long)i[2] * p->n[1] + i[1]) * p->n[0] + i[0];
}

static int check_params(const orc_params* p) {
  if (!p || p->k < 0 || p->k > MAXK) return ORC_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (p->n[a] < 1 || !(p->L[a] > 0)) return ORC_ERR_ARG;
  if (!(p->gamma > 1.0)) return ORC_ERR_ARG;
  if (p->n_force < 0 || (p->n_force > 0 && (!p->force_n || !p->force_a))) return ORC_ERR_ARG;
  if (p->limiter_points != ORC_LIMIT_S && p->limiter_points != ORC_LIMIT_S_VOLUME) return ORC_ERR_ARG;
  return ORC_OK;
}

/* q(xi) = sum_l w_l phi_l(xi), Eq. 1 */
static void eval_at(int k, const double* wK, const double* phi, double* U) {
  int N = orc_nmodes(k);
  for (int i = 0; i < 5; ++i) {
    double s = 0.0;
    for (int l = 0; l < N; ++l) s += wK[i * N + l] * phi[l];
    U[i] = s;
  }
}

void orc_eval(const orc_params* p, const double* w, long cell, const double xi[3], double* U) {
  double phi[MAXN];
  orc_basis(p->k, xi, phi, NULL);
  eval_at(p->k, w + cell * 5 * orc_nmodes(p->k), phi, U);
}

int orc_volume_points(const orc_params* p, double* xyz) {
  if (check_params(p)) return ORC_ERR_ARG;
  int Q = p->k + 1;
  double g[MAXQ], gw[MAXQ];
  orc_gauss(Q, g, gw);
  long nc = ncells(p);
  for (long c = 0; c < nc; ++c) {
    int ijk[3];
    cell_ijk(p, c, ijk);
    for (int cz = 0; cz < Q; ++cz)
      for (int b = 0; b < Q; ++b)
        for (int a = 0; a < Q; ++a) {
          int q = a + Q * (b + Q * cz);
          int ab[3] = {a, b, cz};
          for (int d = 0; d < 3; ++d) {
            double dx = p->L[d] / p->n[d];
            /* inverse of the reference map xi = 2 (x - x^K) / dx */
            xyz[(c * Q * Q * Q + q) * 3 + d] = (ijk[d] + 0.5) * dx + 0.5 * dx * g[ab[d]];
          }
        }
  }
  return ORC_OK;
}

int orc_project(const orc_params* p, const double* f, double* w) {
  if (check_params(p)) return ORC_ERR_ARG;
  int k = p->k, Q = k + 1, N = orc_nmodes(k), Q3 = Q * Q * Q;
  double g[MAXQ], gw[MAXQ];
  orc_gauss(Q, g, gw);
  long nc = ncells(p);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) {
    double acc[5 * MAXN];
    memset(acc, 0, sizeof(acc));
    for (int cz = 0; cz < Q; ++cz)
      for (int b = 0; b < Q; ++b)
        for (int a = 0; a < Q; ++a) {
          int q = a + Q * (b + Q * cz);
          double xi[3] = {g[a], g[b], g[cz]};
          double om = gw[a] * gw[b] * gw[cz];
          double phi[MAXN];
          orc_basis(k, xi, phi, NULL);
          for (int i = 0; i < 5; ++i)
            for (int l = 0; l < N; ++l) acc[i * N + l] += f[(c * 5 + i) * Q3 + q] * phi[l] * om;
        }
    for (int j = 0; j < 5 * N; ++j) w[c * 5 * N + j] = acc[j] / 8.0;
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------- physics */

static double pressure(double gamma, const double* U) {
  double ke = 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0];
  return (gamma - 1.0) * (U[4] - ke);
}

/* F_dir(q) of the Euler equations with an ideal-gas equation of state. */
void orc_euler_flux(int dir, double gamma, const double* U, double* F) {
  double rho = U[0];
  double vel[3] = {U[1] / rho, U[2] / rho, U[3] / rho};
  double p = pressure(gamma, U);
  double un = vel[dir];
  F[0] = U[1 + dir];
  for (int a = 0; a < 3; ++a) F[1 + a] = U[1 + dir] * vel[a] + (a == dir ? p : 0.0);
  F[4] = (U[4] + p) * un;
}

/* HLLC approximate Riemann solver (Toro's formulation) across a face with
 * normal +e_dir; left state = lower cell. Wave speeds: Einfeldt's estimates
 * with Roe averages, S_L = min(u_L - c_L, u~ - c~), S_R = max(u_R + c_R, u~ + c~);
 * middle speed and star states from the jump conditions across the three
 * waves. */
void orc_hllc(int dir, double gamma, const double* UL, const double* UR, double* F) {
  const double* U[2] = {UL, UR};
  double rho[2], vel[2][3], p[2], c[2], H[2], un[2];
  for (int s = 0; s < 2; ++s) {
    rho[s] = U[s][0];
    for (int a = 0; a < 3; ++a) vel[s][a] = U[s][1 + a] / rho[s];
    p[s] = pressure(gamma, U[s]);
    c[s] = sqrt(fmax(gamma * p[s] / rho[s], 0.0)); /* 0 for a pressure rounded to <= 0 */
    H[s] = (U[s][4] + p[s]) / rho[s];
    un[s] = vel[s][dir];
  }
  double sl = sqrt(rho[0]), sr = sqrt(rho[1]);
  double vt[3], v2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    vt[a] = (sl * vel[0][a] + sr * vel[1][a]) / (sl + sr);
    v2 += vt[a] * vt[a];
  }
  double Ht = (sl * H[0] + sr * H[1]) / (sl + sr);
  double c2t = (gamma - 1.0) * (Ht - 0.5 * v2);
  double ct = c2t > 0.0 ? sqrt(c2t) : 0.0;
  double SL = fmin(un[0] - c[0], vt[dir] - ct);
  double SR = fmax(un[1] + c[1], vt[dir] + ct);
  double den = rho[0] * (SL - un[0]) - rho[1] * (SR - un[1]);
  /* den = 0 only when both sound speeds are 0 in a receding flow (S_L = u_L,
   * S_R = u_R): no wave structure, S* = 0 */
  double Ss = den != 0.0 ? (p[1] - p[0] + rho[0] * un[0] * (SL - un[0]) - rho[1] * un[1] * (SR - un[1])) / den : 0.0;
  if (SL >= 0.0) {
    orc_euler_flux(dir, gamma, UL, F);
    return;
  }
  if (SR <= 0.0) {
    orc_euler_flux(dir, gamma, UR, F);
    return;
  }
  int s = (Ss >= 0.0) ? 0 : 1;
  double S = (s == 0) ? SL : SR;
  double Fs[5];
  orc_euler_flux(dir, gamma, U[s], Fs);
  double chi = rho[s] * (S - un[s]) / (S - Ss);
  double Us[5];
  Us[0] = chi;
  for (int a = 0; a < 3; ++a) Us[1 + a] = chi * (a == dir ? Ss : vel[s][a]);
  /* E* = chi (E/rho + (S* - u)(S* + p / (rho (S - u)))), with
   * chi / (rho (S - u)) = 1 / (S - S*) so that it stays defined for S = u */
  Us[4] = chi * (U[s][4] / rho[s] + (Ss - un[s]) * Ss) + (Ss - un[s]) * p[s] / (S - Ss);
  for (int i = 0; i < 5; ++i) F[i] = Fs[i] + S * (Us[i] - U[s][i]);
}

/* a(x) = sum_j Re( ahat_j exp(i k_j . x) ), k_j = 2 pi n_j / L (Sect. 3.1) */
static void forcing_at(const orc_params* p, const double* x, double* a) {
  a[0] = a[1] = a[2] = 0.0;
  for (int j = 0; j < p->n_force; ++j) {
    double ph = 0.0;
    for (int d = 0; d < 3; ++d) ph += 2.0 * M_PI * p->force_n[3 * j + d] / p->L[d] * x[d];
    double cs = cos(ph), sn = sin(ph);
    for (int d = 0; d < 3; ++d) a[d] += p->force_a[6 * j + d] * cs - p->force_a[6 * j + 3 + d] * sn;
  }
}

void orc_forcing_accel(const orc_params* p, long n, const double* xyz, double* a) {
  for (long i = 0; i < n; ++i) forcing_at(p, xyz + 3 * i, a + 3 * i);
}

/* ------------------------------------------------------------------- R(w) */

/* ------------------------------------------------ exact Riemann solver */

/* The exact solution of the one-dimensional Riemann problem of the Euler
 * equations for an ideal gas, the "exact" flux option of Sect. 2.3 (after
 * Eq. dg:eqn:surface_int), built the standard way (Toro, "Riemann Solvers
 * and Numerical Methods for Fluid Dynamics", Ch. 4):
 *  - across the wave of side K, the velocity change as a function of the
 *    star pressure p is f_K(p): the Rankine-Hugoniot shock branch for
 *    p > p_K, the isentropic rarefaction branch (Riemann invariant) for
 *    p <= p_K;
 *  - p* is the root of f(p) = f_L(p) + f_R(p) + u_R - u_L (increasing and
 *    concave), found by Newton's method from the adaptive estimate (the
 *    primitive-variable linearisation when the pressures are close, else the
 *    two-rarefaction or two-shock approximation);
 *  - u* = (u_L + u_R + f_R(p*) - f_L(p*)) / 2;
 *  - the state at x/t = s follows from the wave pattern (shock speeds from
 *    the jump conditions, rarefaction fans from the self-similar solution). */

static void exact_fk(double gamma, double p, double rk, double pk, double ck, double* f, double* df) {
  if (p > pk) {
    double A = 2.0 / ((gamma + 1.0) * rk);
    double B = (gamma - 1.0) / (gamma + 1.0) * pk;
    double q = sqrt(A / (p + B));
    *f = (p - pk) * q;
    *df = q * (1.0 - 0.5 * (p - pk) / (p + B));
  } else {
    double r = pow(p / pk, (gamma - 1.0) / (2.0 * gamma));
    *f = 2.0 * ck / (gamma - 1.0) * (r - 1.0);
    *df = ck * r / (gamma * p);
  }
}

int orc_exact_star(double gamma, const double WL[3], const double WR[3], double* pstar, double* ustar) {
  double rL = WL[0], uL = WL[1], pL = WL[2], rR = WR[0], uR = WR[1], pR = WR[2];
  double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  double du = uR - uL;
  if (2.0 * (cL + cR) / (gamma - 1.0) <= du) {
    *pstar = 0.0;
    *ustar = 0.0;
    return 1;
  }
  /* starting value */
  double ppv = 0.5 * (pL + pR) - 0.125 * du * (rL + rR) * (cL + cR);
  if (ppv < 0.0) ppv = 0.0;
  double pmin = fmin(pL, pR), pmax = fmax(pL, pR);
  double p;
  if (pmax / pmin <= 2.0 && ppv >= pmin && ppv <= pmax) {
    p = ppv;
  } else if (ppv < pmin) {
    double z = (gamma - 1.0) / (2.0 * gamma);
    p = pow((cL + cR - 0.5 * (gamma - 1.0) * du) / (cL / pow(pL, z) + cR / pow(pR, z)), 1.0 / z);
  } else {
    double gL = sqrt(2.0 / ((gamma + 1.0) * rL) / (ppv + (gamma - 1.0) / (gamma + 1.0) * pL));
    double gR = sqrt(2.0 / ((gamma + 1.0) * rR) / (ppv + (gamma - 1.0) / (gamma + 1.0) * pR));
    p = (gL * pL + gR * pR - du) / (gL + gR);
  }
  const double tiny = 1e-14 * pmin;
  if (!(p > tiny)) p = tiny;
  int it;
  for (it = 0; it < 100; ++it) {
    double fL, dfL, fR, dfR;
    exact_fk(gamma, p, rL, pL, cL, &fL, &dfL);
    exact_fk(gamma, p, rR, pR, cR, &fR, &dfR);
    double f = fL + fR + du;
    /* converged: the residual is at the rounding level of its terms (near a
     * vacuum the root is so ill-conditioned that the step itself stays
     * above 1e-14 p), else the relative step is below 1e-14 */
    if (fabs(f) <= 1e-15 * (fabs(fL) + fabs(fR) + fabs(du))) break;
    double pn = p - f / (dfL + dfR);
    if (!(pn > tiny)) pn = tiny;
    double change = fabs(pn - p);
    p = pn;
    if (change <= 1e-14 * p) break;
  }
  if (it == 100 || !isfinite(p)) return ORC_ERR_NEWTON;
  double fL, dfL, fR, dfR;
  exact_fk(gamma, p, rL, pL, cL, &fL, &dfL);
  exact_fk(gamma, p, rR, pR, cR, &fR, &dfR);
  *pstar = p;
  *ustar = 0.5 * (uL + uR) + 0.5 * (fR - fL);
  return ORC_OK;
}

/* state inside the rarefaction fan of side K (sgn = +1 left, -1 right) at x/t = s */
static void exact_fan(double gamma, double rk, double uk, double pk, double ck, double sgn, double s, double W[3]) {
  double c = 2.0 / (gamma + 1.0) * (ck + sgn * 0.5 * (gamma - 1.0) * (uk - s));
  W[1] = s + sgn * c;
  W[0] = rk * pow(c / ck, 2.0 / (gamma - 1.0));
  W[2] = pk * pow(c / ck, 2.0 * gamma / (gamma - 1.0));
}

/* side of the contact the sample lies on: 0 left, 1 right (returned through
 * *side when non-NULL) */
static int exact_sample_side(double gamma, const double WL[3], const double WR[3], double s, double W[3], int* side) {
  double rL = WL[0], uL = WL[1], pL = WL[2], rR = WR[0], uR = WR[1], pR = WR[2];
  double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  double ps, us;
  int st = orc_exact_star(gamma, WL, WR, &ps, &us);
  if (st < 0) return st;
  double g1 = (gamma - 1.0) / (2.0 * gamma), g2 = (gamma + 1.0) / (2.0 * gamma), g6 = (gamma - 1.0) / (gamma + 1.0);
  if (st == 1) {  /* two rarefactions and a vacuum between their tails */
    double sL = uL + 2.0 * cL / (gamma - 1.0), sR = uR - 2.0 * cR / (gamma - 1.0);
    if (s <= uL - cL) { W[0] = rL; W[1] = uL; W[2] = pL; if (side) *side = 0; }
    else if (s < sL) { exact_fan(gamma, rL, uL, pL, cL, 1.0, s, W); if (side) *side = 0; }
    else if (s <= sR) { W[0] = 0.0; W[1] = 0.5 * (sL + sR); W[2] = 0.0; if (side) *side = s <= 0.5 * (sL + sR) ? 0 : 1; }
    else if (s < uR + cR) { exact_fan(gamma, rR, uR, pR, cR, -1.0, s, W); if (side) *side = 1; }
    else { W[0] = rR; W[1] = uR; W[2] = pR; if (side) *side = 1; }
    return 1;
  }
  if (s <= us) {
    if (side) *side = 0;
    if (ps > pL) {
      double SL = uL - cL * sqrt(g2 * ps / pL + g1);
      if (s <= SL) { W[0] = rL; W[1] = uL; W[2] = pL; }
      else { W[0] = rL * (ps / pL + g6) / (g6 * ps / pL + 1.0); W[1] = us; W[2] = ps; }
    } else {
      double cs = cL * pow(ps / pL, g1);
      if (s <= uL - cL) { W[0] = rL; W[1] = uL; W[2] = pL; }
      else if (s > us - cs) { W[0] = rL * pow(ps / pL, 1.0 / gamma); W[1] = us; W[2] = ps; }
      else exact_fan(gamma, rL, uL, pL, cL, 1.0, s, W);
    }
  } else {
    if (side) *side = 1;
    if (ps > pR) {
      double SR = uR + cR * sqrt(g2 * ps / pR + g1);
      if (s >= SR) { W[0] = rR; W[1] = uR; W[2] = pR; }
      else { W[0] = rR * (ps / pR + g6) / (g6 * ps / pR + 1.0); W[1] = us; W[2] = ps; }
    } else {
      double cs = cR * pow(ps / pR, g1);
      if (s >= uR + cR) { W[0] = rR; W[1] = uR; W[2] = pR; }
      else if (s < us + cs) { W[0] = rR * pow(ps / pR, 1.0 / gamma); W[1] = us; W[2] = ps; }
      else exact_fan(gamma, rR, uR, pR, cR, -1.0, s, W);
    }
  }
  return ORC_OK;
}

int orc_exact_sample(double gamma, const double WL[3], const double WR[3], double s, double W[3]) {
  return exact_sample_side(gamma, WL, WR, s, W, NULL);
}

int orc_exact_flux(int dir, double gamma, const double* UL, const double* UR, double* F) {
  const double* U[2] = {UL, UR};
  double W[2][3], vel[2][3];
  for (int s = 0; s < 2; ++s) {
    for (int a = 0; a < 3; ++a) vel[s][a] = U[s][1 + a] / U[s][0];
    W[s][0] = U[s][0];
    W[s][1] = vel[s][dir];
    W[s][2] = pressure(gamma, U[s]);
  }
  double Wf[3];
  int side = 0;
  int st = exact_sample_side(gamma, W[0], W[1], 0.0, Wf, &side);
  if (st < 0) {
    for (int i = 0; i < 5; ++i) F[i] = NAN;
    return st;
  }
  double rho = Wf[0], un = Wf[1], p = Wf[2];
  double v[3];
  for (int a = 0; a < 3; ++a) v[a] = a == dir ? un : vel[side][a];
  double E = p / (gamma - 1.0) + 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  F[0] = rho * un;
  for (int a = 0; a < 3; ++a) F[1 + a] = rho * un * v[a] + (a == dir ? p : 0.0);
  F[4] = (E + p) * un;
  return ORC_OK;
}

/* numerical flux of Sect. 2.3 selected by p->flux */
static int num_flux(const orc_params* p, int dir, const double* UL, const double* UR, double* F) {
  if (p->flux == ORC_FLUX_EXACT) return orc_exact_flux(dir, p->gamma, UL, UR, F) < 0 ? ORC_ERR_NEWTON : ORC_OK;
  orc_hllc(dir, p->gamma, UL, UR, F);
  return ORC_OK;
}

/* dw/dt of one cell:
 *   dw_l/dt = sum_a 1/(4 dx_a) [ sum_{q in G^3} F_a(U_q) dphi_l/dxi_a(xi_q) om_q
 *             - sum_{s=+-1} s sum_{q in face(a,s)} Fhat_a phi_l(xi_{a=s,q}) om_q ]
 *           + 1/8 sum_q S(U_q, x_q) phi_l(xi_q) om_q
 * from Eq. dg:eqn:time_deriv (|K| dw/dt), Eq. dg:eqn:volume_int and
 * Eq. dg:eqn:surface_int divided by |K| = dx dy dz, with the outward normal of
 * each face written as the sign s; source from the forcing integral of
 * Sect. 3.1 (momentum rho a, energy m.a). */
static int cell_dwdt(const orc_params* p, const double* w, long cell, double* dwdt) {
  int status = ORC_OK;
  int k = p->k, Q = k + 1, N = orc_nmodes(k);
  double g[MAXQ], gw[MAXQ];
  orc_gauss(Q, g, gw);
  double dx[3];
  for (int a = 0; a < 3; ++a) dx[a] = p->L[a] / p->n[a];
  const double* wK = w + cell * 5 * N;
  int ijk[3];
  cell_ijk(p, cell, ijk);
  for (int j = 0; j < 5 * N; ++j) dwdt[j] = 0.0;

  /* volume integral */
  for (int cz = 0; cz < Q; ++cz)
    for (int b = 0; b < Q; ++b)
      for (int a = 0; a < Q; ++a) {
        double xi[3] = {g[a], g[b], g[cz]};
        double om = gw[a] * gw[b] * gw[cz];
        double phi[MAXN], dphi[3 * MAXN], U[5];
        orc_basis(k, xi, phi, dphi);
        eval_at(k, wK, phi, U);
        for (int al = 0; al < 3; ++al) {
          double F[5];
          orc_euler_flux(al, p->gamma, U, F);
          for (int i = 0; i < 5; ++i)
            for (int l = 0; l < N; ++l)
              dwdt[i * N + l] += F[i] * dphi[3 * l + al] * om / (4.0 * dx[al]);
        }
        if (p->n_force > 0) {
          double x[3], acc[3], S[5];
          for (int d = 0; d < 3; ++d) x[d] = (ijk[d] + 0.5) * dx[d] + 0.5 * dx[d] * xi[d];
          forcing_at(p, x, acc);
          S[0] = 0.0;
          S[1] = U[0] * acc[0];
          S[2] = U[0] * acc[1];
          S[3] = U[0] * acc[2];
          S[4] = U[1] * acc[0] + U[2] * acc[1] + U[3] * acc[2];
          for (int i = 0; i < 5; ++i)
            for (int l = 0; l < N; ++l) dwdt[i * N + l] += S[i] * phi[l] * om / 8.0;
        }
      }

  /* surface integral: faces (al, s), the other two axes in ascending order */
  for (int al = 0; al < 3; ++al) {
    int ax1 = (al + 1) % 3, ax2 = (al + 2) % 3;
    if (ax1 > ax2) {
      int t = ax1;
      ax1 = ax2;
      ax2 = t;
    }
    for (int s = -1; s <= 1; s += 2) {
      int nb[3] = {ijk[0], ijk[1], ijk[2]};
      nb[al] += s;
      const double* wN = w + cell_index(p, nb) * 5 * N;
      for (int t2 = 0; t2 < Q; ++t2)
        for (int t1 = 0; t1 < Q; ++t1) {
          double xo[3], xn[3];
          xo[al] = (double)s;
          xn[al] = (double)(-s);
          xo[ax1] = xn[ax1] = g[t1];
          xo[ax2] = xn[ax2] = g[t2];
          double om2 = gw[t1] * gw[t2];
          double phio[MAXN], phin[MAXN], Uo[5], Un[5], Fh[5];
          orc_basis(k, xo, phio, NULL);
          orc_basis(k, xn, phin, NULL);
          eval_at(k, wK, phio, Uo);
          eval_at(k, wN, phin, Un);
          int fs = s > 0 ? num_flux(p, al, Uo, Un, Fh) : num_flux(p, al, Un, Uo, Fh);
          if (fs != ORC_OK) status = fs;
          for (int i = 0; i < 5; ++i)
            for (int l = 0; l < N; ++l)
              dwdt[i * N + l] -= s * Fh[i] * phio[l] * om2 / (4.0 * dx[al]);
        }
    }
  }
  return status;
}

int orc_rhs(const orc_params* p, const double* w, double* R) {
  if (check_params(p)) return ORC_ERR_ARG;
  int N = orc_nmodes(p->k);
  long nc = ncells(p);
  int status = ORC_OK;
#pragma omp parallel for schedule(dynamic, 16) reduction(min : status)
  for (long c = 0; c < nc; ++c) {
    double d[5 * MAXN];
    int st = cell_dwdt(p, w, c, d);
    if (st < status) status = st;
    for (int j = 0; j < 5 * N; ++j) R[c * 5 * N + j] = -d[j];
  }
  return status;
}

int orc_rhs_cells(const orc_params* p, const double* w, long n_cells, const int64_t* cells, double* R) {
  if (check_params(p)) return ORC_ERR_ARG;
  int N = orc_nmodes(p->k);
  long nc = ncells(p);
  for (long i = 0; i < n_cells; ++i)
    if (cells[i] < 0 || cells[i] >= nc) return ORC_ERR_ARG;
  int status = ORC_OK;
#pragma omp parallel for schedule(dynamic, 4) reduction(min : status)
  for (long i = 0; i < n_cells; ++i) {
    double d[5 * MAXN];
    int st = cell_dwdt(p, w, cells[i], d);
    if (st < status) status = st;
    for (int j = 0; j < 5 * N; ++j) R[i * 5 * N + j] = -d[j];
  }
  return status;
}

/* ---------------------------------------------------------------- limiter */

/* The positivity point set S = S_x u S_y u S_z of Sect. 2.5: one coordinate
 * from the m GLL points, the other two from the k+1 Gauss points. */
static int limiter_points(int k, double* pts /* [3 m Q^2][3] */) {
  int Q = k + 1, m = orc_gll_count(k);
  double g[MAXQ], gw[MAXQ], h[8], hw[8];
  orc_gauss(Q, g, gw);
  orc_gll(m, h, hw);
  int n = 0;
  for (int al = 0; al < 3; ++al)
    for (int r = 0; r < m; ++r)
      for (int s = 0; s < Q; ++s)
        for (int t = 0; t < Q; ++t) {
          int o1 = (al + 1) % 3, o2 = (al + 2) % 3;
          if (o1 > o2) {
            int tt = o1;
            o1 = o2;
            o2 = tt;
          }
          pts[3 * n + al] = h[r];
          pts[3 * n + o1] = g[s];
          pts[3 * n + o2] = g[t];
          ++n;
        }
  return n;
}

/* P along the segment qbar + tau (q - qbar); Newton from tau = 1. P is
 * concave along the segment while rho > 0, so the iterates decrease
 * monotonically to the root. */
double orc_pressure_tau(double gamma, const double* qbar, const double* q, double eps, int* iters) {
  double d[5];
  for (int i = 0; i < 5; ++i) d[i] = q[i] - qbar[i];
  double tau = 1.0;
  int it;
  for (it = 0; it < 50; ++it) {
    double s[5];
    for (int i = 0; i < 5; ++i) s[i] = qbar[i] + tau * d[i];
    double m2 = s[1] * s[1] + s[2] * s[2] + s[3] * s[3];
    double f = (gamma - 1.0) * (s[4] - 0.5 * m2 / s[0]) - eps;
    /* dP/dtau = (gamma-1) (dE - m.dm/rho + 0.5 |m|^2 drho / rho^2) */
    double md = s[1] * d[1] + s[2] * d[2] + s[3] * d[3];
    double fp = (gamma - 1.0) * (d[4] - md / s[0] + 0.5 * m2 * d[0] / (s[0] * s[0]));
    double tn = tau - f / fp;
    if (!(tn >= 0.0)) tn = 0.0;
    if (tn > tau) tn = tau;
    double step = tau - tn;
    tau = tn;
    if (step <= 1e-15) {
      ++it;
      break;
    }
  }
  if (iters) *iters = it;
  return tau;
}

/* One cell: theta1 from the density minimum over S, then theta2 from the
 * pressure of the theta1-limited polynomial (Sect. 2.5, Eq. p_positivity,
 * with tau solving P(qbar + tau (q - qbar)) = eps). Returns an ORC status and
 * the flag bits. */
static int limit_cell(const orc_params* p, double* wK, const double* pts, int npts,
                      const double* phis, int8_t* flag) {
  int k = p->k, N = orc_nmodes(k);
  double eps_r = p->eps_rho, eps_p = p->eps_p;
  *flag = 0;
  for (int j = 0; j < 5 * N; ++j)
    if (!isfinite(wK[j])) return ORC_ERR_NONFINITE;
  double rbar = wK[0];
  if (!(rbar >= eps_r)) return ORC_ERR_POSITIVITY;
  double qbar[5];
  for (int i = 0; i < 5; ++i) qbar[i] = wK[i * N];
  if (!(pressure(p->gamma, qbar) >= eps_p)) return ORC_ERR_POSITIVITY;
  (void)pts;

  double rmin = rbar;
  for (int s = 0; s < npts; ++s) {
    double r = 0.0;
    for (int l = 0; l < N; ++l) r += wK[l] * phis[s * N + l];
    if (r < rmin) rmin = r;
  }
  double th1 = 1.0;
  if (rmin < eps_r) th1 = fmin(fabs((rbar - eps_r) / (rbar - rmin)), 1.0);
  if (th1 < 1.0) {
    for (int l = 1; l < N; ++l) wK[l] *= th1;
    *flag |= 1;
  }

  double th2 = 1.0;
  int newton_fail = 0;
  for (int s = 0; s < npts; ++s) {
    double U[5];
    eval_at(k, wK, phis + s * N, U);
    if (pressure(p->gamma, U) < eps_p) {
      int it;
      double tau = orc_pressure_tau(p->gamma, qbar, U, eps_p, &it);
      if (it >= 50) newton_fail = 1;
      if (tau < th2) th2 = tau;
    }
  }
  if (th2 < 1.0) {
    for (int i = 0; i < 5; ++i)
      for (int l = 1; l < N; ++l) wK[i * N + l] *= th2;
    *flag |= 2;
  }
  return newton_fail ? ORC_ERR_NEWTON : ORC_OK;
}

static int limit_list(const orc_params* p, double* w, long n, const int64_t* cells, int8_t* flags,
                      int64_t* nlim) {
  int k = p->k, N = orc_nmodes(k), Q = k + 1, m = orc_gll_count(k);
  int nS = 3 * m * Q * Q;
  /* optional: the volume Gauss points, where the volume fluxes are
   * evaluated, join S (Sect. 2.5 asks that S contain every point where
   * fluxes are evaluated; S itself covers the face points only) */
  int npts = nS + (p->limiter_points == ORC_LIMIT_S_VOLUME ? Q * Q * Q : 0);
  double* pts = (double*)malloc(sizeof(double) * 3 * npts);
  double* phis = (double*)malloc(sizeof(double) * npts * N);
  limiter_points(k, pts);
  if (npts > nS) {
    double g[MAXQ], gw[MAXQ];
    orc_gauss(Q, g, gw);
    int s = nS;
    for (int c = 0; c < Q; ++c)
      for (int b = 0; b < Q; ++b)
        for (int a = 0; a < Q; ++a, ++s) {
          pts[3 * s] = g[a];
          pts[3 * s + 1] = g[b];
          pts[3 * s + 2] = g[c];
        }
  }
  for (int s = 0; s < npts; ++s) orc_basis(k, pts + 3 * s, phis + s * N, NULL);
  int status = ORC_OK;
  int64_t count = 0;
#pragma omp parallel for schedule(static) reduction(+ : count)
  for (long i = 0; i < n; ++i) {
    long c = cells ? cells[i] : i;
    int8_t f = 0;
    int st = limit_cell(p, w + c * 5 * N, pts, npts, phis, &f);
    if (flags) flags[i] = f;
    if (f) ++count;
    if (st != ORC_OK) {
#pragma omp critical
      {
        /* report the most severe status: non-finite, positivity, newton */
        if (status == ORC_OK || st > status) status = st;
      }
    }
  }
  free(pts);
  free(phis);
  if (nlim) *nlim = count;
  return status;
}

int orc_limit(const orc_params* p, double* w, int8_t* flags, int64_t* n_limited) {
  if (check_params(p)) return ORC_ERR_ARG;
  return limit_list(p, w, ncells(p), NULL, flags, n_limited);
}

int orc_limit_cells(const orc_params* p, double* w, long n_cells, const int64_t* cells, int8_t* flags) {
  if (check_params(p)) return ORC_ERR_ARG;
  for (long i = 0; i < n_cells; ++i)
    if (cells[i] < 0 || cells[i] >= ncells(p)) return ORC_ERR_ARG;
  return limit_list(p, w, n_cells, cells, flags, NULL);
}

/* ------------------------------------------------------------- time step */

/* Eq. time_step_pos: dt^K = C min(1/(2k+1), w1/2) / sum_a (|v_a| + c)/dx_a
 * with mean velocity and sound speed from the cell means; global minimum. */
int orc_cfl_dt(const orc_params* p, const double* w, double courant, double* dt) {
  if (check_params(p) || !(courant > 0)) return ORC_ERR_ARG;
  int k = p->k, N = orc_nmodes(k), m = orc_gll_count(k);
  double h[8], hw[8];
  orc_gll(m, h, hw);
  double fac = fmin(1.0 / (2 * k + 1), hw[0] / 2.0);
  long nc = ncells(p);
  double best = INFINITY;
  int bad = 0;
  for (long c = 0; c < nc; ++c) {
    double qb[5];
    for (int i = 0; i < 5; ++i) qb[i] = w[c * 5 * N + i * N];
    double pr = pressure(p->gamma, qb);
    if (!(qb[0] > 0) || !(pr > 0)) {
      bad = 1;
      continue;
    }
    double cs = sqrt(p->gamma * pr / qb[0]);
    double sum = 0.0;
    for (int a = 0; a < 3; ++a) sum += (fabs(qb[1 + a] / qb[0]) + cs) / (p->L[a] / p->n[a]);
    double d = courant * fac / sum;
    if (d < best) best = d;
  }
  *dt = best;
  return bad ? ORC_ERR_POSITIVITY : ORC_OK;
}

/* ---------------------------------------------------------------- SSP-RK3 */

/* Shu-Osher SSP-RK3 (Sect. 2.4):
 *   y1 = y0 - dt R(y0); y2 = 3/4 y0 + 1/4 (y1 - dt R(y1));
 *   y3 = 1/3 y0 + 2/3 (y2 - dt R(y2)),
 * with the positivity limiter applied to the state at the beginning of each
 * stage (Sect. 2.5). The returned state is limited as well: it is the state
 * the next step's first stage begins with. */
int orc_step(const orc_params* p, double* w, double dt) {
  if (check_params(p)) return ORC_ERR_ARG;
  long len = ncells(p) * 5 * orc_nmodes(p->k);
  double* y0 = (double*)malloc(sizeof(double) * len);
  double* ys = (double*)malloc(sizeof(double) * len);
  double* R = (double*)malloc(sizeof(double) * len);
  int st = orc_limit(p, w, NULL, NULL);
  memcpy(y0, w, sizeof(double) * len);
  memcpy(ys, w, sizeof(double) * len);
  const double a0[3] = {0.0, 0.75, 1.0 / 3.0};
  const double b0[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int s = 0; s < 3 && st >= ORC_OK; ++s) {
    if (s > 0) st = orc_limit(p, ys, NULL, NULL);
    if (st < ORC_OK && st != ORC_ERR_NEWTON) break;
    int sr = orc_rhs(p, ys, R);
    if (sr != ORC_OK) {
      st = sr;
      break;
    }
    for (long j = 0; j < len; ++j) ys[j] = a0[s] * y0[j] + b0[s] * (ys[j] - dt * R[j]);
  }
  if (st >= ORC_OK || st == ORC_ERR_NEWTON) {
    int st2 = orc_limit(p, ys, NULL, NULL);
    if (st2 != ORC_OK) st = st2;
    memcpy(w, ys, sizeof(double) * len);
  }
  free(y0);
  free(ys);
  free(R);
  return st;
}

/* ----------------------------------------------------------- energy reset */

/* Sect. 3.2: eps = c^2/(gamma-1) (rho/rho0)^(gamma-1) enforced at the volume
 * quadrature points; the energy weights are the projection of
 * 1/2 |m|^2/rho + rho eps. Returns the change of the mean internal energy. */
static double reset_cell(const orc_params* p, double* wK, double c_iso, double rho0) {
  int k = p->k, Q = k + 1, N = orc_nmodes(k);
  double g[MAXQ], gw[MAXQ];
  orc_gauss(Q, g, gw);
  double before = wK[4 * N] - 0.5 * (wK[N] * wK[N] + wK[2 * N] * wK[2 * N] + wK[3 * N] * wK[3 * N]) / wK[0];
  double acc[MAXN];
  for (int l = 0; l < N; ++l) acc[l] = 0.0;
  for (int cz = 0; cz < Q; ++cz)
    for (int b = 0; b < Q; ++b)
      for (int a = 0; a < Q; ++a) {
        double xi[3] = {g[a], g[b], g[cz]};
        double om = gw[a] * gw[b] * gw[cz];
        double phi[MAXN], U[5];
        orc_basis(k, xi, phi, NULL);
        eval_at(k, wK, phi, U);
        double eps = c_iso * c_iso / (p->gamma - 1.0) * pow(U[0] / rho0, p->gamma - 1.0);
        double E = 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0] + U[0] * eps;
        for (int l = 0; l < N; ++l) acc[l] += E * phi[l] * om;
      }
  for (int l = 0; l < N; ++l) wK[4 * N + l] = acc[l] / 8.0;
  double after = wK[4 * N] - 0.5 * (wK[N] * wK[N] + wK[2 * N] * wK[2 * N] + wK[3 * N] * wK[3 * N]) / wK[0];
  return before - after;
}

int orc_energy_reset(const orc_params* p, double* w, double c_iso, double rho0, double* dissipated) {
  if (check_params(p) || !(rho0 > 0) || !(c_iso >= 0)) return ORC_ERR_ARG;
  int N = orc_nmodes(p->k);
  long nc = ncells(p);
  double vol = 1.0;
  for (int a = 0; a < 3; ++a) vol *= p->L[a] / p->n[a];
  double diss = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : diss)
  for (long c = 0; c < nc; ++c) diss += vol * reset_cell(p, w + c * 5 * N, c_iso, rho0);
  if (dissipated) *dissipated = diss;
  return orc_limit(p, w, NULL, NULL);
}

int orc_energy_reset_cells(const orc_params* p, double* w, long n_cells, const int64_t* cells,
                           double c_iso, double rho0) {
  if (check_params(p)) return ORC_ERR_ARG;
  int N = orc_nmodes(p->k);
  for (long i = 0; i < n_cells; ++i) reset_cell(p, w + cells[i] * 5 * N, c_iso, rho0);
  return orc_limit_cells(p, w, n_cells, cells, NULL);
}

void orc_totals(const orc_params* p, const double* w, double* out5) {
  int N = orc_nmodes(p->k);
  long nc = ncells(p);
  double vol = 1.0;
  for (int a = 0; a < 3; ++a) vol *= p->L[a] / p->n[a];
  for (int i = 0; i < 5; ++i) {
    double s = 0.0;
    for (long c = 0; c < nc; ++c) s += w[c * 5 * N + i * N];
    out5[i] = s * vol;
  }
}

/* Sect. 4.1 (rms Mach number) and 4.2 (injected energy), readings in the
 * header. */
void orc_diagnostics(const orc_params* p, const double* w, double* out3) {
  int k = p->k, N = orc_nmodes(k), Q = k + 1;
  long nc = ncells(p);
  double dx[3], vol = 1.0, V = 1.0;
  for (int a = 0; a < 3; ++a) {
    dx[a] = p->L[a] / p->n[a];
    vol *= dx[a];
    V *= p->L[a];
  }
  double g[MAXQ], gw[MAXQ];
  orc_gauss(Q, g, gw);
  double m2 = 0.0, kin = 0.0, pow_ = 0.0;
  for (long c = 0; c < nc; ++c) {
    const double* wK = w + c * 5 * N;
    double rho = wK[0], m[3] = {wK[N], wK[2 * N], wK[3 * N]}, E = wK[4 * N];
    double mm = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
    double pr = (p->gamma - 1.0) * (E - 0.5 * mm / rho);
    double vv = mm / (rho * rho);
    m2 += vol * vv / (p->gamma * pr / rho);
    kin += vol * 0.5 * mm / rho;
    if (p->n_force > 0) {
      int ijk[3];
      cell_ijk(p, c, ijk);
      for (int cz = 0; cz < Q; ++cz)
        for (int b = 0; b < Q; ++b)
          for (int a = 0; a < Q; ++a) {
            double xi[3] = {g[a], g[b], g[cz]};
            double x[3], acc[3], phi[MAXN], U[5];
            for (int d = 0; d < 3; ++d) x[d] = (ijk[d] + 0.5) * dx[d] + 0.5 * dx[d] * xi[d];
            forcing_at(p, x, acc);
            orc_basis(k, xi, phi, NULL);
            eval_at(k, wK, phi, U);
            pow_ += vol * (U[1] * acc[0] + U[2] * acc[1] + U[3] * acc[2]) * gw[a] * gw[b] * gw[cz] / 8.0;
          }
    }
  }
  out3[0] = sqrt(m2 / V);
  out3[1] = kin;
  out3[2] = pow_;
}

/* Sect. 3.3: the velocity field sampled below the cell size for spectra. */
int orc_sample_velocity(const orc_params* p, const double* w, int sub, int comp, double* out) {
  if (check_params(p) || sub < 1 || comp < 0 || comp > 2) return ORC_ERR_ARG;
  if (p->n[0] != p->n[1] || p->n[1] != p->n[2]) return ORC_ERR_ARG;
  int n = p->n[0], M = n * sub;
#pragma omp parallel for schedule(static)
  for (long Z = 0; Z < M; ++Z)
    for (long Y = 0; Y < M; ++Y)
      for (long X = 0; X < M; ++X) {
        double xi[3] = {-1.0 + (2.0 * (X % sub) + 1.0) / sub, -1.0 + (2.0 * (Y % sub) + 1.0) / sub,
                        -1.0 + (2.0 * (Z % sub) + 1.0) / sub};
        long cell = ((Z / sub) * n + Y / sub) * n + X / sub;
        double U[5];
        orc_eval(p, w, cell, xi, U);
        out[(Z * M + Y) * M + X] = U[1 + comp] / U[0];
      }
  return ORC_OK;
}

/* Sect. 4.4: the density field sampled below the cell size for PDFs. */
int orc_sample_density(const orc_params* p, const double* w, int sub, double* out) {
  if (check_params(p) || sub < 1) return ORC_ERR_ARG;
  if (p->n[0] != p->n[1] || p->n[1] != p->n[2]) return ORC_ERR_ARG;
  int n = p->n[0], M = n * sub;
#pragma omp parallel for schedule(static)
  for (long Z = 0; Z < M; ++Z)
    for (long Y = 0; Y < M; ++Y)
      for (long X = 0; X < M; ++X) {
        double xi[3] = {-1.0 + (2.0 * (X % sub) + 1.0) / sub, -1.0 + (2.0 * (Y % sub) + 1.0) / sub,
                        -1.0 + (2.0 * (Z % sub) + 1.0) / sub};
        long cell = ((Z / sub) * n + Y / sub) * n + X / sub;
        double U[5];
        orc_eval(p, w, cell, xi, U);
        out[(Z * M + Y) * M + X] = U[0];
      }
  return ORC_OK;
}
