/*
 * dg_oracle.h -- plain, slow FP64 CPU restatement of the TENET modal DG
 * method for the 3D Euler equations (Bauer et al., arXiv:1602.09079, Sect. 2).
 *
 * TEST INFRASTRUCTURE ONLY. This is the oracle that the CUDA path is checked
 * against. Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference arm may load it. It shares no code, header, table or constant
 * with the CUDA library, and the CUDA library never calls it.
 *
 * Conventions (all written from the paper):
 *   - k: polynomial degree (order O = k+1, Sect. 3), N(k) = (k+1)(k+2)(k+3)/6
 *     modes per variable (Sect. 2.2).
 *   - basis phi_l(xi) = Pt_u(xi1) Pt_v(xi2) Pt_w(xi3), u+v+w <= k, Pt_u the
 *     Legendre polynomial scaled so that (1/8) int phi_l phi_m = delta_lm
 *     (Sect. 2.2, orthonormal basis with w_0 = cell mean).
 *   - mode order: total degree ascending, then u descending, then v
 *     descending.
 *   - state layout: [nz][ny][nx][5][N], variables (rho, rho vx, rho vy,
 *     rho vz, E), cell (ix,iy,iz) centred at ((ix+1/2)dx, ...).
 *   - R follows Eq. "dg:eqn:time": dw/dt + R(w) = 0.
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_ERR_ARG = -1,
  ORC_ERR_NONFINITE = -4,
  ORC_ERR_POSITIVITY = -5,
  ORC_ERR_NEWTON = -6
};

typedef struct {
  int k;              /* polynomial degree 0..3 */
  int n[3];           /* cells per axis */
  double L[3];        /* periodic box lengths, origin at 0 */
  double gamma;       /* ideal-gas adiabatic index */
  double eps_rho;     /* positivity floor for density */
  double eps_p;       /* positivity floor for pressure */
  int n_force;        /* number of forcing Fourier modes (0 = none) */
  const int32_t* force_n;   /* 3*n_force integer wave vectors n, k = 2 pi n / L */
  const double* force_a;    /* 6*n_force: Re a_x,a_y,a_z, Im a_x,a_y,a_z */
  int flux;           /* numerical flux: ORC_FLUX_HLLC or ORC_FLUX_EXACT */
  int limiter_points; /* ORC_LIMIT_S (the paper's S) or ORC_LIMIT_S_VOLUME
                         (S and the (k+1)^3 volume Gauss points) */
} orc_params;

enum { ORC_LIMIT_S = 0, ORC_LIMIT_S_VOLUME = 1 };

enum { ORC_FLUX_HLLC = 0, ORC_FLUX_EXACT = 1 };

int orc_nmodes(int k);
void orc_mode_exponents(int k, int32_t* uvw /* 3*N */);
void orc_gauss(int q, double* x, double* w);
void orc_gll(int m, double* x, double* w);
int orc_gll_count(int k);
void orc_basis(int k, const double xi[3], double* phi, double* dphi /* 3*N, may be NULL */);

/* volume Gauss points (physical coordinates), layout [cell][Q^3][3], point
 * index q = a + Q*(b + Q*c) with a along x */
int orc_volume_points(const orc_params* p, double* xyz);
/* w = (1/8) sum_q f(x_q) phi_l(xi_q) omega_q, Sect. 2.3;
 * f layout [cell][5][Q^3] */
int orc_project(const orc_params* p, const double* f, double* w);
/* evaluate the state polynomial of one cell at reference point xi */
void orc_eval(const orc_params* p, const double* w, long cell, const double xi[3], double* U);

void orc_euler_flux(int dir, double gamma, const double* U, double* F);
void orc_hllc(int dir, double gamma, const double* UL, const double* UR, double* F);

/* Exact Riemann solver, the other flux Sect. 2.3 allows after Eq.
 * dg:eqn:surface_int. Primitive states W = (rho, u_normal, p).
 * orc_exact_star: star pressure and velocity; returns ORC_OK, 1 when the
 * two rarefactions open a vacuum (p* = 0, u* undefined), ORC_ERR_NEWTON when
 * the iteration does not converge in 100 steps.
 * orc_exact_sample: the self-similar solution at x/t = s (status as above).
 * orc_exact_flux: Godunov flux across a face with normal +e_dir from the
 * solution at x/t = 0; tangential velocities from the side of the contact. */
int orc_exact_star(double gamma, const double WL[3], const double WR[3], double* pstar, double* ustar);
int orc_exact_sample(double gamma, const double WL[3], const double WR[3], double s, double W[3]);
int orc_exact_flux(int dir, double gamma, const double* UL, const double* UR, double* F);

/* R(w) for all cells (Eqs. dg:eqn:volume_int, dg:eqn:surface_int) */
int orc_rhs(const orc_params* p, const double* w, double* R);
/* R(w) for a list of cells only; R layout [n_cells][5][N] */
int orc_rhs_cells(const orc_params* p, const double* w, long n_cells, const int64_t* cells, double* R);

/* forcing acceleration a(x) at physical points, xyz [n][3] -> a [n][3] */
void orc_forcing_accel(const orc_params* p, long n, const double* xyz, double* a);

/* Zhang-Shu positivity limiter, Sect. 2.5; flags [n_c] (may be NULL),
 * per cell bit0 = theta1<1, bit1 = theta2<1 */
int orc_limit(const orc_params* p, double* w, int8_t* flags, int64_t* n_limited);
int orc_limit_cells(const orc_params* p, double* w, long n_cells, const int64_t* cells, int8_t* flags);
/* tau solving P(qbar + tau (q - qbar)) = eps by Newton from tau = 1 */
double orc_pressure_tau(double gamma, const double* qbar, const double* q, double eps, int* iters);

/* time step by Eq. time_step_pos with the limited cell means */
int orc_cfl_dt(const orc_params* p, const double* w, double courant, double* dt);
/* one SSP-RK3 step (Shu-Osher form) with the limiter at each stage start */
int orc_step(const orc_params* p, double* w, double dt);
/* isothermal energy reset (Sect. 3.2) followed by the limiter */
int orc_energy_reset(const orc_params* p, double* w, double c_iso, double rho0, double* dissipated);
int orc_energy_reset_cells(const orc_params* p, double* w, long n_cells, const int64_t* cells,
                           double c_iso, double rho0);
/* sum_K |K| w_{i,0} */
void orc_totals(const orc_params* p, const double* w, double* out5);

/* Turbulence diagnostics of Sect. 4.1-4.2 (readings of the paper, which
 * gives no formulas): out[0] = volume-weighted rms Mach number of the cell
 * means, sqrt((1/V) sum_K |K| (|m/rho| / c)^2) with c^2 = gamma p / rho from
 * the means; out[1] = kinetic energy of the means, sum_K |K| |m|^2 / (2 rho);
 * out[2] = rate of work of the driving force (injected power),
 * sum_K int_K m . a dV by the volume Gauss rule with the state polynomial
 * (0 without forcing modes). */
void orc_diagnostics(const orc_params* p, const double* w, double* out3);

/* Velocity component comp (0..2) of the state polynomial, m_comp / rho, at
 * the centres of sub^3 equal sub-cells of every cell of a cubic mesh
 * (Sect. 3.3 spectra sample the solution below the cell size): out [M][M][M]
 * with M = n sub, last index along x. */
int orc_sample_velocity(const orc_params* p, const double* w, int sub, int comp, double* out);
/* The density of the state polynomial on the same grid (Sect. 4.4 PDFs). */
int orc_sample_density(const orc_params* p, const double* w, int sub, double* out);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
