/*
 * dg.h -- C ABI of the GB300 (sm_103a) modal discontinuous Galerkin solver
 * for the 3D Euler equations on a periodic Cartesian mesh, following
 * Bauer et al., "Simulating Turbulence Using the Astrophysical Discontinuous
 * Galerkin Code TENET" (arXiv:1602.09079), Sect. 2 (method) and Sect. 3.1-3.2
 * (driving and energy reset).
 *
 * Conventions
 *   order     paper's convergence order O = k + 1 (Sect. 3), 1..4; k is the
 *             polynomial degree, N(k) = (k+1)(k+2)(k+3)/6 modes (Sect. 2.2).
 *   basis     phi_l = Pt_u(xi1) Pt_v(xi2) Pt_w(xi3), u+v+w <= k, with
 *             Pt_u = sqrt(2u+1) P_u so that (1/8) int phi_l phi_m = delta_lm
 *             and w_0 is the cell mean (Sect. 2.1-2.2). Mode order: total
 *             degree ascending, then u descending, then v descending.
 *   variables (rho, rho vx, rho vy, rho vz, E), ideal gas (Sect. 2.3).
 *   canonical layout (exchange format, host or device):
 *             [nz][ny][nx][5][N] doubles, cell (ix,iy,iz) centred at
 *             ((ix+1/2) dx, (iy+1/2) dy, (iz+1/2) dz), box origin at 0.
 *   state layout (the bound state buffer and dg_rhs operands):
 *             [5][N][n_cells] doubles, cells x-fastest (mode-major,
 *             cell-minor: every row is contiguous over cells).
 *   R         right-hand side of Eq. dg:eqn:time, dw/dt + R(w) = 0.
 *
 * Memory: the library never allocates device memory. The caller allocates
 * the state and one scratch buffer (sizes from dg_sizes), binds them with
 * dg_bind, and owns them; they must stay valid while bound.
 *
 * Streams and errors: every call enqueues on the bound CUDA stream and
 * returns without synchronising, except the calls that return host values
 * (dg_cfl_dt, dg_totals, dg_diagnostics, dg_velocity_spectrum,
 * dg_density_pdf, dg_limit with n_limited, dg_energy_reset with dissipated,
 * dg_get_state to host, dg_indicator_capture, dg_limiter_counts,
 * dg_kernel_stats, dg_check), which synchronise the stream.
 * Conditions found on the device (non-finite values, a cell mean below the
 * positivity floor, Newton non-convergence in the limiter) set a sticky
 * device error word that the next synchronising call reports and clears.
 * All functions return DG_OK (0) or a negative DG_ERR_* code and never
 * throw across the ABI. Functions are not thread-safe on one context.
 */
#ifndef DG_GB300_H
#define DG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DG_OK 0
#define DG_ERR_ARG -1          /* invalid argument or state */
#define DG_ERR_NOT_BOUND -2    /* no state/scratch bound */
#define DG_ERR_CUDA -3         /* a CUDA runtime call failed */
#define DG_ERR_NONFINITE -4    /* NaN/Inf found in the state */
#define DG_ERR_POSITIVITY -5   /* a cell mean density or pressure below eps */
#define DG_ERR_NEWTON -6       /* a Newton iteration (limiter or exact flux) did not converge */
#define DG_ERR_TOO_LARGE -7    /* problem exceeds dg_rhs_noalloc's fixed scratch */

#define DG_PREC_FP64 0   /* every step in FP64 */
#define DG_PREC_MIXED 1  /* quadrature, fluxes and projection in FP32; RK
                            accumulation, limiter, CFL and sums in FP64 */

#define DG_FEATURE_FORCING 1  /* scratch sized for the driving field */

typedef struct {
  int32_t n[3];      /* cells per axis, each >= 1 */
  double length[3];  /* periodic box lengths, each > 0 */
} dg_mesh;

typedef struct dg_ctx dg_ctx; /* opaque, owned by the library */

/* Human-readable text of a status code (static storage). */
const char* dg_strerror(int code);

/* Create a context for a mesh, order O = k+1 in 1..4 (Sect. 3) and adiabatic
 * index gamma > 1 (Sect. 2.3). Uploads the basis/quadrature tables to the
 * current device. Positivity floors default to 1e-12, precision to FP64.
 * Errors: DG_ERR_ARG for bad arguments, DG_ERR_CUDA. */
int dg_init(const dg_mesh* mesh, int order, double gamma, dg_ctx** out);

/* Destroy a context (does not free bound buffers). NULL is ignored. */
void dg_destroy(dg_ctx* ctx);

/* Sizes the caller must allocate: state_len doubles for the state
 * (5 N n_cells) and scratch_bytes bytes of device scratch; features is a
 * bit set of DG_FEATURE_*. */
int dg_sizes(const dg_ctx* ctx, int features, size_t* state_len, size_t* scratch_bytes);

/* Bind caller-owned device buffers and a CUDA stream (cudaStream_t, NULL =
 * legacy default stream). y_dev: state layout, 5 N n_cells doubles, 8-byte
 * aligned; scratch_dev: at least dg_sizes(ctx, 0, ...) bytes, 256-byte
 * aligned; a scratch of dg_sizes(ctx, DG_FEATURE_FORCING, ...) bytes enables
 * dg_set_forcing. Errors: DG_ERR_ARG (NULL, misaligned, too small). */
int dg_bind(dg_ctx* ctx, double* y_dev, void* scratch_dev, size_t scratch_bytes, void* cuda_stream);

/* Copy a canonical-layout state (host if is_device == 0, else device) into
 * the bound state. Marks the state as not yet limited. */
int dg_set_state(dg_ctx* ctx, const double* src, int is_device);

/* Copy the bound state out in canonical layout (host or device). */
int dg_get_state(dg_ctx* ctx, double* dst, int is_device);

/* Physical coordinates of the volume Gauss points, written to host memory
 * as [n_cells][Q^3][3] with Q = k+1 and point index a + Q (b + Q c)
 * (a along x). These are the points at which dg_project expects values. */
int dg_quadrature_points(const dg_ctx* ctx, double* xyz_host);

/* The same for the cells first .. first + count - 1 only (xyz_host holds
 * count * Q^3 * 3 doubles), for meshes whose points do not fit at once. */
int dg_quadrature_points_range(const dg_ctx* ctx, int64_t first, int64_t count, double* xyz_host);

/* Initial L2 projection (Sect. 2.3, w_l = 1/8 sum_q q(x_q) phi_l(xi_q)
 * omega_q): q_points_dev holds conserved variables at the points of
 * dg_quadrature_points, device memory, layout [n_cells][5][Q^3]. Writes the
 * bound state (no limiting). */
int dg_project(dg_ctx* ctx, const double* q_points_dev);

/* dg_project for the cells first .. first + count - 1 (q_points_dev holds
 * their count * 5 * Q^3 values); the other cells are left as they are. */
int dg_project_range(dg_ctx* ctx, const double* q_points_dev, int64_t first, int64_t count);

/* R(y) of Eq. dg:eqn:time: volume integral (Eq. dg:eqn:volume_int) plus
 * surface integral with the numerical flux set by dg_set_flux (HLLC by
 * default; Eq. dg:eqn:surface_int),
 * divided by |K| (Eq. dg:eqn:time_deriv, orthonormal basis), plus the
 * driving source (Sect. 3.1) when set. y_dev and R_dev are device buffers in
 * the state layout; y_dev == NULL means the bound state. No limiting. Uses
 * the current precision mode; R is written in FP64. */
int dg_rhs(dg_ctx* ctx, const double* y_dev, double* R_dev);

/* One SSP-RK3 step (Sect. 2.4, Shu-Osher form) of size dt > 0 on the bound
 * state, in place, with the positivity limiter (Sect. 2.5) applied to the
 * state at the start of every stage; the state left behind is limited (it is
 * the start of the next step's first stage). */
int dg_step(dg_ctx* ctx, double dt);

/* Positivity limiter (Sect. 2.5) on the bound state in place: theta1 from
 * the density minimum over S = S_x u S_y u S_z (m GLL x (k+1)^2 Gauss points
 * per direction), then theta2 from the pressure via Newton-Raphson for tau
 * in P(qbar + tau (q - qbar)) = eps. flags_dev (nullable, device, n_cells
 * int8): bit0 theta1 < 1, bit1 theta2 < 1. n_limited (nullable, host):
 * number of limited cells; non-NULL synchronises. */
int dg_limit(dg_ctx* ctx, int8_t* flags_dev, int64_t* n_limited);

/* Global time step by Eq. time_step_pos: min over cells of
 * C min(1/(2k+1), w1/2) / sum_a (|v_a| + c)/dx_a from the cell means, with
 * w1 the first GLL weight. Synchronises; reports device errors. */
int dg_cfl_dt(dg_ctx* ctx, double courant, double* dt_out);

/* DG_PREC_FP64 or DG_PREC_MIXED. */
int dg_set_precision(dg_ctx* ctx, int mode);

/* Point set of the positivity limiter (Sect. 2.5, which asks that it
 * contain every point where fluxes are evaluated): DG_LIMIT_S (default) is
 * S = S_x u S_y u S_z as the paper writes it, which covers the face
 * quadrature points but not the interior volume Gauss points;
 * DG_LIMIT_S_VOLUME adds the (k+1)^3 volume Gauss points (theta1 and theta2
 * over the union, and the screens use max |phi_l| over the union). Any other
 * value: DG_ERR_ARG. The next dg_step limits its input again. */
#define DG_LIMIT_S 0
#define DG_LIMIT_S_VOLUME 1
int dg_set_limiter_points(dg_ctx* ctx, int mode);

/* Numerical flux of the surface integral (Sect. 2.3, Eq.
 * dg:eqn:surface_int, which allows an exact or an approximate HLLC Riemann
 * solver): DG_FLUX_HLLC (default; Einfeldt wave speeds) or DG_FLUX_EXACT
 * (Godunov flux of the exact Riemann solution, star pressure by Newton's
 * method, at most 50 iterations; a face point whose FP64 iteration does not
 * converge makes the next synchronising call return DG_ERR_NEWTON). Any
 * other value: DG_ERR_ARG. Applies to dg_rhs, dg_step and the indicator
 * capture from the next call on. */
#define DG_FLUX_HLLC 0
#define DG_FLUX_EXACT 1
int dg_set_flux(dg_ctx* ctx, int flux);

/* Positivity floors for density and pressure (Sect. 2.5 "minimum target
 * density"), both > 0. */
int dg_set_eps(dg_ctx* ctx, double eps_rho, double eps_p);

/* Driving acceleration a(x) = sum_j Re(ahat_j exp(i k_j . x)),
 * k_j = 2 pi n_j / L (Sect. 3.1), added as the source (0, rho a, m . a) at
 * the volume points of every stage. nvec_host: 3 n_modes int32 wave numbers;
 * ahat_host: 6 n_modes doubles (Re a_x, a_y, a_z, Im a_x, a_y, a_z).
 * n_modes = 0 switches the driving off. n_modes <= 256. Needs a scratch
 * sized with DG_FEATURE_FORCING (else DG_ERR_ARG). */
int dg_set_forcing(dg_ctx* ctx, int n_modes, const int32_t* nvec_host, const double* ahat_host);

/* Isothermal energy reset (Sect. 3.2): at every volume point enforce
 * eps = c^2/(gamma-1) (rho/rho0)^(gamma-1), re-project the energy weights
 * from 1/2 |m|^2/rho + rho eps, then apply the positivity limiter.
 * dissipated (nullable, host): sum over cells of |K| times the drop of the
 * mean internal energy density; non-NULL synchronises. */
int dg_energy_reset(dg_ctx* ctx, double c_iso, double rho0, double* dissipated);

/* Conserved totals sum_K |K| w_{i,0}, i = 0..4, in FP64 (host out[5]).
 * Synchronises. */
int dg_totals(dg_ctx* ctx, double* out5);

/* Turbulence diagnostics of the bound state (Sect. 4.1, rms Mach number;
 * Sect. 4.2, injected energy; the paper gives no formulas, these are the
 * readings): out3[0] = volume-weighted rms Mach number of the cell means,
 * sqrt((1/V) sum_K |K| (|m|/rho / c)^2), c^2 = gamma p / rho from the means;
 * out3[1] = kinetic energy of the cell means, sum_K |K| |m|^2 / (2 rho);
 * out3[2] = power of the driving force, sum_K int_K m . a dV by the volume
 * Gauss rule on the state polynomial and the cached driving field (0 without
 * forcing); the energy it injects over a step of size dt is about
 * out3[2] dt. Host array of 3 doubles. Synchronises; reports device errors. */
int dg_diagnostics(dg_ctx* ctx, double* out3);

/* Velocity power spectrum of the bound state (Sect. 3.3): the velocity
 * m/rho of the state polynomial is sampled at the centres of sub^3 equal
 * sub-cells of every cell (an M^3 grid, M = n sub), each component is
 * transformed by a 3D real-to-complex FFT (cuFFT), and the power of every
 * integer wave vector n (k = 2 pi n / L) is added to shell round(|n|):
 * spectrum[b] = sum_{round(|n|) = b} |v_hat(n)|^2 / M^6 over the three
 * components, so that sum_b spectrum[b] = mean |v|^2 over the samples (the
 * normalisation that makes the spectrum integrate to the total, as the
 * paper asks). Cubic meshes of a cubic box only (else DG_ERR_ARG); 1 <= sub
 * <= 8. dg_spectrum_sizes gives the device work-area bytes the caller
 * allocates (bins, one real grid, one complex half spectrum, cuFFT's work
 * area; DG_ERR_TOO_LARGE if cuFFT cannot plan the size) and the number of
 * bins, floor(sqrt(3) M / 2) + 2. spectrum: host array of n_bins doubles.
 * Synchronises. */
int dg_spectrum_sizes(const dg_ctx* ctx, int sub, size_t* work_bytes, int* n_bins);
int dg_velocity_spectrum(dg_ctx* ctx, int sub, void* work_dev, size_t work_bytes, double* spectrum);

/* Volume-weighted density PDF of the bound state (Sect. 4.4 density PDFs):
 * counts of s = ln(rho) of the state polynomial at the centres of sub^3
 * equal sub-cells of every cell (cubic mesh of a cubic box, 1 <= sub <= 8)
 * in n_bins (1..4096) equal bins of [lo, hi): counts[1 + j] for
 * floor((s - lo) / (hi - lo) n_bins) = j, counts[0] below lo (and samples
 * whose density is not positive and finite), counts[n_bins + 1] at or above
 * hi; host array of n_bins + 2 int64. Uses the bound scratch; synchronises. */
int dg_density_pdf(dg_ctx* ctx, int sub, double lo, double hi, int n_bins, long long* counts);

/* Synchronise the bound stream and report (and clear) the device error
 * word. */
int dg_check(dg_ctx* ctx);

/* ---- measurement aids (no counterpart in the paper) --------------------
 * Kernel classes: 0 limiter, 1 face flux, 2 volume (RHS or fused stage),
 * 3 CFL reduction, 4 energy reset, 5 other (layout, projection, sums). */
#define DG_KCLASS_COUNT 6

/* When on != 0, every kernel the context launches is bracketed by CUDA
 * events recorded on the bound stream (adds two event records per launch). */
int dg_set_timing(dg_ctx* ctx, int on);

/* Per class: kernel launches since the last call (always counted; the
 * queued limiter's two passes count as two) and, if timing was on, their
 * summed device time in ms (0 otherwise). Synchronises the
 * stream; resets the counters. Arrays of DG_KCLASS_COUNT entries, either may
 * be NULL. */
int dg_kernel_stats(dg_ctx* ctx, int64_t* launches, double* ms);

/* ---- learned troubled-cell indicator -----------------------------------
 * No counterpart in the paper: a small network that predicts, per cell, the
 * flag of the positivity limiter's indicator (Sect. 2.5: the polynomial
 * leaves the positive set on S). Inputs per cell: the high modes scaled by the
 * cell means, log(rho), the mean Mach number, the five excursion bounds
 * sum_{l>=1} |w_il| max_S |phi_l| / s_i, and the 26 neighbour means relative
 * to the cell's (in that order: own modes variable-major, the two scalars,
 * the bounds, then neighbours (dz,dy,dx) lexicographic in
 * {-1,0,1}^3 without the centre, variable-minor), zero-padded to a multiple
 * of 32, in BF16. Network F -> 64 -> 64 -> 1 (ReLU, sigmoid); parameters FP32,
 * flat: W1[64][F], b1[64], W2[64][64], b2[64], w3[64], b3. Orders 2..4. */

/* Feature count, padded width F, parameter count, and the work-buffer bytes
 * dg_indicator_backward needs. */
int dg_indicator_sizes(int order, int* n_features, int* n_padded, size_t* n_params, size_t* work_bytes);

/* Features of every cell of a state (state layout; NULL = the bound state)
 * into X_dev, BF16 [n_cells][F], on the bound stream. */
int dg_indicator_features(dg_ctx* ctx, const double* y_dev, uint16_t* X_dev);

/* logits_dev[r] = network(X_dev[r]) for r < n (FP32), on cuda_stream. */
int dg_indicator_forward(int order, const uint16_t* X_dev, int64_t n, const float* params_dev, float* logits_dev,
                         void* cuda_stream);

/* Gradient of the class-weighted binary cross entropy
 * (1/n) sum_r [pos_weight y_r softplus(-z_r) + (1 - y_r) softplus(z_r)]
 * with respect to every parameter into grads_dev (n_params floats), the loss
 * in grads_dev[n_params]. labels_dev: n floats in {0, 1}. work_dev: at least
 * work_bytes (dg_indicator_sizes). Deterministic (fixed reduction order). */
int dg_indicator_backward(int order, const uint16_t* X_dev, const float* labels_dev, int64_t n, float pos_weight,
                          const float* params_dev, float* grads_dev, void* work_dev, size_t work_bytes,
                          void* cuda_stream);

/* Gate the full positivity limiter with the indicator (params_dev: FP32
 * parameters, caller-owned, valid while set; NULL switches the gate off).
 * In every stage of dg_step, cells that fail the limiter's screen (the
 * plain indicator's cheap sufficient test) are evaluated by the network;
 * only those with probability >= threshold (0 < threshold < 1) go through
 * the full limiter. The limiter itself is unchanged; cells the network
 * passes over are not limited (its misses). */
int dg_set_indicator(dg_ctx* ctx, const float* params_dev, float threshold);

/* Training data from the bound state: one unlimited forward-Euler stage
 * y1 = y - dt R(y) (current precision), its features (X_dev, BF16
 * [n_cells][F]), whether each cell fails the limiter screen (screen_dev,
 * uint8 0/1) and the limiter's flags on y1 (flags_dev, int8: bit0 theta1 < 1,
 * bit1 theta2 < 1). The bound state is unchanged. Synchronises. */
int dg_indicator_capture(dg_ctx* ctx, double dt, uint16_t* X_dev, int8_t* flags_dev, uint8_t* screen_dev);

/* Limiter work since the last call (synchronises, then resets): cells that
 * failed the screen in any stage of dg_step, and cells that went through the
 * full limiter (equal without an indicator). */
int dg_limiter_counts(dg_ctx* ctx, int64_t* queued, int64_t* full);

/* One Adam step (bias-corrected, step >= 1) on FP32 params with moments m, v. */
int dg_indicator_adam(float* params, float* m, float* v, const float* grads, int64_t n_params, float lr,
                      float beta1, float beta2, float eps, int step, void* cuda_stream);

/* ---- allocation-free entry point (no counterpart in the paper) ---------
 * R(y) as dg_rhs computes it (no driving source), for
 * callers that must not allocate device memory themselves: code whose device
 * memory is owned and budgeted by a host application or another framework's
 * allocator, where a cudaMalloc (or the implicit synchronisation of a
 * cudaFree) is not allowed during the run. Instead of a caller-allocated
 * scratch, the face fluxes go to one fixed array in device memory,
 * DG_NOALLOC_SCRATCH_BYTES = 32 MiB, that every GPU which loads the library
 * holds until the process exits. Needs 15 (k+1)^2 n_cells x 8 bytes (FP64)
 * or (15 (k+1)^2 + 5 N) n_cells x 4 bytes (DG_PREC_MIXED), plus 512: e.g. at
 * most 31,000 cells at order 3 in FP64; larger problems return
 * DG_ERR_TOO_LARGE.
 * mesh/order/gamma as in dg_init; precision DG_PREC_FP64 or DG_PREC_MIXED;
 * y_dev (input) and R_dev (output): device, state layout, 5 N n_cells doubles;
 * cuda_stream: cudaStream_t (NULL = legacy default stream), enqueued without
 * synchronising. No context, no dg_bind, no cudaMalloc/cudaFree or any
 * allocating library call. The first call on a device looks up the array's
 * device address and uploads the basis tables of that order (a synchronous
 * copy), so make the first call for each device and order before any stream
 * capture. All calls share the one array: calls that overlap on the GPU (on
 * different streams, or from several threads) race on it; serialise them.
 * The array keeps the last call's contents; every entry a call reads is
 * written by the same call first, and each call clears the array's control
 * block (error bits) on the stream before its kernels run.
 * The numerical flux is always HLLC (there is no context, so dg_set_flux
 * does not apply). FP64: the kernels of dg_rhs, same results. DG_PREC_MIXED:
 * the separate FP32 face and volume kernels, within FP32 rounding of
 * dg_rhs (which runs the fused stage kernel at degree 2).
 * Device-side errors are not reported: a non-finite y gives a non-finite R
 * and DG_OK, so check R where that matters; the return value covers the
 * arguments, the size limit and CUDA launch errors only. */
#define DG_NOALLOC_SCRATCH_BYTES (32u << 20)
int dg_rhs_noalloc(const dg_mesh* mesh, int order, double gamma, int precision, const double* y_dev,
                   double* R_dev, void* cuda_stream);

/* Dense FMA throughput of the current device in FLOP/s (fp64 != 0: FP64,
 * else FP32), measured by a register-resident FMA loop over all SMs timed
 * with CUDA events; takes tens of milliseconds. */
int dg_probe_fma_peak(int fp64, double* flops_per_s);

/* Self-test of the library's integer-pipe IEEE 754 conversions (binary64 ->
 * binary32 round-to-nearest-even, binary32 -> binary64, finite test), which
 * the FP32 path's FP64 stage epilogue uses, against the hardware conversions
 * on n generated values (raw bit patterns, rounding ties and their
 * neighbours, exponents at the binary32 range edges; seed selects them). No
 * counterpart in the paper. *mismatches (host) receives the number of
 * differing results (0 expected). Allocates 8 bytes of device memory for the
 * duration of the call; synchronises. */
int dg_selftest_conversions(long long n, unsigned long long seed, long long* mismatches);

#ifdef __cplusplus
}
#endif
#endif
