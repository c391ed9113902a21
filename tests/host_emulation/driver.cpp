// driver.cpp -- runs the library's DG kernels (dg_kernels.cuh, degree DG_K)
// under the host emulation of emu.h, launched with the grid, block and
// shared-memory sizes of the library's launchers and in the order the C ABI
// issues them (test infrastructure).
//
//   driver rhs  nx ny nz prec gamma in.bin out.bin [flux]
//       R(y): face kernel, then the volume kernel in MODE_RHS (no driving)
//   driver step nx ny nz prec gamma in.bin out.bin dt n_modes modes.bin c_iso rho0 lim_vol [flux]
//       one dg_step (limiter of the input, three stages of face kernel,
//       fused volume/stage kernel and queued limiter, with the driving field
//       when n_modes > 0), then dg_energy_reset and the CFL reduction
//
//   driver analysis n gamma in.bin out.bin sub lo hi nb n_modes modes.bin spec.bin
//       diagnostics, spectrum sampling and shell sums, density histogram
//   driver limit nx ny nz gamma eps lim_vol in.bin out.bin flags.bin
//       dg_limit with per-cell flags
//   driver project nx ny nz gamma first count f.bin out.bin
//       dg_project_range
//   driver layout nx ny nz in.bin out.bin
//       canonical <-> state transposes and the conserved totals
//   driver hllc|exact d gamma UL0..UL4 UR0..UR4
//       the FP32 and FP64 HLLC (or exact-Riemann) fluxes of one face point
//
// prec: 0 FP64, 1 mixed; flux: 0 HLLC (default), 1 exact Riemann solver.
// Degrees 2 and 3 in mixed precision run the fused stage kernel (dg_fused.cuh) as
// the library does; DG_EMU_FUSED=0 in the environment selects the separate
// face and volume kernels instead.
// States in the state layout [5][N][n_cells], FP64.
// Prints "err=<device error word> dissipated=<...> smax=<...>".
#include <type_traits>

#include "dg_kernels.cuh"
#if DG_K >= 2
#include "dg_fused.cuh"
#endif
using namespace dg;
#include "tables.inc"
namespace dg {
namespace spec {
#include "spectrum_kernels.inc"
}  // namespace spec
}  // namespace dg
namespace api {
#include "api_kernels.inc"
}  // namespace api

constexpr int K = DG_K;
using TB = Tab<K>;

static unsigned grid1(long long n, int per) { return (unsigned)((n + per - 1) / per); }

struct Setup {
  std::vector<double> t64;
  std::vector<float> t32;
  Geo g{};
  Ctrl ctrl{};
  long long nc = 0;
};

// the tables as dg_init uploads them (device copies and constant banks)
static void make_setup(Setup& S, int nx, int ny, int nz, double gamma, int lim_vol) {
  S.t64.assign(TAB_STRIDE, 0.0);
  build_tables<K>(S.t64.data());
  S.t32.resize(TAB_STRIDE);
  for (int i = 0; i < TAB_STRIDE; ++i) S.t32[i] = (float)S.t64[i];
  for (int i = 0; i < TB::SIZE; ++i) c_tab32[i] = S.t32[i];
  constexpr int KQ = (K + 1) * (K + 1), NSF = 3 * KQ + 2 * (K + 1);
  for (int i = 0; i < KQ; ++i) {
    c_sf64[i] = S.t64[TB::P1 + i];
    c_sf64[KQ + i] = S.t64[TB::P1W + i];
    c_sf64[2 * KQ + i] = S.t64[TB::D1W + i];
  }
  for (int i = 0; i < 2 * (K + 1); ++i) c_sf64[3 * KQ + i] = S.t64[TB::FEND + i];
  for (int i = 0; i < NSF; ++i) c_sf32[i] = (float)c_sf64[i];
  S.nc = (long long)nx * ny * nz;
  Geo& g = S.g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.nc = S.nc;
  const int n3[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    g.dx[a] = 1.0 / n3[a];
    g.inv_dx[a] = 1.0 / g.dx[a];
  }
  g.gamma = gamma;
  g.eps_rho = 1e-12;
  g.eps_p = 1e-12;
  g.lim_vol = lim_vol;
}

// numerical flux: 0 HLLC, 1 exact Riemann solver (dg_set_flux)
static int g_flux = 0;

static bool use_fused() {
#if DG_K >= 2
  const char* e = std::getenv("DG_EMU_FUSED");
  return !(e && e[0] == '0');
#else
  return false;
#endif
}

#if DG_K >= 2
// the fused kernel's 1D tables (as its upload builds them) and one launch
// with the launcher's grid and planes per segment
static void fused_setup(const Setup& S) {
  using FT = FzTab<K>;
  constexpr int KQ = (K + 1) * (K + 1);
  for (int j = 0; j < KQ; ++j) {
    c_fz[FT::P + j] = (float)S.t64[TB::P1 + j];
    c_fz[FT::PW + j] = (float)S.t64[TB::P1W + j];
    c_fz[FT::DW + j] = (float)S.t64[TB::D1W + j];
  }
  for (int e = 0; e <= K; ++e) {
    c_fz[FT::EM + e] = (float)S.t64[TB::FEND + e];
    c_fz[FT::EP + e] = (float)S.t64[TB::FEND + K + 1 + e];
  }
  for (int l = 0; l < TB::N; ++l) {
    c_fz[FT::LM + l] = (float)S.t64[TB::LMAX + l];
    c_fz[FT::LMV + l] = (float)S.t64[TB::LMAXV + l];
  }
}

template <bool FORCE>
static void fused_launch(Setup& S, FusedArgs a) {
  using FC = FusedCfg<K>;
  a.nbx = (S.g.nx + FC::BX - 1) / FC::BX;
  a.nby = (S.g.ny + FC::BY - 1) / FC::BY;
  // the launcher's choice for meshes that fit one wave: the smallest
  // candidate, 4 planes per segment
  a.lz = 4;
  a.eps_r = (float)S.g.eps_rho;
  a.eps_p = (float)S.g.eps_p;
  const unsigned grid = (unsigned)(a.nbx * a.nby * ((S.g.nz + a.lz - 1) / a.lz));
  a.ctrl = &S.ctrl;
  if (g_flux) emu::launch(grid, FC::THREADS, FC::smem(), [&] { fused_f32_kernel<K, FORCE, 1>(S.g, a); });
  else emu::launch(grid, FC::THREADS, FC::smem(), [&] { fused_f32_kernel<K, FORCE, 0>(S.g, a); });
}
#endif

// face fluxes of the state ys (FP32 path: of its shadow yf)
template <typename T, int FLUX>
static void faces_f(Setup& S, const double* ys, float* yf, T* fh) {
  if constexpr (sizeof(T) == 4)
    emu::launch(grid1(S.nc, 32), 96, 0, [&] { face_flux_f32_kernel<K, FLUX>(yf, fh, S.g, &S.ctrl); });
  else
    emu::launch(grid1(S.nc, 32), FaceSF64<K>::THREADS, FaceSF64<K>::smem(),
                [&] { face_sf64_kernel<K, FLUX>(ys, fh, S.g, &S.ctrl); });
}
template <typename T>
static void faces(Setup& S, const double* ys, float* yf, T* fh) {
  if (g_flux) faces_f<T, 1>(S, ys, yf, fh);
  else faces_f<T, 0>(S, ys, yf, fh);
}

// the volume kernel the launchers pick for (T, K) in MODE
template <typename T, int MODE, bool FORCE>
static void volume(Setup& S, const double* ys, float* yf, const T* fh, const T* field, StageArgs st, double* R) {
  const long long nc = S.nc;
  if constexpr (sizeof(T) == 4 && K <= 2) {
    using CF = VolF32<K>;
    emu::launch(grid1(nc, CF::C), CF::THREADS, CF::smem(FORCE), [&] {
      volume_f32_kernel<K, MODE, FORCE>(yf, fh, field, S.t64.data(), S.g, st, R, &S.ctrl);
    });
  } else if constexpr (sizeof(T) == 4) {
    using CF = VolSF<K, float>;
    emu::launch(grid1(nc, CF::C), kThreads, CF::smem(), [&] {
      volume_sfb_kernel<K, float, MODE, FORCE>(ys, yf, fh, field, S.t32.data(), S.t64.data(), S.g, st, R, &S.ctrl);
    });
  } else if constexpr (K >= 2) {
    using CF = VolSF<K, double>;
    emu::launch(grid1(nc, CF::C), kThreads, CF::smem(), [&] {
      volume_sf_kernel<K, double, MODE, FORCE>(ys, nullptr, fh, field, S.t64.data(), S.t64.data(), S.g, st, R,
                                               &S.ctrl);
    });
  } else {
    using CF = VolCfg<K, double>;
    emu::launch(grid1(nc, CF::C), kThreads, CF::smem(FORCE), [&] {
      volume_kernel<K, double, MODE, FORCE>(ys, fh, field, S.t64.data(), S.t64.data(), S.g, st, R, &S.ctrl);
    });
  }
}

template <typename T>
static void run_rhs(Setup& S, std::vector<double>& y, std::vector<double>& R) {
#if DG_K >= 2
  if (sizeof(T) == 4 && use_fused()) {
    fused_setup(S);
    FusedArgs a{};
    a.ys = y.data();
    a.R = R.data();
    a.stage = 0;
    fused_launch<false>(S, a);
    std::printf("err=%u dissipated=0 smax=0\n", S.ctrl.err);
    return;
  }
#endif
  std::vector<float> yf(sizeof(T) == 4 ? y.size() : 1);
  if (sizeof(T) == 4)
    for (size_t i = 0; i < y.size(); ++i) yf[i] = (float)y[i];  // the library's shadow: round to nearest
  std::vector<T> fh((size_t)15 * TB::Q2 * S.nc, T(std::nan("")));
  faces<T>(S, y.data(), yf.data(), fh.data());
  StageArgs st{};
  volume<T, MODE_RHS, false>(S, y.data(), sizeof(T) == 4 ? yf.data() : nullptr, fh.data(), nullptr, st, R.data());
  std::printf("err=%u dissipated=0 smax=0\n", S.ctrl.err);
}

// the full limiter on the queued cells as the C ABI runs it: the screen pass
// queues the cells that need the FP64 point evaluations into deep, the
// second pass limits them
static void limit_queued(Setup& S, double* y, const int* list, int count_queued, float* yf, const double* y0,
                         float* dinc, std::vector<int>& deep) {
  S.ctrl.n_deep = 0;
  emu::launch(4, ListLim<K>::THREADS, ListLim<K>::smem(), [&] {
    limit_screen_list_kernel<K>(y, list, &S.ctrl.n_flag, S.t64.data(), S.t32.data(), S.g, &S.ctrl, count_queued,
                                deep.data());
  });
  emu::launch(4, ListLim<K>::THREADS, ListLim<K>::smem(), [&] {
    limit_list_kernel<K>(y, deep.data(), &S.ctrl.n_deep, S.t64.data(), S.g, &S.ctrl, yf, y0, dinc);
  });
}

template <typename T>
static void run_step(Setup& S, std::vector<double>& y, double dt, const std::vector<double>& modes, int nm,
                     double c_iso, double rho0) {
  const long long nc = S.nc;
  const bool force = nm > 0;
  std::vector<T> field(force ? (size_t)3 * TB::Q3 * nc : 1, T(std::nan("")));
  if (force)
    emu::launch2(grid1(nc, kThreads), TB::Q3, kThreads, 0, [&] {
      forcing_field_kernel<K, T>(field.data(), modes.data(), nm, S.t64.data(), S.g, 1.0, 1.0, 1.0);
    });
  const T* fld = force ? field.data() : nullptr;
  emu::launch(grid1(nc, kThreads), kThreads, 0,
              [&] { limit_kernel<K>(y.data(), nullptr, S.t64.data(), S.g, &S.ctrl, S.t32.data()); });
  const bool shadow = sizeof(T) == 4;
  std::vector<float> yf(shadow ? y.size() : 1);
  if (shadow)
    for (size_t i = 0; i < y.size(); ++i) yf[i] = (float)y[i];
  float* yfp = shadow ? yf.data() : nullptr;
  std::vector<T> fh((size_t)15 * TB::Q2 * nc, T(std::nan("")));
  std::vector<double> ybuf(y.size(), std::nan(""));
  std::vector<int> list(nc, -1), deep(nc, -1);
  const double a0[3] = {0.0, 0.75, 1.0 / 3.0}, b0[3] = {1.0, 0.25, 2.0 / 3.0};
  const double* ys = y.data();
#if DG_K >= 2
  if (shadow && use_fused()) {
    // the C ABI's fused step: y -> ybuf -> ybuf2 -> y with the FP32
    // increment of the step; the limiter recomputes it for changed cells
    fused_setup(S);
    std::vector<double> ybuf2(y.size(), std::nan(""));
    std::vector<float> dinc(y.size(), std::nanf(""));
    for (int s = 0; s < 3; ++s) {
      double* out = s == 0 ? ybuf.data() : (s == 1 ? ybuf2.data() : y.data());
      FusedArgs a{};
      a.ys = ys;
      a.out = out;
      a.d = dinc.data();
      a.yf = s == 2 ? yfp : nullptr;
      a.field = reinterpret_cast<const float*>(fld);
      a.list = list.data();
      a.b0dt = (float)(b0[s] * dt);
      a.a0 = (float)a0[s];
      a.b0dt_d = b0[s] * dt;
      a.a0_d = a0[s];
      a.b0_d = b0[s];
      a.y0 = y.data();
      a.stage = s + 1;
      S.ctrl.n_flag = 0;
      if (force) fused_launch<true>(S, a);
      else fused_launch<false>(S, a);
      limit_queued(S, out, list.data(), 1, s == 2 ? yfp : nullptr, s < 2 ? y.data() : nullptr,
                   s < 2 ? dinc.data() : nullptr, deep);
      ys = out;
    }
  } else
#endif
  for (int s = 0; s < 3; ++s) {
    double* out = s < 2 ? ybuf.data() : y.data();
    faces<T>(S, ys, yfp, fh.data());
    S.ctrl.n_flag = 0;
    StageArgs st{ys, y.data(), out, a0[s], b0[s], dt, list.data(), yfp};
    if (force) volume<T, MODE_STAGE, true>(S, ys, yfp, fh.data(), fld, st, nullptr);
    else volume<T, MODE_STAGE, false>(S, ys, yfp, fh.data(), fld, st, nullptr);
    limit_queued(S, out, list.data(), 1, yfp, nullptr, nullptr, deep);
    ys = out;
  }
  // energy reset (the shadow stays current on the mixed path) and its limiter
  S.ctrl.n_flag = 0;
  const unsigned nbr = grid1(nc, 32);
  std::vector<double> part(nbr, 0.0);
  ResetConsts<T> rc;
  rc.c2g = (T)(c_iso * c_iso / (S.g.gamma - 1.0));
  rc.inv_rho0 = (T)(1.0 / rho0);
  rc.gm1 = (T)(S.g.gamma - 1.0);
  rc.two_thirds = std::fabs(S.g.gamma - 1.0 - 2.0 / 3.0) < 1e-15 ? 1 : 0;
  const T* tabT = sizeof(T) == 8 ? (const T*)(const void*)S.t64.data() : (const T*)(const void*)S.t32.data();
  emu::launch(nbr, ResetSF<K, T>::THREADS, ResetSF<K, T>::smem(), [&] {
    energy_reset_sf_kernel<K, T>(y.data(), tabT, S.g, rc, part.data(), list.data(), &S.ctrl, yfp);
  });
  limit_queued(S, y.data(), list.data(), 0, yfp, nullptr, nullptr, deep);
  double diss = 0.0;
  for (unsigned b = 0; b < nbr; ++b) diss += part[b];
  diss *= S.g.dx[0] * S.g.dx[1] * S.g.dx[2];
  S.ctrl.cfl_max_bits = 0;
  emu::launch(grid1(nc, kCflThreads), kCflThreads, 0, [&] { cfl_kernel<K>(y.data(), S.g, &S.ctrl); });
  double smax;
  std::memcpy(&smax, &S.ctrl.cfl_max_bits, 8);
  std::printf("err=%u dissipated=%.17g smax=%.17g\n", S.ctrl.err, diss, smax);
}

// diagnostics partial sums (dg_diagnostics): out3 as the C ABI returns it
template <typename T>
static void run_diag(Setup& S, const std::vector<double>& y, const std::vector<double>& modes, int nm, double* out3) {
  const long long nc = S.nc;
  std::vector<T> field(nm > 0 ? (size_t)3 * TB::Q3 * nc : 1, T(0));
  if (nm > 0)
    emu::launch2(grid1(nc, kThreads), TB::Q3, kThreads, 0, [&] {
      forcing_field_kernel<K, T>(field.data(), modes.data(), nm, S.t64.data(), S.g, 1.0, 1.0, 1.0);
    });
  const long long nb = (nc + 255) / 256;
  const int G = (int)(nb < 1024 ? nb : 1024);
  std::vector<double> part((size_t)3 * G, std::nan(""));
  emu::launch(G, 256, 0, [&] {
    diag_partial_kernel<K, T>(y.data(), field.data(), S.t64.data(), S.g, nm > 0 ? 1 : 0, part.data());
  });
  const double vol = S.g.dx[0] * S.g.dx[1] * S.g.dx[2];
  double h[3] = {0, 0, 0};
  for (int j = 0; j < 3; ++j)
    for (int b = 0; b < G; ++b) h[j] += part[(size_t)j * G + b];
  out3[0] = std::sqrt(h[0] * vol);
  out3[1] = h[1] * vol;
  out3[2] = h[2] * vol;
}

static bool read_file(const char* path, double* p, size_t n) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  const bool ok = std::fread(p, 8, n, f) == n;
  std::fclose(f);
  return ok;
}

// driver hllc d gamma UL0..UL4 UR0..UR4: the FP32 and FP64 HLLC fluxes
// (driver exact ...: the exact-Riemann-solver fluxes)
static int run_hllc(int argc, char** argv) {
  if (argc != 14) return 2;
  const bool exact = std::strcmp(argv[1], "exact") == 0;
  const int d = std::atoi(argv[2]);
  const double gamma = std::atof(argv[3]);
  float UL[5], UR[5], F[5];
  double ULd[5], URd[5], Fd[5];
  for (int i = 0; i < 5; ++i) {
    ULd[i] = std::atof(argv[4 + i]);
    URd[i] = std::atof(argv[9 + i]);
    UL[i] = (float)ULd[i];
    UR[i] = (float)URd[i];
  }
  unsigned e32 = 0, e64 = 0;
  if (exact) {
    e32 = riemann_flux<1, float>(d, UL, UR, (float)gamma, F);
    e64 = riemann_flux<1, double>(d, ULd, URd, gamma, Fd);
  } else {
    hllc_flux<float>(d, UL, UR, (float)gamma, F);
    hllc_flux<double>(d, ULd, URd, gamma, Fd);
  }
  std::printf("f32=%.9g,%.9g,%.9g,%.9g,%.9g f64=%.17g,%.17g,%.17g,%.17g,%.17g e32=%u e64=%u\n", F[0], F[1], F[2],
              F[3], F[4], Fd[0], Fd[1], Fd[2], Fd[3], Fd[4], e32, e64);
  return 0;
}

// driver analysis n gamma in.bin out.bin sub lo hi nb n_modes modes.bin spec.bin
//   cubic mesh n^3: diagnostics (FP64 and FP32 field), the velocity samples
//   of the three components, the ln(rho) histogram, and the shell sums of
//   the three half spectra in spec.bin ([3][M][M][M/2+1] complex). out.bin:
//   3 + 3 + 3 M^3 + (nb + 2) + n_bins(M) doubles.
// the spectrum and PDF kernels are grid-stride loops (the library launches
// 2048 / 1024 blocks); a grid of a few blocks runs the same per-thread index
// arithmetic with more iterations per thread at a fraction of the emulation
// cost
constexpr unsigned kStrideGrid = 16;

static int run_analysis(int argc, char** argv) {
  if (argc != 13) return 2;
  const int n = std::atoi(argv[2]), sub = std::atoi(argv[6]), nbins = std::atoi(argv[9]), nm = std::atoi(argv[10]);
  const double gamma = std::atof(argv[3]), lo = std::atof(argv[7]), hi = std::atof(argv[8]);
  Setup S;
  make_setup(S, n, n, n, gamma, 0);
  std::vector<double> y((size_t)5 * TB::N * S.nc), modes((size_t)9 * nm + 1);
  if (!read_file(argv[4], y.data(), y.size())) return 3;
  if (nm > 0 && !read_file(argv[11], modes.data(), (size_t)9 * nm)) return 3;
  const int M = n * sub, H = M / 2 + 1;
  const long long M3 = (long long)M * M * M;
  const int nsh = (int)std::floor(std::sqrt(3.0) * M / 2.0) + 2;
  std::vector<double> out;
  double d3[3];
  run_diag<double>(S, y, modes, nm, d3);
  out.insert(out.end(), d3, d3 + 3);
  run_diag<float>(S, y, modes, nm, d3);
  out.insert(out.end(), d3, d3 + 3);
  for (int comp = 0; comp < 3; ++comp) {
    std::vector<double> v(M3, std::nan(""));
    emu::launch(kStrideGrid, 256, 0, [&] { spec::sample_kernel(y.data(), K, n, sub, comp, v.data()); });
    out.insert(out.end(), v.begin(), v.end());
  }
  std::vector<unsigned long long> counts(nbins + 2, 0);
  emu::launch(kStrideGrid / 2, 256, sizeof(unsigned) * (nbins + 2),
              [&] { spec::density_hist_kernel(y.data(), K, n, sub, lo, hi, nbins, counts.data()); });
  for (auto c : counts) out.push_back((double)c);
  std::vector<double2> sp((size_t)3 * M * M * H);
  if (!read_file(argv[12], reinterpret_cast<double*>(sp.data()), sp.size() * 2)) return 3;
  std::vector<double> bins(nsh, 0.0);
  for (int comp = 0; comp < 3; ++comp)
    emu::launch(kStrideGrid / 2, 256, sizeof(double) * nsh,
                [&] { spec::bin_kernel(sp.data() + (size_t)comp * M * M * H, M, nsh, bins.data()); });
  out.insert(out.end(), bins.begin(), bins.end());
  FILE* f = std::fopen(argv[5], "wb");
  if (!f) return 3;
  std::fwrite(out.data(), 8, out.size(), f);
  std::fclose(f);
  std::printf("err=0 dissipated=0 smax=0\n");
  return 0;
}

// driver limit nx ny nz gamma eps lim_vol in.bin out.bin flags.bin
//   the positivity limiter of dg_limit with per-cell flags (int8 file)
// driver project nx ny nz gamma first count f.bin out.bin
//   dg_project_range: f = [count][5][Q^3] point values of cells first..
static int run_limit_project(int argc, char** argv) {
  const bool lim = std::strcmp(argv[1], "limit") == 0;
  if (argc != 11 && argc != 10) return 2;
  const int nx = std::atoi(argv[2]), ny = std::atoi(argv[3]), nz = std::atoi(argv[4]);
  const double gamma = std::atof(argv[5]);
  Setup S;
  make_setup(S, nx, ny, nz, gamma, lim ? std::atoi(argv[7]) : 0);
  std::vector<double> y((size_t)5 * TB::N * S.nc, std::nan(""));
  const char* out_path;
  if (lim) {
    if (argc != 11) return 2;
    S.g.eps_rho = S.g.eps_p = std::atof(argv[6]);
    if (!read_file(argv[8], y.data(), y.size())) return 3;
    std::vector<int8_t> flags(S.nc, -1);
    emu::launch(grid1(S.nc, kThreads), kThreads, 0,
                [&] { limit_kernel<K>(y.data(), flags.data(), S.t64.data(), S.g, &S.ctrl, S.t32.data()); });
    FILE* f = std::fopen(argv[10], "wb");
    if (!f) return 3;
    std::fwrite(flags.data(), 1, flags.size(), f);
    std::fclose(f);
    out_path = argv[9];
  } else {
    if (argc != 10) return 2;
    const long long first = std::atoll(argv[6]), count = std::atoll(argv[7]);
    std::vector<double> fv((size_t)count * 5 * TB::Q3);
    if (!read_file(argv[8], fv.data(), fv.size())) return 3;
    emu::launch(grid1(5 * count, kThreads), kThreads, 0,
                [&] { project_kernel<K>(fv.data(), y.data(), S.t64.data(), S.g, first, count); });
    out_path = argv[9];
  }
  FILE* f = std::fopen(out_path, "wb");
  if (!f) return 3;
  std::fwrite(y.data(), 8, y.size(), f);
  std::fclose(f);
  std::printf("err=%u n_limited=%llu\n", S.ctrl.err, (unsigned long long)S.ctrl.n_limited);
  return 0;
}

// driver layout nx ny nz in.bin out.bin
//   canonical -> state -> canonical through the C ABI's transpose kernels,
//   then the five conserved totals (means_partial + sum_rows); out.bin: the
//   state layout, the round trip and the totals
static int run_layout(int argc, char** argv) {
  if (argc != 7) return 2;
  const int nx = std::atoi(argv[2]), ny = std::atoi(argv[3]), nz = std::atoi(argv[4]);
  const long long nc = (long long)nx * ny * nz;
  const int N = TB::N, R = 5 * N;
  std::vector<double> canon((size_t)nc * R), st((size_t)nc * R, std::nan("")), back((size_t)nc * R, std::nan(""));
  if (!read_file(argv[5], canon.data(), canon.size())) return 3;
  const unsigned gx = (unsigned)((nc + 31) / 32), gy = (unsigned)((R + 31) / 32);
  emu::launch2(gx, gy, 256, 0, [&] { api::canon_to_state_kernel(canon.data(), st.data(), nc, R); }, 8);
  emu::launch2(gx, gy, 256, 0, [&] { api::state_to_canon_kernel(st.data(), back.data(), nc, R); }, 8);
  const long long nb = (nc + 255) / 256;
  const int G = (int)(nb < api::kRedBlocks ? nb : api::kRedBlocks);
  std::vector<double> part((size_t)5 * G, std::nan("")), sums(5, std::nan(""));
  emu::launch(G, 256, 0, [&] { api::means_partial_kernel(st.data(), nc, N, part.data()); });
  const double vol = 1.0 / (double)nc;
  emu::launch(5, 256, 0, [&] { api::sum_rows_kernel(part.data(), G, vol, sums.data()); });
  std::vector<double> out;
  out.insert(out.end(), st.begin(), st.end());
  out.insert(out.end(), back.begin(), back.end());
  out.insert(out.end(), sums.begin(), sums.end());
  FILE* f = std::fopen(argv[6], "wb");
  if (!f) return 3;
  std::fwrite(out.data(), 8, out.size(), f);
  std::fclose(f);
  std::printf("err=0\n");
  return 0;
}

int main(int argc, char** argv) {
  if (argc >= 2 && (std::strcmp(argv[1], "hllc") == 0 || std::strcmp(argv[1], "exact") == 0))
    return run_hllc(argc, argv);
  if (argc >= 2 && std::strcmp(argv[1], "analysis") == 0) return run_analysis(argc, argv);
  if (argc >= 2 && std::strcmp(argv[1], "layout") == 0) return run_layout(argc, argv);
  if (argc >= 2 && (std::strcmp(argv[1], "limit") == 0 || std::strcmp(argv[1], "project") == 0))
    return run_limit_project(argc, argv);
  if (argc < 9) return 2;
  const bool step = std::strcmp(argv[1], "step") == 0;
  // an optional last argument selects the numerical flux
  const int nargs = step ? 15 : 9;
  if (argc == nargs + 1) g_flux = std::atoi(argv[nargs]);
  else if (argc != nargs) return 2;
  const int nx = std::atoi(argv[2]), ny = std::atoi(argv[3]), nz = std::atoi(argv[4]), prec = std::atoi(argv[5]);
  const double gamma = std::atof(argv[6]);
  Setup S;
  make_setup(S, nx, ny, nz, gamma, step ? std::atoi(argv[14]) : 0);
  std::vector<double> y((size_t)5 * TB::N * S.nc);
  if (!read_file(argv[7], y.data(), y.size())) return 3;
  if (step) {
    const double dt = std::atof(argv[9]), c_iso = std::atof(argv[12]), rho0 = std::atof(argv[13]);
    const int nm = std::atoi(argv[10]);
    std::vector<double> modes((size_t)9 * nm + 1);
    if (nm > 0 && !read_file(argv[11], modes.data(), (size_t)9 * nm)) return 3;
    if (prec) run_step<float>(S, y, dt, modes, nm, c_iso, rho0);
    else run_step<double>(S, y, dt, modes, nm, c_iso, rho0);
  } else {
    std::vector<double> R(y.size(), 0.0);
    if (prec) run_rhs<float>(S, y, R);
    else run_rhs<double>(S, y, R);
    y.swap(R);
  }
  FILE* f = std::fopen(argv[8], "wb");
  if (!f) return 3;
  std::fwrite(y.data(), 8, y.size(), f);
  std::fclose(f);
  return 0;
}
