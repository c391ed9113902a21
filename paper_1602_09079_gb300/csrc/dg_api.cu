// dg_api.cu -- the C ABI of include/dg.h: context, caller-owned buffer
// binding, basis/quadrature tables (closed forms), layout transforms,
// deterministic reductions, and the SSP-RK3 driver (arXiv:1602.09079,
// Sect. 2.4) that sequences the per-degree kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "dg.h"
#include "dg_launch.h"
#include "dg_mlp.h"
#include "dg_spectrum.h"

using namespace dg;

// ----------------------------------------------------------------- tables
namespace {

// Gauss-Legendre nodes (ascending) and weights on [-1,1], closed forms for
// 1..4 points.
void gauss_rule(int q, double* x, double* w) {
  if (q == 1) {
    x[0] = 0.0;
    w[0] = 2.0;
  } else if (q == 2) {
    const double a = 1.0 / std::sqrt(3.0);
    x[0] = -a; x[1] = a;
    w[0] = w[1] = 1.0;
  } else if (q == 3) {
    const double a = std::sqrt(3.0 / 5.0);
    x[0] = -a; x[1] = 0.0; x[2] = a;
    w[0] = w[2] = 5.0 / 9.0;
    w[1] = 8.0 / 9.0;
  } else {
    const double r = 2.0 / 7.0 * std::sqrt(6.0 / 5.0);
    const double xi = std::sqrt(3.0 / 7.0 - r), xo = std::sqrt(3.0 / 7.0 + r);
    const double wi = (18.0 + std::sqrt(30.0)) / 36.0, wo = (18.0 - std::sqrt(30.0)) / 36.0;
    x[0] = -xo; x[1] = -xi; x[2] = xi; x[3] = xo;
    w[0] = wo; w[1] = wi; w[2] = wi; w[3] = wo;
  }
}

// Gauss-Lobatto-Legendre points: m = 2 {-1, 1}, m = 3 {-1, 0, 1}.
void gll_rule(int m, double* x, double* w) {
  if (m == 2) {
    x[0] = -1.0; x[1] = 1.0;
    w[0] = w[1] = 1.0;
  } else {
    x[0] = -1.0; x[1] = 0.0; x[2] = 1.0;
    w[0] = w[2] = 1.0 / 3.0;
    w[1] = 4.0 / 3.0;
  }
}

// sqrt(2u+1) P_u(x) and its derivative, explicit polynomials for u <= 3.
double pt(int u, double x) {
  switch (u) {
    case 0: return 1.0;
    case 1: return std::sqrt(3.0) * x;
    case 2: return std::sqrt(5.0) * 0.5 * (3.0 * x * x - 1.0);
    default: return std::sqrt(7.0) * 0.5 * (5.0 * x * x * x - 3.0 * x);
  }
}
double dpt(int u, double x) {
  switch (u) {
    case 0: return 0.0;
    case 1: return std::sqrt(3.0);
    case 2: return std::sqrt(5.0) * 3.0 * x;
    default: return std::sqrt(7.0) * 0.5 * (15.0 * x * x - 3.0);
  }
}

// Mode exponents in the exchange order: total degree ascending, then u
// descending, then v descending.
void modes(int k, int* e) {
  int l = 0;
  for (int d = 0; d <= k; ++d)
    for (int u = d; u >= 0; --u)
      for (int v = d - u; v >= 0; --v) {
        e[3 * l] = u;
        e[3 * l + 1] = v;
        e[3 * l + 2] = d - u - v;
        ++l;
      }
}

void basis_at(int k, const double xi[3], double* phi, double* grad /*3N or null*/) {
  int e[3 * 20];
  modes(k, e);
  const int N = nmodes(k);
  for (int l = 0; l < N; ++l) {
    const int u = e[3 * l], v = e[3 * l + 1], w = e[3 * l + 2];
    const double a = pt(u, xi[0]), b = pt(v, xi[1]), c = pt(w, xi[2]);
    phi[l] = a * b * c;
    if (grad) {
      grad[3 * l] = dpt(u, xi[0]) * b * c;
      grad[3 * l + 1] = a * dpt(v, xi[1]) * c;
      grad[3 * l + 2] = a * b * dpt(w, xi[2]);
    }
  }
}

template <int K>
void build_tables(double* t) {
  using TB = Tab<K>;
  constexpr int Q = TB::Q, N = TB::N, Q2 = TB::Q2, M = TB::M;
  double g[4], gw[4], h[3], hw[3];
  gauss_rule(Q, g, gw);
  gll_rule(M, h, hw);
  std::memset(t, 0, sizeof(double) * TB::SIZE);
  double phi[20], grad[60];
  for (int c = 0; c < Q; ++c)
    for (int b = 0; b < Q; ++b)
      for (int a = 0; a < Q; ++a) {
        const int q = a + Q * (b + Q * c);
        const double xi[3] = {g[a], g[b], g[c]};
        const double om = gw[a] * gw[b] * gw[c];
        basis_at(K, xi, phi, grad);
        for (int l = 0; l < N; ++l) {
          t[TB::VPHI + q * N + l] = phi[l];
          t[TB::VPHIW + q * N + l] = phi[l] * om / 8.0;
          for (int d = 0; d < 3; ++d) t[TB::VDPHI + (d * TB::Q3 + q) * N + l] = grad[3 * l + d] * om / 4.0;
        }
      }
  for (int d = 0; d < 3; ++d) {
    const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;  // the other two axes, ascending
    for (int s = 0; s < 2; ++s)
      for (int t2 = 0; t2 < Q; ++t2)
        for (int t1 = 0; t1 < Q; ++t1) {
          const int p = t1 + Q * t2;
          double xi[3];
          xi[d] = s ? 1.0 : -1.0;
          xi[o1] = g[t1];
          xi[o2] = g[t2];
          basis_at(K, xi, phi, nullptr);
          for (int l = 0; l < N; ++l) {
            t[TB::FPHI + ((d * 2 + s) * Q2 + p) * N + l] = phi[l];
            t[TB::FPHIW + ((d * 2 + s) * Q2 + p) * N + l] = phi[l] * gw[t1] * gw[t2] / 4.0;
          }
        }
  }
  int n = 0;
  for (int d = 0; d < 3; ++d) {
    const int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
    for (int r = 0; r < M; ++r)
      for (int t2 = 0; t2 < Q; ++t2)
        for (int t1 = 0; t1 < Q; ++t1) {
          double xi[3];
          xi[d] = h[r];
          xi[o1] = g[t1];
          xi[o2] = g[t2];
          basis_at(K, xi, phi, nullptr);
          for (int l = 0; l < N; ++l) {
            t[TB::LPHI + n * N + l] = phi[l];
            t[TB::LMAX + l] = std::fmax(t[TB::LMAX + l], std::fabs(phi[l]));
          }
          ++n;
        }
  }
  // max of |phi_l| over S and the volume Gauss points (the optional point set)
  for (int l = 0; l < N; ++l) {
    double mv = t[TB::LMAX + l];
    for (int q = 0; q < TB::Q3; ++q) mv = std::fmax(mv, std::fabs(t[TB::VPHI + q * N + l]));
    t[TB::LMAXV + l] = mv;
  }
  for (int t2 = 0; t2 < Q; ++t2)
    for (int t1 = 0; t1 < Q; ++t1) {
      int j = 0;
      for (int a = 0; a <= K; ++a)
        for (int b = 0; a + b <= K; ++b) t[TB::F2D + (t1 + Q * t2) * TB::T + j++] = pt(a, g[t1]) * pt(b, g[t2]);
    }
  for (int e = 0; e <= K; ++e) {
    t[TB::FEND + e] = pt(e, -1.0);
    t[TB::FEND + (K + 1) + e] = pt(e, 1.0);
  }
  for (int u = 0; u <= K; ++u)
    for (int a = 0; a < Q; ++a) {
      t[TB::P1 + u * Q + a] = pt(u, g[a]);
      t[TB::P1W + u * Q + a] = pt(u, g[a]) * gw[a];
      t[TB::D1W + u * Q + a] = dpt(u, g[a]) * gw[a];
    }
  for (int a = 0; a < Q; ++a) {
    t[TB::GX + a] = g[a];
    t[TB::GW + a] = gw[a];
  }
}

Launchers launchers_for(int k) {
  switch (k) {
    case 0: return launchers_k0();
    case 1: return launchers_k1();
    case 2: return launchers_k2();
    default: return launchers_k3();
  }
}

// fused FP32-mixed stage kernels exist for degrees 2 and 3
FusedLaunchers fused_for(int k) {
  if (k == 2) return fused_launchers_k2();
  if (k == 3) return fused_launchers_k3();
  FusedLaunchers L{};
  L.k = k;
  return L;
}

std::mutex g_upload_mu;
unsigned long long g_uploaded[4] = {0, 0, 0, 0};  // bit per device

int upload_tables(int k, int dev) {
  std::lock_guard<std::mutex> lock(g_upload_mu);
  if (dev >= 0 && dev < 64 && (g_uploaded[k] >> dev) & 1ull) return DG_OK;
  std::vector<double> t64(TAB_STRIDE, 0.0);
  switch (k) {
    case 0: build_tables<0>(t64.data()); break;
    case 1: build_tables<1>(t64.data()); break;
    case 2: build_tables<2>(t64.data()); break;
    default: build_tables<3>(t64.data()); break;
  }
  std::vector<float> t32(TAB_STRIDE);
  for (int i = 0; i < TAB_STRIDE; ++i) t32[i] = (float)t64[i];
  Launchers L = launchers_for(k);
  if (L.upload(t64.data(), t32.data()) != cudaSuccess) return DG_ERR_CUDA;
  FusedLaunchers F = fused_for(k);
  if (F.upload && F.upload(t64.data()) != cudaSuccess) return DG_ERR_CUDA;
  if (dev >= 0 && dev < 64) g_uploaded[k] |= 1ull << dev;
  return DG_OK;
}

// ------------------------------------------------------ helper kernels
// canonical [nc][R] <-> state [R][nc] (R = 5N), 32x32 tiles
__global__ void canon_to_state_kernel(const double* __restrict__ in, double* __restrict__ out, long long nc, int R) {
  __shared__ double tile[32][33];
  const long long c0 = (long long)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const long long c = c0 + j;
    const int r = r0 + threadIdx.x;
    if (c < nc && r < R) tile[j][threadIdx.x] = in[(size_t)c * R + r];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = r0 + j;
    const long long c = c0 + threadIdx.x;
    if (c < nc && r < R) out[(size_t)r * nc + c] = tile[threadIdx.x][j];
  }
}

__global__ void state_to_canon_kernel(const double* __restrict__ in, double* __restrict__ out, long long nc, int R) {
  __shared__ double tile[32][33];
  const long long c0 = (long long)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int r = r0 + j;
    const long long c = c0 + threadIdx.x;
    if (c < nc && r < R) tile[j][threadIdx.x] = in[(size_t)r * nc + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const long long c = c0 + j;
    const int r = r0 + threadIdx.x;
    if (c < nc && r < R) out[(size_t)c * R + r] = tile[threadIdx.x][j];
  }
}

// FP32 shadow of an FP64 state: yf = float(y)
__global__ void to_f32_kernel(const double* __restrict__ y, float* __restrict__ yf, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) yf[i] = (float)y[i];
}

// out = y - dt * r (one forward-Euler stage, capture of training data)
__global__ void euler_stage_kernel(const double* __restrict__ y, const double* __restrict__ r, double dt,
                                   double* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = y[i] - dt * r[i];
}

constexpr int kRedBlocks = 1024;

// part[i * gridDim.x + b] = sum of the cell means of variable i over block b's
// cells (fixed assignment and tree order: deterministic).
__global__ void __launch_bounds__(256) means_partial_kernel(const double* __restrict__ y, long long nc, int N,
                                                            double* __restrict__ part) {
  __shared__ double s[256];
  for (int i = 0; i < 5; ++i) {
    double acc = 0.0;
    for (long long c = (long long)blockIdx.x * 256 + threadIdx.x; c < nc; c += (long long)gridDim.x * 256)
      acc += y[(size_t)i * N * nc + c];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[i * gridDim.x + blockIdx.x] = s[0];
    __syncthreads();
  }
}

// out[j] = scale * sum_b part[j * n + b], one block per j, fixed order.
__global__ void __launch_bounds__(256) sum_rows_kernel(const double* __restrict__ part, int n, double scale,
                                                       double* __restrict__ out) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int b = threadIdx.x; b < n; b += 256) acc += part[(size_t)blockIdx.x * n + b];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s[0] * scale;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

constexpr int kMaxForce = 256;

}  // namespace

// ------------------------------------------------------------------ context
struct dg_ctx {
  int k = 1;
  int N = 4, Q = 2;
  int device = 0;
  Geo geo{};
  double L[3] = {1, 1, 1};
  Launchers fn{};
  FusedLaunchers fz{};  // fused FP32-mixed stage kernels (fz.run null: none for this degree)
  // binding
  bool bound = false;
  double* y = nullptr;
  unsigned char* scratch = nullptr;
  size_t scratch_bytes = 0;
  cudaStream_t stream = nullptr;
  bool forcing_capable = false;
  // scratch carve-up
  Ctrl* ctrl = nullptr;
  double* part = nullptr;
  double* modes_dev = nullptr;
  double* sums = nullptr;  // 8 doubles
  double* ybuf = nullptr;
  int* list = nullptr;
  int* list2 = nullptr;
  float* yf = nullptr;        // FP32 shadow of the state (FP32 path)
  // fused mixed path: second stage buffer and the FP32 increment y_s - y_0
  // of the step (both carved from the face-flux area, which it does not use)
  double* ybuf2 = nullptr;
  float* dinc = nullptr;
  bool shadow_valid = false;  // yf == float(y)
  // learned indicator gate (caller-owned FP32 parameters)
  const float* ind_params = nullptr;
  float ind_logit_thr = 0.f;
  void* fh = nullptr;
  void* field = nullptr;
  // measurement: launch counts per kernel class, optional event timing
  bool timing = false;
  long long launches[DG_KCLASS_COUNT] = {};
  struct Pending {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  // settings
  int prec = DG_PREC_FP64;
  int flux = DG_FLUX_HLLC;
  bool limited = false;
  int n_force = 0;
  std::vector<double> modes_host;  // 9 per mode
  dg::spec::PlanCache fft;         // cuFFT plan of the velocity spectrum
};

namespace {

struct Layout {
  size_t ctrl, part, modes, sums, ybuf, list, list2, yf, fh, field, base_end, full_end;
};

Layout layout_of(const dg_ctx* c) {
  Layout L{};
  const size_t nc = (size_t)c->geo.nc;
  size_t o = 0;
  L.ctrl = o;
  o += align256(sizeof(Ctrl));
  L.part = o;
  size_t npart = nc / 16 + 2 * kRedBlocks * 5 + 64;
  o += align256(sizeof(double) * npart);
  L.modes = o;
  o += align256(sizeof(double) * 9 * kMaxForce);
  L.sums = o;
  o += align256(sizeof(double) * 8);
  L.ybuf = o;
  o += align256(sizeof(double) * 5 * c->N * nc);
  L.list = o;
  o += align256(sizeof(int) * nc);
  L.list2 = o;
  o += align256(sizeof(int) * nc);
  L.yf = o;
  o += align256(sizeof(float) * 5 * c->N * nc);
  L.fh = o;
  o += align256(sizeof(double) * 15 * c->Q * c->Q * nc);
  L.base_end = o;
  L.field = o;
  o += align256(sizeof(double) * 3 * c->Q * c->Q * c->Q * nc);
  L.full_end = o;
  return L;
}

int cuda_ok(cudaError_t e) { return e == cudaSuccess ? DG_OK : DG_ERR_CUDA; }

#define DG_TRY(expr)                      \
  do {                                    \
    int _st = (expr);                     \
    if (_st != DG_OK) return _st;         \
  } while (0)
#define DG_CUDA(expr) DG_TRY(cuda_ok(expr))

int need_bound(const dg_ctx* c) {
  if (!c) return DG_ERR_ARG;
  return c->bound ? DG_OK : DG_ERR_NOT_BOUND;
}

int err_to_status(unsigned e) {
  if (e & ERRB_NONFINITE) return DG_ERR_NONFINITE;
  if (e & ERRB_POSITIVITY) return DG_ERR_POSITIVITY;
  if (e & ERRB_NEWTON) return DG_ERR_NEWTON;
  return DG_OK;
}

// Synchronise, read and clear the device error word.
int sync_and_check(dg_ctx* c, Ctrl* host_copy) {
  Ctrl h{};
  DG_CUDA(cudaMemcpyAsync(&h, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
  DG_CUDA(cudaStreamSynchronize(c->stream));
  if (host_copy) *host_copy = h;
  if (h.err) {
    DG_CUDA(cudaMemsetAsync(&c->ctrl->err, 0, sizeof(unsigned), c->stream));
    DG_CUDA(cudaStreamSynchronize(c->stream));
  }
  return err_to_status(h.err);
}

int set_device(const dg_ctx* c) { return cuda_ok(cudaSetDevice(c->device)); }

cudaEvent_t take_event(dg_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Every kernel launch of a context goes through here: counted per class (nk
// = the number of kernels f launches) and, with timing on, bracketed by
// events on the bound stream.
template <class F>
int launch(dg_ctx* c, int cls, F&& f, int nk = 1) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (c->timing) {
    a = take_event(c);
    b = take_event(c);
    if (!a || !b) return DG_ERR_CUDA;
    DG_CUDA(cudaEventRecord(a, c->stream));
  }
  cudaError_t e = f();
  c->launches[cls] += nk;
  if (c->timing) {
    DG_CUDA(cudaEventRecord(b, c->stream));
    c->pending.push_back({cls, a, b});
  }
  return cuda_ok(e);
}

enum { KC_LIMIT = 0, KC_FACE = 1, KC_VOLUME = 2, KC_CFL = 3, KC_RESET = 4, KC_OTHER = 5 };

// true when the current precision's kernels read the FP32 shadow
bool uses_shadow(const dg_ctx* c) { return c->prec == DG_PREC_MIXED && c->fn.f32_shadow; }

// true when the mixed path runs the fused stage kernels (they read the FP64
// state; the FP32 shadow is written by the last stage only)
bool uses_fused(const dg_ctx* c) { return c->prec == DG_PREC_MIXED && c->fz.run && c->ybuf2 && c->dinc; }

// yf = float(y) (y: the bound state or any state-layout buffer)
int convert_shadow(dg_ctx* c, const double* y) {
  const long long n = (long long)5 * c->N * c->geo.nc;
  return launch(c, KC_OTHER, [&] {
    to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(y, c->yf, n);
    return cudaGetLastError();
  });
}

int refresh_field(dg_ctx* c) {
  if (c->n_force == 0) return DG_OK;
  return launch(c, KC_OTHER, [&] {
    return c->fn.forcing_field(c->prec, c->field, c->modes_dev, c->n_force, c->geo, c->L, c->stream);
  });
}

// dense FMA throughput probe: 8 independent chains per thread
__device__ double g_probe_sink64;
__device__ float g_probe_sink32;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T a, T b, int write) {
  T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (write) {
    if (sizeof(T) == 8) g_probe_sink64 = (double)s;
    else g_probe_sink32 = (float)s;
  }
}

// One SSP-RK3 step on the fused mixed path: three stage launches
// y -> ybuf -> ybuf2 -> y (a stage never writes the buffer it reads, whose
// neighbours other tiles read), each followed by the full limiter on the
// cells that failed the stage's screen. Stages 1-2 keep the FP32 increment
// d = y_s - y_0 for the next stage's combination; the limiter recomputes it
// for the cells it changes. The last stage writes the FP32 shadow.
int fused_step(dg_ctx* c, double dt, bool force) {
  const double a0[3] = {0.0, 0.75, 1.0 / 3.0};
  const double b0[3] = {1.0, 0.25, 2.0 / 3.0};
  const double* ys = c->y;
  for (int s = 0; s < 3; ++s) {
    double* out = s == 0 ? c->ybuf : (s == 1 ? c->ybuf2 : c->y);
    FusedArgs a{};
    a.ys = ys;
    a.out = out;
    a.d = c->dinc;
    a.yf = s == 2 ? c->yf : nullptr;
    a.field = static_cast<const float*>(c->field);
    a.list = c->list;
    a.ctrl = c->ctrl;
    a.b0dt = (float)(b0[s] * dt);
    a.a0 = (float)a0[s];
    a.b0dt_d = b0[s] * dt;
    a.a0_d = a0[s];
    a.b0_d = b0[s];
    a.y0 = c->y;
    a.stage = s + 1;
    DG_CUDA(cudaMemsetAsync(&c->ctrl->n_flag, 0, sizeof(unsigned), c->stream));
    DG_TRY(launch(c, KC_VOLUME, [&] { return c->fz.run(force, c->flux, c->geo, a, c->stream); }));
    float* yf = s == 2 ? c->yf : nullptr;
    const double* y0 = s < 2 ? c->y : nullptr;
    float* dinc = s < 2 ? c->dinc : nullptr;
    if (c->ind_params) {
      DG_CUDA(cudaMemsetAsync(&c->ctrl->n_gate, 0, sizeof(unsigned), c->stream));
      DG_TRY(launch(c, KC_LIMIT, [&] {
        return dg::mlp::gate_for(c->k, out, c->geo, c->fn.tab64(), c->list, &c->ctrl->n_flag, c->ind_params,
                                 c->ind_logit_thr, c->list2, &c->ctrl->n_gate, &c->ctrl->n_queued_total, c->stream);
      }));
      DG_TRY(launch(c, KC_LIMIT, [&] {
        return c->fn.limit_list(out, c->list2, &c->ctrl->n_gate, c->geo, c->ctrl, 0, yf, y0, dinc, c->list,
                                c->stream);
      }, 2));
    } else {
      DG_TRY(launch(c, KC_LIMIT, [&] {
        return c->fn.limit_list(out, c->list, &c->ctrl->n_flag, c->geo, c->ctrl, 1, yf, y0, dinc, c->list2,
                                c->stream);
      }, 2));
    }
    ys = out;
  }
  c->limited = true;
  c->shadow_valid = true;
  return DG_OK;
}

}  // namespace

extern "C" {

const char* dg_strerror(int code) {
  switch (code) {
    case DG_OK: return "ok";
    case DG_ERR_ARG: return "invalid argument";
    case DG_ERR_NOT_BOUND: return "no state/scratch bound to the context";
    case DG_ERR_CUDA: return "CUDA runtime error";
    case DG_ERR_NONFINITE: return "non-finite value in the state";
    case DG_ERR_POSITIVITY: return "cell mean density or pressure below the positivity floor";
    case DG_ERR_NEWTON: return "positivity-limiter Newton iteration did not converge";
    case DG_ERR_TOO_LARGE: return "problem too large for dg_rhs_noalloc's fixed 32 MiB device scratch";
    default: return "unknown status";
  }
}

int dg_init(const dg_mesh* mesh, int order, double gamma, dg_ctx** out) {
  if (!mesh || !out || order < 1 || order > 4 || !(gamma > 1.0) || !std::isfinite(gamma)) return DG_ERR_ARG;
  long long nc = 1;
  for (int a = 0; a < 3; ++a) {
    if (mesh->n[a] < 1 || !(mesh->length[a] > 0.0) || !std::isfinite(mesh->length[a])) return DG_ERR_ARG;
    // cell counts stay below 2^31 (32-bit cell indices): checked before each
    // product, so the product itself cannot overflow
    if (nc > ((1LL << 31) - 1) / mesh->n[a]) return DG_ERR_ARG;
    nc *= mesh->n[a];
  }
  dg_ctx* c = new (std::nothrow) dg_ctx();
  if (!c) return DG_ERR_ARG;
  c->k = order - 1;
  c->N = nmodes(c->k);
  c->Q = c->k + 1;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return DG_ERR_CUDA;
  }
  c->geo.nx = mesh->n[0];
  c->geo.ny = mesh->n[1];
  c->geo.nz = mesh->n[2];
  c->geo.nc = nc;
  for (int a = 0; a < 3; ++a) {
    c->L[a] = mesh->length[a];
    c->geo.dx[a] = mesh->length[a] / mesh->n[a];
    c->geo.inv_dx[a] = 1.0 / c->geo.dx[a];
  }
  c->geo.gamma = gamma;
  c->geo.eps_rho = 1e-12;
  c->geo.eps_p = 1e-12;
  c->fn = launchers_for(c->k);
  c->fz = fused_for(c->k);
  int st = upload_tables(c->k, c->device);
  if (st != DG_OK) {
    delete c;
    return st;
  }
  *out = c;
  return DG_OK;
}

void dg_destroy(dg_ctx* c) {
  if (!c) return;
  if (c->fft.M && cudaSetDevice(c->device) == cudaSuccess) dg::spec::release(&c->fft);
  for (auto& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  delete c;
}

int dg_sizes(const dg_ctx* c, int features, size_t* state_len, size_t* scratch_bytes) {
  if (!c) return DG_ERR_ARG;
  Layout L = layout_of(c);
  if (state_len) *state_len = (size_t)5 * c->N * (size_t)c->geo.nc;
  if (scratch_bytes) *scratch_bytes = (features & DG_FEATURE_FORCING) ? L.full_end : L.base_end;
  return DG_OK;
}

int dg_bind(dg_ctx* c, double* y_dev, void* scratch_dev, size_t scratch_bytes, void* cuda_stream) {
  if (!c || !y_dev || !scratch_dev) return DG_ERR_ARG;
  if (((uintptr_t)y_dev & 7u) || ((uintptr_t)scratch_dev & 255u)) return DG_ERR_ARG;
  Layout L = layout_of(c);
  if (scratch_bytes < L.base_end) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  c->y = y_dev;
  c->scratch = static_cast<unsigned char*>(scratch_dev);
  c->scratch_bytes = scratch_bytes;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->forcing_capable = scratch_bytes >= L.full_end;
  c->ctrl = reinterpret_cast<Ctrl*>(c->scratch + L.ctrl);
  c->part = reinterpret_cast<double*>(c->scratch + L.part);
  c->modes_dev = reinterpret_cast<double*>(c->scratch + L.modes);
  c->sums = reinterpret_cast<double*>(c->scratch + L.sums);
  c->ybuf = reinterpret_cast<double*>(c->scratch + L.ybuf);
  c->list = reinterpret_cast<int*>(c->scratch + L.list);
  c->list2 = reinterpret_cast<int*>(c->scratch + L.list2);
  c->yf = reinterpret_cast<float*>(c->scratch + L.yf);
  c->shadow_valid = false;
  c->ind_params = nullptr;
  c->fh = c->scratch + L.fh;
  {
    // the fused path's buffers inside the face-flux area (15 Q^2 x 8 bytes
    // per cell >= 5 N x (8 + 4) bytes per cell at every degree)
    const size_t nst = (size_t)5 * c->N * (size_t)c->geo.nc;
    const size_t need = align256(sizeof(double) * nst) + align256(sizeof(float) * nst);
    if (need <= L.base_end - L.fh) {
      c->ybuf2 = reinterpret_cast<double*>(c->scratch + L.fh);
      c->dinc = reinterpret_cast<float*>(c->scratch + L.fh + align256(sizeof(double) * nst));
    } else {
      c->ybuf2 = nullptr;
      c->dinc = nullptr;
    }
  }
  c->field = c->forcing_capable ? c->scratch + L.field : nullptr;
  c->bound = true;
  c->limited = false;
  c->n_force = 0;
  DG_CUDA(cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl), c->stream));
  return DG_OK;
}

int dg_set_state(dg_ctx* c, const double* src, int is_device) {
  DG_TRY(need_bound(c));
  if (!src) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  const int R = 5 * c->N;
  const double* canon = src;
  if (!is_device) {
    DG_CUDA(cudaMemcpyAsync(c->ybuf, src, sizeof(double) * R * c->geo.nc, cudaMemcpyHostToDevice, c->stream));
    canon = c->ybuf;
  }
  dim3 grid((unsigned)((c->geo.nc + 31) / 32), (R + 31) / 32);
  DG_TRY(launch(c, KC_OTHER, [&] {
    canon_to_state_kernel<<<grid, dim3(32, 8), 0, c->stream>>>(canon, c->y, c->geo.nc, R);
    return cudaGetLastError();
  }));
  c->limited = false;
  c->shadow_valid = false;
  return DG_OK;
}

int dg_get_state(dg_ctx* c, double* dst, int is_device) {
  DG_TRY(need_bound(c));
  if (!dst) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  const int R = 5 * c->N;
  double* canon = is_device ? dst : c->ybuf;
  dim3 grid((unsigned)((c->geo.nc + 31) / 32), (R + 31) / 32);
  DG_TRY(launch(c, KC_OTHER, [&] {
    state_to_canon_kernel<<<grid, dim3(32, 8), 0, c->stream>>>(c->y, canon, c->geo.nc, R);
    return cudaGetLastError();
  }));
  if (!is_device) {
    DG_CUDA(cudaMemcpyAsync(dst, c->ybuf, sizeof(double) * R * c->geo.nc, cudaMemcpyDeviceToHost, c->stream));
    DG_CUDA(cudaStreamSynchronize(c->stream));
  }
  return DG_OK;
}

int dg_quadrature_points(const dg_ctx* c, double* xyz) {
  if (!c) return DG_ERR_ARG;
  return dg_quadrature_points_range(c, 0, c->geo.nc, xyz);
}

int dg_quadrature_points_range(const dg_ctx* c, int64_t first, int64_t count, double* xyz) {
  if (!c || !xyz || first < 0 || count < 0 || first + count > c->geo.nc) return DG_ERR_ARG;
  const int Q = c->Q;
  double g[4], w[4];
  gauss_rule(Q, g, w);
  for (long long cell = first; cell < first + count; ++cell) {
    const int ix = (int)(cell % c->geo.nx), iy = (int)((cell / c->geo.nx) % c->geo.ny),
              iz = (int)(cell / ((long long)c->geo.nx * c->geo.ny));
    const int ijk[3] = {ix, iy, iz};
    for (int cc = 0; cc < Q; ++cc)
      for (int b = 0; b < Q; ++b)
        for (int a = 0; a < Q; ++a) {
          const int q = a + Q * (b + Q * cc);
          const int ab[3] = {a, b, cc};
          for (int d = 0; d < 3; ++d)
            xyz[((size_t)(cell - first) * Q * Q * Q + q) * 3 + d] =
                (ijk[d] + 0.5) * c->geo.dx[d] + 0.5 * c->geo.dx[d] * g[ab[d]];
        }
  }
  return DG_OK;
}

int dg_project(dg_ctx* c, const double* q_points_dev) {
  DG_TRY(need_bound(c));
  return dg_project_range(c, q_points_dev, 0, c->geo.nc);
}

int dg_project_range(dg_ctx* c, const double* q_points_dev, int64_t first, int64_t count) {
  DG_TRY(need_bound(c));
  if (!q_points_dev || first < 0 || count < 0 || first + count > c->geo.nc) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  if (count > 0)
    DG_TRY(launch(c, KC_OTHER, [&] { return c->fn.project(q_points_dev, c->y, c->geo, first, count, c->stream); }));
  c->limited = false;
  c->shadow_valid = false;
  return DG_OK;
}

int dg_rhs(dg_ctx* c, const double* y_dev, double* R_dev) {
  DG_TRY(need_bound(c));
  if (!R_dev) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  const double* y = y_dev ? y_dev : c->y;
  const bool force = c->n_force > 0;
  if (uses_fused(c)) {
    FusedArgs a{};
    a.ys = y;
    a.R = R_dev;
    a.field = static_cast<const float*>(c->field);
    a.ctrl = c->ctrl;
    a.stage = 0;
    return launch(c, KC_VOLUME, [&] { return c->fz.run(force, c->flux, c->geo, a, c->stream); });
  }
  if (uses_shadow(c) && !(y == c->y && c->shadow_valid)) {
    DG_TRY(convert_shadow(c, y));
    c->shadow_valid = y == c->y;
  }
  DG_TRY(launch(c, KC_FACE, [&] { return c->fn.face(c->prec, c->flux, y, c->yf, c->fh, c->geo, c->ctrl, c->stream); }));
  DG_TRY(launch(c, KC_VOLUME, [&] {
    return c->fn.volume_rhs(c->prec, force, y, c->yf, c->fh, c->field, c->geo, R_dev, c->ctrl, c->stream);
  }));
  return DG_OK;
}

int dg_step(dg_ctx* c, double dt) {
  DG_TRY(need_bound(c));
  if (!(dt > 0.0) || !std::isfinite(dt)) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  const bool force = c->n_force > 0;
  if (!c->limited) {
    DG_TRY(launch(c, KC_LIMIT, [&] { return c->fn.limit(c->y, nullptr, c->geo, c->ctrl, c->stream); }));
    c->shadow_valid = false;
  }
  if (uses_fused(c)) return fused_step(c, dt, force);
  const bool shadow = uses_shadow(c);
  if (shadow && !c->shadow_valid) DG_TRY(convert_shadow(c, c->y));
  float* yf = shadow ? c->yf : nullptr;
  // Shu-Osher SSP-RK3: y1 = y0 - dt R(y0); y2 = 3/4 y0 + 1/4 (y1 - dt R(y1));
  // y3 = 1/3 y0 + 2/3 (y2 - dt R(y2)); each output limited for the next stage.
  const double a0[3] = {0.0, 0.75, 1.0 / 3.0};
  const double b0[3] = {1.0, 0.25, 2.0 / 3.0};
  const double* ys = c->y;
  for (int s = 0; s < 3; ++s) {
    double* out = s < 2 ? c->ybuf : c->y;
    DG_TRY(launch(c, KC_FACE, [&] { return c->fn.face(c->prec, c->flux, ys, yf, c->fh, c->geo, c->ctrl, c->stream); }));
    DG_CUDA(cudaMemsetAsync(&c->ctrl->n_flag, 0, sizeof(unsigned), c->stream));
    DG_TRY(launch(c, KC_VOLUME, [&] {
      return c->fn.volume_stage(c->prec, force, c->fh, c->field, c->geo, ys, c->y, out, a0[s], b0[s], dt, c->list,
                                yf, c->ctrl, c->stream);
    }));
    // the limiter of the next stage's input: cells that failed the screen,
    // filtered by the learned indicator when one is set
    if (c->ind_params) {
      DG_CUDA(cudaMemsetAsync(&c->ctrl->n_gate, 0, sizeof(unsigned), c->stream));
      DG_TRY(launch(c, KC_LIMIT, [&] {
        return dg::mlp::gate_for(c->k, out, c->geo, c->fn.tab64(), c->list, &c->ctrl->n_flag, c->ind_params,
                                 c->ind_logit_thr, c->list2, &c->ctrl->n_gate, &c->ctrl->n_queued_total, c->stream);
      }));
      DG_TRY(launch(c, KC_LIMIT, [&] {
        return c->fn.limit_list(out, c->list2, &c->ctrl->n_gate, c->geo, c->ctrl, 0, yf, nullptr, nullptr, c->list,
                                c->stream);
      }, 2));
    } else {
      DG_TRY(launch(c, KC_LIMIT, [&] {
        return c->fn.limit_list(out, c->list, &c->ctrl->n_flag, c->geo, c->ctrl, 1, yf, nullptr, nullptr, c->list2,
                                c->stream);
      }, 2));
    }
    ys = out;
  }
  c->limited = true;
  c->shadow_valid = shadow;
  return DG_OK;
}

int dg_limit(dg_ctx* c, int8_t* flags_dev, int64_t* n_limited) {
  DG_TRY(need_bound(c));
  DG_TRY(set_device(c));
  if (n_limited) DG_CUDA(cudaMemsetAsync(&c->ctrl->n_limited, 0, sizeof(unsigned long long), c->stream));
  DG_TRY(launch(c, KC_LIMIT, [&] { return c->fn.limit(c->y, flags_dev, c->geo, c->ctrl, c->stream); }));
  c->limited = true;
  c->shadow_valid = false;
  if (n_limited) {
    Ctrl h{};
    int st = sync_and_check(c, &h);
    *n_limited = (int64_t)h.n_limited;
    return st;
  }
  return DG_OK;
}

int dg_cfl_dt(dg_ctx* c, double courant, double* dt_out) {
  DG_TRY(need_bound(c));
  if (!dt_out || !(courant > 0.0)) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  DG_CUDA(cudaMemsetAsync(&c->ctrl->cfl_max_bits, 0, sizeof(unsigned long long), c->stream));
  DG_TRY(launch(c, KC_CFL, [&] { return c->fn.cfl(c->y, c->geo, c->ctrl, c->stream); }));
  Ctrl h{};
  int st = sync_and_check(c, &h);
  if (st != DG_OK) return st;
  double smax;
  std::memcpy(&smax, &h.cfl_max_bits, sizeof(double));
  if (!(smax > 0.0)) return DG_ERR_POSITIVITY;
  // C min(1/(2k+1), w1/2) with w1 = 1 (m = 2 GLL points), 1/3 (m = 3)
  const double w1 = gll_m(c->k) == 2 ? 1.0 : 1.0 / 3.0;
  const double fac = std::fmin(1.0 / (2 * c->k + 1), w1 / 2.0);
  *dt_out = courant * fac / smax;
  return DG_OK;
}

int dg_set_precision(dg_ctx* c, int mode) {
  if (!c || (mode != DG_PREC_FP64 && mode != DG_PREC_MIXED)) return DG_ERR_ARG;
  const bool changed = c->prec != mode;
  c->prec = mode;
  if (changed && c->bound && c->n_force > 0) {
    DG_TRY(set_device(c));
    DG_TRY(refresh_field(c));
  }
  return DG_OK;
}

int dg_set_limiter_points(dg_ctx* c, int mode) {
  if (!c || (mode != DG_LIMIT_S && mode != DG_LIMIT_S_VOLUME)) return DG_ERR_ARG;
  c->geo.lim_vol = mode == DG_LIMIT_S_VOLUME ? 1 : 0;
  c->limited = false;
  return DG_OK;
}

int dg_set_flux(dg_ctx* c, int flux) {
  if (!c || (flux != DG_FLUX_HLLC && flux != DG_FLUX_EXACT)) return DG_ERR_ARG;
  c->flux = flux;
  return DG_OK;
}

int dg_set_eps(dg_ctx* c, double eps_rho, double eps_p) {
  if (!c || !(eps_rho > 0.0) || !(eps_p > 0.0) || !std::isfinite(eps_rho) || !std::isfinite(eps_p))
    return DG_ERR_ARG;
  c->geo.eps_rho = eps_rho;
  c->geo.eps_p = eps_p;
  c->limited = false;
  return DG_OK;
}

int dg_set_forcing(dg_ctx* c, int n_modes, const int32_t* nvec, const double* ahat) {
  DG_TRY(need_bound(c));
  if (n_modes < 0 || n_modes > kMaxForce) return DG_ERR_ARG;
  if (n_modes > 0 && (!nvec || !ahat || !c->forcing_capable)) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  c->n_force = n_modes;
  if (n_modes == 0) return DG_OK;
  c->modes_host.assign((size_t)9 * n_modes, 0.0);
  for (int j = 0; j < n_modes; ++j) {
    for (int d = 0; d < 3; ++d) c->modes_host[9 * j + d] = (double)nvec[3 * j + d];
    for (int d = 0; d < 6; ++d) {
      if (!std::isfinite(ahat[6 * j + d])) {
        c->n_force = 0;
        return DG_ERR_ARG;
      }
      c->modes_host[9 * j + 3 + d] = ahat[6 * j + d];
    }
  }
  DG_CUDA(cudaMemcpyAsync(c->modes_dev, c->modes_host.data(), sizeof(double) * 9 * n_modes, cudaMemcpyHostToDevice,
                          c->stream));
  DG_CUDA(cudaStreamSynchronize(c->stream));  // host copy may change on the next call
  return refresh_field(c);
}

int dg_energy_reset(dg_ctx* c, double c_iso, double rho0, double* dissipated) {
  DG_TRY(need_bound(c));
  if (!(rho0 > 0.0) || !(c_iso >= 0.0) || !std::isfinite(c_iso) || !std::isfinite(rho0)) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  int n_part = 0;
  const double c2g = c_iso * c_iso / (c->geo.gamma - 1.0);
  // keep the FP32 shadow current if it is (energy rows and limited cells)
  float* yf = (uses_shadow(c) && c->shadow_valid) ? c->yf : nullptr;
  if (!yf) c->shadow_valid = false;
  DG_CUDA(cudaMemsetAsync(&c->ctrl->n_flag, 0, sizeof(unsigned), c->stream));
  DG_TRY(launch(c, KC_RESET, [&] {
    return c->fn.energy_reset(c->prec, c->y, c->geo, c2g, 1.0 / rho0, c->part, &n_part, c->list, c->ctrl, yf,
                              c->stream);
  }));
  // the positivity limiter after the reset (Sect. 3.2): full limiter on the
  // cells that failed the screen
  DG_TRY(launch(c, KC_RESET, [&] {
    return c->fn.limit_list(c->y, c->list, &c->ctrl->n_flag, c->geo, c->ctrl, 0, yf, nullptr, nullptr, c->list2,
                                c->stream);
  }, 2));
  c->limited = true;
  if (dissipated) {
    const double vol = c->geo.dx[0] * c->geo.dx[1] * c->geo.dx[2];
    DG_TRY(launch(c, KC_OTHER, [&] {
      sum_rows_kernel<<<1, 256, 0, c->stream>>>(c->part, n_part, vol, c->sums);
      return cudaGetLastError();
    }));
    double h = 0.0;
    DG_CUDA(cudaMemcpyAsync(&h, c->sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    int st = sync_and_check(c, nullptr);
    *dissipated = h;
    return st;
  }
  return DG_OK;
}

int dg_diagnostics(dg_ctx* c, double* out3) {
  DG_TRY(need_bound(c));
  if (!out3) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  long long nb = (c->geo.nc + 255) / 256;
  const int G = (int)(nb < kRedBlocks ? nb : kRedBlocks);
  const int force = c->n_force > 0 ? 1 : 0;
  DG_TRY(launch(c, KC_OTHER, [&] {
    return c->fn.diagnostics(c->prec, c->y, c->field, force, c->geo, c->part, G, c->stream);
  }));
  const double vol = c->geo.dx[0] * c->geo.dx[1] * c->geo.dx[2];
  DG_TRY(launch(c, KC_OTHER, [&] {
    sum_rows_kernel<<<3, 256, 0, c->stream>>>(c->part, G, vol, c->sums);
    return cudaGetLastError();
  }));
  double h[3];
  DG_CUDA(cudaMemcpyAsync(h, c->sums, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
  const int st = sync_and_check(c, nullptr);
  if (st != DG_OK) return st;
  out3[0] = std::sqrt(h[0] / (c->L[0] * c->L[1] * c->L[2]));
  out3[1] = h[1];
  out3[2] = h[2];
  return DG_OK;
}

namespace {
// the PDF counts live in the partial-sum scratch (at least 2 kRedBlocks x 5 entries)
constexpr int kMaxPdfBins = 4096;

int spectrum_args(const dg_ctx* c, int sub, int* M) {
  if (!c || sub < 1 || sub > 8) return DG_ERR_ARG;
  const Geo& g = c->geo;
  if (g.nx != g.ny || g.ny != g.nz || c->L[0] != c->L[1] || c->L[1] != c->L[2]) return DG_ERR_ARG;
  *M = g.nx * sub;
  return DG_OK;
}
}  // namespace

int dg_spectrum_sizes(const dg_ctx* c, int sub, size_t* work_bytes, int* n_bins) {
  int M = 0;
  DG_TRY(spectrum_args(c, sub, &M));
  if (!work_bytes || !n_bins) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  const size_t b = dg::spec::work_bytes(M, const_cast<dg::spec::PlanCache*>(&c->fft));
  if (b == 0) return DG_ERR_TOO_LARGE;
  *work_bytes = b;
  *n_bins = dg::spec::n_bins(M);
  return DG_OK;
}

int dg_velocity_spectrum(dg_ctx* c, int sub, void* work_dev, size_t work_bytes, double* spectrum) {
  DG_TRY(need_bound(c));
  int M = 0;
  DG_TRY(spectrum_args(c, sub, &M));
  if (!work_dev || !spectrum) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  int cst = 0;
  DG_CUDA(dg::spec::velocity_spectrum(c->k, c->y, c->geo.nx, sub, work_dev, work_bytes, spectrum, c->stream, &cst,
                                      &c->fft));
  if (cst == -1) return DG_ERR_ARG;
  if (cst != 0) return DG_ERR_CUDA;
  return DG_OK;
}

int dg_density_pdf(dg_ctx* c, int sub, double lo, double hi, int n_bins, long long* counts) {
  DG_TRY(need_bound(c));
  int M = 0;
  DG_TRY(spectrum_args(c, sub, &M));
  if (!counts || n_bins < 1 || n_bins > kMaxPdfBins || !(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi))
    return DG_ERR_ARG;
  DG_TRY(set_device(c));
  DG_CUDA(dg::spec::density_pdf(c->k, c->y, c->geo.nx, sub, lo, hi, n_bins,
                                reinterpret_cast<unsigned long long*>(c->part), counts, c->stream));
  return DG_OK;
}

int dg_totals(dg_ctx* c, double* out5) {
  DG_TRY(need_bound(c));
  if (!out5) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  long long nb = (c->geo.nc + 255) / 256;
  const int G = (int)(nb < kRedBlocks ? nb : kRedBlocks);
  DG_TRY(launch(c, KC_OTHER, [&] {
    means_partial_kernel<<<G, 256, 0, c->stream>>>(c->y, c->geo.nc, c->N, c->part);
    return cudaGetLastError();
  }));
  const double vol = c->geo.dx[0] * c->geo.dx[1] * c->geo.dx[2];
  DG_TRY(launch(c, KC_OTHER, [&] {
    sum_rows_kernel<<<5, 256, 0, c->stream>>>(c->part, G, vol, c->sums);
    return cudaGetLastError();
  }));
  DG_CUDA(cudaMemcpyAsync(out5, c->sums, sizeof(double) * 5, cudaMemcpyDeviceToHost, c->stream));
  return sync_and_check(c, nullptr);
}

int dg_check(dg_ctx* c) {
  DG_TRY(need_bound(c));
  DG_TRY(set_device(c));
  return sync_and_check(c, nullptr);
}

int dg_set_indicator(dg_ctx* c, const float* params_dev, float threshold) {
  if (!c) return DG_ERR_ARG;
  if (!params_dev) {
    c->ind_params = nullptr;
    return DG_OK;
  }
  if (c->k < 1 || !(threshold > 0.f) || !(threshold < 1.f)) return DG_ERR_ARG;
  c->ind_params = params_dev;
  c->ind_logit_thr = std::log(threshold / (1.f - threshold));
  return DG_OK;
}

int dg_indicator_capture(dg_ctx* c, double dt, uint16_t* X_dev, int8_t* flags_dev, uint8_t* screen_dev) {
  DG_TRY(need_bound(c));
  if (c->k < 1 || !(dt > 0.0) || !X_dev || !flags_dev || !screen_dev) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  const bool force = c->n_force > 0;
  const long long n = (long long)5 * c->N * c->geo.nc;
  if (uses_shadow(c) && !c->shadow_valid) {
    DG_TRY(convert_shadow(c, c->y));
    c->shadow_valid = true;
  }
  DG_TRY(launch(c, KC_FACE, [&] { return c->fn.face(c->prec, c->flux, c->y, c->yf, c->fh, c->geo, c->ctrl, c->stream); }));
  DG_TRY(launch(c, KC_VOLUME, [&] {
    return c->fn.volume_rhs(c->prec, force, c->y, c->yf, c->fh, c->field, c->geo, c->ybuf, c->ctrl, c->stream);
  }));
  DG_TRY(launch(c, KC_OTHER, [&] {
    euler_stage_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->y, c->ybuf, dt, c->ybuf, n);
    return cudaGetLastError();
  }));
  DG_TRY(launch(c, KC_OTHER, [&] {
    return dg::mlp::features_for(c->k, c->ybuf, c->geo, c->fn.tab64(), X_dev, c->stream);
  }));
  DG_TRY(launch(c, KC_OTHER, [&] { return c->fn.screen(c->ybuf, screen_dev, c->geo, c->stream); }));
  DG_TRY(launch(c, KC_LIMIT, [&] { return c->fn.limit(c->ybuf, flags_dev, c->geo, c->ctrl, c->stream); }));
  return sync_and_check(c, nullptr);
}

int dg_limiter_counts(dg_ctx* c, int64_t* queued, int64_t* full) {
  DG_TRY(need_bound(c));
  DG_TRY(set_device(c));
  Ctrl h{};
  int st = sync_and_check(c, &h);
  if (queued) *queued = (int64_t)h.n_queued_total;
  if (full) *full = (int64_t)h.n_full_total;
  DG_CUDA(cudaMemsetAsync(&c->ctrl->n_queued_total, 0, 2 * sizeof(unsigned long long), c->stream));
  DG_CUDA(cudaStreamSynchronize(c->stream));
  return st;
}

int dg_indicator_features(dg_ctx* c, const double* y_dev, uint16_t* X_dev) {
  DG_TRY(need_bound(c));
  if (!X_dev || c->k < 1) return DG_ERR_ARG;
  DG_TRY(set_device(c));
  const double* y = y_dev ? y_dev : c->y;
  return launch(c, KC_OTHER, [&] { return dg::mlp::features_for(c->k, y, c->geo, c->fn.tab64(), X_dev, c->stream); });
}

int dg_set_timing(dg_ctx* c, int on) {
  if (!c) return DG_ERR_ARG;
  c->timing = on != 0;
  return DG_OK;
}

int dg_kernel_stats(dg_ctx* c, int64_t* launches, double* ms) {
  if (!c) return DG_ERR_ARG;
  double acc[DG_KCLASS_COUNT] = {};
  int st = DG_OK;
  if (c->bound) {
    DG_TRY(set_device(c));
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) st = DG_ERR_CUDA;
  }
  for (auto& p : c->pending) {
    float t = 0.f;
    if (st == DG_OK && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) acc[p.cls] += t;
    c->pool.push_back(p.a);
    c->pool.push_back(p.b);
  }
  c->pending.clear();
  for (int i = 0; i < DG_KCLASS_COUNT; ++i) {
    if (launches) launches[i] = c->launches[i];
    if (ms) ms[i] = acc[i];
    c->launches[i] = 0;
  }
  return st;
}

namespace {
// splitmix64 step (Steele, Lea, Flood 2014) as a counter-based generator
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// every 8th value: a rounding tie or a neighbour of one; every 8th + 1: an
// exponent near the edges of the binary32 range; else raw bit patterns
__global__ void conversion_check_kernel(long long n, unsigned long long seed, unsigned long long* bad) {
  unsigned long long nbad = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long b = mix64(seed ^ mix64((unsigned long long)i));
    if (i % 8 == 0) b = (b & ~0x1fffffffull) | (0x10000000ull + (b >> 62) - 1);
    if (i % 8 == 1) {
      const unsigned long long e = 860 + (b >> 58) % 48 + ((b >> 57) & 1) * 260;  // 860..907 or 1120..1167
      b = (b & 0x800fffffffffffffull) | (e << 52);
    }
    const double x = __longlong_as_double((long long)b);
    const float hw = (float)x, sw = f64_to_f32(x);
    if (!(__float_as_uint(hw) == __float_as_uint(sw) || (isnan(hw) && isnan(sw)))) ++nbad;
    const float f = __uint_as_float((unsigned)(b >> 32));
    const double hw2 = (double)f, sw2 = f32_to_f64(f);
    if (!(__double_as_longlong(hw2) == __double_as_longlong(sw2) || (isnan(hw2) && isnan(sw2)))) ++nbad;
    if (finite64(x) != (bool)isfinite(x)) ++nbad;
  }
  if (nbad) atomicAdd(bad, nbad);
}
}  // namespace

int dg_selftest_conversions(long long n, unsigned long long seed, long long* mismatches) {
  if (n < 0 || !mismatches) return DG_ERR_ARG;
  unsigned long long* d = nullptr;
  DG_CUDA(cudaMalloc(&d, sizeof(unsigned long long)));
  unsigned long long h = 0;
  cudaError_t e = cudaMemset(d, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) {
    conversion_check_kernel<<<1216, 256>>>(n, seed, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return DG_ERR_CUDA;
  *mismatches = (long long)h;
  return DG_OK;
}

int dg_probe_fma_peak(int fp64, double* flops_per_s) {
  if (!flops_per_s) return DG_ERR_ARG;
  int dev = 0, sms = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  const int iters = fp64 ? 4096 : 4096 * 64;
  cudaEvent_t a, b;
  DG_CUDA(cudaEventCreate(&a));
  DG_CUDA(cudaEventCreate(&b));
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(a, 0);
    if (fp64)
      fma_probe_kernel<double><<<blocks, threads>>>(iters, 0.999999, 1e-7, 0);
    else
      fma_probe_kernel<float><<<blocks, threads>>>(iters, 0.999999f, 1e-7f, 0);
    cudaEventRecord(b, 0);
    if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return DG_ERR_CUDA;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    if (rep > 0 && t < best) best = t;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  *flops_per_s = flops / (best * 1e-3);
  return DG_OK;
}

}  // extern "C"

// --------------------------------------------------------------------------
// Allocation-free R(y): the face fluxes of dg_rhs go to one file-scope device
// array instead of a caller-allocated scratch (for callers that may not
// allocate device memory). The array name is a host-side stand-in in host
// code; its device address comes from cudaGetSymbolAddress, looked up once
// per device with that device current.
namespace {

constexpr size_t kNoAllocBytes = DG_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
std::mutex g_noalloc_mu;
void* g_noalloc_dev_ptr[64] = {};
// host staging for a first-call table upload (static: no heap allocation)
double g_noalloc_tab64[TAB_STRIDE];
float g_noalloc_tab32[TAB_STRIDE];

int noalloc_setup(int dev, int k, void** scratch) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_dev_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DG_ERR_CUDA;
    g_noalloc_dev_ptr[dev] = p;
  }
  *scratch = g_noalloc_dev_ptr[dev];
  std::lock_guard<std::mutex> lock2(g_upload_mu);
  if (!((g_uploaded[k] >> dev) & 1ull)) {
    switch (k) {
      case 0: build_tables<0>(g_noalloc_tab64); break;
      case 1: build_tables<1>(g_noalloc_tab64); break;
      case 2: build_tables<2>(g_noalloc_tab64); break;
      default: build_tables<3>(g_noalloc_tab64); break;
    }
    for (int i = 0; i < TAB_STRIDE; ++i) g_noalloc_tab32[i] = (float)g_noalloc_tab64[i];
    if (launchers_for(k).upload(g_noalloc_tab64, g_noalloc_tab32) != cudaSuccess) return DG_ERR_CUDA;
    g_uploaded[k] |= 1ull << dev;
  }
  return DG_OK;
}

}  // namespace

extern "C" int dg_rhs_noalloc(const dg_mesh* mesh, int order, double gamma, int precision, const double* y_dev,
                              double* R_dev, void* cuda_stream) {
  if (!mesh || !y_dev || !R_dev || order < 1 || order > 4 || !(gamma > 1.0) || !std::isfinite(gamma) ||
      (precision != DG_PREC_FP64 && precision != DG_PREC_MIXED))
    return DG_ERR_ARG;
  Geo g{};
  long long nc = 1;
  for (int a = 0; a < 3; ++a) {
    if (mesh->n[a] < 1 || !(mesh->length[a] > 0.0) || !std::isfinite(mesh->length[a])) return DG_ERR_ARG;
    // bounded before each product (as in dg_init), so it cannot overflow
    if (nc > ((1LL << 31) - 1) / mesh->n[a]) return DG_ERR_ARG;
    nc *= mesh->n[a];
    g.dx[a] = mesh->length[a] / mesh->n[a];
    g.inv_dx[a] = 1.0 / g.dx[a];
  }
  const int k = order - 1, Q = k + 1;
  const size_t tsize = precision == DG_PREC_MIXED ? sizeof(float) : sizeof(double);
  const size_t ctrl_bytes = 256;
  const Launchers L = launchers_for(k);
  // FP32 path (every degree): an FP32 copy of y sits behind the face fluxes
  const bool shadow = precision == DG_PREC_MIXED && L.f32_shadow;
  const size_t per_cell = (size_t)15 * Q * Q * tsize + (shadow ? (size_t)5 * nmodes(k) * sizeof(float) : 0);
  if (nc > (long long)(kNoAllocBytes / per_cell) || ctrl_bytes + per_cell * (size_t)nc + 256 > kNoAllocBytes)
    return DG_ERR_TOO_LARGE;
  g.nx = mesh->n[0];
  g.ny = mesh->n[1];
  g.nz = mesh->n[2];
  g.nc = nc;
  g.gamma = gamma;
  g.eps_rho = 1e-12;
  g.eps_p = 1e-12;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DG_ERR_CUDA;
  void* scratch = nullptr;
  DG_TRY(noalloc_setup(dev, k, &scratch));
  Ctrl* ctrl = static_cast<Ctrl*>(scratch);
  void* fh = static_cast<unsigned char*>(scratch) + ctrl_bytes;
  float* yf = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the kernels OR sticky error bits into the control block at the start of
  // the array; clear it on the stream first (a memset allocates nothing), so
  // nothing a previous call left there carries over. No call reads it back:
  // this entry point reports no device-side errors.
  DG_CUDA(cudaMemsetAsync(ctrl, 0, ctrl_bytes, s));
  if (shadow) {
    const size_t fh_bytes = (size_t)15 * Q * Q * tsize * (size_t)nc;
    yf = reinterpret_cast<float*>(static_cast<unsigned char*>(fh) + ((fh_bytes + 255) & ~size_t(255)));
    const long long n = (long long)5 * nmodes(k) * nc;
    to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y_dev, yf, n);
    DG_CUDA(cudaGetLastError());
  }
  DG_CUDA(L.face(precision, DG_FLUX_HLLC, y_dev, yf, fh, g, ctrl, s));
  DG_CUDA(L.volume_rhs(precision, false, y_dev, yf, fh, nullptr, g, R_dev, ctrl, s));
  return DG_OK;
}
