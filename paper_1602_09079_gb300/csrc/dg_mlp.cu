// dg_mlp.cu -- the learned troubled-cell indicator: feature gather, BF16
// MLP forward/backward on the tensor cores (mma.sync m16n8k16, FP32
// accumulation), deterministic gradient reduction, Adam. No counterpart in
// the paper: its labels are the flags of the positivity limiter (Sect. 2.5).
//
// Features per cell (FP64, rounded to BF16): own high modes w_{i,l}/s_i
// (l >= 1, variable-major) with s = (|rho|, sqrt|rho E| x3, |E|) from the cell
// means; log(rho) and the mean Mach number; the excursion bounds
// sum_{l>=1} |w_{i,l}| max_S |phi_l| / s_i (i = 0..4); the 26 neighbour means relative
// to the cell's, (mean_nb - mean)/s, offsets (dz,dy,dx) lexicographic in
// {-1,0,1}^3 without the centre, variable-minor; zero padding to a multiple
// of 32. Network: F -> 64 -> 64 -> 1 with ReLU, sigmoid output.
// Parameters (FP32, flat): W1[64][F], b1[64], W2[64][64], b2[64], w3[64], b3.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "dg.h"
#include "dg_common.cuh"
#include "dg_mlp.h"

namespace dg {
namespace mlp {
namespace {

constexpr int H = 64;
constexpr int kRows = 128;  // cells per tile (8 warps x 16 rows)

__host__ __device__ constexpr int nfeat(int k) { return 5 * (nmodes(k) - 1) + 2 + 5 + 130; }
__host__ __device__ constexpr int nfeat_pad(int k) { return (nfeat(k) + 31) / 32 * 32; }

template <int F>
struct PL {
  static constexpr int W1 = 0, B1 = H * F, W2 = B1 + H, B2 = W2 + H * H, W3 = B2 + H, B3 = W3 + H, TOTAL = B3 + 1;
  static constexpr int LDX = F + 8;   // padded smem leading dimensions (bank spread)
  static constexpr int LDH = H + 8;
};

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack2h(bf16 lo, bf16 hi) {
  __nv_bfloat162 v;
  v.x = lo;
  v.y = hi;
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float lo_f(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float hi_f(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment (16x16) of a row-major matrix M[row][k] in shared memory.
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const bf16* M, int ld, int r0, int k0, int g, int t) {
  a[0] = ld32(M + (r0 + g) * ld + k0 + 2 * t);
  a[1] = ld32(M + (r0 + g + 8) * ld + k0 + 2 * t);
  a[2] = ld32(M + (r0 + g) * ld + k0 + 8 + 2 * t);
  a[3] = ld32(M + (r0 + g + 8) * ld + k0 + 8 + 2 * t);
}
// B fragment (16x8) from Bt[n][k] (k contiguous).
__device__ __forceinline__ void frag_b(uint32_t (&b)[2], const bf16* Bt, int ld, int n0, int k0, int g, int t) {
  b[0] = ld32(Bt + (n0 + g) * ld + k0 + 2 * t);
  b[1] = ld32(Bt + (n0 + g) * ld + k0 + 8 + 2 * t);
}
// A fragment of the transpose of S[k][m] (S row-major, rows = k).
__device__ __forceinline__ void frag_at(uint32_t (&a)[4], const bf16* S, int ld, int m0, int k0, int g, int t) {
  const int k = k0 + 2 * t;
  a[0] = pack2h(S[k * ld + m0 + g], S[(k + 1) * ld + m0 + g]);
  a[1] = pack2h(S[k * ld + m0 + g + 8], S[(k + 1) * ld + m0 + g + 8]);
  a[2] = pack2h(S[(k + 8) * ld + m0 + g], S[(k + 9) * ld + m0 + g]);
  a[3] = pack2h(S[(k + 8) * ld + m0 + g + 8], S[(k + 9) * ld + m0 + g + 8]);
}
// B fragment with B[k][n] = S[k][n] (S row-major, rows = k).
__device__ __forceinline__ void frag_bk(uint32_t (&b)[2], const bf16* S, int ld, int n0, int k0, int g, int t) {
  const int k = k0 + 2 * t;
  b[0] = pack2h(S[k * ld + n0 + g], S[(k + 1) * ld + n0 + g]);
  b[1] = pack2h(S[(k + 8) * ld + n0 + g], S[(k + 9) * ld + n0 + g]);
}

// ------------------------------------------------------------- features
template <int K>
__device__ void cell_features(const double* __restrict__ y, const Geo& g, long long cell, double gamma,
                              const double* __restrict__ tab64, bf16* out) {
  constexpr int N = nmodes(K), F = nfeat_pad(K);
  const long long nc = g.nc;
  double mean[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) mean[i] = y[(size_t)(i * N) * nc + cell];
  const double sm = sqrt(fabs(mean[0] * mean[4]));
  const double inv_s[5] = {1.0 / fabs(mean[0]), 1.0 / sm, 1.0 / sm, 1.0 / sm, 1.0 / fabs(mean[4])};
  int f = 0;
  for (int i = 0; i < 5; ++i)
    for (int l = 1; l < N; ++l) out[f++] = __double2bfloat16(y[(size_t)(i * N + l) * nc + cell] * inv_s[i]);
  const double m2 = mean[1] * mean[1] + mean[2] * mean[2] + mean[3] * mean[3];
  const double p = (gamma - 1.0) * (mean[4] - 0.5 * m2 / mean[0]);
  const double c = sqrt(gamma * p / mean[0]);
  out[f++] = __double2bfloat16(log(mean[0]));
  out[f++] = __double2bfloat16(sqrt(m2) / mean[0] / c);
  for (int i = 0; i < 5; ++i) {
    double b = 0.0;
    for (int l = 1; l < N; ++l) b += fabs(y[(size_t)(i * N + l) * nc + cell]) * __ldg(tab64 + Tab<K>::LMAX + l);
    out[f++] = __double2bfloat16(b * inv_s[i]);
  }
  const int cc = (int)cell;
  const int ix = cc % g.nx, iy = (cc / g.nx) % g.ny, iz = cc / (g.nx * g.ny);
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (dz == 0 && dy == 0 && dx == 0) continue;
        const int jx = (ix + dx + g.nx) % g.nx, jy = (iy + dy + g.ny) % g.ny, jz = (iz + dz + g.nz) % g.nz;
        const long long nb = ((long long)jz * g.ny + jy) * g.nx + jx;
#pragma unroll
        for (int i = 0; i < 5; ++i) out[f++] = __double2bfloat16((y[(size_t)(i * N) * nc + nb] - mean[i]) * inv_s[i]);
      }
  for (; f < F; ++f) out[f] = __float2bfloat16(0.f);
}

template <int K>
__global__ void __launch_bounds__(128) features_kernel(const double* __restrict__ y, Geo g,
                                                       const double* __restrict__ tab64, bf16* __restrict__ X) {
  constexpr int F = nfeat_pad(K);
  const long long cell = (long long)blockIdx.x * 128 + threadIdx.x;
  if (cell >= g.nc) return;
  cell_features<K>(y, g, cell, g.gamma, tab64, X + (size_t)cell * F);
}

// ------------------------------------------------------ weights -> smem
template <int F>
__device__ void load_weights(const float* __restrict__ P, bf16* sW1, bf16* sW2, bf16* sW2T, float* sb1, float* sb2,
                             float* sw3, float* sb3, bool transpose) {
  using L = PL<F>;
  for (int i = threadIdx.x; i < H * F; i += blockDim.x) sW1[(i / F) * L::LDX + (i % F)] = __float2bfloat16(P[L::W1 + i]);
  for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
    const int r = i / H, c = i % H;
    const bf16 v = __float2bfloat16(P[L::W2 + i]);
    sW2[r * L::LDH + c] = v;
    if (transpose) sW2T[c * L::LDH + r] = v;
  }
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    sb1[i] = P[L::B1 + i];
    sb2[i] = P[L::B2 + i];
    sw3[i] = P[L::W3 + i];
  }
  if (threadIdx.x == 0) *sb3 = P[L::B3];
}

// 128 rows of X (row-major, F bf16 per row) -> shared tile
template <int F>
__device__ void load_x_tile(const bf16* __restrict__ X, long long row0, long long n, bf16* sX) {
  using L = PL<F>;
  constexpr int V = F / 8;  // 16-byte vectors per row
  for (int i = threadIdx.x; i < kRows * V; i += blockDim.x) {
    const int r = i / V, v = i % V;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (row0 + r < n) val = *reinterpret_cast<const uint4*>(X + (size_t)(row0 + r) * F + v * 8);
    *reinterpret_cast<uint4*>(sX + r * L::LDX + v * 8) = val;
  }
}

// Forward of one warp's 16 rows: returns the layer-1 activations as BF16 A
// fragments, the layer-2 pre-activations (bias added) and the two logits
// (rows g and g + 8).
template <int F>
__device__ __forceinline__ void warp_forward(const bf16* sX, const bf16* sW1, const bf16* sW2, const float* sb1,
                                             const float* sb2, const float* sw3, float b3, int r0, int g, int t,
                                             uint32_t (&h1a)[4][4], float (&z2)[8][4], float& lg_lo, float& lg_hi) {
  using L = PL<F>;
  float c1[8][4];
#pragma unroll
  for (int n = 0; n < 8; ++n)
#pragma unroll
    for (int e = 0; e < 4; ++e) c1[n][e] = 0.f;
#pragma unroll 4
  for (int kt = 0; kt < F / 16; ++kt) {
    uint32_t a[4];
    frag_a(a, sX, L::LDX, r0, kt * 16, g, t);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      uint32_t b[2];
      frag_b(b, sW1, L::LDX, nt * 8, kt * 16, g, t);
      mma(c1[nt], a, b);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int n0 = 2 * j, n1 = 2 * j + 1;
    const int c0 = n0 * 8 + 2 * t, cq = n1 * 8 + 2 * t;
    h1a[j][0] = pack2(fmaxf(c1[n0][0] + sb1[c0], 0.f), fmaxf(c1[n0][1] + sb1[c0 + 1], 0.f));
    h1a[j][1] = pack2(fmaxf(c1[n0][2] + sb1[c0], 0.f), fmaxf(c1[n0][3] + sb1[c0 + 1], 0.f));
    h1a[j][2] = pack2(fmaxf(c1[n1][0] + sb1[cq], 0.f), fmaxf(c1[n1][1] + sb1[cq + 1], 0.f));
    h1a[j][3] = pack2(fmaxf(c1[n1][2] + sb1[cq], 0.f), fmaxf(c1[n1][3] + sb1[cq + 1], 0.f));
  }
#pragma unroll
  for (int n = 0; n < 8; ++n)
#pragma unroll
    for (int e = 0; e < 4; ++e) z2[n][e] = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      uint32_t b[2];
      frag_b(b, sW2, L::LDH, nt * 8, j * 16, g, t);
      mma(z2[nt], h1a[j], b);
    }
  float slo = 0.f, shi = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int col = nt * 8 + 2 * t + e;
      z2[nt][e] += sb2[col];
      z2[nt][2 + e] += sb2[col];
      slo += fmaxf(z2[nt][e], 0.f) * sw3[col];
      shi += fmaxf(z2[nt][2 + e], 0.f) * sw3[col];
    }
  slo += __shfl_xor_sync(0xffffffffu, slo, 1);
  slo += __shfl_xor_sync(0xffffffffu, slo, 2);
  shi += __shfl_xor_sync(0xffffffffu, shi, 1);
  shi += __shfl_xor_sync(0xffffffffu, shi, 2);
  lg_lo = slo + b3;
  lg_hi = shi + b3;
}

template <int F>
struct FwdSmem {
  using L = PL<F>;
  static constexpr size_t bytes() {
    return sizeof(bf16) * (size_t)(H * L::LDX + H * L::LDH + kRows * L::LDX) + sizeof(float) * (3 * H + 1);
  }
};

template <int F>
__global__ void __launch_bounds__(256) forward_kernel(const bf16* __restrict__ X, long long n,
                                                      const float* __restrict__ P, float* __restrict__ logits) {
  using L = PL<F>;
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* sW1 = reinterpret_cast<bf16*>(smem);
  bf16* sW2 = sW1 + H * L::LDX;
  bf16* sX = sW2 + H * L::LDH;
  float* sb1 = reinterpret_cast<float*>(sX + kRows * L::LDX);
  float* sb2 = sb1 + H;
  float* sw3 = sb2 + H;
  float* sb3 = sw3 + H;
  load_weights<F>(P, sW1, sW2, nullptr, sb1, sb2, sw3, sb3, false);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long ntiles = (n + kRows - 1) / kRows;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    load_x_tile<F>(X, tile * kRows, n, sX);
    __syncthreads();
    uint32_t h1a[4][4];
    float z2[8][4], lo, hi;
    warp_forward<F>(sX, sW1, sW2, sb1, sb2, sw3, *sb3, warp * 16, g, t, h1a, z2, lo, hi);
    if (t == 0) {
      const long long r = tile * kRows + warp * 16 + g;
      if (r < n) logits[r] = lo;
      if (r + 8 < n) logits[r + 8] = hi;
    }
  }
}

// ------------------------------------------------------------- backward
template <int F>
struct BwdSmem {
  using L = PL<F>;
  static constexpr size_t bytes() {
    return sizeof(bf16) * (size_t)(H * L::LDX + 2 * H * L::LDH + kRows * L::LDX + 3 * kRows * L::LDH) +
           sizeof(float) * (3 * H + 1) + sizeof(float) * 8 * (3 * H + 2);
  }
};

// Persistent: each CTA loops over row tiles, accumulates its gradient
// partials (weights in registers, biases per lane) and writes one partial
// row part[blockIdx.x][0 .. TOTAL] (loss in the last entry).
template <int F>
__global__ void __launch_bounds__(256) backward_kernel(const bf16* __restrict__ X, const float* __restrict__ ylab,
                                                       long long n, float pos_weight, float inv_batch,
                                                       const float* __restrict__ P, float* __restrict__ part) {
  using L = PL<F>;
  constexpr int NT1 = F / 8;               // n-tiles of dW1
  constexpr int NTW = (NT1 + 7) / 8;        // per warp
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* sW1 = reinterpret_cast<bf16*>(smem);
  bf16* sW2 = sW1 + H * L::LDX;
  bf16* sW2T = sW2 + H * L::LDH;
  bf16* sX = sW2T + H * L::LDH;
  bf16* sDZ2 = sX + kRows * L::LDX;
  bf16* sDZ1 = sDZ2 + kRows * L::LDH;
  bf16* sH1 = sDZ1 + kRows * L::LDH;
  float* sb1 = reinterpret_cast<float*>(sH1 + kRows * L::LDH);
  float* sb2 = sb1 + H;
  float* sw3 = sb2 + H;
  float* sb3 = sw3 + H;
  float* sred = sb3 + 1;  // [8 warps][3H + 2]
  load_weights<F>(P, sW1, sW2, sW2T, sb1, sb2, sw3, sb3, true);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = warp * 16;
  float gw2[4][4], gw1[4][NTW][4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
#pragma unroll
    for (int e = 0; e < 4; ++e) gw2[m][e] = 0.f;
#pragma unroll
    for (int j = 0; j < NTW; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) gw1[m][j][e] = 0.f;
  }
  float gb1[8][2], gb2[8][2], gw3[8][2];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) gb1[nt][e] = gb2[nt][e] = gw3[nt][e] = 0.f;
  float gb3 = 0.f, lsum = 0.f;
  const long long ntiles = (n + kRows - 1) / kRows;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    load_x_tile<F>(X, tile * kRows, n, sX);
    __syncthreads();
    uint32_t h1a[4][4];
    float z2[8][4], lg_lo, lg_hi;
    warp_forward<F>(sX, sW1, sW2, sb1, sb2, sw3, *sb3, r0, g, t, h1a, z2, lg_lo, lg_hi);
    const long long rlo = tile * kRows + r0 + g, rhi = rlo + 8;
    const bool vlo = rlo < n, vhi = rhi < n;
    // d loss / d logit = (s (a y + 1 - y) - a y) / B
    float dl_lo = 0.f, dl_hi = 0.f;
    if (vlo) {
      const float y = ylab[rlo], s = 1.f / (1.f + __expf(-lg_lo));
      dl_lo = (s * (pos_weight * y + 1.f - y) - pos_weight * y) * inv_batch;
      if (t == 0)
        lsum += pos_weight * y * log1pf(__expf(-fabsf(lg_lo))) + pos_weight * y * fmaxf(-lg_lo, 0.f) +
                (1.f - y) * (log1pf(__expf(-fabsf(lg_lo))) + fmaxf(lg_lo, 0.f));
    }
    if (vhi) {
      const float y = ylab[rhi], s = 1.f / (1.f + __expf(-lg_hi));
      dl_hi = (s * (pos_weight * y + 1.f - y) - pos_weight * y) * inv_batch;
      if (t == 0)
        lsum += pos_weight * y * log1pf(__expf(-fabsf(lg_hi))) + pos_weight * y * fmaxf(-lg_hi, 0.f) +
                (1.f - y) * (log1pf(__expf(-fabsf(lg_hi))) + fmaxf(lg_hi, 0.f));
    }
    if (t == 0) gb3 += dl_lo + dl_hi;
    // layer 3 / layer 2 gradients, dz2 as BF16 A fragments
    float dz2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int col = nt * 8 + 2 * t + e;
        const float hlo = fmaxf(z2[nt][e], 0.f), hhi = fmaxf(z2[nt][2 + e], 0.f);
        gw3[nt][e] += dl_lo * hlo + dl_hi * hhi;
        dz2[nt][e] = z2[nt][e] > 0.f ? dl_lo * sw3[col] : 0.f;
        dz2[nt][2 + e] = z2[nt][2 + e] > 0.f ? dl_hi * sw3[col] : 0.f;
        gb2[nt][e] += dz2[nt][e] + dz2[nt][2 + e];
      }
    uint32_t dza[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      dza[j][0] = pack2(dz2[2 * j][0], dz2[2 * j][1]);
      dza[j][1] = pack2(dz2[2 * j][2], dz2[2 * j][3]);
      dza[j][2] = pack2(dz2[2 * j + 1][0], dz2[2 * j + 1][1]);
      dza[j][3] = pack2(dz2[2 * j + 1][2], dz2[2 * j + 1][3]);
    }
    // dz1 = (dz2 W2) * [z1 > 0]
    float dz1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) dz1[nt][e] = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint32_t b[2];
        frag_b(b, sW2T, L::LDH, nt * 8, j * 16, g, t);
        mma(dz1[nt], dza[j], b);
      }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const uint32_t hlo = h1a[nt >> 1][(nt & 1) * 2 + 0], hhi = h1a[nt >> 1][(nt & 1) * 2 + 1];
      dz1[nt][0] = lo_f(hlo) > 0.f ? dz1[nt][0] : 0.f;
      dz1[nt][1] = hi_f(hlo) > 0.f ? dz1[nt][1] : 0.f;
      dz1[nt][2] = lo_f(hhi) > 0.f ? dz1[nt][2] : 0.f;
      dz1[nt][3] = hi_f(hhi) > 0.f ? dz1[nt][3] : 0.f;
#pragma unroll
      for (int e = 0; e < 2; ++e) gb1[nt][e] += dz1[nt][e] + dz1[nt][2 + e];
    }
    // stage dz2, dz1, h1 (BF16, rows = cells) for the weight gradients
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = nt * 8 + 2 * t;
      const int rl = r0 + g, rh = r0 + g + 8;
      *reinterpret_cast<uint32_t*>(sDZ2 + rl * L::LDH + col) = pack2(dz2[nt][0], dz2[nt][1]);
      *reinterpret_cast<uint32_t*>(sDZ2 + rh * L::LDH + col) = pack2(dz2[nt][2], dz2[nt][3]);
      *reinterpret_cast<uint32_t*>(sDZ1 + rl * L::LDH + col) = pack2(dz1[nt][0], dz1[nt][1]);
      *reinterpret_cast<uint32_t*>(sDZ1 + rh * L::LDH + col) = pack2(dz1[nt][2], dz1[nt][3]);
      *reinterpret_cast<uint32_t*>(sH1 + rl * L::LDH + col) = h1a[nt >> 1][(nt & 1) * 2 + 0];
      *reinterpret_cast<uint32_t*>(sH1 + rh * L::LDH + col) = h1a[nt >> 1][(nt & 1) * 2 + 1];
    }
    __syncthreads();
    // dW2 += dz2^T h1 (warp: n-tile = warp), dW1 += dz1^T X (warp: n-tiles warp + 8 j)
#pragma unroll 2
    for (int kk = 0; kk < kRows / 16; ++kk) {
      uint32_t a2[4][4], a1[4][4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        frag_at(a2[m], sDZ2, L::LDH, m * 16, kk * 16, g, t);
        frag_at(a1[m], sDZ1, L::LDH, m * 16, kk * 16, g, t);
      }
      uint32_t b[2];
      frag_bk(b, sH1, L::LDH, warp * 8, kk * 16, g, t);
#pragma unroll
      for (int m = 0; m < 4; ++m) mma(gw2[m], a2[m], b);
#pragma unroll
      for (int j = 0; j < NTW; ++j) {
        const int nt = warp + 8 * j;
        if (nt < NT1) {
          frag_bk(b, sX, L::LDX, nt * 8, kk * 16, g, t);
#pragma unroll
          for (int m = 0; m < 4; ++m) mma(gw1[m][j], a1[m], b);
        }
      }
    }
  }
  // ---- write this CTA's partial gradient row
  float* out = part + (size_t)blockIdx.x * (L::TOTAL + 1);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int rlo = m * 16 + g, rhi = rlo + 8;
    const int col = warp * 8 + 2 * t;
    out[L::W2 + rlo * H + col] = gw2[m][0];
    out[L::W2 + rlo * H + col + 1] = gw2[m][1];
    out[L::W2 + rhi * H + col] = gw2[m][2];
    out[L::W2 + rhi * H + col + 1] = gw2[m][3];
#pragma unroll
    for (int j = 0; j < NTW; ++j) {
      const int nt = warp + 8 * j;
      if (nt < NT1) {
        const int c1 = nt * 8 + 2 * t;
        out[L::W1 + rlo * F + c1] = gw1[m][j][0];
        out[L::W1 + rlo * F + c1 + 1] = gw1[m][j][1];
        out[L::W1 + rhi * F + c1] = gw1[m][j][2];
        out[L::W1 + rhi * F + c1 + 1] = gw1[m][j][3];
      }
    }
  }
  // per-column vectors: reduce over the 8 row groups (lanes with equal t),
  // then over the warps in a fixed order
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        gb1[nt][e] += __shfl_xor_sync(0xffffffffu, gb1[nt][e], o);
        gb2[nt][e] += __shfl_xor_sync(0xffffffffu, gb2[nt][e], o);
        gw3[nt][e] += __shfl_xor_sync(0xffffffffu, gw3[nt][e], o);
      }
    }
#pragma unroll
  for (int o = 4; o < 32; o <<= 1) {
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  }
  float* red = sred + warp * (3 * H + 2);
  if (g == 0) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int col = nt * 8 + 2 * t + e;
        red[col] = gb1[nt][e];
        red[H + col] = gb2[nt][e];
        red[2 * H + col] = gw3[nt][e];
      }
    if (t == 0) {
      red[3 * H] = gb3;
      red[3 * H + 1] = lsum;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < 3 * H + 2; c += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < 8; ++w) s += sred[w * (3 * H + 2) + c];
    if (c < H) out[L::B1 + c] = s;
    else if (c < 2 * H) out[L::B2 + c - H] = s;
    else if (c < 3 * H) out[L::W3 + c - 2 * H] = s;
    else if (c == 3 * H) out[L::B3] = s;
    else out[L::TOTAL] = s * inv_batch;  // loss
  }
}

// Indicator gate: features and forward pass of the cells queued by a stage
// kernel (list_in, *count_in of them, state y = the stage output); the cells
// whose logit reaches the threshold go on to list_out / *count_out.
template <int K>
__global__ void __launch_bounds__(256) gate_kernel(const double* __restrict__ y, Geo g,
                                                   const double* __restrict__ tab64,
                                                   const int* __restrict__ list_in, const unsigned* count_in,
                                                   const float* __restrict__ P, float logit_thr,
                                                   int* __restrict__ list_out, unsigned* count_out,
                                                   unsigned long long* queued_total) {
  constexpr int F = nfeat_pad(K);
  using L = PL<F>;
  const unsigned n = *count_in;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(queued_total, (unsigned long long)n);
  if (n == 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* sW1 = reinterpret_cast<bf16*>(smem);
  bf16* sW2 = sW1 + H * L::LDX;
  bf16* sX = sW2 + H * L::LDH;
  float* sb1 = reinterpret_cast<float*>(sX + kRows * L::LDX);
  float* sb2 = sb1 + H;
  float* sw3 = sb2 + H;
  float* sb3 = sw3 + H;
  load_weights<F>(P, sW1, sW2, nullptr, sb1, sb2, sw3, sb3, false);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
  const unsigned ntiles = (n + kRows - 1) / kRows;
  for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < kRows) {
      const unsigned r = tile * kRows + threadIdx.x;
      bf16* row = sX + threadIdx.x * L::LDX;
      if (r < n) cell_features<K>(y, g, list_in[r], g.gamma, tab64, row);
      else
        for (int f = 0; f < F; ++f) row[f] = __float2bfloat16(0.f);
    }
    __syncthreads();
    uint32_t h1a[4][4];
    float z2[8][4], lo, hi;
    warp_forward<F>(sX, sW1, sW2, sb1, sb2, sw3, *sb3, warp * 16, gq, t, h1a, z2, lo, hi);
    if (t == 0) {
      const unsigned rl = tile * kRows + warp * 16 + gq, rh = rl + 8;
      if (rl < n && lo >= logit_thr) list_out[atomicAdd(count_out, 1u)] = list_in[rl];
      if (rh < n && hi >= logit_thr) list_out[atomicAdd(count_out, 1u)] = list_in[rh];
    }
  }
}

// grads[j] = sum over partial rows (fixed order)
__global__ void reduce_rows_kernel(const float* __restrict__ part, int rows, int cols, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += part[(size_t)r * cols + j];
  out[j] = s;
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------ dispatch
template <int K>
struct Ops {
  static constexpr int F = nfeat_pad(K);
  static cudaError_t features(const double* y, const Geo& g, const double* tab64, void* X, cudaStream_t s) {
    features_kernel<K><<<(unsigned)((g.nc + 127) / 128), 128, 0, s>>>(y, g, tab64, static_cast<bf16*>(X));
    return cudaGetLastError();
  }
  static cudaError_t forward(const void* X, long long n, const float* P, float* logits, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(forward_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)FwdSmem<F>::bytes());
    if (e != cudaSuccess) return e;
    long long tiles = (n + kRows - 1) / kRows;
    unsigned grid = (unsigned)(tiles < 152 * 2 ? (tiles > 0 ? tiles : 1) : 152 * 2);
    forward_kernel<F><<<grid, 256, FwdSmem<F>::bytes(), s>>>(static_cast<const bf16*>(X), n, P, logits);
    return cudaGetLastError();
  }
  static cudaError_t gate(const double* y, const Geo& g, const double* tab64, const int* list_in,
                          const unsigned* count_in, const float* P, float thr, int* list_out, unsigned* count_out,
                          unsigned long long* queued, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(gate_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)FwdSmem<F>::bytes());
    if (e != cudaSuccess) return e;
    gate_kernel<K><<<152, 256, FwdSmem<F>::bytes(), s>>>(y, g, tab64, list_in, count_in, P, thr, list_out, count_out,
                                                         queued);
    return cudaGetLastError();
  }
  static cudaError_t backward(const void* X, const float* y, long long n, float pw, const float* P, float* grads,
                              float* part, int rows, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(backward_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BwdSmem<F>::bytes());
    if (e != cudaSuccess) return e;
    backward_kernel<F><<<rows, 256, BwdSmem<F>::bytes(), s>>>(static_cast<const bf16*>(X), y, n, pw,
                                                               1.0f / (float)n, P, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int cols = PL<F>::TOTAL + 1;
    reduce_rows_kernel<<<(cols + 255) / 256, 256, 0, s>>>(part, rows, cols, grads);
    return cudaGetLastError();
  }
};

constexpr int kBwdRows = 152 * 2;

int order_ok(int order) { return order >= 2 && order <= 4; }

}  // namespace

int n_params(int order) {
  switch (order) {
    case 2: return PL<nfeat_pad(1)>::TOTAL;
    case 3: return PL<nfeat_pad(2)>::TOTAL;
    default: return PL<nfeat_pad(3)>::TOTAL;
  }
}

}  // namespace mlp
}  // namespace dg

using namespace dg;
using namespace dg::mlp;

extern "C" {

int dg_indicator_sizes(int order, int* n_features, int* n_padded, size_t* n_params_out, size_t* work_bytes) {
  if (!order_ok(order)) return DG_ERR_ARG;
  const int k = order - 1;
  if (n_features) *n_features = nfeat(k);
  if (n_padded) *n_padded = nfeat_pad(k);
  if (n_params_out) *n_params_out = (size_t)mlp::n_params(order);
  if (work_bytes) *work_bytes = sizeof(float) * (size_t)kBwdRows * (mlp::n_params(order) + 1);
  return DG_OK;
}

int dg_indicator_forward(int order, const uint16_t* X_dev, int64_t n, const float* params_dev, float* logits_dev,
                         void* stream) {
  if (!order_ok(order) || !X_dev || !params_dev || !logits_dev || n < 0) return DG_ERR_ARG;
  if (n == 0) return DG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (order) {
    case 2: e = Ops<1>::forward(X_dev, n, params_dev, logits_dev, s); break;
    case 3: e = Ops<2>::forward(X_dev, n, params_dev, logits_dev, s); break;
    default: e = Ops<3>::forward(X_dev, n, params_dev, logits_dev, s); break;
  }
  return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}

int dg_indicator_backward(int order, const uint16_t* X_dev, const float* labels_dev, int64_t n, float pos_weight,
                          const float* params_dev, float* grads_dev, void* work_dev, size_t work_bytes,
                          void* stream) {
  if (!order_ok(order) || !X_dev || !labels_dev || !params_dev || !grads_dev || !work_dev || n <= 0 ||
      !(pos_weight > 0.f))
    return DG_ERR_ARG;
  size_t need = 0;
  dg_indicator_sizes(order, nullptr, nullptr, nullptr, &need);
  if (work_bytes < need) return DG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* part = static_cast<float*>(work_dev);
  cudaError_t e;
  switch (order) {
    case 2: e = Ops<1>::backward(X_dev, labels_dev, n, pos_weight, params_dev, grads_dev, part, kBwdRows, s); break;
    case 3: e = Ops<2>::backward(X_dev, labels_dev, n, pos_weight, params_dev, grads_dev, part, kBwdRows, s); break;
    default: e = Ops<3>::backward(X_dev, labels_dev, n, pos_weight, params_dev, grads_dev, part, kBwdRows, s); break;
  }
  return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}

int dg_indicator_adam(float* params, float* m, float* v, const float* grads, int64_t n_params, float lr,
                      float beta1, float beta2, float eps, int step, void* stream) {
  if (!params || !m || !v || !grads || n_params <= 0 || step < 1) return DG_ERR_ARG;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  adam_kernel<<<(unsigned)((n_params + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      params, m, v, grads, n_params, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}

}  // extern "C"

namespace dg {
namespace mlp {
cudaError_t gate_for(int k, const double* y, const Geo& g, const double* tab64, const int* list_in,
                     const unsigned* count_in, const float* P, float logit_thr, int* list_out, unsigned* count_out,
                     unsigned long long* queued_total, cudaStream_t s) {
  switch (k) {
    case 1: return Ops<1>::gate(y, g, tab64, list_in, count_in, P, logit_thr, list_out, count_out, queued_total, s);
    case 2: return Ops<2>::gate(y, g, tab64, list_in, count_in, P, logit_thr, list_out, count_out, queued_total, s);
    default: return Ops<3>::gate(y, g, tab64, list_in, count_in, P, logit_thr, list_out, count_out, queued_total, s);
  }
}

cudaError_t features_for(int k, const double* y, const Geo& g, const double* tab64, void* X, cudaStream_t s) {
  switch (k) {
    case 1: return Ops<1>::features(y, g, tab64, X, s);
    case 2: return Ops<2>::features(y, g, tab64, X, s);
    default: return Ops<3>::features(y, g, tab64, X, s);
  }
}
}  // namespace mlp
}  // namespace dg
