// emu.h -- host emulation of the CUDA thread model, so that the DG kernels
// can be compiled by g++ under AddressSanitizer / UndefinedBehaviorSanitizer
// / ThreadSanitizer (test infrastructure: checks the kernels' memory accesses
// and shared-memory synchronisation on the CPU; the library never runs on
// the host). Blocks run one after another on one pool of OS threads, one per
// CUDA thread; __syncthreads is a std::barrier of the block, a warp shuffle
// exchanges through a per-warp barrier, __shared__ variables become static
// (one block at a time), atomics are GCC atomic builtins, and the dynamic
// shared memory is a per-block buffer poisoned with 0xCD.
#pragma once
#include <algorithm>
#include <atomic>
#include <barrier>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <thread>
#include <vector>

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __launch_bounds__(...)
#define __align__(n) alignas(n)
#define __constant__
#define __shared__ static

struct emu_uint3 { unsigned x = 0, y = 0, z = 0; };

namespace emu {
struct Block {
  std::unique_ptr<std::barrier<>> bar;
  std::vector<std::unique_ptr<std::barrier<>>> warp;
  std::vector<unsigned char> smem;
  std::vector<uint64_t> shfl;
  std::vector<uint32_t> mma;  // per thread: 4 A and 2 B fragment registers
};
inline emu_uint3 g_blockIdx, g_blockDim, g_gridDim;
inline thread_local emu_uint3 t_threadIdx;
inline Block* g_block = nullptr;
inline unsigned char* dyn_smem() { return g_block->smem.data(); }

// run f() as grid x block threads (1D), dynamic shared memory of smem bytes
template <class F>
void launch2(unsigned grid, unsigned gridy, unsigned block, size_t smem, F&& f, unsigned blocky = 1) {
  // block = threads per block; with blocky > 1 the block is (block / blocky) x blocky
  g_gridDim = {grid, gridy, 1};
  g_blockDim = {block / blocky, blocky, 1};
  const unsigned nblocks = grid * gridy, nw = (block + 31) / 32;
  // one pool of `block` threads walks the blocks; the main thread sets each
  // block up (fresh barriers, poisoned shared memory) between two pool-wide
  // barriers
  std::barrier<> start(block + 1), done(block + 1);
  Block B;
  auto setup = [&](unsigned bb) {
    g_blockIdx = {bb % grid, bb / grid, 0};
    B.bar = std::make_unique<std::barrier<>>(block);
    B.warp.clear();
    for (unsigned w = 0; w < nw; ++w)
      B.warp.push_back(std::make_unique<std::barrier<>>(std::min(32u, block - 32 * w)));
    B.smem.assign(smem + 16, 0xCD);  // poison: reads before writes show up
    B.shfl.assign(block, 0);
    B.mma.assign((size_t)6 * block, 0);
    g_block = &B;
  };
  std::vector<std::thread> th;
  th.reserve(block);
  for (unsigned t = 0; t < block; ++t)
    th.emplace_back([&, t] {
      t_threadIdx = {t % (block / blocky), t / (block / blocky), 0};
      for (unsigned bb = 0; bb < nblocks; ++bb) {
        start.arrive_and_wait();
        f();
        B.bar->arrive_and_drop();
        B.warp[t / 32]->arrive_and_drop();
        done.arrive_and_wait();
      }
    });
  for (unsigned bb = 0; bb < nblocks; ++bb) {
    setup(bb);
    start.arrive_and_wait();
    done.arrive_and_wait();
  }
  for (auto& x : th) x.join();
  g_block = nullptr;
}
template <class F>
void launch(unsigned grid, unsigned block, size_t smem, F&& f) {
  launch2(grid, 1, block, smem, f);
}
}  // namespace emu

#define threadIdx (emu::t_threadIdx)
#define blockIdx (emu::g_blockIdx)
#define blockDim (emu::g_blockDim)
#define gridDim (emu::g_gridDim)

inline void __syncthreads() { emu::g_block->bar->arrive_and_wait(); }
// linear thread index within the block (warps are formed from it)
inline unsigned emu_linear_tid() { return threadIdx.x + threadIdx.y * blockDim.x; }

template <class T>
inline T __shfl_xor_sync(unsigned, T v, int m) {
  const unsigned t = emu_linear_tid(), w = t / 32, lane = t % 32;
  auto& B = *emu::g_block;
  uint64_t bits = 0;
  std::memcpy(&bits, &v, sizeof(T));
  B.shfl[t] = bits;
  B.warp[w]->arrive_and_wait();
  const uint64_t o = B.shfl[w * 32 + (lane ^ (unsigned)m)];
  B.warp[w]->arrive_and_wait();
  T r;
  std::memcpy(&r, &o, sizeof(T));
  return r;
}

template <class T> inline T __ldg(const T* p) { return *p; }
template <class T> inline T __ldcg(const T* p) { return *p; }

inline unsigned atomicAdd(unsigned* p, unsigned v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline int atomicAdd(int* p, int v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
  return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST);
}
inline double atomicAdd(double* p, double v) {
  double old = __atomic_load_n((long long*)p, __ATOMIC_SEQ_CST), nw;
  long long ob, nb;
  do {
    std::memcpy(&ob, p, 8);
    std::memcpy(&old, &ob, 8);
    nw = old + v;
    std::memcpy(&nb, &nw, 8);
  } while (!__atomic_compare_exchange_n((long long*)p, &ob, nb, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST));
  return old;
}
inline unsigned atomicOr(unsigned* p, unsigned v) { return __atomic_fetch_or(p, v, __ATOMIC_SEQ_CST); }
inline unsigned long long atomicMax(unsigned long long* p, unsigned long long v) {
  unsigned long long o = __atomic_load_n(p, __ATOMIC_SEQ_CST);
  while (o < v && !__atomic_compare_exchange_n(p, &o, v, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST)) {
  }
  return o;
}

inline long long __double_as_longlong(double x) { long long r; std::memcpy(&r, &x, 8); return r; }
inline double __longlong_as_double(long long x) { double r; std::memcpy(&r, &x, 8); return r; }
inline unsigned __float_as_uint(float x) { unsigned r; std::memcpy(&r, &x, 4); return r; }
inline float __uint_as_float(unsigned x) { float r; std::memcpy(&r, &x, 4); return r; }
inline int __double2hiint(double x) { return (int)(unsigned)((unsigned long long)__double_as_longlong(x) >> 32); }
inline int __double2loint(double x) { return (int)(unsigned)((unsigned long long)__double_as_longlong(x) & 0xffffffffull); }
inline double __hiloint2double(int hi, int lo) {
  return __longlong_as_double((long long)(((unsigned long long)(unsigned)hi << 32) | (unsigned)lo));
}
inline float atomicAdd(float* p, float v) {
  float old, nw;
  unsigned ob, nb;
  do {
    std::memcpy(&ob, p, 4);
    std::memcpy(&old, &ob, 4);
    nw = old + v;
    std::memcpy(&nb, &nw, 4);
  } while (!__atomic_compare_exchange_n((unsigned*)p, &ob, nb, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST));
  return old;
}

// BF16 storage type and round-to-nearest-even conversions
struct __nv_bfloat16 {
  uint16_t x;
};
struct __nv_bfloat162 {
  __nv_bfloat16 x, y;
};
inline __nv_bfloat16 __float2bfloat16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  __nv_bfloat16 h;
  if ((u & 0x7fffffffu) > 0x7f800000u) {
    h.x = 0x7fc0;  // NaN
    return h;
  }
  u += 0x7fffu + ((u >> 16) & 1u);
  h.x = (uint16_t)(u >> 16);
  return h;
}
inline __nv_bfloat16 __double2bfloat16(double d) {
  // round the binary64 significand to 8 bits directly (no intermediate
  // binary32 rounding); normal range of the test data only
  uint64_t u;
  std::memcpy(&u, &d, 8);
  if (d != d) return __float2bfloat16(NAN);
  if (d == 0.0) return __float2bfloat16(std::signbit(d) ? -0.f : 0.f);
  int e;
  const double m = std::frexp(std::fabs(d), &e);       // |d| = m 2^e, m in [0.5, 1)
  const double q = std::nearbyint(std::ldexp(m, 8));    // 8 significant bits, ties to even
  return __float2bfloat16((float)std::copysign(std::ldexp(q, e - 8), d));
}
inline float __bfloat162float(__nv_bfloat16 h) {
  const uint32_t u = (uint32_t)h.x << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
inline __nv_bfloat162 __floats2bfloat162_rn(float lo, float hi) { return {__float2bfloat16(lo), __float2bfloat16(hi)}; }
struct uint4 {
  unsigned x, y, z, w;
};
inline uint4 make_uint4(unsigned x, unsigned y, unsigned z, unsigned w) { return {x, y, z, w}; }
inline float __expf(float x) { return std::exp(x); }
inline float __fdividef(float a, float b) { return a / b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
// hi:lo shifted left by s mod 32, upper 32 bits
inline unsigned __funnelshift_l(unsigned lo, unsigned hi, unsigned s) {
  return (unsigned)(((((unsigned long long)hi << 32) | lo) << (s & 31)) >> 32);
}

namespace emu {
// mma.sync m16n8k16 row.col, BF16 inputs, FP32 accumulate, over the warp:
// lane (g = lane / 4, t = lane % 4) holds A[g][2t..2t+1], A[g+8][2t..],
// A[g][2t+8..], A[g+8][2t+8..] (a0..a3), B[2t..2t+1][g], B[2t+8..][g]
// (b0, b1), and D[g][2t..2t+1], D[g+8][2t..2t+1] (d0..d3); the lower 16 bits
// of a register hold the element with the even k
inline float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
inline float bf_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }
inline void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  const unsigned tid = emu_linear_tid(), w = tid / 32, lane = tid % 32;
  auto& B = *g_block;
  uint32_t* mine = &B.mma[(size_t)6 * tid];
  for (int i = 0; i < 4; ++i) mine[i] = a[i];
  mine[4] = b[0];
  mine[5] = b[1];
  B.warp[w]->arrive_and_wait();
  const uint32_t* base = &B.mma[(size_t)6 * (w * 32)];
  auto A = [&](int r, int k) {
    const uint32_t reg = base[6 * ((r % 8) * 4 + (k % 8) / 2) + (r >= 8 ? 1 : 0) + (k >= 8 ? 2 : 0)];
    return (k % 2) ? bf_hi(reg) : bf_lo(reg);
  };
  auto Bm = [&](int k, int n) {
    const uint32_t reg = base[6 * (n * 4 + (k % 8) / 2) + 4 + (k >= 8 ? 1 : 0)];
    return (k % 2) ? bf_hi(reg) : bf_lo(reg);
  };
  const int g = lane / 4, t = lane % 4;
  for (int i = 0; i < 4; ++i) {
    const int r = g + (i >= 2 ? 8 : 0), n = 2 * t + (i % 2);
    float acc = d[i];
    for (int k = 0; k < 16; ++k) acc += A(r, k) * Bm(k, n);
    d[i] = acc;
  }
  B.warp[w]->arrive_and_wait();
}
}  // namespace emu

inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
inline float __frcp_rn(float x) { return 1.0f / x; }
using std::cbrt;
using std::max;
using std::min;
using std::fmax;
using std::fmin;
using std::isfinite;
using std::pow;
using std::sqrt;
