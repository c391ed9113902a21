// mlp_driver.cpp -- runs the learned indicator's kernels (dg_mlp.cu, the
// features of degree DG_K and the BF16 network) under the host emulation of
// emu.h, with the library's launch sizes (test infrastructure).
//
//   mlp_driver features nx ny nz gamma in.bin X.bin
//       features_kernel: state [5][N][n_cells] FP64 -> X [n_cells][F] BF16
//   mlp_driver forward n X.bin P.bin logits.bin
//       forward_kernel: X [n][F] BF16, P FP32 -> n FP32 logits
//   mlp_driver backward n pos_weight X.bin y.bin P.bin grads.bin
//       backward_kernel + reduce_rows_kernel: gradient and loss, FP32
//   mlp_driver gate nx ny nz gamma in.bin list.bin n_list P.bin thr out.bin
//       gate_kernel: the queued cells whose logit reaches thr
//   mlp_driver adam n step lr p.bin m.bin v.bin g.bin
//       adam_kernel: p, m, v after one step, written over g.bin
#include "dg_common.cuh"
namespace dg {
namespace mlp {
namespace {
#include "mlp_kernels.inc"
}  // namespace
}  // namespace mlp
}  // namespace dg
using namespace dg;
#include "tables.inc"
using namespace dg::mlp;
constexpr int K = DG_K;
constexpr int F = nfeat_pad(K);
using L = PL<F>;

template <class T>
static bool rd(const char* path, T* p, size_t n) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  const bool ok = std::fread(p, sizeof(T), n, f) == n;
  std::fclose(f);
  return ok;
}
template <class T>
static bool wr(const char* path, const T* p, size_t n) {
  FILE* f = std::fopen(path, "wb");
  if (!f) return false;
  std::fwrite(p, sizeof(T), n, f);
  std::fclose(f);
  return true;
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const std::string mode = argv[1];
  if (mode == "features" && argc == 8) {
    const int nx = std::atoi(argv[2]), ny = std::atoi(argv[3]), nz = std::atoi(argv[4]);
    std::vector<double> t64(TAB_STRIDE, 0.0);
    build_tables<K>(t64.data());
    Geo g{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.nc = (long long)nx * ny * nz;
    g.gamma = std::atof(argv[5]);
    std::vector<double> y((size_t)5 * nmodes(K) * g.nc);
    if (!rd(argv[6], y.data(), y.size())) return 3;
    std::vector<bf16> X((size_t)g.nc * F, __float2bfloat16(NAN));
    emu::launch((unsigned)((g.nc + 127) / 128), 128, 0,
                [&] { features_kernel<K>(y.data(), g, t64.data(), X.data()); });
    return wr(argv[7], X.data(), X.size()) ? 0 : 3;
  }
  if (mode == "forward" && argc == 6) {
    const long long n = std::atoll(argv[2]);
    std::vector<bf16> X((size_t)n * F);
    std::vector<float> P(L::TOTAL), out(n, NAN);
    if (!rd(argv[3], X.data(), X.size()) || !rd(argv[4], P.data(), P.size())) return 3;
    const long long tiles = (n + kRows - 1) / kRows;
    const unsigned grid = (unsigned)(tiles < 152 * 2 ? (tiles > 0 ? tiles : 1) : 152 * 2);
    emu::launch(grid, 256, FwdSmem<F>::bytes(), [&] { forward_kernel<F>(X.data(), n, P.data(), out.data()); });
    return wr(argv[5], out.data(), out.size()) ? 0 : 3;
  }
  if (mode == "backward" && argc == 8) {
    const long long n = std::atoll(argv[2]);
    const float pw = (float)std::atof(argv[3]);
    std::vector<bf16> X((size_t)n * F);
    std::vector<float> y(n), P(L::TOTAL);
    if (!rd(argv[4], X.data(), X.size()) || !rd(argv[5], y.data(), y.size()) || !rd(argv[6], P.data(), P.size()))
      return 3;
    // the library launches 304 blocks; the kernel is a grid-stride loop over
    // 128-row tiles whose per-block partial sums reduce_rows adds up, so a
    // few blocks run the same index arithmetic at a fraction of the
    // emulation cost
    const int rows = 8, cols = L::TOTAL + 1;
    std::vector<float> part((size_t)rows * cols, NAN), grads(cols, NAN);
    emu::launch(rows, 256, BwdSmem<F>::bytes(),
                [&] { backward_kernel<F>(X.data(), y.data(), n, pw, 1.0f / (float)n, P.data(), part.data()); });
    emu::launch((cols + 255) / 256, 256, 0, [&] { reduce_rows_kernel(part.data(), rows, cols, grads.data()); });
    return wr(argv[7], grads.data(), grads.size()) ? 0 : 3;
  }
  if (mode == "gate" && argc == 12) {
    // gate nx ny nz gamma in.bin list.bin n_list P.bin thr out.bin
    const int nx = std::atoi(argv[2]), ny = std::atoi(argv[3]), nz = std::atoi(argv[4]);
    std::vector<double> t64(TAB_STRIDE, 0.0);
    build_tables<K>(t64.data());
    Geo g{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.nc = (long long)nx * ny * nz;
    g.gamma = std::atof(argv[5]);
    const unsigned nl = (unsigned)std::atoi(argv[8]);
    std::vector<double> y((size_t)5 * nmodes(K) * g.nc);
    std::vector<int> list_in(nl), list_out(nl + 1, -1);
    std::vector<float> P(L::TOTAL);
    if (!rd(argv[6], y.data(), y.size()) || !rd(argv[7], list_in.data(), nl) || !rd(argv[9], P.data(), P.size()))
      return 3;
    unsigned count_in = nl, count_out = 0;
    unsigned long long queued = 0;
    const float thr = (float)std::atof(argv[10]);
    // the library launches 152 blocks over the 128-cell tiles of the queue
    emu::launch(4, 256, FwdSmem<F>::bytes(), [&] {
      gate_kernel<K>(y.data(), g, t64.data(), list_in.data(), &count_in, P.data(), thr, list_out.data(), &count_out,
                     &queued);
    });
    if (queued != nl) return 4;
    list_out.resize(count_out);
    return wr(argv[11], list_out.data(), list_out.size()) ? 0 : 3;
  }
  if (mode == "adam" && argc == 9) {
    // adam n step lr p.bin m.bin v.bin g.bin out.bin (out: p, m, v)
    const long long n = std::atoll(argv[2]);
    const int step = std::atoi(argv[3]);
    const float lr = (float)std::atof(argv[4]), b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    std::vector<float> p(n), m(n), v(n), gr(n);
    if (!rd(argv[5], p.data(), n) || !rd(argv[6], m.data(), n) || !rd(argv[7], v.data(), n) ||
        !rd(argv[8], gr.data(), n))
      return 3;
    const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
    emu::launch((unsigned)((n + 255) / 256), 256, 0,
                [&] { adam_kernel(p.data(), m.data(), v.data(), gr.data(), n, lr, b1, b2, eps, c1, c2); });
    std::vector<float> out;
    out.insert(out.end(), p.begin(), p.end());
    out.insert(out.end(), m.begin(), m.end());
    out.insert(out.end(), v.begin(), v.end());
    return wr(argv[8], out.data(), out.size()) ? 0 : 3;
  }
  return 2;
}
