// Instantiations of the full-FFT variant of the fused PIE kernel.
#include <vector>

#include "pie_kernels.cuh"

using namespace pftk;

namespace {

constexpr int kThreads = 256;

struct Entry {
  int N, mode, C;
  bool claim;
  PieKernel k;
};

template <int N, int MODE, int C, bool CLAIM = false>
void add(std::vector<Entry>& v) {
  if constexpr (PieFullShape<N, C>::VALID && PieFullShape<N, C>::FITS) {
    PieKernel k;
    k.fn = (const void*)k_pie_full<N, MODE, C, kThreads, CLAIM>;
    k.smem = PieFullShape<N, C>::SMEM;
    k.cluster = C;
    k.threads = kThreads;
    v.push_back(Entry{N, MODE, C, CLAIM, k});
  }
}

template <int N>
void add_size(std::vector<Entry>& v) {
  add<N, MODE_COLOURED, 1>(v);
  add<N, MODE_COLOURED, 2>(v);
  add<N, MODE_COLOURED, 4>(v);
  add<N, MODE_COLOURED, 8>(v);
  add<N, MODE_COLOURED, 4, true>(v);
  add<N, MODE_COLOURED, 8, true>(v);
  add<N, MODE_BATCHED, 1>(v);
  add<N, MODE_BATCHED, 2>(v);
  add<N, MODE_BATCHED, 4>(v);
}

// 256 x 256 frames: the spectrum fits shared memory only when each of 8 CTAs
// holds an eighth of it (about 167 KB per CTA), so only clusters of 8 exist.
void add_size_256(std::vector<Entry>& v) {
  add<256, MODE_COLOURED, 8>(v);
  add<256, MODE_COLOURED, 8, true>(v);
  add<256, MODE_BATCHED, 8>(v);
}

std::vector<Entry> build_table() {
  std::vector<Entry> v;
  add_size<16>(v);
  add_size<32>(v);
  add_size<64>(v);
  add_size<128>(v);
  add_size_256(v);
  return v;
}

}  // namespace

namespace pfth {
PieKernel pie_full_kernel(int N, int mode, int C, bool claim) {
  static const std::vector<Entry> table = build_table();
  for (const Entry& e : table)
    if (e.N == N && e.mode == mode && e.C == C && e.claim == claim) return e.k;
  return PieKernel{};
}
}  // namespace pfth
