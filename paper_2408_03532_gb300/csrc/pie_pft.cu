// Instantiations of the PFT variant of the fused PIE kernel.
#include <vector>

#include "pie_kernels.cuh"

using namespace pftk;

namespace {

constexpr int kThreads = 256;

struct Entry {
  int P, Q, MP, mode, C;
  bool claim;
  PieKernel k;
};

template <int P, int Q, int MP, int MODE, int C, bool CLAIM = false>
void add(std::vector<Entry>& v) {
  if constexpr (PiePftShape<P, Q, MP, C>::VALID) {
    PieKernel k;
    k.fn = (const void*)k_pie_pft<P, Q, MP, MODE, C, kThreads, CLAIM>;
    k.smem = PiePftShape<P, Q, MP, C>::SMEM;
    k.cluster = C;
    k.threads = kThreads;
    v.push_back(Entry{P, Q, MP, MODE, C, CLAIM, k});
  }
}

template <int P, int Q, int MP>
void add_shape(std::vector<Entry>& v) {
  add<P, Q, MP, MODE_COLOURED, 1>(v);
  add<P, Q, MP, MODE_COLOURED, 2>(v);
  add<P, Q, MP, MODE_COLOURED, 4>(v);
  add<P, Q, MP, MODE_COLOURED, 8>(v);
  add<P, Q, MP, MODE_COLOURED, 4, true>(v);
  add<P, Q, MP, MODE_COLOURED, 8, true>(v);
  add<P, Q, MP, MODE_BATCHED, 1>(v);
  add<P, Q, MP, MODE_BATCHED, 2>(v);
  add<P, Q, MP, MODE_BATCHED, 4>(v);
  add<P, Q, MP, MODE_GRAD, 1>(v);
}

std::vector<Entry> build_table() {
  std::vector<Entry> v;
  add_shape<8, 4, 2>(v);    // n = 32,  M = 16
  add_shape<8, 8, 2>(v);    // n = 64,  M = 16
  add_shape<16, 4, 2>(v);   // n = 64,  M = 32
  add_shape<8, 16, 2>(v);   // n = 128, M = 16
  add_shape<16, 8, 2>(v);   // n = 128, M = 32
  add_shape<32, 4, 2>(v);   // n = 128, M = 64
  add_shape<16, 16, 2>(v);  // n = 256, M = 32
  add_shape<32, 8, 2>(v);   // n = 256, M = 64
  add_shape<32, 2, 2>(v);   // n = 64,  M = 64
  add_shape<8, 32, 2>(v);   // n = 256, M = 16
  return v;
}

}  // namespace

namespace pfth {
PieKernel pie_pft_kernel(int P, int Q, int MP, int mode, int C, bool claim) {
  static const std::vector<Entry> table = build_table();
  for (const Entry& e : table)
    if (e.P == P && e.Q == Q && e.MP == MP && e.mode == mode && e.C == C && e.claim == claim) return e.k;
  return PieKernel{};
}
}  // namespace pfth
