// N-point FFTs on one warp (N = L * E, L = min(N, 32) lanes, E per lane), the
// building block of the full 2-D transform used by the refine phase of the
// hybrid (Algorithm 3, step 3) and by the FFT-then-crop baseline.
//
// A row held as x[e] = v[lane + L e] is transformed in three steps:
//   1. an E-point DFT over e in registers,
//   2. the twiddles w_N^{lane k1},
//   3. an L-point DFT across the lanes for each k1,
// after which register pos of lane l holds V[bitrev_E(pos) + E bitrev_L(l)].
// That value is kept in "slot" pos * L + l (so stores stay conflict-free) and
// the adjoint transform takes slot order straight back to natural order.
#pragma once

#include "common.cuh"

namespace pftk {

template <int N>
struct Fft {
  static constexpr int L = N < 32 ? N : 32;
  static constexpr int E = N / L;
  static constexpr int G = 32 / L;  // rows per warp
  static constexpr int S = N + 1;   // shared row stride (odd: column access conflict-free)

  __device__ __forceinline__ static int freq_of_slot(int s) {
    return bitrev<E>(s / L) + E * bitrev<L>(s % L);
  }
  __device__ __forceinline__ static int slot_of_freq(int f) {
    return bitrev<E>(f % E) * L + bitrev<L>(f / E);
  }

  // natural order in, slot order out; twN[m] = e^{-2 pi i m / N}
  __device__ __forceinline__ static void fwd(float2 (&x)[E], int lane, const float2* __restrict__ twN) {
    reg_dif<E, false>(x, twN, N);
#pragma unroll
    for (int pos = 0; pos < E; ++pos) {
      const int idx = (lane * bitrev<E>(pos)) & (N - 1);
      if (idx) x[pos] = cmul(x[pos], twN[idx]);
    }
#pragma unroll
    for (int pos = 0; pos < E; ++pos) x[pos] = lane_dif<L, false, N / L>(x[pos], lane, twN);
  }

  // exact adjoint of fwd: slot order in, natural order out (F^H = N F^{-1})
  __device__ __forceinline__ static void adj(float2 (&x)[E], int lane, const float2* __restrict__ twN) {
#pragma unroll
    for (int pos = 0; pos < E; ++pos) x[pos] = lane_dif_adj<L, false, N / L>(x[pos], lane, twN);
#pragma unroll
    for (int pos = 0; pos < E; ++pos) {
      const int idx = (lane * bitrev<E>(pos)) & (N - 1);
      if (idx) x[pos] = cmulc(x[pos], twN[idx]);
    }
    reg_dif_adj<E, false>(x, twN, N);
  }
};

// Centred crop index of frequency f (0 <= f < N) for an M-wide output, or -1.
template <int N, int M>
__device__ __forceinline__ int crop_index(int f) {
  return f < M / 2 ? f + M / 2 : (f >= N - M / 2 ? f - N + M / 2 : -1);
}

}  // namespace pftk

namespace pfth {
// Device table e^{-2 pi i m / N}, m < N, computed once per N in FP64 with
// exact integer reduction and rounded to FP32 (N a power of two <= 256).
const float2* twiddles(int N);
}  // namespace pfth
