// N-point FFTs on one warp (N = L * E: L lanes, min(N, 32) by default, E values
// per lane), the building block of the full 2-D transform used by the refine
// phase of the hybrid (the full-FFT phase of Algorithm 3) and by the FFT-then-crop
// baseline.
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

template <int N, int LANES = (N < 32 ? N : 32)>
struct Fft {
  static_assert(LANES >= 2 && LANES <= 32 && N % LANES == 0, "lanes per row");
  static constexpr int L = LANES;
  static constexpr int E = N / L;
  static constexpr int G = 32 / L;  // rows per warp
  static constexpr int S = N + 1;   // shared row stride (odd: column access conflict-free)

  __device__ __forceinline__ static int freq_of_slot(int s) {
    return bitrev<E>(s / L) + E * bitrev<L>(s % L);
  }
  __device__ __forceinline__ static int slot_of_freq(int f) {
    return bitrev<E>(f % E) * L + bitrev<L>(f / E);
  }

  // Shared tables of one N: twN[m] = e^{-2 pi i m / N} (N entries, read with
  // warp-uniform indices), the lane network's stage table (L - 1 entries) and
  // the twiddles between the two steps, tw2[k1 L + lane] = w_N^{lane k1}.
  static constexpr int TAB = N + 32 + E * L;
  __device__ __forceinline__ static void fill(float2* tab, const float2* __restrict__ gtw) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) tab[i] = gtw[i];
    fill_stage_table<L>(tab + N, gtw, N);
    for (int i = threadIdx.x; i < E * L; i += blockDim.x) tab[N + 32 + i] = gtw[((i % L) * (i / L)) & (N - 1)];
  }
  // The same through cp.async (the caller commits and waits).
  __device__ __forceinline__ static void fill_async(float2* tab, const float2* __restrict__ gtw) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) cp_async8(tab + i, gtw + i);
    fill_stage_table_async<L>(tab + N, gtw, N);
    for (int i = threadIdx.x; i < E * L; i += blockDim.x) cp_async8(tab + N + 32 + i, gtw + (((i % L) * (i / L)) & (N - 1)));
  }

  using Net = LaneNet<L, false>;
  __device__ __forceinline__ static void init_net(Net& net, int lane, const float2* __restrict__ tab) {
    net.init(lane, tab + N);
  }

  // natural order in, slot order out
  __device__ __forceinline__ static void fwd(float2 (&x)[E], int lane, const float2* __restrict__ tab,
                                             const Net& net) {
    reg_dif<E, false>(x, tab, N);
#pragma unroll
    for (int pos = 0; pos < E; ++pos)
      if (bitrev<E>(pos)) x[pos] = cmul(x[pos], tab[N + 32 + bitrev<E>(pos) * L + lane]);
#pragma unroll
    for (int pos = 0; pos < E; ++pos) x[pos] = net.fwd(x[pos]);
  }

  // exact adjoint of fwd: slot order in, natural order out (F^H = N F^{-1})
  __device__ __forceinline__ static void adj(float2 (&x)[E], int lane, const float2* __restrict__ tab,
                                             const Net& net) {
#pragma unroll
    for (int pos = 0; pos < E; ++pos) x[pos] = net.adj(x[pos]);
#pragma unroll
    for (int pos = 0; pos < E; ++pos)
      if (bitrev<E>(pos)) x[pos] = cmulc(x[pos], tab[N + 32 + bitrev<E>(pos) * L + lane]);
    reg_dif_adj<E, false>(x, tab, N);
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
