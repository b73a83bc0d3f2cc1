// Device building blocks of the factorised PFT (Algorithm 5) on sm_103a.
//
// A 2-D PFT is separable: z^ = A1 Z A2^T with each A_nu an M x n operator of
// the 1-D form of Algorithm 2, so a frame is transformed row by row (axis 2)
// into an n x M intermediate Y and then column by column (axis 1).
//
// One 1-D transform of a length-n vector (n = P Q) runs on a group of P lanes
// of a warp; lane k owns the block x[Q k .. Q k + Q - 1]:
//   stage A of Algorithm 2 (the compression C = Z B): C[k][j] = sum_l B[l][j] x[Q k + l],
//     with B[l][j] = a_j (1 - 2 l / Q)^j real. Rows l and Q - l have opposite
//     abscissae, so even j use x_l + x_{Q-l} and odd j use x_l - x_{Q-l},
//     halving the multiply-adds. B sits in the kernel's parameter space and
//     every index is a compile-time constant, so it is read as a constant
//     operand of the FMA instructions.
//   stage B of Algorithm 2 (the expansion): a P-point DFT over k for each j, across the P
//     lanes by a radix-2 butterfly network with shuffles and per-lane register
//     twiddles (lane k then holds residue v = bitrev(k)), followed by
//     z^[t] = sum_j W'[t][j] C^[t mod P][j] for the M/P outputs t = v mod P,
//     where W'[t][j] = i^j (t/P)^j e^{-i pi t/P} carries the factor i^j of
//     w_j = i^j a_j.
// The adjoint runs the exact transpose of each step in reverse order.
#pragma once

#include "common.cuh"

namespace pftk {

constexpr int RMAX = 13;       // polynomial terms the kernels are built for (r <= 13)
constexpr int BH_ROWS = 17;    // Q/2 + 1 rows of B kept (Q <= 32)

// Per-plan constants passed by value (kernel parameter space).
struct PftConst {
  float bh[2][BH_ROWS][RMAX];  // [axis][l][j] = a_j (1 - 2l/Q)^j, l = 0..Q/2
};

// Column slot -> column index: places the columns that share a half-warp at
// indices that differ in bits log2(P)..3, so that with the XOR swizzle below
// the column reads of one half-warp hit 16 different bank pairs.
template <int P>
__device__ __forceinline__ int col_of(int cs) {
  if (P >= 16) return cs;
  constexpr int C = P >= 16 ? 1 : 16 / P;  // columns per half-warp
  int base = cs & ~15, r = cs & 15;
  return base | ((r % C) * P + r / C);
}

// Row-major n x M intermediate with row stride M + 8 and an XOR swizzle of the
// column by the row's block index (u / Q) & 15: row writes stay a permutation
// of one row, column reads of one block-column spread over all banks.
template <int Q, int M>
struct YLayout {
  static constexpr int S = M + 8;
  __device__ __forceinline__ static int at(int u, int t) { return u * S + (t ^ ((u / Q) & 15)); }
};

// ---------------------------------------------------------------- stage A
template <int Q>
__device__ __forceinline__ void stageA_fwd(const float2 (&x)[Q], float2 (&C)[RMAX],
                                           const float (&bh)[BH_ROWS][RMAX]) {
  constexpr int H = Q / 2;
  float2 s[H > 1 ? H : 1], d[H > 1 ? H : 1];
  float2 tot = cadd(x[0], x[H]);
#pragma unroll
  for (int l = 1; l < H; ++l) {
    s[l] = cadd(x[l], x[Q - l]);
    d[l] = csub(x[l], x[Q - l]);
    tot = cadd(tot, s[l]);
  }
  C[0] = cscale(tot, bh[0][0]);
#pragma unroll
  for (int j = 1; j < RMAX; ++j) {
    float2 acc = cscale(x[0], bh[0][j]);
#pragma unroll
    for (int l = 1; l < H; ++l) {
      const float2 v = (j & 1) ? d[l] : s[l];
      acc.x = fmaf(bh[l][j], v.x, acc.x);
      acc.y = fmaf(bh[l][j], v.y, acc.y);
    }
    C[j] = acc;
  }
}

template <int Q>
__device__ __forceinline__ void stageA_adj(const float2 (&E)[RMAX], float2 (&x)[Q],
                                           const float (&bh)[BH_ROWS][RMAX]) {
  constexpr int H = Q / 2;
  float2 x0 = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < RMAX; ++j) {
    x0.x = fmaf(bh[0][j], E[j].x, x0.x);
    x0.y = fmaf(bh[0][j], E[j].y, x0.y);
  }
  x[0] = x0;
  x[H] = cscale(E[0], bh[0][0]);  // abscissa 0: only j = 0
#pragma unroll
  for (int l = 1; l < H; ++l) {
    float2 e = make_float2(0.f, 0.f), o = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
      if (j & 1) {
        o.x = fmaf(bh[l][j], E[j].x, o.x);
        o.y = fmaf(bh[l][j], E[j].y, o.y);
      } else {
        e.x = fmaf(bh[l][j], E[j].x, e.x);
        e.y = fmaf(bh[l][j], E[j].y, e.y);
      }
    }
    x[l] = cadd(e, o);
    x[Q - l] = csub(e, o);
  }
}

// ----------------------------------------------------------- 1-D transform
template <int P, int Q, int MP>
struct Pft1D {
  static constexpr int N = P * Q;
  static constexpr int M = MP * P;

  // index of the first output of lane k's residue (outputs are c P + w, c < MP)
  __device__ __forceinline__ static int first_out(int k) { return (bitrev<P>(k) + M / 2) % P; }

  // Forward: lane k holds x[Qk .. Qk+Q-1]; calls store(t_idx, value) for the
  // outputs t_idx (= t + M/2) of its residue. sW: [RMAX][M] (j-major).
  template <class Store>
  __device__ __forceinline__ static void forward(const float2 (&x)[Q], int k,
                                                 const float (&bh)[BH_ROWS][RMAX],
                                                 const float2* __restrict__ sW,
                                                 const LaneNet<P, false>& net, Store store) {
    float2 C[RMAX];
    stageA_fwd<Q>(x, C, bh);
#pragma unroll
    for (int j = 0; j < RMAX; ++j) C[j] = net.fwd(C[j]);
    const int w = first_out(k);
#pragma unroll
    for (int c = 0; c < MP; ++c) {
      const int t = c * P + w;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < RMAX; ++j) acc = cfma(acc, sW[j * M + t], C[j]);
      store(t, acc);
    }
  }

  // Adjoint: load(t_idx) returns the input at output index t_idx of lane k's
  // residue; on exit x[l] = (A^H y)[Qk + l].
  template <class Load>
  __device__ __forceinline__ static void adjoint(Load load, int k,
                                                 const float (&bh)[BH_ROWS][RMAX],
                                                 const float2* __restrict__ sW,
                                                 const LaneNet<P, false>& net, float2 (&x)[Q]) {
    const int w = first_out(k);
    float2 yv[MP];
#pragma unroll
    for (int c = 0; c < MP; ++c) yv[c] = load(c * P + w);
    float2 E[RMAX];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < MP; ++c) acc = cfmac(acc, sW[j * M + c * P + w], yv[c]);
      E[j] = net.adj(acc);
    }
    stageA_adj<Q>(E, x, bh);
  }
};

// The same 1-D transform on 2P lanes (P <= 16): the two P-lane halves of the
// group hold the same block and split the r terms between them, half h taking
// j = h JH ... h JH + JH - 1 (JH = 7; half 1's seventh term is a zero pad).
// Stage A runs in both halves; the lane network and the W' combine run on half
// the terms each, and one shuffle across the halves adds the partial sums.
template <int P, int Q, int MP>
struct Pft1DSplit {
  static_assert(P <= 16, "two halves of P lanes share a warp");
  static constexpr int N = P * Q;
  static constexpr int M = MP * P;
  static constexpr int JH = (RMAX + 1) / 2;

  // Forward: both halves hold x[Qk .. Qk+Q-1]; half h stores the outputs c of
  // its residue with c % 2 == h.
  template <class Store>
  __device__ __forceinline__ static void forward(const float2 (&x)[Q], int k, int h,
                                                 const float (&bh)[BH_ROWS][RMAX],
                                                 const float2* __restrict__ sW,
                                                 const LaneNet<P, false>& net, Store store) {
    float2 C[RMAX];
    stageA_fwd<Q>(x, C, bh);
    float2 Ch[JH];
#pragma unroll
    for (int i = 0; i < JH; ++i) {
      const float2 hi = (i + JH < RMAX) ? C[i + JH] : make_float2(0.f, 0.f);
      Ch[i] = net.fwd(h ? hi : C[i]);
    }
    const int w = Pft1D<P, Q, MP>::first_out(k);
    const int j0 = h * JH;
#pragma unroll
    for (int c = 0; c < MP; ++c) {
      const int t = c * P + w;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < JH; ++i) {
        const int j = min(j0 + i, RMAX - 1);  // half 1's pad term multiplies a zero
        acc = cfma(acc, sW[j * M + t], Ch[i]);
      }
      acc.x += __shfl_xor_sync(PFT_FULL_MASK, acc.x, P);
      acc.y += __shfl_xor_sync(PFT_FULL_MASK, acc.y, P);
      if ((c & 1) == h) store(t, acc);
    }
  }

  // Adjoint: both halves load the inputs of their residue and end with the
  // whole x[l] = (A^H y)[Qk + l].
  template <class Load>
  __device__ __forceinline__ static void adjoint(Load load, int k, int h, const float (&bh)[BH_ROWS][RMAX],
                                                 const float2* __restrict__ sW,
                                                 const LaneNet<P, false>& net, float2 (&x)[Q]) {
    const int w = Pft1D<P, Q, MP>::first_out(k);
    float2 yv[MP];
#pragma unroll
    for (int c = 0; c < MP; ++c) yv[c] = load(c * P + w);
    const int j0 = h * JH;
    float2 Eh[JH];
#pragma unroll
    for (int i = 0; i < JH; ++i) {
      const int j = min(j0 + i, RMAX - 1);
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < MP; ++c) acc = cfmac(acc, sW[j * M + c * P + w], yv[c]);
      Eh[i] = net.adj(acc);
      if (j0 + i >= RMAX) Eh[i] = make_float2(0.f, 0.f);
    }
    float2 E[RMAX];
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
      const float2 mine = j < JH ? Eh[j] : Eh[j - JH];
      E[j] = ((j < JH) == (h == 0)) ? mine : make_float2(0.f, 0.f);
    }
    stageA_adj<Q>(E, x, bh);
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      x[l].x += __shfl_xor_sync(PFT_FULL_MASK, x[l].x, P);
      x[l].y += __shfl_xor_sync(PFT_FULL_MASK, x[l].y, P);
    }
  }
};

// The same 1-D transform on 32 lanes for P = 8: four 8-lane groups hold the
// same block and take four of the r terms each (group h: j = 4h .. 4h + 3;
// j >= r are zero pads), in stage A, the lane network and the W' sums; two
// shuffles across the groups add the partial sums. B comes from shared memory
// (sB[l * RMAX + j], rows l = 0 .. Q/2) because each group reads other terms.
template <int Q, int MP>
struct Pft1DSplit4 {
  static constexpr int P = 8;
  static constexpr int N = P * Q;
  static constexpr int M = MP * P;
  static constexpr int JH = 4;

  // Forward: every group holds x[Qk .. Qk+Q-1]; group h stores output c = h.
  template <class Store>
  __device__ __forceinline__ static void forward(const float2 (&x)[Q], int k, int h, const float* __restrict__ sB,
                                                 const float2* __restrict__ sW, const LaneNet<P, false>& net,
                                                 Store store) {
    constexpr int H = Q / 2;
    float2 s[H > 1 ? H : 1], d[H > 1 ? H : 1];
#pragma unroll
    for (int l = 1; l < H; ++l) {
      s[l] = cadd(x[l], x[Q - l]);
      d[l] = csub(x[l], x[Q - l]);
    }
    const int j0 = JH * h;  // even, so the parity of j is the parity of i
    float2 C[JH];
#pragma unroll
    for (int i = 0; i < JH; ++i) {
      const int j = min(j0 + i, RMAX - 1);
      float2 acc = cscale(x[0], sB[j]);
      if ((i & 1) == 0) {  // abscissa 0 (row Q/2) contributes to j = 0 only: B[Q/2][j] = a_j 0^j
        const float b = sB[H * RMAX + j];
        acc.x = fmaf(b, x[H].x, acc.x);
        acc.y = fmaf(b, x[H].y, acc.y);
      }
#pragma unroll
      for (int l = 1; l < H; ++l) {
        const float b = sB[l * RMAX + j];
        const float2 v = (i & 1) ? d[l] : s[l];
        acc.x = fmaf(b, v.x, acc.x);
        acc.y = fmaf(b, v.y, acc.y);
      }
      const float2 v = net.fwd(acc);
      C[i] = (j0 + i < RMAX) ? v : make_float2(0.f, 0.f);
    }
    const int w = Pft1D<P, Q, MP>::first_out(k);
#pragma unroll
    for (int c = 0; c < MP; ++c) {
      const int t = c * P + w;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < JH; ++i) acc = cfma(acc, sW[min(j0 + i, RMAX - 1) * M + t], C[i]);
#pragma unroll
      for (int o = 8; o <= 16; o <<= 1) {
        acc.x += __shfl_xor_sync(PFT_FULL_MASK, acc.x, o);
        acc.y += __shfl_xor_sync(PFT_FULL_MASK, acc.y, o);
      }
      if (c == h) store(t, acc);
    }
  }

  // Adjoint: every group loads the inputs of its residue; group h ends with
  // xq[i] = (A^H y)[Qk + h Q/4 + i], a quarter of the block.
  template <class Load>
  __device__ __forceinline__ static void adjoint(Load load, int k, int h, const float* __restrict__ sB,
                                                 const float2* __restrict__ sW, const LaneNet<P, false>& net,
                                                 float2 (&xq)[Q / 4]) {
    constexpr int H = Q / 2, QQ = Q / 4;
    const int w = Pft1D<P, Q, MP>::first_out(k);
    float2 yv[MP];
#pragma unroll
    for (int c = 0; c < MP; ++c) yv[c] = load(c * P + w);
    const int j0 = JH * h;
    float2 E[JH];
#pragma unroll
    for (int i = 0; i < JH; ++i) {
      const int jj = min(j0 + i, RMAX - 1);
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < MP; ++c) acc = cfmac(acc, sW[jj * M + c * P + w], yv[c]);
      const float2 v = net.adj(acc);
      E[i] = (j0 + i < RMAX) ? v : make_float2(0.f, 0.f);
    }
    // every term's E from its group (lane k of group g holds terms 4g .. 4g + 3)
    float2 Ea[4 * JH];
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
      for (int i = 0; i < JH; ++i) {
        Ea[JH * g + i].x = __shfl_sync(PFT_FULL_MASK, E[i].x, k + 8 * g);
        Ea[JH * g + i].y = __shfl_sync(PFT_FULL_MASK, E[i].y, k + 8 * g);
      }
    // x[l] = sum_j B[l][j] E[j]; B[Q - l][j] = (-1)^j B[l][j]
#pragma unroll
    for (int i = 0; i < QQ; ++i) {
      const int l = h * QQ + i;
      const bool up = l > H;
      const float* row = sB + (up ? Q - l : l) * RMAX;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < RMAX; ++j) {
        const float b = (up && (j & 1)) ? -row[j] : row[j];
        acc.x = fmaf(b, Ea[j].x, acc.x);
        acc.y = fmaf(b, Ea[j].y, acc.y);
      }
      xq[i] = acc;
    }
  }
};

}  // namespace pftk
