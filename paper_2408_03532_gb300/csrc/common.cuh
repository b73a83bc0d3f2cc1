// Shared device helpers of the GB300 PFT / PIE library (sm_103a).
//
// Complex numbers are float2 (x = real, y = imaginary). The DFT networks below
// are radix-2 decimation-in-frequency butterflies either across the lanes of a
// warp (lane_dif) or across the registers of one thread (reg_dif), and their
// exact adjoints (the same butterflies in reverse order with conjugated
// twiddles). Forward networks take natural order and leave bit-reversed order;
// the adjoint networks take that bit-reversed order back to natural order, so
// forward and adjoint passes never need an explicit permutation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pft.h"

#define PFT_FULL_MASK 0xffffffffu

namespace pftk {

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// acc + a * b
__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
// acc + conj(a) * b
__device__ __forceinline__ float2 cfmac(float2 acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  v.x = __shfl_xor_sync(PFT_FULL_MASK, v.x, m);
  v.y = __shfl_xor_sync(PFT_FULL_MASK, v.y, m);
  return v;
}

template <int L>
__host__ __device__ constexpr int ilog2() { return L <= 1 ? 0 : 1 + ilog2<L / 2>(); }

template <int L>
__host__ __device__ __forceinline__ int bitrev(int k) {
  int r = 0;
#pragma unroll
  for (int b = 0; b < ilog2<L>(); ++b) r |= ((k >> b) & 1) << (ilog2<L>() - 1 - b);
  return r;
}

// ------------------------------------------------------- lane DFT network
// Stage table of an L-lane network: entry (h - 1) + m holds w_{2h}^m =
// e^{-2 pi i m / (2h)} for h = 1, 2, 4, ..., L/2 and m < h (L - 1 entries), so
// the lanes of one stage read consecutive entries (no bank conflicts).
// src[i] = e^{-2 pi i i / NS}; NS is a multiple of L.
template <int L>
__device__ __forceinline__ void fill_stage_table(float2* tws, const float2* __restrict__ src, int NS) {
  for (int i = threadIdx.x; i < L - 1; i += blockDim.x) {
    int h = 1;
    while (2 * h <= i + 1) h *= 2;
    tws[i] = src[(i + 1 - h) * (NS / (2 * h))];
  }
}

// Asynchronous global -> shared copies (cp.async, L1-allocating): the caller
// commits the group and waits for it before the data are read.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// fill_stage_table through cp.async.
template <int L>
__device__ __forceinline__ void fill_stage_table_async(float2* tws, const float2* __restrict__ src, int NS) {
  for (int i = threadIdx.x; i < L - 1; i += blockDim.x) {
    int h = 1;
    while (2 * h <= i + 1) h *= 2;
    cp_async8(tws + i, src + (i + 1 - h) * (NS / (2 * h)));
  }
}

// L-point DFT across groups of L consecutive lanes (L <= 32, a power of two).
// In: lane k (= lane % L) holds x[k]. Out: lane k holds X[bitrev_L(k)], with
// X[f] = sum_k x[k] w^{f k}, w = e^{-2 pi i / L} (conjugated when INV).
// tws: the stage table above (shared memory).
template <int L, bool INV>
__device__ __forceinline__ float2 lane_dif(float2 v, int k, const float2* __restrict__ tws) {
#pragma unroll
  for (int h = L / 2; h >= 1; h >>= 1) {
    float2 o = shfl_xor2(v, h);
    if (k & h) {
      float2 w = tws[h - 1 + (k & (h - 1))];
      if (INV) w.y = -w.y;
      v = cmul(csub(o, v), w);
    } else {
      v = cadd(v, o);
    }
  }
  return v;
}

// Exact adjoint of lane_dif<L, INV>: lane k holds Y[bitrev(k)] on entry and
// sum_f conj(w)^{f k} Y[f] on exit (natural order).
template <int L, bool INV>
__device__ __forceinline__ float2 lane_dif_adj(float2 v, int k, const float2* __restrict__ tws) {
#pragma unroll
  for (int h = 1; h <= L / 2; h <<= 1) {
    float2 s = v;
    if (k & h) {
      float2 w = tws[h - 1 + (k & (h - 1))];
      if (!INV) w.y = -w.y;
      s = cmul(v, w);
    }
    float2 o = shfl_xor2(s, h);
    v = (k & h) ? csub(o, s) : cadd(v, o);
  }
  return v;
}

// The same network with each lane's twiddles and signs held in registers.
// Lane k's twiddle and sign at every stage depend only on k, so they are
// loaded once; each butterfly is then branch-free: two shuffles, d = o + sg v,
// and a complex multiply by the lane's twiddle (1 for the lower lane, and
// skipped at the last stage where every twiddle is 1).
template <int L, bool INV>
struct LaneNet {
  static constexpr int S = ilog2<L>() > 0 ? ilog2<L>() : 1;
  float2 w[S];
  float sg[S];
  __device__ __forceinline__ void init(int k, const float2* __restrict__ tws) {
#pragma unroll
    for (int s = 0; s < ilog2<L>(); ++s) {
      const int h = L >> (s + 1);
      const bool up = (k & h) != 0;
      float2 t = up ? tws[h - 1 + (k & (h - 1))] : make_float2(1.f, 0.f);
      if (INV) t.y = -t.y;
      w[s] = t;
      sg[s] = up ? -1.f : 1.f;
    }
  }
  // = lane_dif<L, INV>
  __device__ __forceinline__ float2 fwd(float2 v) const {
#pragma unroll
    for (int s = 0; s < ilog2<L>(); ++s) {
      const int h = L >> (s + 1);
      const float2 o = shfl_xor2(v, h);
      const float2 d = make_float2(fmaf(sg[s], v.x, o.x), fmaf(sg[s], v.y, o.y));
      v = (h == 1) ? d : cmul(d, w[s]);
    }
    return v;
  }
  // = lane_dif_adj<L, INV> (the exact adjoint of fwd)
  __device__ __forceinline__ float2 adj(float2 v) const {
#pragma unroll
    for (int s = ilog2<L>() - 1; s >= 0; --s) {
      const int h = L >> (s + 1);
      const float2 t = (h == 1) ? v : cmulc(v, w[s]);
      const float2 o = shfl_xor2(t, h);
      v = make_float2(fmaf(sg[s], t.x, o.x), fmaf(sg[s], t.y, o.y));
    }
    return v;
  }
};

// ---------------------------------------------------- register DFT network
// E-point DFT over the registers of one thread (E a power of two <= 16).
// In: x[e] natural. Out: x[pos] = X[bitrev_E(pos)]. twN[m] = e^{-2 pi i m / N}
// with N a multiple of E (so w_E^m = twN[m N / E]).
template <int E, bool INV>
__device__ __forceinline__ void reg_dif(float2 (&x)[E], const float2* __restrict__ twN, int N) {
#pragma unroll
  for (int h = E / 2; h >= 1; h >>= 1) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      if ((i & h) == 0) {
        float2 a = x[i], b = x[i + h];
        x[i] = cadd(a, b);
        int m = i & (h - 1);
        float2 d = csub(a, b);
        if (m == 0) {
          x[i + h] = d;
        } else {
          float2 w = twN[m * (N / (2 * h))];
          if (INV) w.y = -w.y;
          x[i + h] = cmul(d, w);
        }
      }
    }
  }
}

// Exact adjoint of reg_dif<E, INV>.
template <int E, bool INV>
__device__ __forceinline__ void reg_dif_adj(float2 (&x)[E], const float2* __restrict__ twN, int N) {
#pragma unroll
  for (int h = 1; h <= E / 2; h <<= 1) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      if ((i & h) == 0) {
        int m = i & (h - 1);
        float2 U = x[i + h];
        if (m != 0) {
          float2 w = twN[m * (N / (2 * h))];
          if (!INV) w.y = -w.y;
          U = cmul(U, w);
        }
        float2 Lv = x[i];
        x[i] = cadd(Lv, U);
        x[i + h] = csub(Lv, U);
      }
    }
  }
}

// ------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(PFT_FULL_MASK, v, o);
  return v;
}

// Block-wide sum of one double per thread; result valid in thread 0.
// `red` is shared scratch of at least blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

}  // namespace pftk

// ----------------------------------------------------------- host errors
namespace pfth {
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);
int sm_count();
}  // namespace pfth

#define PFT_CUDA_TRY(call)                                   \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return pfth::cuda_error(_e, #call); \
  } while (0)
