// FP64 entries of the folded 1-D PFT operator and their BF16 hi / lo split,
// shared by the tensor-core forward and adjoint table builders.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace tc {

// A[t][v] for the 1-D PFT of Algorithm 5 with v = q k + l, t = ti - M/2:
//   A[t][v] = e^{-2 pi i t k / p} sum_j W'[t, j] B[l, j],
//   W'[t, j] = (t / p)^j e^{i pi m / p}, m = (j p / 2 - t) mod 2p  (= i^j (t/p)^j e^{-i pi t / p}),
//   B[l, j]  = a_j (1 - 2 l / q)^j,
// in FP64 with the phases reduced exactly in integers (p even).
__device__ inline void operator_entry(int M, int p, int q, int r, const double* __restrict__ a, int ti, int v,
                                      double& ar, double& ai) {
  const long long t = (long long)ti - M / 2;
  const int kb = v / q, l = v % q;
  double sr = 0.0, si = 0.0;
  for (int j = 0; j < r; ++j) {
    const double wmag = (j == 0) ? 1.0 : pow((double)t / (double)p, (double)j);
    const double bval = a[j] * ((j == 0) ? 1.0 : pow((double)(q - 2 * l) / (double)q, (double)j));
    long long m = ((long long)j * (p / 2) - t) % (2LL * p);
    if (m < 0) m += 2LL * p;
    double s, c;
    sincospi((double)m / (double)p, &s, &c);
    sr += wmag * bval * c;
    si += wmag * bval * s;
  }
  long long mm = (t * kb) % p;
  if (mm < 0) mm += p;
  double s, c;
  sincospi(-2.0 * (double)mm / (double)p, &s, &c);
  ar = sr * c - si * s;
  ai = sr * s + si * c;
}

// v = hi + lo + O(2^-17 |v|), hi and lo BF16 (bit patterns).
__device__ inline void split_bf16(double v, uint16_t& hi, uint16_t& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
  const __nv_bfloat16 l = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
  hi = __bfloat16_as_ushort(h);
  lo = __bfloat16_as_ushort(l);
}

}  // namespace tc
