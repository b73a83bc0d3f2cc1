// Split-BF16 tensor-core adjoint PFT (tcgen05, sm_103a) for 256 x 256 frames
// with a 64 x 64 input (p = 32): x = A^H y conj(A) per frame, the exact
// conjugate transpose of the forward Y = A X A^T of pft_tc64.cu.
//
// Folding. A[-t] = conj(A[t]) for t = 1 .. 31, so per axis
//   x[v] = sum_t conj(A[t][v]) y[t]
//        = sum_{s in S} A_re[s][v] u[s] + A_im[s][v] w[s],   S = {0 .. 31, -32},
//   u[s] = y[s] + y[-s],  w[s] = -i (y[s] - y[-s])            (s = 1 .. 31),
//   u[s] = y[s],          w[s] = -i y[s]                      (s = 0, -32).
// The adjoint becomes a REAL table T[v][k] (K = 66, padded to 80: k < 32 holds
// A_re[k], 32 <= k < 64 A_im[k - 32], k = 64 / 65 A_re / A_im of row -32)
// applied to folded complex data, so T hi / lo takes 80 KB of shared memory
// instead of the 128 KB of the complex table.
//
// Per frame, in two column tiles h (v2 in [128 h, 128 h + 128)):
//   pass 1  U^T[v2][t1] = sum_k T[v2][k] F[t1][k]     F = Y folded along t2
//           (M = v2, N = [t1 re | t1 im] = 128, K = 80)
//   fold    G[v2][k]    = U^T[v2][.] folded along t1 (per TMEM lane, in registers)
//   pass 2  X^T[v2][v1] = sum_k G[v2][k] T[v1][k]     (M = v2, N = v1 in blocks
//           of 64, K = 80; D_re from G_re, D_im from G_im)
// TMEM lane = image column v2 in pass 2, so a warp stores 32 consecutive
// columns of one output row (256 contiguous bytes) per instruction. Every
// product is formed from three BF16 partial products (hi hi, lo hi, hi lo)
// with FP32 accumulation, as in the forward.
//
// Roles (persistent, one CTA per SM, 16 warps, tiles in order):
//   warps 12-15  load Y (64 x 64 complex), fold it along t2 and split it into
//                the pass-1 B operand;
//   warp 8       allocates tensor memory; one lane issues P1(tile 0), then per
//                tile: P1(next tile), P2(this tile);
//   warps 4-7    fold the pass-1 accumulators along t1 into the pass-2 A
//                operand G;
//   warps 0-3    read the pass-2 accumulators (three 128 x 64 tiles in
//                flight) and store X;
//   warps 9-11   pad the block to whole warp groups.
// Every wait is bounded (2 s); a timeout sets the plan's status word.
#include <cuda_bf16.h>

#include "coeffs.h"
#include "plan.cuh"
#include "tc.cuh"
#include "tc_table.cuh"

namespace {

using namespace tc;

constexpr int kN = 256, kM = 64, kK = 80;
constexpr uint32_t CM = 128;
// table T: [v: 256][k: 80] K-major in core matrices [k / 8][v / 8][8][16 B]; hi, lo
constexpr uint32_t T_LBO = (kN / 8) * CM;        // 4096
constexpr uint32_t T_COMP = (kK / 8) * T_LBO;    // 40960
constexpr uint32_t T_BYTES = 2 * T_COMP;
// pass-1 B operand F: rows [t1 re 0..63 | t1 im 0..63], K = 80; hi, lo
constexpr uint32_t F_LBO = (128 / 8) * CM;       // 2048
constexpr uint32_t F_COMP = (kK / 8) * F_LBO;    // 20480
constexpr uint32_t F_BYTES = 2 * F_COMP;
// pass-2 A operand G: rows v2 (128 of one tile), K = 80; re hi, re lo, im hi, im lo
constexpr uint32_t G_LBO = F_LBO;
constexpr uint32_t G_COMP = F_COMP;
constexpr uint32_t G_BYTES = 4 * G_COMP;
constexpr uint32_t OFF_TAB = 0;
constexpr uint32_t OFF_F = OFF_TAB + T_BYTES;
constexpr uint32_t OFF_G = OFF_F + F_BYTES;
constexpr uint32_t OFF_BAR = OFF_G + G_BYTES;
constexpr int kOBufs = 3;
constexpr int NBAR = 6 + 2 * kOBufs + 1;
constexpr uint32_t OFF_SLOT = OFF_BAR + 8 * NBAR;
constexpr uint32_t OFF_ABORT = OFF_SLOT + 8;
constexpr uint32_t SMEM_BYTES = OFF_ABORT + 8;
static_assert(SMEM_BYTES <= 232448, "shared memory layout too large");

constexpr int kE2Warp0 = 0, kE1Warp0 = 4, kMmaWarp = 8, kLdWarp0 = 12, kLdWarps = 4;
constexpr int kThreadsAdj = 32 * 16;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t P1_COLS = 128;     // U^T re (64) | U^T im (64)
constexpr uint32_t P2_BASE = P1_COLS;
constexpr uint32_t P2_COLS = 128;     // per output block: D_re (64) | D_im (64)
constexpr int kVBlocks = kN / 64;     // output blocks per tile (64 rows v1 each)
constexpr int kKSteps = kK / 16;
constexpr uint64_t kWaitNs = 2000000000ull;

static_assert(P2_BASE + kOBufs * P2_COLS <= TMEM_COLS, "tensor memory");

__device__ __forceinline__ uint4 split8(const float (&v)[8], uint4& lo) {
  __nv_bfloat162 h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(h[i]);
    l[i] = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
  }
  lo = *reinterpret_cast<uint4*>(l);
  return *reinterpret_cast<uint4*>(h);
}

// Writes 8 values as one 16-byte core-matrix row, hi at `hi_at`, lo `lo_off` later.
__device__ __forceinline__ void put8(uint8_t* hi_at, uint32_t lo_off, const float (&v)[8]) {
  uint4 lo;
  const uint4 hi = split8(v, lo);
  *reinterpret_cast<uint4*>(hi_at) = hi;
  *reinterpret_cast<uint4*>(hi_at + lo_off) = lo;
}

__global__ void __launch_bounds__(kThreadsAdj, 1)
    k_pft_tc64_adj(const float2* __restrict__ y, float2* __restrict__ x, long long batch,
                   const uint4* __restrict__ tab, int* status) {
  extern __shared__ __align__(128) uint8_t sm[];
  const uint32_t sb = smem_u32(sm);
  const uint32_t bar = sb + OFF_BAR;
  const uint32_t F_FULL = bar, F_EMPTY = bar + 8, P1_FULL = bar + 16, P1_EMPTY = bar + 24, G_FULL = bar + 32,
                 G_EMPTY = bar + 40, O_FULL = bar + 48, O_EMPTY = O_FULL + 8 * kOBufs,
                 DONE = O_EMPTY + 8 * kOBufs;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF_ABORT);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + OFF_SLOT);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int i = threadIdx.x; i < (int)(T_BYTES / 16); i += blockDim.x)
    reinterpret_cast<uint4*>(sm + OFF_TAB)[i] = __ldg(tab + i);
  // the padding columns k = 66 .. 79 of F and G are never written again
  for (int i = threadIdx.x; i < (int)((F_BYTES + G_BYTES) / 16); i += blockDim.x)
    reinterpret_cast<uint4*>(sm + OFF_F)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    mbar_init(F_FULL, kLdWarps);
    mbar_init(F_EMPTY, 1);
    mbar_init(P1_FULL, 1);
    mbar_init(P1_EMPTY, 4);
    mbar_init(G_FULL, 4);
    mbar_init(G_EMPTY, 1);
    for (int d = 0; d < kOBufs; ++d) {
      mbar_init(O_FULL + 8 * d, 1);
      mbar_init(O_EMPTY + 8 * d, 4);
    }
    mbar_init(DONE, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {
    tmem_alloc(smem_u32(tslot), TMEM_COLS);
    tmem_relinquish();
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const long long nloc = blockIdx.x < batch ? (batch - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const long long ntiles = 2 * nloc;

  if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc1 = idesc_bf16(128, 128), idesc2 = idesc_bf16(128, 64);
      const uint32_t tb = sb + OFF_TAB, fb = sb + OFF_F, gb = sb + OFF_G;
      auto pass1 = [&](long long tau) -> bool {
        const long long fi = tau >> 1;
        const int h = (int)(tau & 1);
        if (h == 0 && !mbar_wait(F_FULL, (uint32_t)fi & 1u, abort_flag, kWaitNs)) return false;
        if (!mbar_wait(P1_EMPTY, ((uint32_t)tau & 1u) ^ 1u, abort_flag, kWaitNs)) return false;
        tc_fence_after();
#pragma unroll
        for (int ks = 0; ks < kKSteps; ++ks) {
          const uint32_t acc = ks;
          const uint32_t ta = tb + ks * 2 * T_LBO + h * 16 * CM;
          const uint64_t th = sdesc(ta, T_LBO, CM), tl = sdesc(ta + T_COMP, T_LBO, CM);
          const uint32_t fa = fb + ks * 2 * F_LBO;
          const uint64_t fh = sdesc(fa, F_LBO, CM), fl = sdesc(fa + F_COMP, F_LBO, CM);
          mma_bf16(tmem, th, fh, idesc1, acc);
          mma_bf16(tmem, tl, fh, idesc1, 1);
          mma_bf16(tmem, th, fl, idesc1, 1);
        }
        if (h == 1) mma_commit(F_EMPTY);
        mma_commit(P1_FULL);
        return true;
      };
      auto pass2 = [&](long long tau) -> bool {
        for (int b = 0; b < kVBlocks; ++b) {
          const long long T2 = tau * kVBlocks + b;
          const int d = (int)(T2 % kOBufs);
          const uint32_t use = (uint32_t)(T2 / kOBufs);
          if (!mbar_wait(O_EMPTY + 8 * d, (use & 1u) ^ 1u, abort_flag, kWaitNs)) return false;
          tc_fence_after();
          const uint32_t dr = tmem + P2_BASE + d * P2_COLS, di = dr + 64;
#pragma unroll
          for (int ks = 0; ks < kKSteps; ++ks) {
            const uint32_t acc = ks;
            const uint32_t ga = gb + ks * 2 * G_LBO;
            const uint64_t grh = sdesc(ga, G_LBO, CM), grl = sdesc(ga + G_COMP, G_LBO, CM);
            const uint64_t gih = sdesc(ga + 2 * G_COMP, G_LBO, CM), gil = sdesc(ga + 3 * G_COMP, G_LBO, CM);
            const uint32_t ta = tb + ks * 2 * T_LBO + b * 8 * CM;
            const uint64_t th = sdesc(ta, T_LBO, CM), tl = sdesc(ta + T_COMP, T_LBO, CM);
            mma_bf16(dr, grh, th, idesc2, acc);
            mma_bf16(dr, grl, th, idesc2, 1);
            mma_bf16(dr, grh, tl, idesc2, 1);
            mma_bf16(di, gih, th, idesc2, acc);
            mma_bf16(di, gil, th, idesc2, 1);
            mma_bf16(di, gih, tl, idesc2, 1);
          }
          mma_commit(O_FULL + 8 * d);
        }
        mma_commit(G_EMPTY);
        return true;
      };
      bool ok = ntiles == 0 || pass1(0);
      for (long long tau = 0; tau < ntiles && ok; ++tau) {
        ok = mbar_wait(G_FULL, (uint32_t)tau & 1u, abort_flag, kWaitNs);
        if (ok) tc_fence_after();
        if (ok && tau + 1 < ntiles) ok = pass1(tau + 1);
        if (ok) ok = pass2(tau);
      }
      volatile int never = 0;
      mma_commit(DONE);
      mbar_wait(DONE, 0, &never, kWaitNs);
    }
    __syncwarp();
  } else if (warp >= kE1Warp0 && warp < kE1Warp0 + 4) {
    // ------------------------------- pass-1 accumulators -> folded operand G
    const int q = warp - kE1Warp0;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    uint8_t* g = sm + OFF_G + (uint32_t)(q * 32 + lane) * 16;
    for (long long tau = 0; tau < ntiles; ++tau) {
      if (!mbar_wait(P1_FULL, (uint32_t)tau & 1u, abort_flag, kWaitNs)) break;
      tc_fence_after();
      // U^T[v2][t1] sits at column t1 + 32 (re) and 64 + t1 + 32 (im). Per
      // component, columns 16 .. 47 give the fold groups j0 = 0, 8 and
      // columns 0 .. 16, 48 .. 63 the groups j0 = 16, 24 and the row -32.
      // The real parts give G_re[j] = U_re[j] + U_re[-j] and
      // G_im[32 + j] = -(U_re[j] - U_re[-j]); the imaginary parts
      // G_im[j] = U_im[j] + U_im[-j] and G_re[32 + j] = U_im[j] - U_im[-j].
      bool ok = true;
      float c0v[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const uint32_t col = tmem + lane_off + 64 * c;
        uint8_t* gs = g + (c == 0 ? 0u : 2 * G_COMP);      // sums
        uint8_t* gd = g + (c == 0 ? 2 * G_COMP : 0u);      // differences
        const float sgn = c == 0 ? -1.f : 1.f;
        float lo[16], hi[16];
        tmem_ld16(col + 16, lo);
        tmem_ld16(col + 32, hi);
        tmem_wait_ld();
        if (c == 0 && !mbar_wait(G_EMPTY, ((uint32_t)tau & 1u) ^ 1u, abort_flag, kWaitNs)) {
          ok = false;
          break;
        }
        const float c16 = lo[0];
#pragma unroll
        for (int j0 = 0; j0 < 16; j0 += 8) {
          float s[8], d[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const int j = j0 + m;
            const float pv = hi[j], mv = j == 0 ? 0.f : lo[16 - j];
            s[m] = pv + mv;
            d[m] = sgn * (pv - mv);
          }
          put8(gs + (j0 / 8) * G_LBO, G_COMP, s);
          put8(gd + (4 + j0 / 8) * G_LBO, G_COMP, d);
        }
        tmem_ld16(col, lo);
        tmem_ld16(col + 48, hi);
        tmem_wait_ld();
        if (c == 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(P1_EMPTY);
        }
        c0v[c] = lo[0];
#pragma unroll
        for (int j0 = 16; j0 < 32; j0 += 8) {
          float s[8], d[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const int j = j0 + m;
            const float pv = hi[j - 16], mv = j == 16 ? c16 : lo[32 - j];
            s[m] = pv + mv;
            d[m] = sgn * (pv - mv);
          }
          put8(gs + (j0 / 8) * G_LBO, G_COMP, s);
          put8(gd + (4 + j0 / 8) * G_LBO, G_COMP, d);
        }
      }
      if (!ok) break;
      const float ur0 = c0v[0], ui0 = c0v[1];
      // row -32: u = U[-32] at k = 64, w = -i U[-32] at k = 65
      const float tre[8] = {ur0, ui0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const float tim[8] = {ui0, -ur0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      put8(g + 8 * G_LBO, G_COMP, tre);
      put8(g + 2 * G_COMP + 8 * G_LBO, G_COMP, tim);
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(G_FULL);
    }
  } else if (warp < kE2Warp0 + 4) {
    // ------------------------------------------ pass-2 accumulators -> X
    const int q = warp - kE2Warp0;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    bool ok = true;
    for (long long tau = 0; tau < ntiles && ok; ++tau) {
      const long long f = blockIdx.x + (tau >> 1) * gridDim.x;
      const int v2 = (int)(tau & 1) * 128 + q * 32 + lane;
      float2* xf = x + f * (long long)(kN * kN) + v2;
      for (int b = 0; b < kVBlocks; ++b) {
        const long long T2 = tau * kVBlocks + b;
        const int d = (int)(T2 % kOBufs);
        if (!mbar_wait(O_FULL + 8 * d, (uint32_t)(T2 / kOBufs) & 1u, abort_flag, kWaitNs)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dr = tmem + lane_off + P2_BASE + d * P2_COLS, di = dr + 64;
#pragma unroll
        for (int pc = 0; pc < 4; ++pc) {
          float re[16], im[16];
          tmem_ld16(dr + 16 * pc, re);
          tmem_ld16(di + 16 * pc, im);
          tmem_wait_ld();
          if (pc == 3) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(O_EMPTY + 8 * d);
          }
          float2* dst = xf + (long long)(b * 64 + 16 * pc) * kN;
#pragma unroll
          for (int j = 0; j < 16; ++j) dst[j * kN] = make_float2(re[j], im[j]);
        }
      }
    }
  } else if (warp >= kLdWarp0) {
    // ------------------------ Y -> folded pass-1 B operand F (rows t1 re | t1 im)
    const int i = threadIdx.x - kLdWarp0 * 32;   // 0..127
    const int t1 = i & 63;                       // row index t1 + 32 of Y
    const int jh = i >> 6;                       // fold groups j0 = 16 jh, 16 jh + 8
    uint8_t* fre = sm + OFF_F + (uint32_t)t1 * 16;
    uint8_t* fim = fre + 64 * 16;
    for (long long fi = 0; fi < nloc; ++fi) {
      const long long f = blockIdx.x + fi * gridDim.x;
      const float2* row = y + f * (long long)(kM * kM) + t1 * kM;
      // per group: Y[t1][32 + j0 ..] (plus), Y[t1][24 - j0 .. 31 - j0] and Y[t1][32 - j0] (minus side)
      float4 pl[2][4], mi[2][4];
      float2 edge[2];
#pragma unroll
      for (int gi = 0; gi < 2; ++gi) {
        const int j0 = 16 * jh + 8 * gi;
        const float4* p4 = reinterpret_cast<const float4*>(row + 32 + j0);
        const float4* m4 = reinterpret_cast<const float4*>(row + 24 - j0);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          pl[gi][e] = __ldg(p4 + e);
          mi[gi][e] = __ldg(m4 + e);
        }
        edge[gi] = __ldg(row + 32 - j0);
      }
      const float2 tail = __ldg(row);   // t2 = -32
      if (!mbar_wait(F_EMPTY, ((uint32_t)fi & 1u) ^ 1u, abort_flag, kWaitNs)) break;
#pragma unroll
      for (int gi = 0; gi < 2; ++gi) {
        const int j0 = 16 * jh + 8 * gi;
        float ur[8], ui[8], wr[8], wi[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          // plus: Y[t1][j0 + m]; minus: Y[t1][-(j0 + m)] (column 32 - j0 - m)
          const float4 pq = pl[gi][m >> 1];
          const float pr = (m & 1) ? pq.z : pq.x, pi = (m & 1) ? pq.w : pq.y;
          float mr, mim;
          if (m == 0) {
            mr = edge[gi].x;
            mim = edge[gi].y;
            if (j0 == 0) mr = mim = 0.f;   // t2 = 0 has no partner
          } else {
            const float4 mq = mi[gi][(8 - m) >> 1];
            mr = ((8 - m) & 1) ? mq.z : mq.x;
            mim = ((8 - m) & 1) ? mq.w : mq.y;
          }
          ur[m] = pr + mr;
          ui[m] = pi + mim;
          wr[m] = pi - mim;      // w = -i (plus - minus)
          wi[m] = mr - pr;
        }
        put8(fre + (j0 / 8) * F_LBO, F_COMP, ur);
        put8(fim + (j0 / 8) * F_LBO, F_COMP, ui);
        put8(fre + (4 + j0 / 8) * F_LBO, F_COMP, wr);
        put8(fim + (4 + j0 / 8) * F_LBO, F_COMP, wi);
      }
      if (jh == 1) {
        const float tre[8] = {tail.x, tail.y, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const float tim[8] = {tail.y, -tail.x, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        put8(fre + 8 * F_LBO, F_COMP, tre);
        put8(fim + 8 * F_LBO, F_COMP, tim);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(F_FULL);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
  if (threadIdx.x == 0 && *abort_flag) {
    *reinterpret_cast<volatile int*>(status) = PFT_ERR_TIMEOUT;
    __threadfence_system();
  }
}

// Real adjoint table T[v][k] split into BF16 hi / lo: for the stored rows
// s = 0 .. 31 (t = s) and s = 32 (t = -32), A_re[s][v] at k = s (64 for
// t = -32) and A_im[s][v] at k = 32 + s (65 for t = -32). The buffer is
// zeroed before, so k = 66 .. 79 stay 0.
__global__ void k_tc64_table_adj(int p, int q, int r, const double* __restrict__ a, uint16_t* __restrict__ tab) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (kM / 2 + 1) * kN) return;
  const int s = id / kN, v = id % kN;
  const int t = s < kM / 2 ? s : -kM / 2;
  double ar, ai;
  operator_entry(kM, p, q, r, a, t + kM / 2, v, ar, ai);
  auto at = [&](int k) {
    return ((uint32_t)(k / 8) * T_LBO + (uint32_t)(v / 8) * CM + (uint32_t)(v % 8) * 16 + (uint32_t)(k % 8) * 2) / 2;
  };
  const int kr = s < kM / 2 ? s : 64, ki = s < kM / 2 ? kM / 2 + s : 65;
  uint16_t hi, lo;
  split_bf16(ar, hi, lo);
  tab[at(kr)] = hi;
  tab[T_COMP / 2 + at(kr)] = lo;
  split_bf16(ai, hi, lo);
  tab[at(ki)] = hi;
  tab[T_COMP / 2 + at(ki)] = lo;
}

}  // namespace

namespace pfth {

int tc64_build_adjoint_table(pft_plan* plan) {
  double xi = 0.0, a[pftc::kMaxTerms] = {0};
  if (!pftc::design(plan->eps, plan->r1, &xi, a, nullptr))
    return set_error(PFT_ERR_INVALID_ARG, "coefficient design failed (eps=%g r=%d)", plan->eps, plan->r1);
  double* d_a = nullptr;
  PFT_CUDA_TRY(cudaMalloc(&d_a, sizeof(double) * pftc::kMaxTerms));
  PFT_CUDA_TRY(cudaMemcpy(d_a, a, sizeof(double) * plan->r1, cudaMemcpyHostToDevice));
  PFT_CUDA_TRY(cudaMalloc(&plan->d_tc_adj, T_BYTES));
  PFT_CUDA_TRY(cudaMemset(plan->d_tc_adj, 0, T_BYTES));
  k_tc64_table_adj<<<((kM / 2 + 1) * kN + 127) / 128, 128>>>(plan->p1, plan->q1, plan->r1, d_a,
                                                              reinterpret_cast<uint16_t*>(plan->d_tc_adj));
  PFT_CUDA_TRY(cudaGetLastError());
  PFT_CUDA_TRY(cudaDeviceSynchronize());
  PFT_CUDA_TRY(cudaFree(d_a));
  return PFT_OK;
}

int tc64_adjoint(const pft_plan* plan, const void* y, void* x, int64_t batch, void* stream) {
  if (*plan->h_status != PFT_OK) {
    const int st = *plan->h_status;
    *plan->h_status = PFT_OK;
    return set_error(st, "a device-side wait of an earlier split-BF16 launch timed out");
  }
  static bool attr_set = false;
  if (!attr_set) {
    PFT_CUDA_TRY(
        cudaFuncSetAttribute(k_pft_tc64_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
    attr_set = true;
  }
  long long grid = sm_count();
  if (grid > batch) grid = batch;
  k_pft_tc64_adj<<<(unsigned)grid, kThreadsAdj, SMEM_BYTES, (cudaStream_t)stream>>>(
      (const float2*)y, (float2*)x, (long long)batch, (const uint4*)plan->d_tc_adj, plan->d_status);
  PFT_CUDA_TRY(cudaGetLastError());
  return PFT_OK;
}

}  // namespace pfth
