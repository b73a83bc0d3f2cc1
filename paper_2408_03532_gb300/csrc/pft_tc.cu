// Split-BF16 tensor-core PFT (tcgen05, sm_103a) for batches of 256 x 256
// frames with a 32 x 32 output.
//
// Operator. Per axis the PFT of Algorithm 5 is a linear map C^n -> C^M,
//   A[t, q k + l] = e^{-2 pi i t k / p} sum_j W'[t, j] B[l, j]
// (stage A contracts l with B, stage B is the p-point DFT over k followed by
// the W' combine; W' carries i^j so that B is real). The 2-D transform is
// Y = A X A^T. On tensor cores both passes run as dense contractions against
// this folded expansion table, built once per plan in FP64 (integer phase
// reduction) and stored as BF16 hi + lo parts: at n / M = 8 the contraction
// is far from the bound, which is the HBM read of the frames.
//
// Precision. Every operand v is split as v = hi + lo + O(2^-17 |v|) with hi
// and lo BF16; each product is formed as hi*hi + lo*hi + hi*lo with FP32
// accumulation in tensor memory (three MMAs into one accumulator), so each
// product carries a relative error of about 3 * 2^-18.
//
// Work split per CTA (persistent, one CTA per SM, 24 warps):
//   warps 8-23  load 4 frames x 32 rows x 32 columns of X per stage from HBM
//               (coalesced 16-byte loads, two stages in flight per thread),
//               split them into Re/Im hi/lo BF16 and store the MMA A-operand
//               tiles (warps 5-7 only pad the block to whole warp groups);
//   warp 4      allocates tensor memory; one lane issues all MMAs:
//               row pass   T[(f, u), t2] = sum_v X_f[u, v] A[t2, v]
//               column pass Y_f[t1, t2] = sum_u T[(f, u), t2] A[t1, u]
//               (the row-pass tile of 4 frames x 32 rows is the column pass's
//               K chunk, so T never leaves the SM);
//   warps 0-3   read the row-pass accumulators (TMEM lane = (frame, row)),
//               combine Re/Im, split T into BF16 hi/lo column-pass operands,
//               and after the last row tile write Y (lane = (frame, t2)).
// Accumulators: Z1 = X_re [A_re | A_im], Z2 = X_im [A_re | A_im] (N = 64),
// T_re = Z1[:, 0:32] - Z2[:, 32:64], T_im = Z1[:, 32:64] + Z2[:, 0:32].
// Every wait is bounded (2 s); a timeout sets the plan's status word and all
// roles leave their loops; tensor memory is always released.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>

#include "coeffs.h"
#include "plan.cuh"
#include "tc.cuh"
#include "tc_table.cuh"

namespace {

using namespace tc;

constexpr int kN = 256;                 // frame side
constexpr int kM = 32;                  // output side
constexpr int kF = 128 / kM;            // frames per group (column-pass M = 128)
constexpr int kR = 128 / kF;            // rows per frame in one row tile
constexpr int kTiles = kN / kR;         // row tiles per group
constexpr int kC = 32;                  // K columns per X stage
constexpr int kChunks = kN / kC;        // X stages per row tile
constexpr int kStages = 4;
constexpr int kA2 = 1;                  // column-pass operand buffers
constexpr int kTabRows = 4 * kM;        // A_re hi, A_im hi, A_re lo, A_im lo
constexpr uint32_t CM = 128;            // bytes of one 8 x 16-byte core matrix
constexpr uint32_t TAB_LBO = (kTabRows / 8) * CM;        // 2048
constexpr uint32_t TAB_BYTES = (kN / 8) * TAB_LBO;       // 65536
constexpr uint32_t TAB_B2 = (2 * kM / 8) * CM;           // offset of the lo half (rows 2M..4M)
constexpr uint32_t X_LBO = 16 * CM + 32;                 // padded: conflict-free 4-byte stores
constexpr uint32_t X_COMP = (kC / 8) * X_LBO;
constexpr uint32_t X_STAGE = 4 * X_COMP;
constexpr uint32_t A2_LBO = 16 * CM + 32;
constexpr uint32_t A2_COMP = (kR / 8) * A2_LBO + 16;  // +16: hi / lo words on different banks
constexpr uint32_t A2_STAGE = 4 * A2_COMP;
constexpr uint32_t OFF_TAB = 0;
constexpr uint32_t OFF_X = OFF_TAB + TAB_BYTES;
constexpr uint32_t OFF_A2 = OFF_X + kStages * X_STAGE;
constexpr uint32_t OFF_BAR = OFF_A2 + kA2 * A2_STAGE;
constexpr int NBAR = 2 * kStages + 8 + 3;
constexpr uint32_t OFF_SLOT = OFF_BAR + 8 * NBAR;
constexpr uint32_t OFF_ABORT = OFF_SLOT + 8;
constexpr uint32_t SMEM_USED = OFF_ABORT + 8;
// The full opt-in shared memory is requested: every descriptor read then stays
// inside the CTA's allocation even under the other reading of LBO and SBO.
constexpr uint32_t SMEM_BYTES = 232448;
static_assert(SMEM_USED <= SMEM_BYTES, "shared memory layout too large");

constexpr int kEpiWarps = 4, kMmaWarp = 4, kCvtWarp0 = 8, kCvtWarps = 16;  // warps 5-7 idle
constexpr int kThreadsTC = 32 * (kCvtWarp0 + kCvtWarps);
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COLS = 4 * kM;   // Z1 | Z2 of one row tile
constexpr uint32_t COL_ACC = 2 * ACC_COLS;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kRowsPerThread = 128 / (2 * kCvtWarps);  // 4
constexpr int kDepth = 3;  // X stages held in registers per loader thread (2 in flight)

static_assert(kF * kR == 128 && kTiles * kR == kN && kChunks * kC == kN, "tiling");
static_assert(COL_ACC + ACC_COLS <= TMEM_COLS, "tensor memory");
static_assert(kA2 == 1 || kA2 == 2, "column-pass operand buffers");

__device__ __forceinline__ void split_store(uint8_t* base, uint32_t comp_bytes, uint32_t off, float a, float b) {
  const __nv_bfloat162 hi = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(hi);
  const __nv_bfloat162 lo = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  *reinterpret_cast<__nv_bfloat162*>(base + off) = hi;
  *reinterpret_cast<__nv_bfloat162*>(base + comp_bytes + off) = lo;
}

// Each lane stores its own BF16 hi and lo parts (2-byte stores): lanes are
// K-adjacent rows, so a warp fills whole 16-byte core-matrix rows without any
// lane exchange.
__device__ __forceinline__ void own_store(uint8_t* base, uint32_t off, uint32_t lo_off, float v) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
  *reinterpret_cast<__nv_bfloat16*>(base + off) = hi;
  *reinterpret_cast<__nv_bfloat16*>(base + lo_off + off) = lo;
}

__global__ void __launch_bounds__(kThreadsTC, 1)
    k_pft_tc_fwd(const float2* __restrict__ x, float2* __restrict__ y, long long batch,
                 const uint4* __restrict__ tab, int* status) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t* sm = smem_raw;  // no-swizzle operands need 16-byte alignment only
  const uint32_t sb = smem_u32(sm);
  const uint32_t bar = sb + OFF_BAR;
  const uint32_t X_FULL = bar, X_EMPTY = bar + 8 * kStages, ACC_FULL = bar + 16 * kStages,
                 ACC_EMPTY = ACC_FULL + 16, A2_FULL = ACC_FULL + 32, A2_EMPTY = ACC_FULL + 48,
                 COL_FULL = ACC_FULL + 64, COL_EMPTY = ACC_FULL + 72, DONE = ACC_FULL + 80;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF_ABORT);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + OFF_SLOT);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int i = threadIdx.x; i < (int)(TAB_BYTES / 16); i += blockDim.x)
    reinterpret_cast<uint4*>(sm + OFF_TAB)[i] = __ldg(tab + i);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(X_FULL + 8 * s, kCvtWarps);
      mbar_init(X_EMPTY + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(ACC_FULL + 8 * b, 1);
      mbar_init(ACC_EMPTY + 8 * b, kEpiWarps);
      mbar_init(A2_FULL + 8 * b, kEpiWarps);
      mbar_init(A2_EMPTY + 8 * b, 1);
    }
    mbar_init(COL_FULL, 1);
    mbar_init(COL_EMPTY, kEpiWarps);
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
  const long long ngroups = (batch + kF - 1) / kF;
  const long long nloc = blockIdx.x < ngroups ? (ngroups - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const long long ntiles = nloc * kTiles;

  if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(128, 2 * kM);
      bool ok = true;
      auto col_pass = [&](long long Tp) -> bool {
        const int ip = (int)(Tp % kTiles);
        const int b = (int)(Tp % kA2);
        const uint32_t v = (uint32_t)(Tp / kA2);
        if (ip == 0 && !mbar_wait(COL_EMPTY, ((uint32_t)(Tp / kTiles) & 1u) ^ 1u, abort_flag, kWaitNs)) return false;
        if (!mbar_wait(A2_FULL + 8 * b, v & 1u, abort_flag, kWaitNs)) return false;
        tc_fence_after();
        const uint32_t a2 = sb + OFF_A2 + b * A2_STAGE;
#pragma unroll
        for (int ks = 0; ks < kR / 16; ++ks) {
          const int kg = ip * (kR / 16) + ks;
          const uint32_t acc = (ip | ks) != 0;
          const uint32_t tb = sb + OFF_TAB + kg * 2 * TAB_LBO;
          const uint64_t b1 = sdesc(tb, TAB_LBO, CM), b2 = sdesc(tb + TAB_B2, TAB_LBO, CM);
          const uint32_t ka = a2 + ks * 2 * A2_LBO;
          const uint64_t rh = sdesc(ka, A2_LBO, CM), rl = sdesc(ka + A2_COMP, A2_LBO, CM);
          const uint64_t ih = sdesc(ka + 2 * A2_COMP, A2_LBO, CM), il = sdesc(ka + 3 * A2_COMP, A2_LBO, CM);
          const uint32_t d1 = tmem + COL_ACC, d2 = d1 + 2 * kM;
          mma_bf16(d1, rh, b1, idesc, acc);
          mma_bf16(d1, rl, b1, idesc, 1);
          mma_bf16(d1, rh, b2, idesc, 1);
          mma_bf16(d2, ih, b1, idesc, acc);
          mma_bf16(d2, il, b1, idesc, 1);
          mma_bf16(d2, ih, b2, idesc, 1);
        }
        mma_commit(A2_EMPTY + 8 * b);
        if (ip == kTiles - 1) mma_commit(COL_FULL);
        return true;
      };
      long long T = 0;
      for (; T < ntiles && ok; ++T) {
        const int b = (int)(T & 1);
        const uint32_t v = (uint32_t)(T >> 1);
        if (!mbar_wait(ACC_EMPTY + 8 * b, (v & 1u) ^ 1u, abort_flag, kWaitNs)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d1 = tmem + b * ACC_COLS, d2 = d1 + 2 * kM;
        for (int c = 0; c < kChunks; ++c) {
          const long long Cn = T * kChunks + c;
          const int s = (int)(Cn % kStages);
          const uint32_t u = (uint32_t)(Cn / kStages);
          if (!mbar_wait(X_FULL + 8 * s, u & 1u, abort_flag, kWaitNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t xs = sb + OFF_X + s * X_STAGE;
#pragma unroll
          for (int ks = 0; ks < kC / 16; ++ks) {
            const int kg = c * (kC / 16) + ks;
            const uint32_t acc = (c | ks) != 0;
            const uint32_t tb = sb + OFF_TAB + kg * 2 * TAB_LBO;
            const uint64_t b1 = sdesc(tb, TAB_LBO, CM), b2 = sdesc(tb + TAB_B2, TAB_LBO, CM);
            const uint32_t ka = xs + ks * 2 * X_LBO;
            const uint64_t rh = sdesc(ka, X_LBO, CM), rl = sdesc(ka + X_COMP, X_LBO, CM);
            const uint64_t ih = sdesc(ka + 2 * X_COMP, X_LBO, CM), il = sdesc(ka + 3 * X_COMP, X_LBO, CM);
            mma_bf16(d1, rh, b1, idesc, acc);
            mma_bf16(d1, rl, b1, idesc, 1);
            mma_bf16(d1, rh, b2, idesc, 1);
            mma_bf16(d2, ih, b1, idesc, acc);
            mma_bf16(d2, il, b1, idesc, 1);
            mma_bf16(d2, ih, b2, idesc, 1);
          }
          mma_commit(X_EMPTY + 8 * s);
        }
        if (!ok) break;
        mma_commit(ACC_FULL + 8 * b);
        if (T > 0 && !col_pass(T - 1)) ok = false;
      }
      if (ok && ntiles > 0) col_pass(ntiles - 1);
      // Drain: every MMA issued has completed before tensor memory is freed.
      volatile int never = 0;
      mma_commit(DONE);
      mbar_wait(DONE, 0, &never, kWaitNs);
    }
    __syncwarp();
  } else if (warp < kEpiWarps) {
    // ------------------------------------------------------------- epilogue
    const int q = warp;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const uint32_t kofs = (uint32_t)(lane >> 3) * A2_LBO + (uint32_t)(lane & 7) * 2;
    long long T = 0;
    for (long long it = 0; it < nloc; ++it) {
      const long long g = blockIdx.x + it * gridDim.x;
      for (int i = 0; i < kTiles; ++i, ++T) {
        const int b = (int)(T & 1);
        const uint32_t v = (uint32_t)(T >> 1);
        const int ba = (int)(T % kA2);
        const uint32_t va = (uint32_t)(T / kA2);
        if (!mbar_wait(ACC_FULL + 8 * b, v & 1u, abort_flag, kWaitNs)) goto epi_done;
        if (!mbar_wait(A2_EMPTY + 8 * ba, (va & 1u) ^ 1u, abort_flag, kWaitNs)) goto epi_done;
        tc_fence_after();
        {
          uint8_t* a2 = sm + OFF_A2 + ba * A2_STAGE;
          const uint32_t z1 = tmem + lane_off + b * ACC_COLS, z2 = z1 + 2 * kM;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float p0[16], p1[16];
            tmem_ld16(z1 + 16 * h, p0);
            tmem_ld16(z2 + kM + 16 * h, p1);
            tmem_wait_ld();
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const uint32_t m2 = (uint32_t)(q * kM + 16 * h + t);
              own_store(a2, kofs + (m2 >> 3) * CM + (m2 & 7) * 16, A2_COMP, p0[t] - p1[t]);
            }
            tmem_ld16(z1 + kM + 16 * h, p0);
            tmem_ld16(z2 + 16 * h, p1);
            tmem_wait_ld();
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const uint32_t m2 = (uint32_t)(q * kM + 16 * h + t);
              own_store(a2 + 2 * A2_COMP, kofs + (m2 >> 3) * CM + (m2 & 7) * 16, A2_COMP, p0[t] + p1[t]);
            }
          }
        }
        tc_fence_before();
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(ACC_EMPTY + 8 * b);
          mbar_arrive(A2_FULL + 8 * ba);
        }
        if (i == kTiles - 1) {
          if (!mbar_wait(COL_FULL, (uint32_t)(it & 1), abort_flag, kWaitNs)) goto epi_done;
          tc_fence_after();
          const uint32_t y1 = tmem + lane_off + COL_ACC, y2 = y1 + 2 * kM;
          const long long f = g * kF + q;
          float2* yf = y + f * (long long)(kM * kM) + lane;  // lane = t2
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float a[16], b[16], c[16], d[16];
            tmem_ld16(y1 + 16 * h, a);
            tmem_ld16(y2 + kM + 16 * h, b);
            tmem_ld16(y1 + kM + 16 * h, c);
            tmem_ld16(y2 + 16 * h, d);
            tmem_wait_ld();
            if (f < batch) {
#pragma unroll
              for (int t = 0; t < 16; ++t) yf[(16 * h + t) * kM] = make_float2(a[t] - b[t], c[t] + d[t]);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(COL_EMPTY);
        }
      }
    }
  epi_done:;
    // ------------------------------------------------------ load + convert
  } else if (warp >= kCvtWarp0) {
    const int cw = warp - kCvtWarp0;
    const int half = lane >> 4, e = lane & 15;
    const uint32_t kk = (uint32_t)(e >> 2), wd = (uint32_t)(e & 3);
    const long long total = ntiles * kChunks;
    using Buf = float4[kRowsPerThread];
    auto load = [&](long long L, Buf& r) {
      if (L >= total) return;
      const long long T = L / kChunks;
      const int c = (int)(L % kChunks);
      const long long g = blockIdx.x + (T / kTiles) * gridDim.x;
      const int i = (int)(T % kTiles);
#pragma unroll
      for (int j = 0; j < kRowsPerThread; ++j) {
        const int m = cw * (2 * kRowsPerThread) + 2 * j + half;
        const long long f = g * kF + (m / kR);
        const int row = i * kR + (m % kR);
        if (f < batch) {
          const float2* src = x + (f * kN + row) * (long long)kN + c * kC + 2 * e;
          r[j] = __ldg(reinterpret_cast<const float4*>(src));
        } else {
          r[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    };
    // Converts stage L from `r`, then refills `r` with stage L + kDepth, so
    // that kDepth - 1 stages stay in flight while one is converted.
    auto step = [&](long long L, Buf& r) -> bool {
      if (L >= total) return true;
      const int s = (int)(L % kStages);
      const uint32_t u = (uint32_t)(L / kStages);
      if (!mbar_wait(X_EMPTY + 8 * s, (u & 1u) ^ 1u, abort_flag, kWaitNs)) return false;
      uint8_t* xs = sm + OFF_X + s * X_STAGE;
#pragma unroll
      for (int j = 0; j < kRowsPerThread; ++j) {
        const uint32_t m = (uint32_t)(cw * (2 * kRowsPerThread) + 2 * j + half);
        const uint32_t off = kk * X_LBO + m * 16 + wd * 4;
        split_store(xs, X_COMP, off, r[j].x, r[j].z);
        split_store(xs + 2 * X_COMP, X_COMP, off, r[j].y, r[j].w);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(X_FULL + 8 * s);
      load(L + kDepth, r);
      return true;
    };
    static_assert(kDepth == 3 || kDepth == 4, "the loop below is unrolled for three or four register stages");
    Buf b0, b1, b2, b3;
    load(0, b0);
    load(1, b1);
    load(2, b2);
    if constexpr (kDepth == 4) load(3, b3);
    for (long long L = 0; L < total; L += kDepth) {
      if (!step(L, b0) || !step(L + 1, b1) || !step(L + 2, b2)) break;
      if constexpr (kDepth == 4) {
        if (!step(L + 3, b3)) break;
      }
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

// Folded expansion table A[t][v] (t = -M/2 .. M/2-1, v = q k + l) in FP64,
// split into BF16 hi / lo and written in the MMA B-operand layout: rows
// [0, M) A_re hi, [M, 2M) A_im hi, [2M, 3M) A_re lo, [3M, 4M) A_im lo; K = v.
__global__ void k_tc_table(int p, int q, int r, const double* __restrict__ a, uint16_t* __restrict__ tab) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= kM * kN) return;
  const int ti = id / kN, v = id % kN;
  double ar, ai;
  operator_entry(kM, p, q, r, a, ti, v, ar, ai);
  auto at = [&](int rr) {
    return ((uint32_t)(v / 8) * TAB_LBO + (uint32_t)(rr / 8) * CM + (uint32_t)(rr % 8) * 16 + (uint32_t)(v % 8) * 2) / 2;
  };
  uint16_t hi, lo;
  split_bf16(ar, hi, lo);
  tab[at(ti)] = hi;
  tab[at(ti + 2 * kM)] = lo;
  split_bf16(ai, hi, lo);
  tab[at(kM + ti)] = hi;
  tab[at(3 * kM + ti)] = lo;
}

}  // namespace

namespace pfth {

bool tc_supported(int n, int M, int p) { return n == kN && (M == kM || M == 2 * kM) && p == M / 2; }

int tc_build_tables(pft_plan* plan) {
  double xi = 0.0, a[pftc::kMaxTerms] = {0};
  if (!pftc::design(plan->eps, plan->r1, &xi, a, nullptr))
    return set_error(PFT_ERR_INVALID_ARG, "coefficient design failed (eps=%g r=%d)", plan->eps, plan->r1);
  double* d_a = nullptr;
  PFT_CUDA_TRY(cudaMalloc(&d_a, sizeof(double) * pftc::kMaxTerms));
  PFT_CUDA_TRY(cudaMemcpy(d_a, a, sizeof(double) * plan->r1, cudaMemcpyHostToDevice));
  PFT_CUDA_TRY(cudaMalloc(&plan->d_tc, TAB_BYTES));
  PFT_CUDA_TRY(cudaMemset(plan->d_tc, 0, TAB_BYTES));
  k_tc_table<<<(kM * kN + 127) / 128, 128>>>(plan->p1, plan->q1, plan->r1, d_a,
                                             reinterpret_cast<uint16_t*>(plan->d_tc));
  PFT_CUDA_TRY(cudaGetLastError());
  int rc = tc_build_adjoint_table(plan, d_a);
  if (rc != PFT_OK) return rc;
  PFT_CUDA_TRY(cudaDeviceSynchronize());
  PFT_CUDA_TRY(cudaFree(d_a));
  PFT_CUDA_TRY(cudaHostAlloc(&plan->h_status, sizeof(int), cudaHostAllocMapped));
  *plan->h_status = PFT_OK;
  PFT_CUDA_TRY(cudaHostGetDevicePointer(&plan->d_status, plan->h_status, 0));
  return PFT_OK;
}

int tc_forward(const pft_plan* plan, const void* x, void* y, int64_t batch, void* stream) {
  if (*plan->h_status != PFT_OK) {
    const int st = *plan->h_status;
    *plan->h_status = PFT_OK;
    return set_error(st, "a device-side wait of an earlier split-BF16 launch timed out");
  }
  static bool attr_set = false;
  if (!attr_set) {
    PFT_CUDA_TRY(cudaFuncSetAttribute(k_pft_tc_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
    attr_set = true;
  }
  const long long groups = (batch + kF - 1) / kF;
  long long grid = sm_count();
  if (grid > groups) grid = groups;
  k_pft_tc_fwd<<<(unsigned)grid, kThreadsTC, SMEM_BYTES, (cudaStream_t)stream>>>(
      (const float2*)x, (float2*)y, (long long)batch, (const uint4*)plan->d_tc, plan->d_status);
  PFT_CUDA_TRY(cudaGetLastError());
  return PFT_OK;
}

}  // namespace pfth
