// Split-BF16 tensor-core PFT forward (tcgen05, sm_103a) for batches of
// 256 x 256 frames with a 64 x 64 output (p = 32).
//
// The same scheme as the M = 32 kernel (pft_tc.cu): Y = A X A^T with the
// folded per-axis operator A (Algorithm 5), split-BF16 operands, FP32
// accumulation in tensor memory, a row pass over tiles of 2 frames x 64 rows
// whose column pass consumes the tile without leaving the SM. To keep the
// BF16 hi / lo table in shared memory, only the rows t = 0 .. 31 and
// t = -32 of A are stored: A[-t] = conj(A[t]) (W'[-t, j] = conj(W'[t, j]), B
// real), so for s = 1 .. 31 the products X A_re[s] and X A_im[s] give both
// Y[s] = X A_re + i X A_im and Y[-s] = X A_re - i X A_im.
// Accumulators per row tile: Z1 = X_re [A_re | A_im], Z2 = X_im [A_re | A_im]
// (N = 80: 33 + 33 rows, padded), and for t = t(s):
//   Y[t]  = (Z1[s] - Z2[33 + s]) + i (Z1[33 + s] + Z2[s]),
//   Y[-t] = (Z1[s] + Z2[33 + s]) + i (Z2[s] - Z1[33 + s])     (s = 1 .. 31).
// Every wait is bounded (2 s); a timeout sets the plan's status word.
#include <cuda_bf16.h>

#include "coeffs.h"
#include "plan.cuh"
#include "tc.cuh"
#include "tc_table.cuh"

namespace {

using namespace tc;

constexpr int kN = 256, kM = 64;
constexpr int kF = 128 / kM;            // frames per group (2)
constexpr int kR = 128 / kF;            // rows per frame in a row tile (64)
constexpr int kTiles = kN / kR;         // 4
constexpr int kC = 32, kChunks = kN / kC, kStages = 2;
constexpr int kS = kM / 2 + 1;          // stored rows of A: t = 0 .. 31 and -32
constexpr int kNt = 80;                 // [A_re (33) | A_im (33) | 0], a multiple of 16
constexpr uint32_t CM = 128;
constexpr uint32_t TAB_LBO = (kNt / 8) * CM;         // 1280
constexpr uint32_t TAB_REGION = (kN / 8) * TAB_LBO;  // 40960: hi, then lo
constexpr uint32_t TAB_BYTES = 2 * TAB_REGION;
constexpr uint32_t X_LBO = 16 * CM + 32;
constexpr uint32_t X_COMP = (kC / 8) * X_LBO;
constexpr uint32_t X_STAGE = 4 * X_COMP;
constexpr uint32_t A2_LBO = 16 * CM + 32;            // column-pass operand: one K half (32 rows)
constexpr uint32_t A2_COMP = 4 * A2_LBO + 16;
constexpr uint32_t A2_STAGE = 4 * A2_COMP;
constexpr uint32_t OFF_TAB = 0, OFF_X = TAB_BYTES, OFF_A2 = OFF_X + kStages * X_STAGE;
constexpr uint32_t OFF_BAR = OFF_A2 + 2 * A2_STAGE;
constexpr int NBAR = 2 * kStages + 8 + 3;
constexpr uint32_t OFF_SLOT = OFF_BAR + 8 * NBAR, OFF_ABORT = OFF_SLOT + 8, SMEM_USED = OFF_ABORT + 8;
constexpr uint32_t SMEM_BYTES = 232448;
static_assert(SMEM_USED <= SMEM_BYTES, "shared memory layout too large");

constexpr int kEpiWarps = 4, kMmaWarp = 4, kCvtWarp0 = 8, kCvtWarps = 16;  // warps 5-7 idle
constexpr int kThreads = 32 * (kCvtWarp0 + kCvtWarps);
constexpr int kRowsPerThread = 128 / (2 * kCvtWarps);
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COLS = 2 * kNt;     // Z1 | Z2
constexpr uint32_t COL_ACC = 2 * ACC_COLS;
constexpr uint64_t kWaitNs = 2000000000ull;
static_assert(COL_ACC + ACC_COLS <= TMEM_COLS, "tensor memory");

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

// Reads Z1[s], Z1[33 + s], Z2[s], Z2[33 + s] for s = s0 .. s0 + 15 (s0 < 32)
// from an accumulator at column `z` and forms the outputs of t(s) and -t(s).
// emit(t_idx, re, im) is called with t_idx = t + 32.
template <class Emit>
__device__ __forceinline__ void recombine(uint32_t z, Emit&& emit) {
#pragma unroll
  for (int s0 = 0; s0 < 32; s0 += 16) {
    float a[16], b[16], c[16], d[16];
    tmem_ld16(z + s0, a);               // X_re A_re
    tmem_ld16(z + kS + s0, b);          // X_re A_im
    tmem_ld16(z + kNt + s0, c);         // X_im A_re
    tmem_ld16(z + kNt + kS + s0, d);    // X_im A_im
    tmem_wait_ld();
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int s = s0 + e;
      emit(s + 32, a[e] - d[e], b[e] + c[e]);
      if (s > 0) emit(32 - s, a[e] + d[e], c[e] - b[e]);
    }
  }
  // s = 32 holds A[-32] itself
  const float a = tmem_ld1(z + 32), b = tmem_ld1(z + kS + 32), c = tmem_ld1(z + kNt + 32),
              d = tmem_ld1(z + kNt + kS + 32);
  tmem_wait_ld();
  emit(0, a - d, b + c);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_pft_tc64_fwd(const float2* __restrict__ x, float2* __restrict__ y, long long batch,
                   const uint4* __restrict__ tab, int* status) {
  extern __shared__ __align__(128) uint8_t sm[];
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
      mbar_init(A2_FULL + 8 * b, 2);  // the two warps of one K half
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
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(128, kNt);
      bool ok = true;
      auto mma6 = [&](uint32_t d1, uint32_t ka, uint32_t lbo, uint32_t comp, uint32_t tb, uint32_t acc) {
        const uint64_t b1 = sdesc(tb, TAB_LBO, CM), b2 = sdesc(tb + TAB_REGION, TAB_LBO, CM);
        const uint64_t rh = sdesc(ka, lbo, CM), rl = sdesc(ka + comp, lbo, CM);
        const uint64_t ih = sdesc(ka + 2 * comp, lbo, CM), il = sdesc(ka + 3 * comp, lbo, CM);
        const uint32_t d2 = d1 + kNt;
        mma_bf16(d1, rh, b1, idesc, acc);
        mma_bf16(d1, rl, b1, idesc, 1);
        mma_bf16(d1, rh, b2, idesc, 1);
        mma_bf16(d2, ih, b1, idesc, acc);
        mma_bf16(d2, il, b1, idesc, 1);
        mma_bf16(d2, ih, b2, idesc, 1);
      };
      auto col_pass = [&](long long Tp) -> bool {
        const int ip = (int)(Tp % kTiles);
        for (int h = 0; h < 2; ++h) {
          if (ip == 0 && h == 0 &&
              !mbar_wait(COL_EMPTY, ((uint32_t)(Tp / kTiles) & 1u) ^ 1u, abort_flag, kWaitNs))
            return false;
          if (!mbar_wait(A2_FULL + 8 * h, (uint32_t)Tp & 1u, abort_flag, kWaitNs)) return false;
          tc_fence_after();
          const uint32_t a2 = sb + OFF_A2 + h * A2_STAGE;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const int kg = 4 * ip + 2 * h + ks;
            mma6(tmem + COL_ACC, a2 + ks * 2 * A2_LBO, A2_LBO, A2_COMP, sb + OFF_TAB + kg * 2 * TAB_LBO,
                 (ip | h | ks) != 0);
          }
          mma_commit(A2_EMPTY + 8 * h);
        }
        if (ip == kTiles - 1) mma_commit(COL_FULL);
        return true;
      };
      long long T = 0;
      for (; T < ntiles && ok; ++T) {
        const int b = (int)(T & 1);
        if (!mbar_wait(ACC_EMPTY + 8 * b, ((uint32_t)(T >> 1) & 1u) ^ 1u, abort_flag, kWaitNs)) break;
        tc_fence_after();
        for (int c = 0; c < kChunks; ++c) {
          const long long L = T * kChunks + c;
          const int s = (int)(L % kStages);
          if (!mbar_wait(X_FULL + 8 * s, (uint32_t)(L / kStages) & 1u, abort_flag, kWaitNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t xs = sb + OFF_X + s * X_STAGE;
#pragma unroll
          for (int ks = 0; ks < kC / 16; ++ks) {
            const int kg = c * (kC / 16) + ks;
            mma6(tmem + b * ACC_COLS, xs + ks * 2 * X_LBO, X_LBO, X_COMP, sb + OFF_TAB + kg * 2 * TAB_LBO,
                 (c | ks) != 0);
          }
          mma_commit(X_EMPTY + 8 * s);
        }
        if (!ok) break;
        mma_commit(ACC_FULL + 8 * b);
        if (T > 0 && !col_pass(T - 1)) ok = false;
      }
      if (ok && ntiles > 0) col_pass(ntiles - 1);
      volatile int never = 0;
      mma_commit(DONE);
      mbar_wait(DONE, 0, &never, kWaitNs);
    }
    __syncwarp();
  } else if (warp < kEpiWarps) {
    // TMEM lane 32 q + lane = (frame q >> 1, row 32 (q & 1) + lane of the tile)
    const int q = warp, h = q & 1;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const uint32_t kofs = (uint32_t)(lane >> 3) * A2_LBO + (uint32_t)(lane & 7) * 2;
    long long T = 0;
    for (long long it = 0; it < nloc; ++it) {
      const long long g = blockIdx.x + it * gridDim.x;
      for (int i = 0; i < kTiles; ++i, ++T) {
        const int b = (int)(T & 1);
        if (!mbar_wait(ACC_FULL + 8 * b, (uint32_t)(T >> 1) & 1u, abort_flag, kWaitNs)) goto done;
        if (!mbar_wait(A2_EMPTY + 8 * h, ((uint32_t)T & 1u) ^ 1u, abort_flag, kWaitNs)) goto done;
        tc_fence_after();
        {
          uint8_t* a2 = sm + OFF_A2 + h * A2_STAGE;
          const uint32_t fbase = (uint32_t)((q >> 1) * kM);
          recombine(tmem + lane_off + b * ACC_COLS, [&](int ti, float re, float im) {
            const uint32_t m2 = fbase + (uint32_t)ti;
            const uint32_t off = kofs + (m2 >> 3) * CM + (m2 & 7) * 16;
            own_store(a2, off, A2_COMP, re);
            own_store(a2 + 2 * A2_COMP, off, A2_COMP, im);
          });
        }
        tc_fence_before();
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(ACC_EMPTY + 8 * b);
          mbar_arrive(A2_FULL + 8 * h);
        }
        if (i == kTiles - 1) {
          if (!mbar_wait(COL_FULL, (uint32_t)(it & 1), abort_flag, kWaitNs)) goto done;
          tc_fence_after();
          // D2 lane 32 q + lane = (frame q >> 1, t2_idx = 32 (q & 1) + lane); columns over t1
          const long long f = g * kF + (q >> 1);
          float2* yf = y + f * (long long)(kM * kM) + 32 * (q & 1) + lane;
          const bool write = f < batch;
          recombine(tmem + lane_off + COL_ACC, [&](int t1, float re, float im) {
            if (write) yf[t1 * kM] = make_float2(re, im);
          });
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(COL_EMPTY);
        }
      }
    }
  done:;
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
        r[j] = f < batch ? __ldg(reinterpret_cast<const float4*>(x + (f * kN + row) * (long long)kN + c * kC + 2 * e))
                         : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    auto step = [&](long long L, Buf& r) -> bool {
      if (L >= total) return true;
      const int s = (int)(L % kStages);
      if (!mbar_wait(X_EMPTY + 8 * s, ((uint32_t)(L / kStages) & 1u) ^ 1u, abort_flag, kWaitNs)) return false;
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
      load(L + 3, r);
      return true;
    };
    Buf b0, b1, b2;
    load(0, b0);
    load(1, b1);
    load(2, b2);
    for (long long L = 0; L < total; L += 3)
      if (!step(L, b0) || !step(L + 1, b1) || !step(L + 2, b2)) break;
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

// Rows s of the stored table: t(s) = s (s < 32), t(32) = -32; [A_re | A_im]
// in each of the hi and lo regions, [v / 8][row / 8][8][16 B].
__global__ void k_tc64_table(int p, int q, int r, const double* __restrict__ a, uint16_t* __restrict__ tab) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= kS * kN) return;
  const int s = id / kN, v = id % kN;
  const int t = s < kM / 2 ? s : -kM / 2;
  double ar, ai;
  operator_entry(kM, p, q, r, a, t + kM / 2, v, ar, ai);
  auto at = [&](int row) {
    return ((uint32_t)(v / 8) * TAB_LBO + (uint32_t)(row / 8) * CM + (uint32_t)(row % 8) * 16 + (uint32_t)(v % 8) * 2) / 2;
  };
  uint16_t hi, lo;
  split_bf16(ar, hi, lo);
  tab[at(s)] = hi;
  tab[TAB_REGION / 2 + at(s)] = lo;
  split_bf16(ai, hi, lo);
  tab[at(kS + s)] = hi;
  tab[TAB_REGION / 2 + at(kS + s)] = lo;
}

}  // namespace

namespace pfth {

int tc64_build_tables(pft_plan* plan) {
  double xi = 0.0, a[pftc::kMaxTerms] = {0};
  if (!pftc::design(plan->eps, plan->r1, &xi, a, nullptr))
    return set_error(PFT_ERR_INVALID_ARG, "coefficient design failed (eps=%g r=%d)", plan->eps, plan->r1);
  double* d_a = nullptr;
  PFT_CUDA_TRY(cudaMalloc(&d_a, sizeof(double) * pftc::kMaxTerms));
  PFT_CUDA_TRY(cudaMemcpy(d_a, a, sizeof(double) * plan->r1, cudaMemcpyHostToDevice));
  PFT_CUDA_TRY(cudaMalloc(&plan->d_tc, TAB_BYTES));
  PFT_CUDA_TRY(cudaMemset(plan->d_tc, 0, TAB_BYTES));
  k_tc64_table<<<(kS * kN + 127) / 128, 128>>>(plan->p1, plan->q1, plan->r1, d_a,
                                               reinterpret_cast<uint16_t*>(plan->d_tc));
  PFT_CUDA_TRY(cudaGetLastError());
  PFT_CUDA_TRY(cudaDeviceSynchronize());
  PFT_CUDA_TRY(cudaFree(d_a));
  PFT_CUDA_TRY(cudaHostAlloc(&plan->h_status, sizeof(int), cudaHostAllocMapped));
  *plan->h_status = PFT_OK;
  PFT_CUDA_TRY(cudaHostGetDevicePointer(&plan->d_status, plan->h_status, 0));
  return PFT_OK;
}

int tc64_forward(const pft_plan* plan, const void* x, void* y, int64_t batch, void* stream) {
  if (*plan->h_status != PFT_OK) {
    const int st = *plan->h_status;
    *plan->h_status = PFT_OK;
    return set_error(st, "a device-side wait of an earlier split-BF16 launch timed out");
  }
  static bool attr_set = false;
  if (!attr_set) {
    PFT_CUDA_TRY(cudaFuncSetAttribute(k_pft_tc64_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
    attr_set = true;
  }
  const long long groups = (batch + kF - 1) / kF;
  long long grid = sm_count();
  if (grid > groups) grid = groups;
  k_pft_tc64_fwd<<<(unsigned)grid, kThreads, SMEM_BYTES, (cudaStream_t)stream>>>(
      (const float2*)x, (float2*)y, (long long)batch, (const uint4*)plan->d_tc, plan->d_status);
  PFT_CUDA_TRY(cudaGetLastError());
  return PFT_OK;
}

}  // namespace pfth
