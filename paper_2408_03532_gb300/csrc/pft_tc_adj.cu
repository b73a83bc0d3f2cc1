// Split-BF16 tensor-core adjoint PFT (tcgen05, sm_103a) for 256 x 256 frames
// with a 32 x 32 input: x = A^H y conj(A) per frame, the exact conjugate
// transpose of Y = A X A^T (A the folded 1-D PFT operator, M x n).
//
// Per frame, with the adjoint table Ac[v][t] = conj(A[t][v]) (n x M):
//   pass 1  U^T[v][t1] = sum_t2 Ac[v][t2] Y[t1][t2]          (M = v, N = t1, K = t2)
//   pass 2  X^T[v][u]  = sum_t1 U^T[v][t1] Ac[u][t1]         (M = v, N = u,  K = t1)
// so that TMEM lane = image column v in pass 2 and a warp stores 32
// consecutive columns of one output row (256 contiguous bytes) per
// instruction. Both passes use BF16 hi + lo splits of both operands with
// three partial products per term and FP32 accumulation, as the forward.
// Pass 1 accumulates Z1 = Ac_re [Y_re | Y_im], Z2 = Ac_im [Y_re | Y_im];
// pass 2 accumulates D_re = U_re Ac_re - U_im Ac_im (the second product with
// the instruction's negate-B bit) and D_im = U_re Ac_im + U_im Ac_re directly.
//
// Roles (persistent, one CTA per SM, 16 warps, one frame per iteration):
//   warps 12-15  load Y (32 x 32 complex) and split it into the pass-1
//                B operand (two stages);
//   warp 8       allocates tensor memory; one lane issues the MMAs in the
//                order P1(f), P2(f-1), P1(f+1), P2(f), ...;
//   warps 4-7    turn the pass-1 accumulators into the pass-2 A operand U^T
//                (BF16 hi / lo, two buffers);
//   warps 0-3    read the pass-2 accumulators (two tiles of 128 v x 64 u in
//                flight) and store X;
//   warps 9-11   pad the block to whole warp groups.
// Every wait is bounded (2 s); a timeout sets the plan's status word.
#include <cuda_bf16.h>

#include "plan.cuh"
#include "tc.cuh"
#include "tc_table.cuh"

namespace {

using namespace tc;

constexpr int kN = 256, kM = 32;
constexpr uint32_t CM = 128;
// adjoint table: 4 components (Ac_re hi, Ac_im hi, Ac_re lo, Ac_im lo), each
// [v: 256][t: 32] K-major in core matrices [t / 8][v / 8][8][16 B]
constexpr uint32_t T_LBO = (kN / 8) * CM;          // 4096
constexpr uint32_t T_COMP = (kM / 8) * T_LBO;      // 16384
constexpr uint32_t T_BYTES = 4 * T_COMP;           // 65536
// pass-1 B operand: rows [Y_re t1 0..31 | Y_im t1 0..31], K = t2; hi then lo
constexpr uint32_t Y_LBO = (2 * kM / 8) * CM;      // 1024
constexpr uint32_t Y_HALF = (kM / 8) * Y_LBO;      // 4096
constexpr uint32_t Y_STAGE = 2 * Y_HALF;           // 8192
constexpr int kYStages = 2;
// pass-2 A operand U^T: 4 components (U_re hi, U_re lo, U_im hi, U_im lo),
// each [v: 256][t1: 32] like the table
constexpr uint32_t U_COMP = T_COMP;
constexpr uint32_t U_BUF = 4 * U_COMP;             // 65536
constexpr int kUBufs = 2;
constexpr uint32_t OFF_TAB = 0;
constexpr uint32_t OFF_Y = OFF_TAB + T_BYTES;
constexpr uint32_t OFF_U = OFF_Y + kYStages * Y_STAGE;
constexpr uint32_t OFF_BAR = OFF_U + kUBufs * U_BUF;
constexpr int NBAR = 15;
constexpr uint32_t OFF_SLOT = OFF_BAR + 8 * NBAR;
constexpr uint32_t OFF_ABORT = OFF_SLOT + 8;
constexpr uint32_t SMEM_BYTES = OFF_ABORT + 8;
static_assert(SMEM_BYTES <= 232448, "shared memory layout too large");

constexpr int kE2Warp0 = 0, kE1Warp0 = 4, kMmaWarp = 8, kLdWarp0 = 12, kLdWarps = 4;
constexpr int kThreadsAdj = 32 * 16;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t P1_COLS = 128;     // per v tile: Z1 (64) | Z2 (64)
constexpr uint32_t P2_BASE = 2 * P1_COLS;
constexpr uint32_t P2_COLS = 128;     // per output tile: D_re (64) | D_im (64)
constexpr int kUBlocks = kN / 64;     // output tiles per v tile (64 rows u each)
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint32_t kNegB = 1u << 14;

static_assert(P2_BASE + 2 * P2_COLS <= TMEM_COLS, "tensor memory");

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

__global__ void __launch_bounds__(kThreadsAdj, 1)
    k_pft_tc_adj(const float2* __restrict__ y, float2* __restrict__ x, long long batch,
                 const uint4* __restrict__ tab, int* status) {
  extern __shared__ __align__(128) uint8_t sm[];
  const uint32_t sb = smem_u32(sm);
  const uint32_t bar = sb + OFF_BAR;
  const uint32_t Y_FULL = bar, Y_EMPTY = bar + 16, P1_FULL = bar + 32, P1_EMPTY = bar + 40, U_FULL = bar + 48,
                 U_EMPTY = bar + 64, O_FULL = bar + 80, O_EMPTY = bar + 96, DONE = bar + 112;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF_ABORT);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + OFF_SLOT);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int i = threadIdx.x; i < (int)(T_BYTES / 16); i += blockDim.x)
    reinterpret_cast<uint4*>(sm + OFF_TAB)[i] = __ldg(tab + i);
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(Y_FULL + 8 * s, kLdWarps);
      mbar_init(Y_EMPTY + 8 * s, 1);
      mbar_init(U_FULL + 8 * s, 4);
      mbar_init(U_EMPTY + 8 * s, 1);
      mbar_init(O_FULL + 8 * s, 1);
      mbar_init(O_EMPTY + 8 * s, 4);
    }
    mbar_init(P1_FULL, 1);
    mbar_init(P1_EMPTY, 4);
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

  if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(128, 64);
      const uint32_t tb = sb + OFF_TAB;
      bool ok = true;
      auto pass1 = [&](long long fi) -> bool {
        const int s = (int)(fi % kYStages);
        if (!mbar_wait(Y_FULL + 8 * s, (uint32_t)(fi / kYStages) & 1u, abort_flag, kWaitNs)) return false;
        if (!mbar_wait(P1_EMPTY, ((uint32_t)fi & 1u) ^ 1u, abort_flag, kWaitNs)) return false;
        tc_fence_after();
        const uint32_t ys = sb + OFF_Y + s * Y_STAGE;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t z1 = tmem + h * P1_COLS, z2 = z1 + 64;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint32_t acc = ks;
            const uint32_t ta = tb + ks * 2 * T_LBO + h * 16 * CM;
            const uint64_t rh = sdesc(ta, T_LBO, CM), ih = sdesc(ta + T_COMP, T_LBO, CM);
            const uint64_t rl = sdesc(ta + 2 * T_COMP, T_LBO, CM), il = sdesc(ta + 3 * T_COMP, T_LBO, CM);
            const uint32_t yb = ys + ks * 2 * Y_LBO;
            const uint64_t yh = sdesc(yb, Y_LBO, CM), yl = sdesc(yb + Y_HALF, Y_LBO, CM);
            mma_bf16(z1, rh, yh, idesc, acc);
            mma_bf16(z1, rl, yh, idesc, 1);
            mma_bf16(z1, rh, yl, idesc, 1);
            mma_bf16(z2, ih, yh, idesc, acc);
            mma_bf16(z2, il, yh, idesc, 1);
            mma_bf16(z2, ih, yl, idesc, 1);
          }
        }
        mma_commit(Y_EMPTY + 8 * s);
        mma_commit(P1_FULL);
        return true;
      };
      auto pass2 = [&](long long fi) -> bool {
        const int ub = (int)(fi % kUBufs);
        if (!mbar_wait(U_FULL + 8 * ub, (uint32_t)(fi / kUBufs) & 1u, abort_flag, kWaitNs)) return false;
        tc_fence_after();
        const uint32_t ua = sb + OFF_U + ub * U_BUF;
        for (int h = 0; h < 2; ++h) {
          for (int b = 0; b < kUBlocks; ++b) {
            const long long T2 = fi * (2 * kUBlocks) + h * kUBlocks + b;
            const int d = (int)(T2 & 1);
            if (!mbar_wait(O_EMPTY + 8 * d, ((uint32_t)(T2 >> 1) & 1u) ^ 1u, abort_flag, kWaitNs)) return false;
            tc_fence_after();
            const uint32_t dr = tmem + P2_BASE + d * P2_COLS, di = dr + 64;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint32_t acc = ks;
              const uint32_t a0 = ua + ks * 2 * T_LBO + h * 16 * CM;
              const uint64_t urh = sdesc(a0, T_LBO, CM), url = sdesc(a0 + U_COMP, T_LBO, CM);
              const uint64_t uih = sdesc(a0 + 2 * U_COMP, T_LBO, CM), uil = sdesc(a0 + 3 * U_COMP, T_LBO, CM);
              const uint32_t b0 = tb + ks * 2 * T_LBO + b * 8 * CM;
              const uint64_t crh = sdesc(b0, T_LBO, CM), cih = sdesc(b0 + T_COMP, T_LBO, CM);
              const uint64_t crl = sdesc(b0 + 2 * T_COMP, T_LBO, CM), cil = sdesc(b0 + 3 * T_COMP, T_LBO, CM);
              mma_bf16(dr, urh, crh, idesc, acc);
              mma_bf16(dr, url, crh, idesc, 1);
              mma_bf16(dr, urh, crl, idesc, 1);
              mma_bf16(dr, uih, cih, idesc | kNegB, 1);
              mma_bf16(dr, uil, cih, idesc | kNegB, 1);
              mma_bf16(dr, uih, cil, idesc | kNegB, 1);
              mma_bf16(di, urh, cih, idesc, acc);
              mma_bf16(di, url, cih, idesc, 1);
              mma_bf16(di, urh, cil, idesc, 1);
              mma_bf16(di, uih, crh, idesc, 1);
              mma_bf16(di, uil, crh, idesc, 1);
              mma_bf16(di, uih, crl, idesc, 1);
            }
            mma_commit(O_FULL + 8 * d);
          }
        }
        mma_commit(U_EMPTY + 8 * ub);
        return true;
      };
      for (long long fi = 0; fi < nloc && ok; ++fi) {
        ok = pass1(fi);
        if (ok && fi > 0) ok = pass2(fi - 1);
      }
      if (ok && nloc > 0) pass2(nloc - 1);
      volatile int never = 0;
      mma_commit(DONE);
      mbar_wait(DONE, 0, &never, kWaitNs);
    }
    __syncwarp();
  } else if (warp >= kE1Warp0 && warp < kE1Warp0 + 4) {
    // ------------------------------------- pass-1 accumulators -> U^T operand
    const int q = warp - kE1Warp0;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    for (long long fi = 0; fi < nloc; ++fi) {
      const int ub = (int)(fi % kUBufs);
      if (!mbar_wait(P1_FULL, (uint32_t)fi & 1u, abort_flag, kWaitNs)) break;
      if (!mbar_wait(U_EMPTY + 8 * ub, ((uint32_t)(fi / kUBufs) & 1u) ^ 1u, abort_flag, kWaitNs)) break;
      tc_fence_after();
      uint8_t* ubuf = sm + OFF_U + ub * U_BUF;
      for (int h = 0; h < 2; ++h) {
        const uint32_t z1 = tmem + lane_off + h * P1_COLS, z2 = z1 + 64;
        const uint32_t v = (uint32_t)(h * 128 + q * 32 + lane);
#pragma unroll
        for (int pc = 0; pc < 2; ++pc) {
          float a[16], b[16], c[16], d[16];
          tmem_ld16(z1 + 16 * pc, a);        // Ac_re Y_re
          tmem_ld16(z2 + 32 + 16 * pc, b);   // Ac_im Y_im
          tmem_ld16(z1 + 32 + 16 * pc, c);   // Ac_re Y_im
          tmem_ld16(z2 + 16 * pc, d);        // Ac_im Y_re
          tmem_wait_ld();
          if (h == 1 && pc == 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(P1_EMPTY);
          }
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            float r8[8], i8[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              r8[e] = a[8 * g + e] - b[8 * g + e];
              i8[e] = c[8 * g + e] + d[8 * g + e];
            }
            const uint32_t off = (uint32_t)(2 * pc + g) * T_LBO + v * 16;
            uint4 lo;
            uint4 hi = split8(r8, lo);
            *reinterpret_cast<uint4*>(ubuf + off) = hi;
            *reinterpret_cast<uint4*>(ubuf + U_COMP + off) = lo;
            hi = split8(i8, lo);
            *reinterpret_cast<uint4*>(ubuf + 2 * U_COMP + off) = hi;
            *reinterpret_cast<uint4*>(ubuf + 3 * U_COMP + off) = lo;
          }
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(U_FULL + 8 * ub);
    }
  } else if (warp < kE2Warp0 + 4) {
    // ------------------------------------------ pass-2 accumulators -> X
    const int q = warp - kE2Warp0;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    bool ok = true;
    for (long long fi = 0; fi < nloc && ok; ++fi) {
      const long long f = blockIdx.x + fi * gridDim.x;
      float2* xf = x + f * (long long)(kN * kN);
      for (int h = 0; h < 2 && ok; ++h) {
        const int v = h * 128 + q * 32 + lane;
        for (int b = 0; b < kUBlocks; ++b) {
          const long long T2 = fi * (2 * kUBlocks) + h * kUBlocks + b;
          const int d = (int)(T2 & 1);
          if (!mbar_wait(O_FULL + 8 * d, (uint32_t)(T2 >> 1) & 1u, abort_flag, kWaitNs)) {
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
            float2* dst = xf + (long long)(b * 64 + 16 * pc) * kN + v;
#pragma unroll
            for (int j = 0; j < 16; ++j) dst[j * kN] = make_float2(re[j], im[j]);
          }
        }
      }
    }
  } else if (warp >= kLdWarp0) {
    // ------------------------------------------------ Y -> pass-1 B operand
    const int i = threadIdx.x - kLdWarp0 * 32;   // 0..127
    const int kk = (i & 31) >> 3;                // t2 group of 8
    const int t1 = (i >> 5) * 8 + (i & 7);       // 0..31
    for (long long fi = 0; fi < nloc; ++fi) {
      const long long f = blockIdx.x + fi * gridDim.x;
      const float4* src = reinterpret_cast<const float4*>(y + f * (long long)(kM * kM) + t1 * kM + kk * 8);
      float4 v4[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v4[j] = __ldg(src + j);
      const int s = (int)(fi % kYStages);
      if (!mbar_wait(Y_EMPTY + 8 * s, ((uint32_t)(fi / kYStages) & 1u) ^ 1u, abort_flag, kWaitNs)) break;
      float r8[8], i8[8];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        r8[2 * j] = v4[j].x;
        i8[2 * j] = v4[j].y;
        r8[2 * j + 1] = v4[j].z;
        i8[2 * j + 1] = v4[j].w;
      }
      uint8_t* ys = sm + OFF_Y + s * Y_STAGE;
      uint4 lo;
      uint4 hi = split8(r8, lo);
      *reinterpret_cast<uint4*>(ys + kk * Y_LBO + t1 * 16) = hi;
      *reinterpret_cast<uint4*>(ys + Y_HALF + kk * Y_LBO + t1 * 16) = lo;
      hi = split8(i8, lo);
      *reinterpret_cast<uint4*>(ys + kk * Y_LBO + (kM + t1) * 16) = hi;
      *reinterpret_cast<uint4*>(ys + Y_HALF + kk * Y_LBO + (kM + t1) * 16) = lo;
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(Y_FULL + 8 * s);
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

// Adjoint table Ac[v][t] = conj(A[t][v]) split into BF16 hi / lo, in the
// layout above: components Ac_re hi, Ac_im hi, Ac_re lo, Ac_im lo.
__global__ void k_tc_table_adj(int p, int q, int r, const double* __restrict__ a, uint16_t* __restrict__ tab) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= kM * kN) return;
  const int ti = id / kN, v = id % kN;
  double ar, ai;
  operator_entry(kM, p, q, r, a, ti, v, ar, ai);
  const uint32_t at = ((uint32_t)(ti / 8) * T_LBO + (uint32_t)(v / 8) * CM + (uint32_t)(v % 8) * 16 +
                       (uint32_t)(ti % 8) * 2) / 2;
  uint16_t hi, lo;
  split_bf16(ar, hi, lo);
  tab[at] = hi;
  tab[at + 2 * T_COMP / 2] = lo;
  split_bf16(-ai, hi, lo);
  tab[at + T_COMP / 2] = hi;
  tab[at + 3 * T_COMP / 2] = lo;
}

}  // namespace

namespace pfth {

int tc_build_adjoint_table(pft_plan* plan, const double* d_a) {
  PFT_CUDA_TRY(cudaMalloc(&plan->d_tc_adj, T_BYTES));
  k_tc_table_adj<<<(kM * kN + 127) / 128, 128>>>(plan->p1, plan->q1, plan->r1, d_a,
                                                 reinterpret_cast<uint16_t*>(plan->d_tc_adj));
  PFT_CUDA_TRY(cudaGetLastError());
  return PFT_OK;
}

int tc_adjoint(const pft_plan* plan, const void* y, void* x, int64_t batch, void* stream) {
  if (*plan->h_status != PFT_OK) {
    const int st = *plan->h_status;
    *plan->h_status = PFT_OK;
    return set_error(st, "a device-side wait of an earlier split-BF16 launch timed out");
  }
  static bool attr_set = false;
  if (!attr_set) {
    PFT_CUDA_TRY(cudaFuncSetAttribute(k_pft_tc_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
    attr_set = true;
  }
  long long grid = sm_count();
  if (grid > batch) grid = batch;
  k_pft_tc_adj<<<(unsigned)grid, kThreadsAdj, SMEM_BYTES, (cudaStream_t)stream>>>(
      (const float2*)y, (float2*)x, (long long)batch, (const uint4*)plan->d_tc_adj, plan->d_status);
  PFT_CUDA_TRY(cudaGetLastError());
  return PFT_OK;
}

}  // namespace pfth
