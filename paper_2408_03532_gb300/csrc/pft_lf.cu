// Large-frame PFT (the paper's regime n >> M): n = 2048 ... 16384 with
// M = 128, p = 64 (m~/p = 1, so r = 13 at eps = 1e-7) and q = n / 64, in
// split-BF16 tensor-core arithmetic for stage A and FP32 for stage B.
//
// Each axis applies Algorithm 2 to every row (Algorithm 5 is the tensor
// product of the two axes):
//   stage A  C[k][j]  = sum_l x[q k + l] B[l][j]          (k < 64, j < 13)
//   stage B  C^[rho][j] = sum_k C[k][j] e^{-2 pi i rho k / 64},
//            y[t]     = sum_j W'[t][j] C^[t mod 64][j]      (t = -64 .. 63)
// Stage A is the O(n r) main cost and streams the frame from HBM; it runs on
// tcgen05 (M = 128 blocks (row, k) of q contiguous values, K = l, N = 16 for
// the 13 terms), with every operand split into BF16 hi + lo and three partial
// products per term. Stage B (13 FFTs of size 64 per row and the W' combine)
// runs in FP32 on CUDA cores in the same kernel's epilogue, straight from the
// tensor-memory accumulators, and writes the row's M outputs transposed, so
// the second axis is the same kernel applied to the rows of the transposed
// intermediate T^T[t2][u]:
//   k_lf_stage_a(x rows)   -> T^T  [frame][128][n]
//   k_lf_stage_a(T^T rows) -> Y    [frame][128][128]
// Every wait is bounded (2 s); a timeout sets the plan's status word.
#include <cuda_bf16.h>

#include <algorithm>

#include "coeffs.h"
#include "fft_core.cuh"
#include "plan.cuh"
#include "tc.cuh"
#include "tc_table.cuh"

namespace {

using namespace tc;
using namespace pftk;

constexpr int kP = 64;                 // blocks per row (p)
constexpr int kMl = 128;               // output side M
constexpr int kRt = 13;                // polynomial terms r
constexpr int kJ = 16;                 // r padded to the MMA N
constexpr int kC = 32;                 // K values (l) per operand stage
constexpr int kStages = 5;
constexpr int kAccBufs = 4;
constexpr uint32_t CM = 128;
constexpr uint32_t X_LBO = 16 * CM + 32;          // padded: conflict-free 4-byte stores
constexpr uint32_t X_COMP = (kC / 8) * X_LBO;
constexpr uint32_t X_STAGE = 4 * X_COMP;
constexpr uint32_t B_LBO = (kJ / 8) * CM;         // 256: table core matrices along K
constexpr uint32_t TAB_MAX = 2 * (256 / 8) * B_LBO;  // hi + lo at q = 256: 16 KB
constexpr uint32_t OFF_TAB = 0;
constexpr uint32_t OFF_X = TAB_MAX;
// stage B in the epilogue: Fft<64> tables, W' in slot order, the half-row
// exchange of C between the two warps of a row, and their partial sums
constexpr uint32_t OFF_TW = OFF_X + kStages * X_STAGE;
constexpr uint32_t OFF_W = OFF_TW + 160 * 8;
constexpr uint32_t OFF_XCH = OFF_W + kRt * kMl * 8;
constexpr uint32_t OFF_PS = OFF_XCH + 4 * kRt * 32 * 8;  // two epilogue groups x two rows
constexpr uint32_t OFF_BAR = OFF_PS + 4 * kMl * 8;
constexpr int NBAR = 2 * kStages + 2 * kAccBufs + 1;
constexpr uint32_t OFF_SLOT = OFF_BAR + 8 * NBAR;
constexpr uint32_t OFF_ABORT = OFF_SLOT + 8;
constexpr uint32_t SMEM_A = OFF_ABORT + 8;
static_assert(SMEM_A <= 232448, "shared memory layout too large");

// Two epilogue groups of four warps take alternate tiles (group 0: warps 0-3,
// group 1: warps 8, 5, 6, 7, so that each group covers the four TMEM lane
// quadrants, warp % 4); warp 4 issues the MMAs; warps 9-24 load.
constexpr int kEpiWarps = 4, kMmaWarp = 4, kLdWarp0 = 9, kLdWarps = 16;
constexpr int kThreadsA = 32 * (kLdWarp0 + kLdWarps);
constexpr int kRowsPerThread = 128 / (2 * kLdWarps);  // 4
constexpr uint32_t TMEM_COLS = 128;
constexpr uint32_t ACC_COLS = 2 * kJ;                  // D_re | D_im
constexpr uint64_t kWaitNs = 2000000000ull;
static_assert(kAccBufs * ACC_COLS <= TMEM_COLS, "tensor memory");

__device__ __forceinline__ void split_store2(uint8_t* base, uint32_t comp_bytes, uint32_t off, float a, float b) {
  const __nv_bfloat162 hi = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(hi);
  const __nv_bfloat162 lo = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  *reinterpret_cast<__nv_bfloat162*>(base + off) = hi;
  *reinterpret_cast<__nv_bfloat162*>(base + comp_bytes + off) = lo;
}

using F64 = Fft<kP>;

// W'[j][t_idx] (t_idx < 128) in "slot" order s = (2 pos + hi) 32 + l, where
// lane l ends the 64-point FFT holding rho = 2 bitrev(l) + pos and owns the
// outputs t_idx = rho + 64 hi: a warp then reads 32 consecutive entries.
__device__ __forceinline__ void fill_w_slots(float2* sW, const float2* __restrict__ gW) {
  for (int i = threadIdx.x; i < kRt * kMl; i += blockDim.x) {
    const int j = i / kMl, sl = i % kMl, l = sl % 32, pos = (sl / 32) >> 1, hi = (sl / 32) & 1;
    sW[i] = gW[j * kMl + 2 * bitrev<32>(l) + pos + kP * hi];
  }
}

__device__ __forceinline__ void pair_barrier(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// Both warps of a pair get the AND of their flags (so that they leave the
// tile loop together and never wait at a pair barrier the other skips).
__device__ __forceinline__ bool pair_all(bool v, int id) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, 64, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ float4 ld_stream(const float2* p, uint64_t pol) {
  float4 r;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "l"(p), "l"(pol));
  return r;
}

// Stages A and B of `nrows` rows of length 64 Q (row stride = row length);
// the tile t covers rows 2t, 2t + 1, i.e. 128 blocks (row, k) of Q values.
// Stage A runs on tensor cores; the four epilogue warps (two per row) then
// run stage B on the accumulators and write the row's 128 outputs to
// out[frame][t_idx][row in frame] (rows_per_frame rows per frame).
template <int Q>
__global__ void __launch_bounds__(kThreadsA, 1)
    k_lf_stage_a(const float2* __restrict__ x, long long nrows, int rows_per_frame, float2* __restrict__ out,
                 const uint4* __restrict__ tab, const float2* __restrict__ gW, const float2* __restrict__ gtw,
                 int* status) {
  constexpr int N = kP * Q;
  constexpr int kChunks = Q / kC;
  constexpr uint32_t TAB_BYTES = 2 * (Q / 8) * B_LBO;
  constexpr uint32_t TAB_LO = TAB_BYTES / 2;
  static_assert(Q % kC == 0 && TAB_BYTES <= TAB_MAX, "block length");
  extern __shared__ __align__(128) uint8_t sm[];
  const uint32_t sb = smem_u32(sm);
  const uint32_t bar = sb + OFF_BAR;
  const uint32_t X_FULL = bar, X_EMPTY = bar + 8 * kStages, ACC_FULL = bar + 16 * kStages,
                 ACC_EMPTY = ACC_FULL + 8 * kAccBufs, DONE = ACC_EMPTY + 8 * kAccBufs;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF_ABORT);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + OFF_SLOT);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int i = threadIdx.x; i < (int)(TAB_BYTES / 16); i += blockDim.x)
    reinterpret_cast<uint4*>(sm + OFF_TAB)[i] = __ldg(tab + i);
  float2* s_tw = reinterpret_cast<float2*>(sm + OFF_TW);
  float2* s_w = reinterpret_cast<float2*>(sm + OFF_W);
  F64::fill(s_tw, gtw);
  fill_w_slots(s_w, gW);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(X_FULL + 8 * s, kLdWarps);
      mbar_init(X_EMPTY + 8 * s, 1);
    }
    for (int b = 0; b < kAccBufs; ++b) {
      mbar_init(ACC_FULL + 8 * b, 1);
      mbar_init(ACC_EMPTY + 8 * b, kEpiWarps);
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
  const long long ntile_all = nrows / 2;
  const long long ntiles = blockIdx.x < ntile_all ? (ntile_all - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (warp == kMmaWarp) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(128, kJ);
      bool ok = true;
      for (long long T = 0; T < ntiles && ok; ++T) {
        const int b = (int)(T % kAccBufs);
        const uint32_t v = (uint32_t)(T / kAccBufs);
        if (!mbar_wait(ACC_EMPTY + 8 * b, (v & 1u) ^ 1u, abort_flag, kWaitNs)) break;
        tc_fence_after();
        const uint32_t dr = tmem + b * ACC_COLS, di = dr + kJ;
        for (int c = 0; c < kChunks; ++c) {
          const long long L = T * kChunks + c;
          const int s = (int)(L % kStages);
          const uint32_t u = (uint32_t)(L / kStages);
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
            const uint32_t tb = sb + OFF_TAB + kg * 2 * B_LBO;
            const uint64_t bh = sdesc(tb, B_LBO, CM), bl = sdesc(tb + TAB_LO, B_LBO, CM);
            const uint32_t ka = xs + ks * 2 * X_LBO;
            const uint64_t rh = sdesc(ka, X_LBO, CM), rl = sdesc(ka + X_COMP, X_LBO, CM);
            const uint64_t ih = sdesc(ka + 2 * X_COMP, X_LBO, CM), il = sdesc(ka + 3 * X_COMP, X_LBO, CM);
            mma_bf16(dr, rh, bh, idesc, acc);
            mma_bf16(dr, rl, bh, idesc, 1);
            mma_bf16(dr, rh, bl, idesc, 1);
            mma_bf16(di, ih, bh, idesc, acc);
            mma_bf16(di, il, bh, idesc, 1);
            mma_bf16(di, ih, bl, idesc, 1);
          }
          mma_commit(X_EMPTY + 8 * s);
        }
        if (!ok) break;
        mma_commit(ACC_FULL + 8 * b);
      }
      volatile int never = 0;
      mma_commit(DONE);
      mbar_wait(DONE, 0, &never, kWaitNs);
    }
    __syncwarp();
  } else if (warp < kLdWarp0) {
    // TMEM lane m = 32 q + lane: block k = 32 h + lane of row r = q >> 1
    // (h = q & 1). Warp h = 0 of a row runs the FFTs of j = 0..6, warp h = 1
    // those of j = 7..12; each first hands the other the half of C it lacks.
    // Group g takes tiles g, g + 2, ...
    const int grp = warp < kEpiWarps ? 0 : 1;
    const int q = warp % 4, r = q >> 1, h = q & 1;
    const int pid = 1 + 2 * grp + r;  // named barrier of the row's warp pair
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    constexpr int kJ0 = 7;
    const int jlo = h ? kJ0 : 0, jhi = h ? kRt : kJ0;
    float2* xch = reinterpret_cast<float2*>(sm + OFF_XCH) + (2 * grp + r) * kRt * 32;
    float2* ps = reinterpret_cast<float2*>(sm + OFF_PS) + (2 * grp + r) * kMl;
    typename F64::Net net;
    F64::init_net(net, lane, s_tw);
    for (long long T = grp; T < ntiles; T += 2) {
      const long long tile = blockIdx.x + T * gridDim.x;
      const int b = (int)(T % kAccBufs);
      const uint32_t v = (uint32_t)(T / kAccBufs);
      const bool got = mbar_wait(ACC_FULL + 8 * b, v & 1u, abort_flag, kWaitNs);
      if (!pair_all(got, pid)) break;
      tc_fence_after();
      float re[16], im[16];
      tmem_ld16(tmem + lane_off + b * ACC_COLS, re);
      tmem_ld16(tmem + lane_off + b * ACC_COLS + kJ, im);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(ACC_EMPTY + 8 * b);
#pragma unroll
      for (int j = 0; j < kRt; ++j)
        if (j < jlo || j >= jhi) xch[j * 32 + lane] = make_float2(re[j], im[j]);
      pair_barrier(pid);
      float2 acc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < kRt; ++j) {
        if (j < jlo || j >= jhi) continue;
        const float2 mine = make_float2(re[j], im[j]), other = xch[j * 32 + lane];
        float2 cv[2] = {h ? other : mine, h ? mine : other};  // k = lane, k = lane + 32
        F64::fwd(cv, lane, s_tw, net);                          // cv[pos] = C^[2 bitrev(lane) + pos][j]
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 w = s_w[j * kMl + i * 32 + lane], c = cv[i >> 1];
          acc[i].x = fmaf(w.x, c.x, fmaf(-w.y, c.y, acc[i].x));
          acc[i].y = fmaf(w.x, c.y, fmaf(w.y, c.x, acc[i].y));
        }
      }
      if (h) {
#pragma unroll
        for (int i = 0; i < 4; ++i) ps[i * 32 + lane] = acc[i];
      }
      pair_barrier(pid);
      if (!h) {
        const long long row = 2 * tile + r;
        const long long f = row / rows_per_frame;
        const long long rin = row % rows_per_frame;
        float2* o = out + f * (long long)kMl * rows_per_frame + rin;
        const int rho0 = 2 * bitrev<32>(lane);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 p2 = ps[i * 32 + lane];
          const int ti = rho0 + (i >> 1) + kP * (i & 1);   // slot i * 32 + lane
          o[(long long)ti * rows_per_frame] = make_float2(acc[i].x + p2.x, acc[i].y + p2.y);
        }
      }
    }
  } else if (warp >= kLdWarp0) {
    const int cw = warp - kLdWarp0;
    const int half = lane >> 4, e = lane & 15;
    const uint32_t kk = (uint32_t)(e >> 2), wd = (uint32_t)(e & 3);
    const long long total = ntiles * kChunks;
    // the frames are read once: mark them first to leave L2, so that the
    // stage-A output C stays there for stage B
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    using Buf = float4[kRowsPerThread];
    auto load = [&](long long L, Buf& r) {
      if (L >= total) return;
      const long long tile = blockIdx.x + (L / kChunks) * gridDim.x;
      const int c = (int)(L % kChunks);
#pragma unroll
      for (int j = 0; j < kRowsPerThread; ++j) {
        const int m = cw * (2 * kRowsPerThread) + 2 * j + half;
        const long long row = 2 * tile + (m >> 6);
        const float2* src = x + row * (long long)N + (m & 63) * Q + c * kC + 2 * e;
        r[j] = ld_stream(src, pol);
      }
    };
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
        split_store2(xs, X_COMP, off, r[j].x, r[j].z);
        split_store2(xs + 2 * X_COMP, X_COMP, off, r[j].y, r[j].w);
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

// Stage-A table B[l][j] = a_j (1 - 2 l / q)^j (j < 13, zero for j = 13..15) in
// FP64, split into BF16 hi / lo: [hi | lo], each [l / 8][j / 8][8][16 B].
__global__ void k_lf_table(int q, int r, const double* __restrict__ a, uint16_t* __restrict__ tab) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= q * kJ) return;
  const int l = id / kJ, j = id % kJ;
  const double v = j < r ? a[j] * ((j == 0) ? 1.0 : pow((double)(q - 2 * l) / (double)q, (double)j)) : 0.0;
  uint16_t hi, lo;
  split_bf16(v, hi, lo);
  const uint32_t at = ((uint32_t)(l / 8) * B_LBO + (uint32_t)(j / 8) * CM + (uint32_t)(j % 8) * 16 +
                       (uint32_t)(l % 8) * 2) / 2;
  tab[at] = hi;
  tab[at + (uint32_t)(q / 8) * B_LBO / 2] = lo;
}

template <int Q>
int launch_stage_a(const float2* x, long long nrows, int rows_per_frame, float2* out, const void* tab,
                   const float2* W, int* status, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    PFT_CUDA_TRY(cudaFuncSetAttribute(k_lf_stage_a<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_A));
    attr = true;
  }
  const float2* tw = pfth::twiddles(kP);
  if (!tw) return PFT_ERR_CUDA;
  long long grid = pfth::sm_count();
  if (grid > nrows / 2) grid = nrows / 2;
  if (grid < 1) return PFT_OK;
  k_lf_stage_a<Q><<<(unsigned)grid, kThreadsA, SMEM_A, st>>>(x, nrows, rows_per_frame, out, (const uint4*)tab, W,
                                                               tw, status);
  PFT_CUDA_TRY(cudaGetLastError());
  return PFT_OK;
}

int stage_ab(int q, const float2* x, long long nrows, int rows_per_frame, float2* out, const void* tab,
             const float2* W, int* status, cudaStream_t st) {
  switch (q) {
    case 32: return launch_stage_a<32>(x, nrows, rows_per_frame, out, tab, W, status, st);
    case 64: return launch_stage_a<64>(x, nrows, rows_per_frame, out, tab, W, status, st);
    case 128: return launch_stage_a<128>(x, nrows, rows_per_frame, out, tab, W, status, st);
    case 256: return launch_stage_a<256>(x, nrows, rows_per_frame, out, tab, W, status, st);
    default: return pfth::set_error(PFT_ERR_UNSUPPORTED, "large-frame block length q=%d not built", q);
  }
}



// ============================================================== adjoint
// Per axis the adjoint of Algorithm 2 reverses each step:
//   H[rho][j] = sum_{t = rho mod 64} conj(W'[t][j]) y[t]
//   E[k][j]   = sum_rho e^{+2 pi i rho k / 64} H[rho][j]        (F^H)
//   x[q k + l] = sum_j B[l][j] E[k][j]                         (B real)
// k_lf_expand reads each row's M inputs transposed (the layout the forward
// writes), runs the first two steps in its loader warps and the last on
// tensor cores (M = 128 blocks, N = q values l, K = 16 terms j).

constexpr int kStagesE = 4;
constexpr uint32_t E_LBO = 16 * CM;               // K-direction step (j 0..7 -> 8..15)
constexpr uint32_t E_COMP = 2 * E_LBO;            // [128 blocks][16 j] BF16
constexpr uint32_t E_STAGE = 4 * E_COMP;          // re hi, re lo, im hi, im lo
constexpr int kStgStride = 17;                    // staging row stride (complex), odd
constexpr uint32_t OFF2_TAB = 0;                  // B^T hi | lo, up to 16 KB
constexpr uint32_t OFF2_E = 16384;
constexpr uint32_t OFF2_STG = OFF2_E + kStagesE * E_STAGE;
constexpr uint32_t STG_BYTES = 4 * 32 * kStgStride * 8;
constexpr uint32_t OFF2_TW = OFF2_STG + STG_BYTES;
constexpr uint32_t OFF2_W = OFF2_TW + 160 * 8;
constexpr uint32_t OFF2_BAR = OFF2_W + kRt * kMl * 8;
constexpr int NBAR2 = 2 * kStagesE + 2 * 4 + 1;
constexpr uint32_t OFF2_SLOT = OFF2_BAR + 8 * NBAR2;
constexpr uint32_t OFF2_ABORT = OFF2_SLOT + 8;
constexpr uint32_t SMEM_E = OFF2_ABORT + 8;
static_assert(SMEM_E <= 232448, "shared memory layout too large");
// Loader warps: three groups of four (warps 8-19) that take every third tile,
// each filling the operand stage of its tile (warps 5-7 idle). At small q the
// stage-B adjoint of a tile's two rows costs more than its expansion, so more
// groups keep the tensor cores and the stores fed.
constexpr int kLdWarpsE = 4, kLdWarp0E = 8, kLdGroupsE = 3;
constexpr int kThreadsE = 32 * (kLdWarp0E + kLdGroupsE * kLdWarpsE);

__device__ __forceinline__ void split8_store(uint8_t* hi_base, uint32_t comp_bytes, uint32_t off, const float (&v)[8]) {
  __nv_bfloat162 h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(h[i]);
    l[i] = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
  }
  *reinterpret_cast<uint4*>(hi_base + off) = *reinterpret_cast<uint4*>(h);
  *reinterpret_cast<uint4*>(hi_base + comp_bytes + off) = *reinterpret_cast<uint4*>(l);
}

// The adjoint of one axis for `nrows` rows, read transposed from
// in[frame][t_idx][row in frame]: the loader warps run the stage-B adjoint of
// two rows per tile (warp pair per row, j = 0..7 and 8..15) straight into the
// BF16 operand of the tensor-core expansion
//   x[row][q k + l] = sum_j B[l][j] E[row][k][j].
template <int Q>
__global__ void __launch_bounds__(kThreadsE, 1)
    k_lf_expand(const float2* __restrict__ in, long long nrows, int rows_per_frame, float2* __restrict__ x,
                const uint4* __restrict__ tab, const float2* __restrict__ gW, const float2* __restrict__ gtw,
                int* status) {
  constexpr int N = kP * Q;
  constexpr uint32_t T_LBO = (Q / 8) * CM;         // B^T: [j / 8][l / 8][8][16 B]
  constexpr uint32_t T_HALF = 2 * T_LBO;
  constexpr uint32_t ACC = 2 * Q;                  // D_re | D_im
  constexpr int kBufs = (512 / ACC) < 4 ? (512 / ACC) : 4;
  constexpr uint32_t TCOLS = kBufs * ACC <= 32 ? 32 : (kBufs * ACC <= 64 ? 64 : (kBufs * ACC <= 128 ? 128 :
                             (kBufs * ACC <= 256 ? 256 : 512)));
  static_assert(2 * T_HALF <= OFF2_E && Q % 16 == 0 && Q <= 256, "block length");
  extern __shared__ __align__(128) uint8_t sm[];
  const uint32_t sb = smem_u32(sm);
  const uint32_t bar = sb + OFF2_BAR;
  const uint32_t E_FULL = bar, E_EMPTY = bar + 8 * kStagesE, ACC_FULL = bar + 16 * kStagesE,
                 ACC_EMPTY = ACC_FULL + 32, DONE = ACC_FULL + 64;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF2_ABORT);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + OFF2_SLOT);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int i = threadIdx.x; i < (int)(2 * T_HALF / 16); i += blockDim.x)
    reinterpret_cast<uint4*>(sm + OFF2_TAB)[i] = __ldg(tab + i);
  float2* s_tw = reinterpret_cast<float2*>(sm + OFF2_TW);
  float2* s_w = reinterpret_cast<float2*>(sm + OFF2_W);
  F64::fill(s_tw, gtw);
  fill_w_slots(s_w, gW);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesE; ++s) {
      mbar_init(E_FULL + 8 * s, kLdWarpsE);
      mbar_init(E_EMPTY + 8 * s, 1);
    }
    for (int b = 0; b < 4; ++b) {
      mbar_init(ACC_FULL + 8 * b, 1);
      mbar_init(ACC_EMPTY + 8 * b, kEpiWarps);
    }
    mbar_init(DONE, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {
    tmem_alloc(smem_u32(tslot), TCOLS);
    tmem_relinquish();
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const long long ntile_all = nrows / 2;
  const long long ntiles = blockIdx.x < ntile_all ? (ntile_all - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (warp == kMmaWarp) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(128, Q);
      const uint64_t th = sdesc(sb + OFF2_TAB, T_LBO, CM), tl = sdesc(sb + OFF2_TAB + T_HALF, T_LBO, CM);
      for (long long T = 0; T < ntiles; ++T) {
        const int b = (int)(T % kBufs);
        const uint32_t v = (uint32_t)(T / kBufs);
        const int s = (int)(T % kStagesE);
        const uint32_t u = (uint32_t)(T / kStagesE);
        if (!mbar_wait(ACC_EMPTY + 8 * b, (v & 1u) ^ 1u, abort_flag, kWaitNs)) break;
        if (!mbar_wait(E_FULL + 8 * s, u & 1u, abort_flag, kWaitNs)) break;
        tc_fence_after();
        const uint32_t es = sb + OFF2_E + s * E_STAGE;
        const uint64_t rh = sdesc(es, E_LBO, CM), rl = sdesc(es + E_COMP, E_LBO, CM);
        const uint64_t ih = sdesc(es + 2 * E_COMP, E_LBO, CM), il = sdesc(es + 3 * E_COMP, E_LBO, CM);
        const uint32_t dr = tmem + b * ACC, di = dr + Q;
        mma_bf16(dr, rh, th, idesc, 0);
        mma_bf16(dr, rl, th, idesc, 1);
        mma_bf16(dr, rh, tl, idesc, 1);
        mma_bf16(di, ih, th, idesc, 0);
        mma_bf16(di, il, th, idesc, 1);
        mma_bf16(di, ih, tl, idesc, 1);
        mma_commit(E_EMPTY + 8 * s);
        mma_commit(ACC_FULL + 8 * b);
      }
      volatile int never = 0;
      mma_commit(DONE);
      mbar_wait(DONE, 0, &never, kWaitNs);
    }
    __syncwarp();
  } else if (warp < kEpiWarps) {
    // TMEM lane 32 q + lane = block k = 32 (q & 1) + lane of row 2t + (q >> 1)
    const int q = warp;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    float2* stg = reinterpret_cast<float2*>(sm + OFF2_STG) + q * 32 * kStgStride;
    for (long long T = 0; T < ntiles; ++T) {
      const long long tile = blockIdx.x + T * gridDim.x;
      const int b = (int)(T % kBufs);
      const uint32_t v = (uint32_t)(T / kBufs);
      if (!mbar_wait(ACC_FULL + 8 * b, v & 1u, abort_flag, kWaitNs)) break;
      tc_fence_after();
      const long long row = 2 * tile + (q >> 1);
      float2* xr = x + row * (long long)N + (q & 1) * 32 * Q;
      for (int c = 0; c < Q / 16; ++c) {
        float re[16], im[16];
        tmem_ld16(tmem + lane_off + b * ACC + 16 * c, re);
        tmem_ld16(tmem + lane_off + b * ACC + Q + 16 * c, im);
        tmem_wait_ld();
        if (c == Q / 16 - 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(ACC_EMPTY + 8 * b);
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) stg[lane * kStgStride + e] = make_float2(re[e], im[e]);
        __syncwarp();
        // 32 blocks x 16 values: 8 lanes per block, 16 bytes each, 4 blocks per step
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int blk = it * 4 + (lane >> 3), part = lane & 7;
          const float2 a = stg[blk * kStgStride + 2 * part], b2 = stg[blk * kStgStride + 2 * part + 1];
          *reinterpret_cast<float4*>(xr + blk * Q + 16 * c + 2 * part) = make_float4(a.x, a.y, b2.x, b2.y);
        }
        __syncwarp();
      }
    }
  } else if (warp >= kLdWarp0E) {
    // warp pair per row r of the tile; warp h fills the K core-matrix column
    // j = 8h .. 8h + 7 of blocks k = lane and lane + 32 (terms j >= 13 are 0)
    const int grp = (warp - kLdWarp0E) / kLdWarpsE;
    const int w = (warp - kLdWarp0E) % kLdWarpsE, r = w >> 1, h = w & 1;
    typename F64::Net net;
    F64::init_net(net, lane, s_tw);
    const int rho0 = 2 * bitrev<32>(lane);
    for (long long T = grp; T < ntiles; T += kLdGroupsE) {
      const long long tile = blockIdx.x + T * gridDim.x;
      const int s = (int)(T % kStagesE);
      const uint32_t u = (uint32_t)(T / kStagesE);
      const long long row = 2 * tile + r;
      const long long f = row / rows_per_frame, rin = row % rows_per_frame;
      const float2* ip = in + f * (long long)kMl * rows_per_frame + rin;
      float2 yv[4];  // slot i * 32 + lane: t_idx = rho0 + (i >> 1) + 64 (i & 1)
#pragma unroll
      for (int i = 0; i < 4; ++i) yv[i] = __ldg(ip + (long long)(rho0 + (i >> 1) + kP * (i & 1)) * rows_per_frame);
      float er0[8], ei0[8], er1[8], ei1[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int j = 8 * h + jj;
        float2 hv[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (j < kRt) {
#pragma unroll
          for (int pos = 0; pos < 2; ++pos) {
#pragma unroll
            for (int hi = 0; hi < 2; ++hi) {
              const float2 wv = s_w[j * kMl + (2 * pos + hi) * 32 + lane], yy = yv[2 * pos + hi];
              hv[pos].x = fmaf(wv.x, yy.x, fmaf(wv.y, yy.y, hv[pos].x));   // conj(W') y
              hv[pos].y = fmaf(wv.x, yy.y, fmaf(-wv.y, yy.x, hv[pos].y));
            }
          }
          F64::adj(hv, lane, s_tw, net);  // hv[e] = E[lane + 32 e][j]
        }
        er0[jj] = hv[0].x;
        ei0[jj] = hv[0].y;
        er1[jj] = hv[1].x;
        ei1[jj] = hv[1].y;
      }
      if (!mbar_wait(E_EMPTY + 8 * s, (u & 1u) ^ 1u, abort_flag, kWaitNs)) break;
      uint8_t* es = sm + OFF2_E + s * E_STAGE;
      const uint32_t m0 = (uint32_t)(64 * r + lane), m1 = m0 + 32;
      split8_store(es, E_COMP, (uint32_t)h * E_LBO + m0 * 16, er0);
      split8_store(es + 2 * E_COMP, E_COMP, (uint32_t)h * E_LBO + m0 * 16, ei0);
      split8_store(es, E_COMP, (uint32_t)h * E_LBO + m1 * 16, er1);
      split8_store(es + 2 * E_COMP, E_COMP, (uint32_t)h * E_LBO + m1 * 16, ei1);
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(E_FULL + 8 * s);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, TCOLS);
  }
  if (threadIdx.x == 0 && *abort_flag) {
    *reinterpret_cast<volatile int*>(status) = PFT_ERR_TIMEOUT;
    __threadfence_system();
  }
}

// B^T for the expansion: [N = l][K = j] K-major, hi | lo, each
// [j / 8][l / 8][8][16 B].
__global__ void k_lf_table_adj(int q, int r, const double* __restrict__ a, uint16_t* __restrict__ tab) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= q * kJ) return;
  const int l = id / kJ, j = id % kJ;
  const double v = j < r ? a[j] * ((j == 0) ? 1.0 : pow((double)(q - 2 * l) / (double)q, (double)j)) : 0.0;
  uint16_t hi, lo;
  split_bf16(v, hi, lo);
  const uint32_t t_lbo = (uint32_t)(q / 8) * CM;
  const uint32_t at = ((uint32_t)(j / 8) * t_lbo + (uint32_t)(l / 8) * CM + (uint32_t)(l % 8) * 16 +
                       (uint32_t)(j % 8) * 2) / 2;
  tab[at] = hi;
  tab[at + t_lbo] = lo;  // lo half starts 2 t_lbo bytes = t_lbo entries later
}

template <int Q>
int launch_expand(const float2* in, long long nrows, int rows_per_frame, float2* x, const void* tab, const float2* W,
                  int* status, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    PFT_CUDA_TRY(cudaFuncSetAttribute(k_lf_expand<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_E));
    attr = true;
  }
  long long grid = pfth::sm_count();
  if (grid > nrows / 2) grid = nrows / 2;
  if (grid < 1) return PFT_OK;
  const float2* tw = pfth::twiddles(kP);
  if (!tw) return PFT_ERR_CUDA;
  k_lf_expand<Q><<<(unsigned)grid, kThreadsE, SMEM_E, st>>>(in, nrows, rows_per_frame, x, (const uint4*)tab, W, tw,
                                                              status);
  PFT_CUDA_TRY(cudaGetLastError());
  return PFT_OK;
}

int expand(int q, const float2* in, long long nrows, int rows_per_frame, float2* x, const void* tab, const float2* W,
           int* status, cudaStream_t st) {
  switch (q) {
    case 32: return launch_expand<32>(in, nrows, rows_per_frame, x, tab, W, status, st);
    case 64: return launch_expand<64>(in, nrows, rows_per_frame, x, tab, W, status, st);
    case 128: return launch_expand<128>(in, nrows, rows_per_frame, x, tab, W, status, st);
    case 256: return launch_expand<256>(in, nrows, rows_per_frame, x, tab, W, status, st);
    default: return pfth::set_error(PFT_ERR_UNSUPPORTED, "large-frame block length q=%d not built", q);
  }
}


}  // namespace

namespace pfth {

bool lf_supported(int n, int M, int p) {
  return M == kMl && (p == 0 || p == kP) && (n == 2048 || n == 4096 || n == 8192 || n == 16384);
}

int lf_build(pft_plan* plan) {
  const int n = plan->n1, q = plan->q1;
  double xi = 0.0, a[pftc::kMaxTerms] = {0};
  if (!pftc::design(plan->eps, plan->r1, &xi, a, nullptr))
    return set_error(PFT_ERR_INVALID_ARG, "coefficient design failed (eps=%g r=%d)", plan->eps, plan->r1);
  if (plan->r1 != kRt) return set_error(PFT_ERR_UNSUPPORTED, "large frames are built for r = %d terms", kRt);
  double* d_a = nullptr;
  PFT_CUDA_TRY(cudaMalloc(&d_a, sizeof(double) * pftc::kMaxTerms));
  PFT_CUDA_TRY(cudaMemcpy(d_a, a, sizeof(double) * plan->r1, cudaMemcpyHostToDevice));
  PFT_CUDA_TRY(cudaMalloc(&plan->d_tc, 2 * (q / 8) * B_LBO));
  k_lf_table<<<(q * kJ + 127) / 128, 128>>>(q, plan->r1, d_a, reinterpret_cast<uint16_t*>(plan->d_tc));
  PFT_CUDA_TRY(cudaGetLastError());
  PFT_CUDA_TRY(cudaMalloc(&plan->d_tc_adj, 4 * (q / 8) * CM));
  k_lf_table_adj<<<(q * kJ + 127) / 128, 128>>>(q, plan->r1, d_a, reinterpret_cast<uint16_t*>(plan->d_tc_adj));
  PFT_CUDA_TRY(cudaGetLastError());
  PFT_CUDA_TRY(cudaDeviceSynchronize());
  PFT_CUDA_TRY(cudaFree(d_a));
  // frames per pass: the transposed intermediate T^T (128 x n per frame) of a
  // pass stays well inside L2
  const long long t_bytes = (long long)kMl * n * sizeof(float2);
  plan->lf_chunk = (int)std::max(1LL, (32LL << 20) / t_bytes);
  const long long f = plan->lf_chunk;
  const size_t ws = (size_t)f * (size_t)kMl * n * sizeof(float2);
  PFT_CUDA_TRY(cudaMalloc(&plan->d_ws, ws));
  PFT_CUDA_TRY(cudaHostAlloc(&plan->h_status, sizeof(int), cudaHostAllocMapped));
  *plan->h_status = PFT_OK;
  PFT_CUDA_TRY(cudaHostGetDevicePointer(&plan->d_status, plan->h_status, 0));
  return PFT_OK;
}

int lf_forward(const pft_plan* plan, const void* x, void* y, int64_t batch, void* stream) {
  if (*plan->h_status != PFT_OK) {
    const int st = *plan->h_status;
    *plan->h_status = PFT_OK;
    return set_error(st, "a device-side wait of an earlier large-frame launch timed out");
  }
  const cudaStream_t st = (cudaStream_t)stream;
  const int n = plan->n1;
  const long long f = plan->lf_chunk;
  float2* TT = (float2*)plan->d_ws;
  const float2* W = plan->d_W;  // axis 0: W'[j][t_idx], j < RMAX, t_idx < 128
  for (long long f0 = 0; f0 < batch; f0 += f) {
    const long long nf = std::min<long long>(f, batch - f0);
    const float2* xf = (const float2*)x + f0 * (long long)n * n;
    float2* yf = (float2*)y + f0 * (long long)kMl * kMl;
    int rc = stage_ab(plan->q1, xf, nf * n, n, TT, plan->d_tc, W, plan->d_status, st);
    if (rc == PFT_OK) rc = stage_ab(plan->q1, TT, nf * kMl, kMl, yf, plan->d_tc, W, plan->d_status, st);
    if (rc != PFT_OK) return rc;
  }
  return PFT_OK;
}

int lf_adjoint(const pft_plan* plan, const void* y, void* x, int64_t batch, void* stream) {
  if (*plan->h_status != PFT_OK) {
    const int st = *plan->h_status;
    *plan->h_status = PFT_OK;
    return set_error(st, "a device-side wait of an earlier large-frame launch timed out");
  }
  const cudaStream_t st = (cudaStream_t)stream;
  const int n = plan->n1;
  const long long f = plan->lf_chunk;
  float2* TT = (float2*)plan->d_ws;
  const float2* W = plan->d_W;
  for (long long f0 = 0; f0 < batch; f0 += f) {
    const long long nf = std::min<long long>(f, batch - f0);
    const float2* yf = (const float2*)y + f0 * (long long)kMl * kMl;
    float2* xf = (float2*)x + f0 * (long long)n * n;
    int rc = expand(plan->q1, yf, nf * kMl, kMl, TT, plan->d_tc_adj, W, plan->d_status, st);
    if (rc == PFT_OK) rc = expand(plan->q1, TT, nf * n, n, xf, plan->d_tc_adj, W, plan->d_status, st);
    if (rc != PFT_OK) return rc;
  }
  return PFT_OK;
}

}  // namespace pfth
