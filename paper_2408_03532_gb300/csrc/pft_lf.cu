// Large-frame PFT (the paper's regime n >> M): n = 2048, 4096 or 8192 with
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
// runs on CUDA cores in FP32 and writes the row's M outputs transposed, so
// the second axis is the same two kernels applied to the rows of the
// transposed intermediate T^T[t2][u]:
//   k_lf_stage_a(x rows)   -> C    [rows][13][64]
//   k_lf_stage_b(C)        -> T^T  [frame][128][n]
//   k_lf_stage_a(T^T rows) -> C'   [rows][13][64]
//   k_lf_stage_b(C')       -> Y    [frame][128][128]
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
constexpr int kStages = 6;
constexpr int kAccBufs = 4;
constexpr uint32_t CM = 128;
constexpr uint32_t X_LBO = 16 * CM + 32;          // padded: conflict-free 4-byte stores
constexpr uint32_t X_COMP = (kC / 8) * X_LBO;
constexpr uint32_t X_STAGE = 4 * X_COMP;
constexpr uint32_t B_LBO = (kJ / 8) * CM;         // 256: table core matrices along K
constexpr uint32_t TAB_MAX = 2 * (128 / 8) * B_LBO;  // hi + lo at q = 128: 8 KB
constexpr uint32_t OFF_TAB = 0;
constexpr uint32_t OFF_X = TAB_MAX;
constexpr uint32_t OFF_BAR = OFF_X + kStages * X_STAGE;
constexpr int NBAR = 2 * kStages + 2 * kAccBufs + 1;
constexpr uint32_t OFF_SLOT = OFF_BAR + 8 * NBAR;
constexpr uint32_t OFF_ABORT = OFF_SLOT + 8;
constexpr uint32_t SMEM_A = OFF_ABORT + 8;
static_assert(SMEM_A <= 232448, "shared memory layout too large");

constexpr int kEpiWarps = 4, kMmaWarp = 4, kLdWarp0 = 8, kLdWarps = 16;  // warps 5-7 idle
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

// Stage A of `nrows` rows of length 64 Q (row stride = row length); the tile
// t covers rows 2t, 2t + 1, i.e. 128 blocks (row, k) of Q values.
template <int Q>
__global__ void __launch_bounds__(kThreadsA, 1)
    k_lf_stage_a(const float2* __restrict__ x, long long nrows, float2* __restrict__ C,
                 const uint4* __restrict__ tab, int* status) {
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
  } else if (warp < kEpiWarps) {
    // TMEM lane m = 32 q + lane: block k = 32 (q & 1) + lane of row 2t + (q >> 1)
    const int q = warp;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    for (long long T = 0; T < ntiles; ++T) {
      const long long tile = blockIdx.x + T * gridDim.x;
      const int b = (int)(T % kAccBufs);
      const uint32_t v = (uint32_t)(T / kAccBufs);
      if (!mbar_wait(ACC_FULL + 8 * b, v & 1u, abort_flag, kWaitNs)) break;
      tc_fence_after();
      float re[16], im[16];
      tmem_ld16(tmem + lane_off + b * ACC_COLS, re);
      tmem_ld16(tmem + lane_off + b * ACC_COLS + kJ, im);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(ACC_EMPTY + 8 * b);
      const long long row = 2 * tile + (q >> 1);
      float2* dst = C + row * (long long)(kRt * kP) + (q & 1) * 32 + lane;
#pragma unroll
      for (int j = 0; j < kRt; ++j) dst[j * kP] = make_float2(re[j], im[j]);
    }
  } else if (warp >= kLdWarp0) {
    const int cw = warp - kLdWarp0;
    const int half = lane >> 4, e = lane & 15;
    const uint32_t kk = (uint32_t)(e >> 2), wd = (uint32_t)(e & 3);
    const long long total = ntiles * kChunks;
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
        r[j] = __ldg(reinterpret_cast<const float4*>(src));
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

// Stage B of `nrows` rows (rows_per_frame rows per frame): one warp per row,
// eight consecutive rows per CTA; writes out[frame][t_idx][row in frame].
constexpr int kThreadsB = 256;
constexpr int kRowsB = kThreadsB / 32;
using F64 = Fft<kP>;

__global__ void __launch_bounds__(kThreadsB)
    k_lf_stage_b(const float2* __restrict__ C, long long nrows, int rows_per_frame, float2* __restrict__ out,
                 const float2* __restrict__ gW, const float2* __restrict__ gtw) {
  __shared__ float2 tw[F64::TAB];
  __shared__ float2 sW[kRt * kMl];
  __shared__ float2 stage[kMl][kRowsB];
  F64::fill(tw, gtw);
  for (int i = threadIdx.x; i < kRt * kMl; i += blockDim.x) sW[i] = gW[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  typename F64::Net net;
  F64::init_net(net, lane, tw);
  const int rho0 = 2 * bitrev<32>(lane);
  for (long long r0 = (long long)blockIdx.x * kRowsB; r0 < nrows; r0 += (long long)gridDim.x * kRowsB) {
    const long long row = r0 + warp;
    float2 ch[kRt][2];
    const float2* src = C + row * (long long)(kRt * kP);
#pragma unroll
    for (int j = 0; j < kRt; ++j) {
      float2 v[2] = {__ldg(src + j * kP + lane), __ldg(src + j * kP + lane + 32)};
      F64::fwd(v, lane, tw, net);  // v[pos] = C^[pos + 2 bitrev(lane)][j]
      ch[j][0] = v[0];
      ch[j][1] = v[1];
    }
#pragma unroll
    for (int pos = 0; pos < 2; ++pos) {
      const int rho = rho0 + pos;
#pragma unroll
      for (int hi = 0; hi < 2; ++hi) {
        const int ti = rho + hi * kP;  // t = ti - 64, t mod 64 = rho
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < kRt; ++j) {
          const float2 w = sW[j * kMl + ti];
          acc.x = fmaf(w.x, ch[j][pos].x, fmaf(-w.y, ch[j][pos].y, acc.x));
          acc.y = fmaf(w.x, ch[j][pos].y, fmaf(w.y, ch[j][pos].x, acc.y));
        }
        stage[ti][warp] = acc;
      }
    }
    __syncthreads();
    const long long f = r0 / rows_per_frame;
    const int rin = (int)(r0 % rows_per_frame);
    float2* o = out + f * (long long)kMl * rows_per_frame + rin;
    for (int i = threadIdx.x; i < kMl * kRowsB / 2; i += blockDim.x) {
      const int ti = i / (kRowsB / 2), part = i % (kRowsB / 2);
      const float2 a = stage[ti][2 * part], b = stage[ti][2 * part + 1];
      *reinterpret_cast<float4*>(o + (long long)ti * rows_per_frame + 2 * part) = make_float4(a.x, a.y, b.x, b.y);
    }
    __syncthreads();
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
int launch_stage_a(const float2* x, long long nrows, float2* C, const void* tab, int* status, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    PFT_CUDA_TRY(cudaFuncSetAttribute(k_lf_stage_a<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_A));
    attr = true;
  }
  long long grid = pfth::sm_count();
  if (grid > nrows / 2) grid = nrows / 2;
  if (grid < 1) return PFT_OK;
  k_lf_stage_a<Q><<<(unsigned)grid, kThreadsA, SMEM_A, st>>>(x, nrows, C, (const uint4*)tab, status);
  PFT_CUDA_TRY(cudaGetLastError());
  return PFT_OK;
}

int stage_a(int q, const float2* x, long long nrows, float2* C, const void* tab, int* status, cudaStream_t st) {
  switch (q) {
    case 32: return launch_stage_a<32>(x, nrows, C, tab, status, st);
    case 64: return launch_stage_a<64>(x, nrows, C, tab, status, st);
    case 128: return launch_stage_a<128>(x, nrows, C, tab, status, st);
    default: return pfth::set_error(PFT_ERR_UNSUPPORTED, "large-frame block length q=%d not built", q);
  }
}

int stage_b(const float2* C, long long nrows, int rows_per_frame, float2* out, const float2* W, cudaStream_t st) {
  const float2* tw = pfth::twiddles(kP);
  if (!tw) return PFT_ERR_CUDA;
  long long groups = nrows / kRowsB;
  long long grid = groups < 8LL * pfth::sm_count() ? groups : 8LL * pfth::sm_count();
  k_lf_stage_b<<<(unsigned)grid, kThreadsB, 0, st>>>(C, nrows, rows_per_frame, out, W, tw);
  PFT_CUDA_TRY(cudaGetLastError());
  return PFT_OK;
}

}  // namespace

namespace pfth {

bool lf_supported(int n, int M, int p) {
  return M == kMl && (p == 0 || p == kP) && (n == 2048 || n == 4096 || n == 8192);
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
  PFT_CUDA_TRY(cudaDeviceSynchronize());
  PFT_CUDA_TRY(cudaFree(d_a));
  // frames per chunk: keep the stage-A intermediate of a chunk near 128 MB (L2-sized)
  const long long c_bytes = (long long)n * kRt * kP * sizeof(float2);
  plan->lf_chunk = (int)std::max(1LL, (128LL << 20) / c_bytes);
  const long long f = plan->lf_chunk;
  const size_t ws = (size_t)f * ((size_t)n * kRt * kP + (size_t)kMl * n + (size_t)kMl * kRt * kP) * sizeof(float2);
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
  float2* Cw = (float2*)plan->d_ws;
  float2* TT = Cw + f * (long long)n * kRt * kP;
  float2* C2 = TT + f * (long long)kMl * n;
  const float2* W = plan->d_W;  // axis 0: W'[j][t_idx], j < RMAX, t_idx < 128
  for (long long f0 = 0; f0 < batch; f0 += f) {
    const long long nf = std::min<long long>(f, batch - f0);
    const float2* xf = (const float2*)x + f0 * (long long)n * n;
    float2* yf = (float2*)y + f0 * (long long)kMl * kMl;
    int rc = stage_a(plan->q1, xf, nf * n, Cw, plan->d_tc, plan->d_status, st);
    if (rc == PFT_OK) rc = stage_b(Cw, nf * n, n, TT, W, st);
    if (rc == PFT_OK) rc = stage_a(plan->q1, TT, nf * kMl, C2, plan->d_tc, plan->d_status, st);
    if (rc == PFT_OK) rc = stage_b(C2, nf * kMl, kMl, yf, W, st);
    if (rc != PFT_OK) return rc;
  }
  return PFT_OK;
}

}  // namespace pfth
