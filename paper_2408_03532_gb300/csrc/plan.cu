// PFT plans (Algorithm 4) and the batched forward / adjoint transforms
// (Algorithm 5 and its exact adjoint) on sm_103a.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "coeffs.h"
#include "plan.cuh"

using namespace pftk;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// ------------------------------------------------------------ FP64 tables
// Algorithm 1 / 4 tables for one axis, in FP64 with exact integer phase
// reduction, rounded once to FP32:
//   B[l][j]   = a_j (1 - 2 l / q)^j                    (real; w_j = i^j a_j)
//   W'[j][t]  = i^j (t / p)^j e^{-i pi t / p},  t = t_idx - M/2
//             = (t / p)^j e^{i pi m / p},  m = (j p / 2 - t) mod 2p
//   tw[m]     = e^{-2 pi i m / p}
__global__ void k_tables(int q, int p, int M, int r, const double* __restrict__ a, float* __restrict__ B,
                         float2* __restrict__ W, float2* __restrict__ tw) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nB = q * RMAX, nW = RMAX * M;
  if (tid < nB) {
    const int l = tid / RMAX, j = tid % RMAX;
    double v = 0.0;
    if (j < r) v = a[j] * pow((double)(q - 2 * l) / (double)q, (double)j);
    B[tid] = (float)v;
  } else if (tid < nB + nW) {
    const int i = tid - nB, j = i / M, ti = i % M;
    const long long t = (long long)ti - M / 2;
    float2 out = make_float2(0.f, 0.f);
    if (j < r) {
      const double mag = (j == 0) ? 1.0 : pow((double)t / (double)p, (double)j);
      long long m = ((long long)j * (p / 2) - t) % (2LL * p);
      if (m < 0) m += 2LL * p;
      double s, c;
      sincospi((double)m / (double)p, &s, &c);
      out = make_float2((float)(mag * c), (float)(mag * s));
    }
    W[i] = out;
  } else if (tid < nB + nW + p / 2) {
    const int m = tid - nB - nW;
    double s, c;
    sincospi(-2.0 * (double)m / (double)p, &s, &c);
    tw[m] = make_float2((float)c, (float)s);
  }
}

// --------------------------------------------------------- frame kernels
// A frame is n1 x n2 (rows u < n1 of length n2). Axis 2 (along a row) uses the
// 1-D shape (P2, Q2, M2/P2), axis 1 (along a column) the shape (P1, Q1, M1/P1);
// a square plan is the case where both are the same.
template <int P1, int Q1, int MP1, int P2, int Q2, int MP2>
struct FrameShape {
  static constexpr int N1 = P1 * Q1, M1 = MP1 * P1, G1 = 32 / P1;
  static constexpr int N2 = P2 * Q2, M2 = MP2 * P2, G2 = 32 / P2;
  static constexpr bool SAME = (P1 == P2);  // one stage table and lane network serve both axes
  using L = YLayout<Q1, M2>;                // the n1 x M2 intermediate, read by columns in blocks of Q1
  static constexpr int OFF_W1 = 0;
  static constexpr int OFF_W2 = OFF_W1 + RMAX * M1;
  static constexpr int OFF_TW1 = OFF_W2 + RMAX * M2;
  static constexpr int OFF_TW2 = SAME ? OFF_TW1 : OFF_TW1 + 32;
  static constexpr int OFF_Y = OFF_TW2 + 32;
  static constexpr int OFF_Z = OFF_Y + N1 * L::S;
  static constexpr int ZS = M2 + 1;
  static constexpr int FLOATS2 = OFF_Z + M1 * ZS;
  static constexpr size_t SMEM = sizeof(float2) * FLOATS2;
};

template <int Q>
__device__ __forceinline__ void load_block_v4(const float2* __restrict__ src, float2 (&x)[Q]) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int i = 0; i < Q / 2; ++i) {
    float4 v = __ldg(s4 + i);
    x[2 * i] = make_float2(v.x, v.y);
    x[2 * i + 1] = make_float2(v.z, v.w);
  }
}

template <int Q>
__device__ __forceinline__ void store_block_v4(float2* dst, const float2 (&x)[Q]) {
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int i = 0; i < Q / 2; ++i) d4[i] = make_float4(x[2 * i].x, x[2 * i].y, x[2 * i + 1].x, x[2 * i + 1].y);
}

// W' of both axes (axis 1 then axis 2, RMAX x M each, j-major) and the stage
// tables of the lane networks (axis 2's at gtw + 32 when P1 != P2).
template <class S, int P1, int P2>
__device__ __forceinline__ void load_tables(float2* sm, const float2* __restrict__ gW,
                                            const float2* __restrict__ gtw) {
  for (int i = threadIdx.x; i < RMAX * (S::M1 + S::M2); i += blockDim.x) sm[i] = gW[i];
  fill_stage_table<P1>(sm + S::OFF_TW1, gtw, P1);
  if constexpr (!S::SAME) fill_stage_table<P2>(sm + S::OFF_TW2, gtw + 32, P2);
}

// y[f] = A1 x[f] A2^T  (Algorithm 5), one frame per CTA iteration.
template <int P1, int Q1, int MP1, int P2, int Q2, int MP2>
__global__ void __launch_bounds__(kThreads) k_pft_fwd(const float2* __restrict__ x, float2* __restrict__ y,
                                                      long long batch, const __grid_constant__ PftConst c,
                                                      const float2* __restrict__ gW, const float2* __restrict__ gtw) {
  using S = FrameShape<P1, Q1, MP1, P2, Q2, MP2>;
  using T1 = Pft1D<P1, Q1, MP1>;
  using T2 = Pft1D<P2, Q2, MP2>;
  constexpr int N1 = S::N1, N2 = S::N2, M1 = S::M1, M2 = S::M2, G1 = S::G1, G2 = S::G2;
  extern __shared__ __align__(16) float2 sm[];
  float2* sW1 = sm + S::OFF_W1;
  float2* sW2 = sm + S::OFF_W2;
  float2* sY = sm + S::OFF_Y;
  float2* sZ = sm + S::OFF_Z;
  load_tables<S, P1, P2>(sm, gW, gtw);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k1 = lane % P1, g1 = lane / P1, k2 = lane % P2, g2 = lane / P2;
  LaneNet<P1, false> net1;
  net1.init(k1, sm + S::OFF_TW1);
  LaneNet<P2, false> net2;
  if constexpr (S::SAME) net2 = net1;
  else net2.init(k2, sm + S::OFF_TW2);
  // Each warp keeps the next row block's loads in flight while it computes the
  // current one (also across frames, so they overlap the column pass).
  constexpr int STEP = kWarps * G2;
  float2 xn[Q2];
  long long fn = blockIdx.x;
  int un = warp * G2;
  if (fn < batch) load_block_v4<Q2>(x + fn * (long long)(N1 * N2) + (un + g2) * N2 + Q2 * k2, xn);
  for (long long f = blockIdx.x; f < batch; f += gridDim.x) {
    // rows: axis 2
    for (int u0 = warp * G2; u0 < N1; u0 += STEP) {
      const int u = u0 + g2;
      float2 xv[Q2];
#pragma unroll
      for (int l = 0; l < Q2; ++l) xv[l] = xn[l];
      un = u0 + STEP;
      fn = f;
      if (un >= N1) {
        un = warp * G2;
        fn = f + gridDim.x;
      }
      if (fn < batch) load_block_v4<Q2>(x + fn * (long long)(N1 * N2) + (un + g2) * N2 + Q2 * k2, xn);
      T2::forward(xv, k2, c.bh[1], sW2, net2, [&](int t, float2 v) { sY[S::L::at(u, t)] = v; });
    }
    __syncthreads();
    // columns: axis 1
    for (int cs0 = warp * G1; cs0 < M2; cs0 += kWarps * G1) {
      const int t2 = col_of<P1>(cs0 + g1);
      float2 xv[Q1];
#pragma unroll
      for (int l = 0; l < Q1; ++l) xv[l] = sY[S::L::at(Q1 * k1 + l, t2)];
      T1::forward(xv, k1, c.bh[0], sW1, net1, [&](int t1, float2 v) { sZ[t1 * S::ZS + t2] = v; });
    }
    __syncthreads();
    float2* yf = y + f * (long long)(M1 * M2);
    for (int i = threadIdx.x; i < M1 * M2; i += kThreads) yf[i] = sZ[(i / M2) * S::ZS + (i % M2)];
    __syncthreads();
  }
}

// x[f] = A1^H y[f] conj(A2)  (exact adjoint of k_pft_fwd).
template <int P1, int Q1, int MP1, int P2, int Q2, int MP2>
__global__ void __launch_bounds__(kThreads) k_pft_adj(const float2* __restrict__ y, float2* __restrict__ x,
                                                      long long batch, const __grid_constant__ PftConst c,
                                                      const float2* __restrict__ gW, const float2* __restrict__ gtw) {
  using S = FrameShape<P1, Q1, MP1, P2, Q2, MP2>;
  using T1 = Pft1D<P1, Q1, MP1>;
  using T2 = Pft1D<P2, Q2, MP2>;
  constexpr int N1 = S::N1, N2 = S::N2, M1 = S::M1, M2 = S::M2, G1 = S::G1, G2 = S::G2;
  extern __shared__ __align__(16) float2 sm[];
  float2* sW1 = sm + S::OFF_W1;
  float2* sW2 = sm + S::OFF_W2;
  float2* sY = sm + S::OFF_Y;
  float2* sZ = sm + S::OFF_Z;
  load_tables<S, P1, P2>(sm, gW, gtw);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k1 = lane % P1, g1 = lane / P1, k2 = lane % P2, g2 = lane / P2;
  LaneNet<P1, false> net1;
  net1.init(k1, sm + S::OFF_TW1);
  LaneNet<P2, false> net2;
  if constexpr (S::SAME) net2 = net1;
  else net2.init(k2, sm + S::OFF_TW2);
  for (long long f = blockIdx.x; f < batch; f += gridDim.x) {
    const float2* yf = y + f * (long long)(M1 * M2);
    for (int i = threadIdx.x; i < M1 * M2; i += kThreads) sZ[(i / M2) * S::ZS + (i % M2)] = __ldg(yf + i);
    __syncthreads();
    // columns: adjoint of axis 1
    for (int cs0 = warp * G1; cs0 < M2; cs0 += kWarps * G1) {
      const int t2 = col_of<P1>(cs0 + g1);
      float2 xv[Q1];
      T1::adjoint([&](int t1) { return sZ[t1 * S::ZS + t2]; }, k1, c.bh[0], sW1, net1, xv);
#pragma unroll
      for (int l = 0; l < Q1; ++l) sY[S::L::at(Q1 * k1 + l, t2)] = xv[l];
    }
    __syncthreads();
    // rows: adjoint of axis 2
    float2* xf = x + f * (long long)(N1 * N2);
    for (int u0 = warp * G2; u0 < N1; u0 += kWarps * G2) {
      const int u = u0 + g2;
      float2 xv[Q2];
      T2::adjoint([&](int t) { return sY[S::L::at(u, t)]; }, k2, c.bh[1], sW2, net2, xv);
      store_block_v4<Q2>(xf + u * N2 + Q2 * k2, xv);
    }
    __syncthreads();
  }
}

template <int P1, int Q1, int MP1, int P2 = P1, int Q2 = Q1, int MP2 = MP1>
pfth::FrameKernels make_frame_kernels() {
  return pfth::FrameKernels{P1, Q1, MP1, P2, Q2, MP2,
                            (const void*)k_pft_fwd<P1, Q1, MP1, P2, Q2, MP2>,
                            (const void*)k_pft_adj<P1, Q1, MP1, P2, Q2, MP2>,
                            FrameShape<P1, Q1, MP1, P2, Q2, MP2>::SMEM};
}

// Shapes built: M = 2P (m~/p = 1, the paper's choice) for the frame sizes of
// the workloads (n = 32 ... 256, M = 16 ... 64), square, and a few rectangular
// frames (axis 1 first): the rectangle's sides and outputs per axis differ, and
// so may p.
const pfth::FrameKernels g_frame_kernels[] = {
    make_frame_kernels<8, 4, 2>(),   // n = 32,  M = 16
    make_frame_kernels<8, 8, 2>(),   // n = 64,  M = 16
    make_frame_kernels<16, 4, 2>(),  // n = 64,  M = 32
    make_frame_kernels<8, 16, 2>(),  // n = 128, M = 16
    make_frame_kernels<16, 8, 2>(),  // n = 128, M = 32
    make_frame_kernels<32, 4, 2>(),  // n = 128, M = 64
    make_frame_kernels<16, 16, 2>(), // n = 256, M = 32
    make_frame_kernels<32, 8, 2>(),  // n = 256, M = 64
    make_frame_kernels<32, 2, 2>(),  // n = 64,  M = 64
    make_frame_kernels<8, 32, 2>(),  // n = 256, M = 16
    make_frame_kernels<16, 8, 2, 16, 16, 2>(),  // 128 x 256, M 32 x 32
    make_frame_kernels<16, 16, 2, 16, 8, 2>(),  // 256 x 128, M 32 x 32
    make_frame_kernels<16, 4, 2, 16, 8, 2>(),   // 64 x 128,  M 32 x 32
    make_frame_kernels<16, 8, 2, 32, 4, 2>(),   // 128 x 128, M 32 x 64
    make_frame_kernels<32, 8, 2, 16, 16, 2>(),  // 256 x 256, M 64 x 32
    make_frame_kernels<8, 16, 2, 16, 8, 2>(),   // 128 x 128, M 16 x 32
};

}  // namespace

namespace pfth {

int frame_kernel_count() { return (int)(sizeof(g_frame_kernels) / sizeof(g_frame_kernels[0])); }
const FrameKernels* frame_kernels(int id) { return &g_frame_kernels[id]; }
int find_frame_kernels(int P1, int Q1, int MP1, int P2, int Q2, int MP2) {
  for (int i = 0; i < frame_kernel_count(); ++i) {
    const FrameKernels& f = g_frame_kernels[i];
    if (f.P1 == P1 && f.Q1 == Q1 && f.MP1 == MP1 && f.P2 == P2 && f.Q2 == Q2 && f.MP2 == MP2) return i;
  }
  return -1;
}

namespace {

// Algorithm 4 for one axis: p, q and r (r_force > 0 fixes r), checked against
// what the kernels are built for.
struct AxisPlan {
  int n, M, P, Q, r;
  double xi;
  double a[pftc::kMaxTerms];
};

int plan_axis(int n, int M, int P, double eps, int r_force, AxisPlan* ax) {
  if (n <= 0 || M <= 0 || M % 2 || M > n)
    return set_error(PFT_ERR_INVALID_ARG, "need n > 0 and even 0 < M <= n (n=%d M=%d)", n, M);
  if (P == 0) P = M / 2;
  if (P < 2 || n % P)
    return set_error(PFT_ERR_INVALID_ARG, "p=%d must divide n=%d and be >= 2", P, n);
  const int Q = n / P;
  if (Q < 2 || (Q & (Q - 1)) || (P & (P - 1)))
    return set_error(PFT_ERR_UNSUPPORTED, "p=%d, q=%d: powers of two >= 2 are built", P, Q);
  if (M % P) return set_error(PFT_ERR_UNSUPPORTED, "M=%d must be a multiple of p=%d", M, P);
  int r = r_force;
  if (r <= 0) {
    r = pftc::choose_r(eps, (M / 2.0) / P);
    if (r < 0) return set_error(PFT_ERR_INVALID_ARG, "no r reaches eps=%g at m~/p=%g", eps, (M / 2.0) / P);
  }
  if (r > RMAX)
    return set_error(PFT_ERR_UNSUPPORTED, "r=%d > %d terms (eps=%g, m~/p=%g): use a larger p", r, RMAX, eps,
                     (M / 2.0) / P);
  ax->n = n;
  ax->M = M;
  ax->P = P;
  ax->Q = Q;
  ax->r = r;
  std::fill(ax->a, ax->a + pftc::kMaxTerms, 0.0);
  if (!pftc::design(eps, r, &ax->xi, ax->a, nullptr))
    return set_error(PFT_ERR_INVALID_ARG, "coefficient design failed (eps=%g r=%d)", eps, r);
  return PFT_OK;
}

}  // namespace

int build_plan2(pft_plan* p, int n1, int n2, int M1, int M2, int P1, int P2, double eps, int r1, int r2) {
  AxisPlan ax[2];
  int rc = plan_axis(n1, M1, P1, eps, r1, &ax[0]);
  if (rc != PFT_OK) return rc;
  rc = plan_axis(n2, M2, P2, eps, r2, &ax[1]);
  if (rc != PFT_OK) return rc;
  const bool square = n1 == n2 && M1 == M2 && ax[0].P == ax[1].P;
  const int kid = find_frame_kernels(ax[0].P, ax[0].Q, M1 / ax[0].P, ax[1].P, ax[1].Q, M2 / ax[1].P);
  if (kid < 0 && !(square && lf_supported(n1, M1, ax[0].P)))
    return set_error(PFT_ERR_UNSUPPORTED, "no kernel built for %d x %d frames, M = %d x %d, p = %d, %d", n1, n2, M1,
                     M2, ax[0].P, ax[1].P);
  p->n1 = n1;
  p->n2 = n2;
  p->M1 = M1;
  p->M2 = M2;
  p->p1 = ax[0].P;
  p->p2 = ax[1].P;
  p->q1 = ax[0].Q;
  p->q2 = ax[1].Q;
  p->r1 = ax[0].r;
  p->r2 = ax[1].r;
  p->xi1 = ax[0].xi;
  p->xi2 = ax[1].xi;
  p->eps = eps;
  p->kid = kid;

  double* d_a = nullptr;
  PFT_CUDA_TRY(cudaMalloc(&d_a, sizeof(double) * pftc::kMaxTerms));
  PFT_CUDA_TRY(cudaMalloc(&p->d_W, sizeof(float2) * RMAX * (M1 + M2)));
  PFT_CUDA_TRY(cudaMalloc(&p->d_twp, sizeof(float2) * 64));
  PFT_CUDA_TRY(cudaMalloc(&p->d_B, sizeof(float) * (ax[0].Q + ax[1].Q) * RMAX));
  PFT_CUDA_TRY(cudaMemset(p->d_twp, 0, sizeof(float2) * 64));
  std::memset(&p->cst, 0, sizeof(p->cst));
  float2* W = p->d_W;
  float* B = p->d_B;
  for (int k = 0; k < 2; ++k) {
    const AxisPlan& x = ax[k];
    PFT_CUDA_TRY(cudaMemcpy(d_a, x.a, sizeof(double) * pftc::kMaxTerms, cudaMemcpyHostToDevice));
    const int total = x.Q * RMAX + RMAX * x.M + x.P / 2;
    k_tables<<<(total + 127) / 128, 128>>>(x.Q, x.P, x.M, x.r, d_a, B, W, p->d_twp + 32 * k);
    PFT_CUDA_TRY(cudaGetLastError());
    // the kernels keep rows 0 .. q/2 of each axis's B as constants (q <= 32)
    std::vector<float> hB(x.Q * RMAX);
    PFT_CUDA_TRY(cudaMemcpy(hB.data(), B, sizeof(float) * x.Q * RMAX, cudaMemcpyDeviceToHost));
    if (x.Q / 2 < (int)(sizeof(p->cst.bh[0]) / sizeof(p->cst.bh[0][0])))
      for (int l = 0; l <= x.Q / 2; ++l)
        for (int j = 0; j < RMAX; ++j) p->cst.bh[k][l][j] = hB[l * RMAX + j];
    W += RMAX * x.M;
    B += x.Q * RMAX;
  }
  PFT_CUDA_TRY(cudaFree(d_a));
  return PFT_OK;
}

int build_plan(pft_plan* p, int n, int M, int P, double eps, int r_force) {
  return build_plan2(p, n, n, M, M, P, P, eps, r_force, r_force);
}

}  // namespace pfth

// ------------------------------------------------------------------ C ABI
namespace {

int launch_frames(const pft_plan* plan, const void* in, void* out, int64_t batch, void* stream, bool adjoint) {
  if (!plan || (!in && batch) || (!out && batch)) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (batch < 0) return pfth::set_error(PFT_ERR_INVALID_ARG, "batch < 0");
  if (batch == 0) return PFT_OK;
  const pfth::FrameKernels* fk = pfth::frame_kernels(plan->kid);
  const void* fn = adjoint ? fk->adj : fk->fwd;
  static bool attr_set[64][2] = {};
  if (!attr_set[plan->kid][adjoint]) {
    PFT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fk->smem));
    attr_set[plan->kid][adjoint] = true;
  }
  int per_sm = 0;
  PFT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, fk->smem));
  if (per_sm < 1) return pfth::set_error(PFT_ERR_UNSUPPORTED, "frame kernel does not fit on an SM");
  long long grid = (long long)per_sm * pfth::sm_count();
  if (grid > batch) grid = batch;
  const float2* a = (const float2*)in;
  float2* b = (float2*)out;
  long long nb = batch;
  PftConst cst = plan->cst;
  const float2* W = plan->d_W;
  const float2* tw = plan->d_twp;
  void* args[] = {(void*)&a, (void*)&b, (void*)&nb, (void*)&cst, (void*)&W, (void*)&tw};
  PFT_CUDA_TRY(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kThreads), args, fk->smem, (cudaStream_t)stream));
  return PFT_OK;
}

}  // namespace

extern "C" {

int pft_plan_create(pft_plan** out, int n1, int n2, int M1, int M2, int p1, int p2, double eps, int r1, int r2,
                    int path, int precision) {
  if (!out) return pfth::set_error(PFT_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  if (eps == 0.0) eps = 1e-7;
  if (!(eps > 0.0 && eps < 1.0)) return pfth::set_error(PFT_ERR_INVALID_ARG, "need 0 < eps < 1");
  if (path != PFT_PATH_AUTO && path != PFT_PATH_FACTORISED && path != PFT_PATH_DIRECT)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "unknown path %d", path);
  if (precision != PFT_PREC_FP32 && precision != PFT_PREC_SPLIT_BF16)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "unknown precision %d", precision);
  if (path == PFT_PATH_DIRECT) return pfth::set_error(PFT_ERR_UNSUPPORTED, "the direct path is not built");
  const bool square = n1 == n2 && M1 == M2 && p1 == p2 && r1 == r2;
  if (!square && precision != PFT_PREC_FP32)
    return pfth::set_error(PFT_ERR_UNSUPPORTED, "rectangular plans are built for PFT_PREC_FP32");
  pft_plan* p = new (std::nothrow) pft_plan();
  if (!p) return pfth::set_error(PFT_ERR_OOM, "host allocation failed");
  int rc = pfth::build_plan2(p, n1, n2, M1, M2, p1, p2, eps, r1, r2);
  if (rc != PFT_OK) {
    pft_plan_destroy(p);
    return rc;
  }
  p->path = PFT_PATH_FACTORISED;
  p->precision = precision;
  if (p->kid < 0) {  // large frames: split-BF16 stage A on tensor cores
    if (precision != PFT_PREC_SPLIT_BF16) {
      pft_plan_destroy(p);
      return pfth::set_error(PFT_ERR_UNSUPPORTED, "n=%d frames are built for PFT_PREC_SPLIT_BF16 only", n1);
    }
    p->lf = true;
    rc = pfth::lf_build(p);
    if (rc != PFT_OK) {
      pft_plan_destroy(p);
      return rc;
    }
    *out = p;
    return PFT_OK;
  }
  if (precision == PFT_PREC_SPLIT_BF16) {
    if (!pfth::tc_supported(p->n1, p->M1, p->p1)) {
      pft_plan_destroy(p);
      return pfth::set_error(PFT_ERR_UNSUPPORTED,
                             "split-BF16 is built for n=256 with M=32 (p=16) or M=64 (p=32), and for large frames "
                             "(got n=%d M=%d p=%d)", n1, M1, p1 ? p1 : M1 / 2);
    }
    rc = p->M1 == 64 ? pfth::tc64_build_tables(p) : pfth::tc_build_tables(p);
    if (rc == PFT_OK && p->M1 == 64) rc = pfth::tc64_build_adjoint_table(p);
    if (rc != PFT_OK) {
      pft_plan_destroy(p);
      return rc;
    }
  }
  *out = p;
  return PFT_OK;
}

int pft_plan_destroy(pft_plan* p) {
  if (!p) return PFT_OK;
  cudaFree(p->d_W);
  cudaFree(p->d_twp);
  cudaFree(p->d_B);
  cudaFree(p->d_tc);
  cudaFree(p->d_tc_adj);
  cudaFree(p->d_ws);
  if (p->h_status) cudaFreeHost(p->h_status);
  delete p;
  return PFT_OK;
}

int pft_plan_info_get(const pft_plan* p, pft_plan_info* info) {
  if (!p || !info) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  info->n1 = p->n1; info->n2 = p->n2; info->M1 = p->M1; info->M2 = p->M2;
  info->p1 = p->p1; info->p2 = p->p2; info->q1 = p->q1; info->q2 = p->q2;
  info->r1 = p->r1; info->r2 = p->r2; info->xi1 = p->xi1; info->xi2 = p->xi2;
  info->eps = p->eps; info->path = p->path; info->precision = p->precision;
  return PFT_OK;
}

int pft_plan_tables(const pft_plan* p, int axis, float* B, float* W) {
  if (!p || axis < 0 || axis > 1) return pfth::set_error(PFT_ERR_INVALID_ARG, "bad plan or axis");
  const int q = axis ? p->q2 : p->q1, M = axis ? p->M2 : p->M1, r = axis ? p->r2 : p->r1;
  if (B) {
    std::vector<float> hB(q * RMAX);
    PFT_CUDA_TRY(cudaMemcpy(hB.data(), p->d_B + axis * p->q1 * RMAX, sizeof(float) * q * RMAX,
                            cudaMemcpyDeviceToHost));
    for (int l = 0; l < q; ++l)
      for (int j = 0; j < r; ++j) B[l * r + j] = hB[l * RMAX + j];
  }
  if (W) {
    std::vector<float2> hW(RMAX * M);
    PFT_CUDA_TRY(cudaMemcpy(hW.data(), p->d_W + axis * RMAX * p->M1, sizeof(float2) * RMAX * M,
                            cudaMemcpyDeviceToHost));
    for (int t = 0; t < M; ++t)
      for (int j = 0; j < r; ++j) {
        W[2 * (t * r + j)] = hW[j * M + t].x;
        W[2 * (t * r + j) + 1] = hW[j * M + t].y;
      }
  }
  return PFT_OK;
}

int pft_forward(const pft_plan* plan, const void* x, void* y, int64_t batch, void* stream) {
  if (plan && plan->precision == PFT_PREC_SPLIT_BF16) {
    if ((!x || !y) && batch) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
    if (batch < 0) return pfth::set_error(PFT_ERR_INVALID_ARG, "batch < 0");
    if (batch == 0) return PFT_OK;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15)
      return pfth::set_error(PFT_ERR_INVALID_ARG, "x and y must be 16-byte aligned");
    if (plan->lf) return pfth::lf_forward(plan, x, y, batch, stream);
    if (plan->M1 == 64) return pfth::tc64_forward(plan, x, y, batch, stream);
    return pfth::tc_forward(plan, x, y, batch, stream);
  }
  return launch_frames(plan, x, y, batch, stream, false);
}

int pft_adjoint(const pft_plan* plan, const void* y, void* x, int64_t batch, void* stream) {
  if (plan && plan->precision == PFT_PREC_SPLIT_BF16) {
    if ((!x || !y) && batch) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
    if (batch < 0) return pfth::set_error(PFT_ERR_INVALID_ARG, "batch < 0");
    if (batch == 0) return PFT_OK;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15)
      return pfth::set_error(PFT_ERR_INVALID_ARG, "x and y must be 16-byte aligned");
    if (plan->lf) return pfth::lf_adjoint(plan, y, x, batch, stream);
    if (plan->M1 == 64) return pfth::tc64_adjoint(plan, y, x, batch, stream);
    return pfth::tc_adjoint(plan, y, x, batch, stream);
  }
  return launch_frames(plan, y, x, batch, stream, true);
}

}  // extern "C"
