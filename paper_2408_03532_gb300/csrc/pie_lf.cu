// PIE sweeps over large frames (the paper's regime n >> M, Section 4's
// 8192^2 windows): Eq. pie_update with the PFT of Algorithm 5 (reading R4 for
// its inverse), on frames too large for one thread-block cluster.
//
// A colour's positions have disjoint patches, so the colour is one batch of
// frames for the large-frame transforms of pft_lf.cu:
//   1. k_lf_exit     psi_b = w . Q_b z                          (n x n per position)
//   2. pft_forward   Psi_b = A psi_b                             (M x M, split-BF16 tensor cores)
//   3. k_lf_project  R_b = Psi_b - d_b^crop sgn(Psi_b), Phi += |R_b|^2  (in place)
//   4. pft_adjoint   dpsi_b = A^H R_b                            (n x n, into the exit-wave buffer)
//   5. k_lf_update   Q_b z -= beta conj(w) / (max|w|^2 n^2) dpsi_b
// Colours run in colour-major order, so a sweep is sequential PIE in that
// order, as in the fused kernels for small frames.
#include <algorithm>
#include <cmath>
#include <vector>

#include "plan.cuh"

namespace {

constexpr int kThreads = 256;

long long grid_for(long long n) {
  const long long per = (n + kThreads - 1) / kThreads;
  return std::max<long long>(1, std::min<long long>(per, 152LL * 16));
}

// d^crop[j][t1][t2] = sqrt(I[j][t1 mod n][t2 mod n]) (centred M x M, FFT-order
// input); a NaN or infinite count is flagged.
__global__ void k_lf_crop(const float* __restrict__ I, float* __restrict__ dc, int npos, int n, int M,
                          unsigned* __restrict__ nonfinite) {
  const long long tot = (long long)npos * M * M;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long j = i / ((long long)M * M);
    const int r = (int)(i % ((long long)M * M));
    const int t1 = r / M - M / 2, t2 = r % M - M / 2;
    const int f1 = (t1 % n + n) % n, f2 = (t2 % n + n) % n;
    const float v = I[j * (long long)n * n + (long long)f1 * n + f2];
    bad |= !isfinite(v);
    dc[i] = sqrtf(fmaxf(v, 0.f));
  }
  if (bad) atomicOr(nonfinite, 1u);
}

// psi[b][u][v] = w[u][v] z[r_b + u][c_b + v]: float4 = two pixels per access.
__global__ void k_lf_exit(const float2* __restrict__ z, long long obj_w, const float2* __restrict__ w,
                          const int2* __restrict__ pos, const int* __restrict__ list, int count, int n,
                          float2* __restrict__ psi) {
  const long long half = (long long)n * n / 2;
  const long long tot = (long long)count * half;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / half);
    const long long e = 2 * (i % half);
    const int u = (int)(e / n), v = (int)(e % n);
    const int2 rc = pos[list[b]];
    const float4 zz = __ldg(reinterpret_cast<const float4*>(z + (rc.x + u) * obj_w + rc.y + v));
    const float4 ww = __ldg(reinterpret_cast<const float4*>(w + e));
    reinterpret_cast<float4*>(psi)[(long long)b * half + e / 2] =
        make_float4(ww.x * zz.x - ww.y * zz.y, ww.x * zz.y + ww.y * zz.x,
                    ww.z * zz.z - ww.w * zz.w, ww.z * zz.w + ww.w * zz.z);
  }
}

// Modulus projection (Eq. 3) on the M x M coefficients of each frame, in place:
// R = Psi - d sgn(Psi), theta(0) = 0 (a zero coefficient becomes -d); the
// objective's sum of |R|^2 in FP64.
__global__ void k_lf_project(float2* __restrict__ Y, const float* __restrict__ dc, const int* __restrict__ list,
                             int count, int M, double* __restrict__ phi) {
  __shared__ double red[kThreads / 32];
  const long long mm = (long long)M * M, tot = (long long)count * mm;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / mm, r = i % mm;
    const float d = dc[(long long)list[b] * mm + r];
    const float2 p = Y[i];
    const float m2 = p.x * p.x + p.y * p.y;
    float2 R;
    if (m2 != 0.f) {  // != rather than >: a NaN coefficient stays NaN
      const float s = 1.f - d * rsqrtf(m2);
      R = make_float2(p.x * s, p.y * s);
    } else {
      R = make_float2(-d, 0.f);
    }
    Y[i] = R;
    acc += (double)R.x * R.x + (double)R.y * R.y;
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s += red[k];
    atomicAdd(phi, s);
  }
}

// z[r_b + u][c_b + v] -= coef conj(w[u][v]) dpsi[b][u][v]; the patches of a
// colour are disjoint, so plain read-modify-writes.
__global__ void k_lf_update(float2* __restrict__ z, long long obj_w, const float2* __restrict__ w,
                            const int2* __restrict__ pos, const int* __restrict__ list, int count, int n,
                            const float2* __restrict__ dpsi, float coef) {
  const long long half = (long long)n * n / 2;
  const long long tot = (long long)count * half;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / half);
    const long long e = 2 * (i % half);
    const int u = (int)(e / n), v = (int)(e % n);
    const int2 rc = pos[list[b]];
    float4* zp = reinterpret_cast<float4*>(z + (rc.x + u) * obj_w + rc.y + v);
    const float4 ww = __ldg(reinterpret_cast<const float4*>(w + e));
    const float4 d = __ldg(reinterpret_cast<const float4*>(dpsi) + (long long)b * half + e / 2);
    float4 o = *zp;
    // conj(w) dpsi
    const float ux = ww.x * d.x + ww.y * d.y, uy = ww.x * d.y - ww.y * d.x;
    const float vx = ww.z * d.z + ww.w * d.w, vy = ww.z * d.w - ww.w * d.z;
    o.x = fmaf(-coef, ux, o.x);
    o.y = fmaf(-coef, uy, o.y);
    o.z = fmaf(-coef, vx, o.z);
    o.w = fmaf(-coef, vy, o.w);
    *zp = o;
  }
}

// ||z - z_prev||^2 and ||z_prev||^2 (the stopping rule's relative change).
__global__ void k_lf_change(const float2* __restrict__ z, const float2* __restrict__ prev, long long n,
                            double* __restrict__ out) {
  __shared__ double red[2][kThreads / 32];
  double d2 = 0.0, p2 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 a = z[i], b = prev[i];
    const double dx = (double)a.x - b.x, dy = (double)a.y - b.y;
    d2 += dx * dx + dy * dy;
    p2 += (double)b.x * b.x + (double)b.y * b.y;
  }
  for (int o = 16; o; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    p2 += __shfl_xor_sync(0xffffffffu, p2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = d2;
    red[1][threadIdx.x >> 5] = p2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) {
      a += red[0][k];
      b += red[1][k];
    }
    atomicAdd(out, a);
    atomicAdd(out + 1, b);
  }
}

}  // namespace

struct pie_lf {
  int n = 0, M = 0, npos = 0, H = 0, W = 0, ncol = 0, max_colour = 0;
  pft_plan* plan = nullptr;
  float probe_max2 = 0.f;
  std::vector<int> col_off;  // colour k is sched[col_off[k] .. col_off[k + 1])
  float2* d_probe = nullptr;
  int2* d_pos = nullptr;
  int* d_sched = nullptr;
  float* d_ampc = nullptr;   // [N][M][M] centred cropped amplitudes
  float2* d_frames = nullptr;  // [max colour][n][n]: exit waves, then A^H R
  float2* d_Y = nullptr;       // [max colour][M][M]
  float2* d_prev = nullptr;    // object before the sweep (statistics)
  double* d_red = nullptr;     // [4]: Phi, ||dz||^2, ||z||^2, non-finite flag
  double* h_red = nullptr;
};

extern "C" {

int pie_lf_destroy(pie_lf* c) {
  if (!c) return PFT_OK;
  if (c->plan) pft_plan_destroy(c->plan);
  cudaFree(c->d_probe);
  cudaFree(c->d_pos);
  cudaFree(c->d_sched);
  cudaFree(c->d_ampc);
  cudaFree(c->d_frames);
  cudaFree(c->d_Y);
  cudaFree(c->d_prev);
  cudaFree(c->d_red);
  if (c->h_red) cudaFreeHost(c->h_red);
  delete c;
  return PFT_OK;
}

int pie_lf_create(pie_lf** out, const pie_problem* pb, const void* probe, const int32_t* positions,
                  const float* intensities, void* stream) {
  if (!out || !pb || !probe || !positions || !intensities)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const int n = pb->n, N = pb->npos, H = pb->obj_h, W = pb->obj_w, M = pb->M;
  if (n <= 0 || N <= 0 || H < n || W < n) return pfth::set_error(PFT_ERR_INVALID_ARG, "bad problem sizes");
  if (M <= 0 || M % 2 || M > n) return pfth::set_error(PFT_ERR_INVALID_ARG, "need even 0 < M <= n");
  if (W % 2) return pfth::set_error(PFT_ERR_INVALID_ARG, "the object width must be even");
  if (pb->mode != PIE_MODE_COLOURED)
    return pfth::set_error(PFT_ERR_UNSUPPORTED, "large-frame PIE sweeps are coloured (sequential PIE)");
  cudaStream_t st = (cudaStream_t)stream;
  pie_lf* c = new (std::nothrow) pie_lf();
  if (!c) return pfth::set_error(PFT_ERR_OOM, "host allocation failed");
  c->n = n;
  c->M = M;
  c->npos = N;
  c->H = H;
  c->W = W;
  int rc = PFT_OK;
#define LF_CUDA(x)                                                    \
  do {                                                                \
    cudaError_t e_ = (x);                                             \
    if (e_ != cudaSuccess) {                                          \
      rc = pfth::cuda_error(e_, #x);                                  \
      pie_lf_destroy(c);                                              \
      return rc;                                                      \
    }                                                                 \
  } while (0)
  // the transform: the large-frame split-BF16 PFT (refuses shapes it does not build)
  rc = pft_plan_create(&c->plan, n, n, M, M, pb->p, pb->p, pb->eps > 0 ? pb->eps : 1e-7, 0, 0, PFT_PATH_AUTO,
                       PFT_PREC_SPLIT_BF16);
  if (rc != PFT_OK || !pfth::lf_supported(n, M, c->plan->p1)) {
    pie_lf_destroy(c);
    return rc != PFT_OK ? rc
                        : pfth::set_error(PFT_ERR_UNSUPPORTED, "large-frame PIE is built for n >= 2048, M = 128");
  }
  // positions (v even, so that every float4 access stays inside one row) and the colour-major schedule
  std::vector<int32_t> colour(N), sched(N);
  for (int j = 0; j < N; ++j)
    if (positions[2 * j + 1] % 2) {
      pie_lf_destroy(c);
      return pfth::set_error(PFT_ERR_INVALID_ARG, "position %d: the column must be even", j);
    }
  int ncol = 0;
  int64_t ndep = 0;
  rc = pie_scan_schedule(positions, N, n, H, W, nullptr, 0, &ncol, colour.data(), sched.data(), nullptr, nullptr, 0,
                         &ndep);
  if (rc != PFT_OK) {
    pie_lf_destroy(c);
    return rc;
  }
  c->ncol = ncol;
  c->col_off.assign(ncol + 1, 0);
  for (int j = 0; j < N; ++j) c->col_off[colour[j] + 1]++;
  for (int k = 0; k < ncol; ++k) c->col_off[k + 1] += c->col_off[k];
  for (int k = 0; k < ncol; ++k) c->max_colour = std::max(c->max_colour, c->col_off[k + 1] - c->col_off[k]);
  std::vector<int2> pos(N);
  for (int j = 0; j < N; ++j) pos[j] = make_int2(positions[2 * j], positions[2 * j + 1]);
  const size_t n2 = (size_t)n * n, m2 = (size_t)M * M;
  LF_CUDA(cudaMalloc(&c->d_pos, sizeof(int2) * N));
  LF_CUDA(cudaMalloc(&c->d_sched, sizeof(int) * N));
  LF_CUDA(cudaMalloc(&c->d_probe, sizeof(float2) * n2));
  LF_CUDA(cudaMalloc(&c->d_ampc, sizeof(float) * N * m2));
  LF_CUDA(cudaMalloc(&c->d_frames, sizeof(float2) * c->max_colour * n2));
  LF_CUDA(cudaMalloc(&c->d_Y, sizeof(float2) * c->max_colour * m2));
  LF_CUDA(cudaMalloc(&c->d_red, sizeof(double) * 4));
  LF_CUDA(cudaMallocHost(&c->h_red, sizeof(double) * 4));
  LF_CUDA(cudaMemcpyAsync(c->d_pos, pos.data(), sizeof(int2) * N, cudaMemcpyHostToDevice, st));
  LF_CUDA(cudaMemcpyAsync(c->d_sched, sched.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  LF_CUDA(cudaMemcpyAsync(c->d_probe, probe, sizeof(float2) * n2, cudaMemcpyDeviceToDevice, st));
  LF_CUDA(cudaMemsetAsync(c->d_red, 0, sizeof(double) * 4, st));
  k_lf_crop<<<grid_for((long long)N * m2), kThreads, 0, st>>>(intensities, c->d_ampc, N, n, M,
                                                             reinterpret_cast<unsigned*>(c->d_red + 3));
  LF_CUDA(cudaGetLastError());
  std::vector<float2> hp(n2);
  LF_CUDA(cudaMemcpyAsync(hp.data(), probe, sizeof(float2) * n2, cudaMemcpyDeviceToHost, st));
  LF_CUDA(cudaMemcpyAsync(c->h_red, c->d_red, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
  LF_CUDA(cudaStreamSynchronize(st));
  if (*reinterpret_cast<const unsigned*>(c->h_red + 3) != 0u) {
    pie_lf_destroy(c);
    return pfth::set_error(PFT_ERR_NONFINITE, "the intensities hold a NaN or infinite value");
  }
  for (const float2& v : hp) c->probe_max2 = std::max(c->probe_max2, v.x * v.x + v.y * v.y);
  if (!(c->probe_max2 > 0.f) || !std::isfinite(c->probe_max2)) {
    pie_lf_destroy(c);
    return pfth::set_error(PFT_ERR_NONFINITE, "probe is zero or not finite");
  }
#undef LF_CUDA
  *out = c;
  return PFT_OK;
}

int pie_lf_colours(const pie_lf* c, int* ncolours, int* max_colour) {
  if (!c || !ncolours) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  *ncolours = c->ncol;
  if (max_colour) *max_colour = c->max_colour;
  return PFT_OK;
}

int pie_lf_iteration(pie_lf* c, void* object, double beta, pie_stats* stats, void* stream) {
  if (!c || !object) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (reinterpret_cast<uintptr_t>(object) & 15) return pfth::set_error(PFT_ERR_INVALID_ARG, "object must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  const long long HW = (long long)c->H * c->W;
  float2* z = (float2*)object;
  if (stats) {
    if (!c->d_prev) PFT_CUDA_TRY(cudaMalloc(&c->d_prev, sizeof(float2) * HW));
    PFT_CUDA_TRY(cudaMemcpyAsync(c->d_prev, z, sizeof(float2) * HW, cudaMemcpyDeviceToDevice, st));
  }
  PFT_CUDA_TRY(cudaMemsetAsync(c->d_red, 0, sizeof(double) * 3, st));
  const long long n2 = (long long)c->n * c->n;
  const float coef = (float)(beta / ((double)c->probe_max2 * (double)n2));
  for (int k = 0; k < c->ncol; ++k) {
    const int* list = c->d_sched + c->col_off[k];
    const int cnt = c->col_off[k + 1] - c->col_off[k];
    k_lf_exit<<<grid_for(cnt * n2 / 2), kThreads, 0, st>>>(z, c->W, c->d_probe, c->d_pos, list, cnt, c->n,
                                                            c->d_frames);
    PFT_CUDA_TRY(cudaGetLastError());
    int rc = pft_forward(c->plan, c->d_frames, c->d_Y, cnt, stream);
    if (rc != PFT_OK) return rc;
    k_lf_project<<<grid_for((long long)cnt * c->M * c->M), kThreads, 0, st>>>(c->d_Y, c->d_ampc, list, cnt, c->M,
                                                                               c->d_red);
    PFT_CUDA_TRY(cudaGetLastError());
    rc = pft_adjoint(c->plan, c->d_Y, c->d_frames, cnt, stream);
    if (rc != PFT_OK) return rc;
    k_lf_update<<<grid_for(cnt * n2 / 2), kThreads, 0, st>>>(z, c->W, c->d_probe, c->d_pos, list, cnt, c->n,
                                                              c->d_frames, coef);
    PFT_CUDA_TRY(cudaGetLastError());
  }
  if (stats) {
    k_lf_change<<<grid_for(HW), kThreads, 0, st>>>(z, c->d_prev, HW, c->d_red + 1);
    PFT_CUDA_TRY(cudaGetLastError());
    PFT_CUDA_TRY(cudaMemcpyAsync(c->h_red, c->d_red, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    PFT_CUDA_TRY(cudaStreamSynchronize(st));
    stats->phi = c->h_red[0] / ((double)c->npos * (double)n2);
    stats->rel_change = c->h_red[2] > 0 ? std::sqrt(c->h_red[1] / c->h_red[2]) : 0.0;
    if (!std::isfinite(c->h_red[0]) || !std::isfinite(c->h_red[1]) || !std::isfinite(c->h_red[2]))
      return pfth::set_error(PFT_ERR_NONFINITE, "non-finite objective or object change");
  }
  return PFT_OK;
}

}  // extern "C"
