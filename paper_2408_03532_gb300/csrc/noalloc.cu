// Allocation-free variant of the phase-aligned error reduction.
//
// Some callers cannot call cudaMalloc at the moment they need a result: a
// plug-in running inside a host framework that owns every device allocation
// through its own pool (an allocation behind the pool's back breaks its
// accounting, or is forbidden outright), and latency-critical loops, where
// cudaMalloc and cudaFree can synchronise the whole device. pie_nrmse_noalloc
// serves them: it takes only caller-owned inputs and keeps its intermediate
// sums in a fixed array compiled into this library, which every GPU that loads
// the library holds until the process exits.
//
// The error is found in two passes over the data, both on the device: the
// first sums <z, t> and |t|^2 and turns <z, t> into the aligning phase, the
// second sums |e^{i phi} z - t|^2 directly, so small errors are not lost to
// the cancellation of |z|^2 + |t|^2 - 2 |<z, t>|.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr long long kPerBlock = (long long)kThreads * kPerThread;  // elements per block
constexpr int kMaxBlocks = 4096;
constexpr long long kMaxCount = kPerBlock * kMaxBlocks;          // 16,777,216 elements

// Layout of the fixed array (doubles):
//   [0, 3 kMaxBlocks)                per-block Re<z,t>, Im<z,t>, |t|^2 (pass 1)
//   [3 kMaxBlocks, 4 kMaxBlocks)     per-block |e^{i phi} z - t|^2 (pass 2)
//   kFinal + 0 .. 5                  Re<z,t>, Im<z,t>, |t|^2, cos phi, sin phi, error^2
// 16,390 doubles (128 KiB + 48 B). Every slot that a call reads is written
// earlier in the same call, so nothing needs clearing between calls; two calls
// that overlap on the GPU race on this array.
constexpr int kPass2 = 3 * kMaxBlocks;
constexpr int kFinal = 4 * kMaxBlocks;
static __device__ __align__(256) double g_scratch[kFinal + 6];

__global__ void __launch_bounds__(kThreads) k_inner(const float2* __restrict__ z, const float2* __restrict__ t,
                                                   const unsigned char* __restrict__ mask, long long count,
                                                   double* __restrict__ scratch) {
  __shared__ double s[kThreads / 32];
  double v[3] = {0.0, 0.0, 0.0};
  const long long base = (long long)blockIdx.x * kPerBlock;
  for (int k = 0; k < kPerThread; ++k) {
    const long long i = base + (long long)k * kThreads + threadIdx.x;
    if (i >= count || (mask && !mask[i])) continue;
    const double zr = z[i].x, zi = z[i].y, tr = t[i].x, ti = t[i].y;
    v[0] += zr * tr + zi * ti;  // conj(z) t
    v[1] += zr * ti - zi * tr;
    v[2] += tr * tr + ti * ti;
  }
  for (int q = 0; q < 3; ++q) {
    const double tot = pftk::block_sum(v[q], s);
    if (threadIdx.x == 0) scratch[3 * blockIdx.x + q] = tot;
  }
}

// Sums pass 1's partials and stores the aligning phase e^{i phi} = <z,t>/|<z,t>|
// (1 when <z,t> = 0).
__global__ void __launch_bounds__(kThreads) k_phase(int nblocks, double* __restrict__ scratch) {
  __shared__ double s[kThreads / 32];
  double tot[3];
  for (int q = 0; q < 3; ++q) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) v += scratch[3 * b + q];
    tot[q] = pftk::block_sum(v, s);
  }
  if (threadIdx.x == 0) {
    const double a = hypot(tot[0], tot[1]);
    scratch[kFinal + 0] = tot[0];
    scratch[kFinal + 1] = tot[1];
    scratch[kFinal + 2] = tot[2];
    scratch[kFinal + 3] = a > 0.0 ? tot[0] / a : 1.0;
    scratch[kFinal + 4] = a > 0.0 ? tot[1] / a : 0.0;
  }
}

__global__ void __launch_bounds__(kThreads) k_residual(const float2* __restrict__ z, const float2* __restrict__ t,
                                                      const unsigned char* __restrict__ mask, long long count,
                                                      double* __restrict__ scratch) {
  __shared__ double s[kThreads / 32];
  const double c = scratch[kFinal + 3], sn = scratch[kFinal + 4];
  double v = 0.0;
  const long long base = (long long)blockIdx.x * kPerBlock;
  for (int k = 0; k < kPerThread; ++k) {
    const long long i = base + (long long)k * kThreads + threadIdx.x;
    if (i >= count || (mask && !mask[i])) continue;
    const double zr = z[i].x, zi = z[i].y;
    const double dr = c * zr - sn * zi - t[i].x;  // e^{i phi} z - t
    const double di = c * zi + sn * zr - t[i].y;
    v += dr * dr + di * di;
  }
  const double tot = pftk::block_sum(v, s);
  if (threadIdx.x == 0) scratch[kPass2 + blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) k_error(int nblocks, double* __restrict__ scratch) {
  __shared__ double s[kThreads / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) v += scratch[kPass2 + b];
  const double tot = pftk::block_sum(v, s);
  if (threadIdx.x == 0) scratch[kFinal + 5] = tot;
}

// Device address of g_scratch for each device, looked up once per device with
// that device current (in host code the symbol itself is only a stand-in, not
// a device address). The address belongs to the device's primary context as it
// was at the lookup; it is not looked up again after cudaDeviceReset.
std::mutex g_mu;
double* g_ptr[64] = {};

int scratch_for_current_device(double** out) {
  int dev = 0;
  PFT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return pfth::set_error(PFT_ERR_UNSUPPORTED, "device index %d beyond 63", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    PFT_CUDA_TRY(cudaGetSymbolAddress(&p, g_scratch));
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return PFT_OK;
}

}  // namespace

extern "C" int pie_nrmse_noalloc(const void* object, const void* truth, const uint8_t* mask, int64_t count,
                                 double* out, void* stream) {
  if (!object || !truth || !out) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (count <= 0) return pfth::set_error(PFT_ERR_INVALID_ARG, "count must be positive");
  if (count > kMaxCount)
    return pfth::set_error(PFT_ERR_INVALID_ARG,
                           "count %lld exceeds the allocation-free maximum of %lld elements (4096 x 4096)",
                           (long long)count, kMaxCount);
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != PFT_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int nblocks = (int)((count + kPerBlock - 1) / kPerBlock);
  const float2* z = (const float2*)object;
  const float2* t = (const float2*)truth;
  k_inner<<<nblocks, kThreads, 0, st>>>(z, t, mask, count, scratch);
  PFT_CUDA_TRY(cudaGetLastError());
  k_phase<<<1, kThreads, 0, st>>>(nblocks, scratch);
  PFT_CUDA_TRY(cudaGetLastError());
  k_residual<<<nblocks, kThreads, 0, st>>>(z, t, mask, count, scratch);
  PFT_CUDA_TRY(cudaGetLastError());
  k_error<<<1, kThreads, 0, st>>>(nblocks, scratch);
  PFT_CUDA_TRY(cudaGetLastError());
  double fin[6];
  PFT_CUDA_TRY(cudaMemcpyAsync(fin, scratch + kFinal, sizeof(fin), cudaMemcpyDeviceToHost, st));
  PFT_CUDA_TRY(cudaStreamSynchronize(st));
  *out = fin[2] > 0 ? std::sqrt(fin[5] / fin[2]) : 0.0;
  if (!std::isfinite(*out)) return pfth::set_error(PFT_ERR_NONFINITE, "non-finite error norm");
  return PFT_OK;
}
