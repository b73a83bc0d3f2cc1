// Allocation-free variant of the phase-aligned error reduction.
//
// Some callers cannot allocate device memory at the moment they need a result:
// code recorded into a CUDA graph (cudaMalloc and cudaFree are not allowed
// while a stream is being captured), latency-critical loops (both calls can
// synchronise the whole device), and plug-ins inside a host framework that owns
// every device allocation through its own pool. pie_nrmse_noalloc serves them:
// it takes only caller-owned inputs and keeps its intermediate sums in a
// fixed array compiled into this library, which every GPU that loads the
// library holds until the process exits.
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
constexpr int kSums = 4;                                          // Re<z,t>, Im<z,t>, |z|^2, |t|^2

// Per-block partial sums followed by the 4 final sums: 16388 doubles (128 KiB).
// Every slot that a call reads is written earlier in the same call, so nothing
// needs clearing; two calls that overlap on the GPU race on this array.
static __device__ __align__(256) double g_scratch[kSums * kMaxBlocks + kSums];

__global__ void __launch_bounds__(kThreads) k_partials(const float2* __restrict__ z, const float2* __restrict__ t,
                                                      const unsigned char* __restrict__ mask, long long count,
                                                      double* __restrict__ scratch) {
  __shared__ double s[kThreads / 32];
  double v[kSums] = {0.0, 0.0, 0.0, 0.0};
  const long long base = (long long)blockIdx.x * kPerBlock;
  for (int k = 0; k < kPerThread; ++k) {
    const long long i = base + (long long)k * kThreads + threadIdx.x;
    if (i >= count || (mask && !mask[i])) continue;
    const double zr = z[i].x, zi = z[i].y, tr = t[i].x, ti = t[i].y;
    v[0] += zr * tr + zi * ti;  // conj(z) t
    v[1] += zr * ti - zi * tr;
    v[2] += zr * zr + zi * zi;
    v[3] += tr * tr + ti * ti;
  }
  for (int q = 0; q < kSums; ++q) {
    const double tot = pftk::block_sum(v[q], s);
    if (threadIdx.x == 0) scratch[kSums * blockIdx.x + q] = tot;
  }
}

__global__ void __launch_bounds__(kThreads) k_final(int nblocks, double* __restrict__ scratch) {
  __shared__ double s[kThreads / 32];
  for (int q = 0; q < kSums; ++q) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) v += scratch[kSums * b + q];
    const double tot = pftk::block_sum(v, s);
    if (threadIdx.x == 0) scratch[kSums * kMaxBlocks + q] = tot;
  }
}

// Device address of g_scratch for each device, looked up once per device with
// that device current (in host code the symbol itself is only a stand-in).
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
  k_partials<<<nblocks, kThreads, 0, st>>>((const float2*)object, (const float2*)truth, mask, count, scratch);
  PFT_CUDA_TRY(cudaGetLastError());
  k_final<<<1, kThreads, 0, st>>>(nblocks, scratch);
  PFT_CUDA_TRY(cudaGetLastError());
  double sums[kSums];
  PFT_CUDA_TRY(cudaMemcpyAsync(sums, scratch + kSums * kMaxBlocks, sizeof(sums), cudaMemcpyDeviceToHost, st));
  PFT_CUDA_TRY(cudaStreamSynchronize(st));
  const double ip = std::hypot(sums[0], sums[1]);
  const double e2 = std::max(0.0, sums[2] + sums[3] - 2.0 * ip);
  *out = sums[3] > 0 ? std::sqrt(e2 / sums[3]) : 0.0;
  if (!std::isfinite(*out)) return pfth::set_error(PFT_ERR_NONFINITE, "non-finite error norm");
  return PFT_OK;
}
