// Full 2-D FFT of n x n frames and the FFT-then-crop baseline (the route the
// PFT replaces: Section 3.1, computing the FFT and then cropping costs
// O(n log n)).
#include <mutex>

#include "fft_core.cuh"

using namespace pftk;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__global__ void k_twiddles(int N, float2* out) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < N) {
    double s, c;
    sincospi(-2.0 * (double)m / (double)N, &s, &c);
    out[m] = make_float2((float)c, (float)s);
  }
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_fft2(const float2* in, float2* out, long long batch, int inverse,
                                                   const float2* __restrict__ gtw) {
  using F = Fft<N>;
  constexpr int L = F::L, E = F::E, G = F::G, S = F::S;
  extern __shared__ __align__(16) float2 sm[];
  float2* tw = sm;
  float2* sF = sm + F::TAB;
  F::fill(tw, gtw);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = lane % L, g = lane / L;
  typename F::Net net;
  F::init_net(net, l, tw);
  for (long long f = blockIdx.x; f < batch; f += gridDim.x) {
    const float2* src = in + f * (long long)(N * N);
    float2* dst = out + f * (long long)(N * N);
    if (!inverse) {
      for (int u0 = warp * G; u0 < N; u0 += kWarps * G) {
        const int u = u0 + g;
        float2 x[E];
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = src[u * N + l + L * e];
        F::fwd(x, l, tw, net);
#pragma unroll
        for (int p = 0; p < E; ++p) sF[u * S + p * L + l] = x[p];
      }
      __syncthreads();
      for (int b0 = warp * G; b0 < N; b0 += kWarps * G) {
        const int b = b0 + g;
        float2 x[E];
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = sF[(l + L * e) * S + b];
        F::fwd(x, l, tw, net);
#pragma unroll
        for (int p = 0; p < E; ++p) sF[(p * L + l) * S + b] = x[p];
      }
      __syncthreads();
      for (int i = threadIdx.x; i < N * N; i += kThreads)
        dst[i] = sF[F::slot_of_freq(i / N) * S + F::slot_of_freq(i % N)];
    } else {
      for (int i = threadIdx.x; i < N * N; i += kThreads)
        sF[F::slot_of_freq(i / N) * S + F::slot_of_freq(i % N)] = src[i];
      __syncthreads();
      for (int b0 = warp * G; b0 < N; b0 += kWarps * G) {
        const int b = b0 + g;
        float2 x[E];
#pragma unroll
        for (int p = 0; p < E; ++p) x[p] = sF[(p * L + l) * S + b];
        F::adj(x, l, tw, net);
#pragma unroll
        for (int e = 0; e < E; ++e) sF[(l + L * e) * S + b] = x[e];
      }
      __syncthreads();
      for (int u0 = warp * G; u0 < N; u0 += kWarps * G) {
        const int u = u0 + g;
        float2 x[E];
#pragma unroll
        for (int p = 0; p < E; ++p) x[p] = sF[u * S + p * L + l];
        F::adj(x, l, tw, net);
#pragma unroll
        for (int e = 0; e < E; ++e) dst[u * N + l + L * e] = x[e];
      }
    }
    __syncthreads();
  }
}

// Full FFT of every row, keep the M centred columns, FFT those columns, keep
// the M centred rows: out[f] is the centred M x M crop of FFT2(in[f]).
template <int N, int M>
__global__ void __launch_bounds__(kThreads) k_fft_crop(const float2* __restrict__ in, float2* __restrict__ out,
                                                       long long batch, const float2* __restrict__ gtw) {
  using F = Fft<N>;
  constexpr int L = F::L, E = F::E, G = F::G;
  constexpr int SM = M + 1;
  extern __shared__ __align__(16) float2 sm[];
  float2* tw = sm;
  float2* sR = sm + F::TAB;     // [N][M+1] rows after the row FFT, kept columns
  float2* sO = sR + N * SM;     // [M][M+1]
  F::fill(tw, gtw);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = lane % L, g = lane / L;
  typename F::Net net;
  F::init_net(net, l, tw);
  for (long long f = blockIdx.x; f < batch; f += gridDim.x) {
    const float2* src = in + f * (long long)(N * N);
    for (int u0 = warp * G; u0 < N; u0 += kWarps * G) {
      const int u = u0 + g;
      float2 x[E];
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = __ldg(src + u * N + l + L * e);
      F::fwd(x, l, tw, net);
#pragma unroll
      for (int p = 0; p < E; ++p) {
        const int ci = crop_index<N, M>(F::freq_of_slot(p * L + l));
        if (ci >= 0) sR[u * SM + ci] = x[p];
      }
    }
    __syncthreads();
    for (int c0 = warp * G; c0 < M; c0 += kWarps * G) {
      const int ci = c0 + g;
      float2 x[E];
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = sR[(l + L * e) * SM + ci];
      F::fwd(x, l, tw, net);
#pragma unroll
      for (int p = 0; p < E; ++p) {
        const int ri = crop_index<N, M>(F::freq_of_slot(p * L + l));
        if (ri >= 0) sO[ri * SM + ci] = x[p];
      }
    }
    __syncthreads();
    float2* dst = out + f * (long long)(M * M);
    for (int i = threadIdx.x; i < M * M; i += kThreads) dst[i] = sO[(i / M) * SM + (i % M)];
    __syncthreads();
  }
}

template <class K>
int launch_persistent(K fn, size_t smem, long long batch, void** args, cudaStream_t st) {
  PFT_CUDA_TRY(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PFT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem));
  if (per_sm < 1) return pfth::set_error(PFT_ERR_UNSUPPORTED, "FFT kernel does not fit on an SM");
  long long grid = (long long)per_sm * pfth::sm_count();
  if (grid > batch) grid = batch;
  PFT_CUDA_TRY(cudaLaunchKernel((const void*)fn, dim3((unsigned)grid), dim3(kThreads), args, smem, st));
  return PFT_OK;
}

template <int N>
int run_fft2(const void* in, void* out, long long batch, int inverse, cudaStream_t st) {
  const float2* tw = pfth::twiddles(N);
  if (!tw) return PFT_ERR_CUDA;
  size_t smem = sizeof(float2) * (Fft<N>::TAB + N * Fft<N>::S);
  void* args[] = {(void*)&in, (void*)&out, (void*)&batch, (void*)&inverse, (void*)&tw};
  return launch_persistent(k_fft2<N>, smem, batch, args, st);
}

template <int N, int M>
int run_fft_crop(const void* in, void* out, long long batch, cudaStream_t st) {
  const float2* tw = pfth::twiddles(N);
  if (!tw) return PFT_ERR_CUDA;
  size_t smem = sizeof(float2) * (Fft<N>::TAB + N * (M + 1) + M * (M + 1));
  void* args[] = {(void*)&in, (void*)&out, (void*)&batch, (void*)&tw};
  return launch_persistent(k_fft_crop<N, M>, smem, batch, args, st);
}

}  // namespace

namespace pfth {

const float2* twiddles(int N) {
  static std::mutex mu;
  static float2* tabs[10] = {};
  static int dev_of[10] = {};
  if (N < 2 || N > 512 || (N & (N - 1))) return nullptr;
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (tabs[lg] && dev_of[lg] == dev) return tabs[lg];
  float2* t = nullptr;
  if (cudaMalloc(&t, sizeof(float2) * N) != cudaSuccess) {
    set_error(PFT_ERR_OOM, "twiddle table allocation failed");
    return nullptr;
  }
  k_twiddles<<<(N + 127) / 128, 128>>>(N, t);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error(PFT_ERR_CUDA, "twiddle table generation failed");
    return nullptr;
  }
  tabs[lg] = t;
  dev_of[lg] = dev;
  return t;
}

}  // namespace pfth

extern "C" {

int pft_fft2(const void* in, void* out, int n, int64_t batch, int inverse, void* stream) {
  if (batch < 0 || (batch && (!in || !out))) return pfth::set_error(PFT_ERR_INVALID_ARG, "bad arguments");
  if (batch == 0) return PFT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  switch (n) {
    case 16: return run_fft2<16>(in, out, batch, inverse != 0, st);
    case 32: return run_fft2<32>(in, out, batch, inverse != 0, st);
    case 64: return run_fft2<64>(in, out, batch, inverse != 0, st);
    case 128: return run_fft2<128>(in, out, batch, inverse != 0, st);
    default: return pfth::set_error(PFT_ERR_UNSUPPORTED, "pft_fft2: n=%d not built (16..128)", n);
  }
}

int pft_fft_crop(const void* in, void* out, int n, int M, int64_t batch, void* stream) {
  if (batch < 0 || (batch && (!in || !out))) return pfth::set_error(PFT_ERR_INVALID_ARG, "bad arguments");
  if (batch == 0) return PFT_OK;
  cudaStream_t st = (cudaStream_t)stream;
#define PFT_CROP_CASE(NN, MM) \
  if (n == NN && M == MM) return run_fft_crop<NN, MM>(in, out, batch, st);
  PFT_CROP_CASE(256, 32)
  PFT_CROP_CASE(256, 64)
  PFT_CROP_CASE(128, 32)
  PFT_CROP_CASE(64, 32)
  PFT_CROP_CASE(32, 16)
#undef PFT_CROP_CASE
  return pfth::set_error(PFT_ERR_UNSUPPORTED, "pft_fft_crop: (n=%d, M=%d) not built", n, M);
}

}  // extern "C"
