// PIE on the GPU: one fused kernel per scan position computes
//   psi = w . Q_j z                         (exit wave, Eq. 1)
//   Psi = A psi                             (PFT of Algorithm 5, or the full FFT)
//   R = Psi - d_j . sgn(Psi)                (modulus projection residual, Eq. 3)
//   dpsi = A^H R / n^2                      (= psi - P_M(psi) for A = F)
//   z_j <- z_j - beta conj(w) / max|w|^2 . dpsi   (Eq. pie_update)
// and accumulates ||R||^2 for the objective of Eq. 4. Positions are grouped in
// colours whose patches do not overlap; the colours run one after another, so a
// sweep is exactly sequential PIE in colour-major order. The batched mode lets
// all positions read the same object and sums their updates instead.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "pie_kernels.cuh"
#include "plan.cuh"

using namespace pftk;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// ------------------------------------------------------------ helper kernels
__global__ void k_amplitudes(const float* __restrict__ I, float* __restrict__ d, float* __restrict__ dc,
                             int npos, int n, int M, unsigned* __restrict__ nonfinite) {
  const long long tot = (long long)npos * n * n;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const float v = I[i];
    bad |= !isfinite(v);  // fmaxf below would turn a NaN count into 0
    d[i] = sqrtf(fmaxf(v, 0.f));
  }
  if (bad) atomicOr(nonfinite, 1u);
  const long long totc = (long long)npos * M * M;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < totc; i += (long long)gridDim.x * blockDim.x) {
    const long long j = i / (M * M);
    const int r = (int)(i % (M * M));
    const int t1 = r / M - M / 2, t2 = r % M - M / 2;
    const int f1 = (t1 % n + n) % n, f2 = (t2 % n + n) % n;
    dc[i] = sqrtf(fmaxf(I[j * n * n + f1 * n + f2], 0.f));
  }
}

__global__ void k_illumination(const float2* __restrict__ probe, const int2* __restrict__ pos, int npos, int n,
                               long long W, float* __restrict__ illum) {
  const long long tot = (long long)npos * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / (n * n)), r = (int)(i % (n * n));
    const int u = r / n, v = r % n;
    const int2 rc = pos[j];
    atomicAdd(illum + (long long)(rc.x + u) * W + rc.y + v, cabs2(probe[r]));
  }
}

__global__ void k_max(const float* __restrict__ x, long long n, unsigned int* out) {
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, x[i]);
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(PFT_FULL_MASK, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // m >= 0
}

__global__ void k_finish_illum(float* __restrict__ illum, long long n, const unsigned int* __restrict__ mx,
                               float delta_rel, unsigned char* __restrict__ mask) {
  const float m = __uint_as_float(*mx);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = illum[i];
    mask[i] = (m > 0.f && v >= 1e-3f * m) ? 1 : 0;
    illum[i] = 1.f / (v + delta_rel * m);  // becomes the inverse illumination
  }
}

// red[0] += sum |a - b|^2, red[1] += sum |b|^2   (FP64)
__global__ void k_diff_norms(const float2* __restrict__ a, const float2* __restrict__ b, long long n, double* red) {
  __shared__ double s[kWarps];
  double d2 = 0.0, b2 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 x = a[i], y = b[i];
    const double dx = (double)x.x - y.x, dy = (double)x.y - y.y;
    d2 += dx * dx + dy * dy;
    b2 += (double)y.x * y.x + (double)y.y * y.y;
  }
  double t = block_sum(d2, s);
  if (threadIdx.x == 0) atomicAdd(red, t);
  t = block_sum(b2, s);
  if (threadIdx.x == 0) atomicAdd(red + 1, t);
}

// masked sums for the phase-aligned error: red += [Re <z,t>, Im <z,t>, |z|^2, |t|^2]
__global__ void k_align_sums(const float2* __restrict__ z, const float2* __restrict__ t,
                             const unsigned char* __restrict__ mask, long long n, double* red) {
  __shared__ double s[kWarps];
  double v[4] = {0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (!mask[i]) continue;
    const double zr = z[i].x, zi = z[i].y, tr = t[i].x, ti = t[i].y;
    v[0] += zr * tr + zi * ti;  // conj(z) t
    v[1] += zr * ti - zi * tr;
    v[2] += zr * zr + zi * zi;
    v[3] += tr * tr + ti * ti;
  }
  for (int q = 0; q < 4; ++q) {
    double tt = block_sum(v[q], s);
    if (threadIdx.x == 0) atomicAdd(red + q, tt);
  }
}

// z <- z - beta * acc * inv_illum  (batched update)
__global__ void k_apply_batched(float2* __restrict__ z, const float2* __restrict__ acc,
                                const float* __restrict__ inv_illum, float beta, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float s = beta * inv_illum[i];
    float2 o = z[i];
    const float2 u = acc[i];
    o.x = fmaf(-s, u.x, o.x);
    o.y = fmaf(-s, u.y, o.y);
    z[i] = o;
  }
}

// One gradient step of the smoothed isotropic total variation,
//   out = z - lambda (D_x^H(D_x z / s) + D_y^H(D_y z / s)),
//   s = sqrt(|D_x z|^2 + |D_y z|^2 + eps^2),
// forward differences with zero flux across the last row and column.
__device__ __forceinline__ void tv_terms(const float2* __restrict__ z, int H, int W, int i, int j, float eps2,
                                         float2& u, float2& v) {
  const float2 c = z[(long long)i * W + j];
  const float2 a = j + 1 < W ? csub(z[(long long)i * W + j + 1], c) : make_float2(0.f, 0.f);
  const float2 b = i + 1 < H ? csub(z[(long long)(i + 1) * W + j], c) : make_float2(0.f, 0.f);
  const float inv = rsqrtf(cabs2(a) + cabs2(b) + eps2);
  u = cscale(a, inv);
  v = cscale(b, inv);
}

__global__ void k_tv_step(const float2* __restrict__ z, float2* __restrict__ out, int H, int W, float lam,
                          float eps) {
  const long long n = (long long)H * W;
  const float eps2 = eps * eps;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p / W), j = (int)(p % W);
    float2 u, v, ul, vu, tmp;
    tv_terms(z, H, W, i, j, eps2, u, v);
    float2 g = make_float2(0.f, 0.f);
    if (j + 1 < W) g = csub(g, u);          // -u[i, j]
    if (i + 1 < H) g = csub(g, v);          // -v[i, j]
    if (j > 0) {                            // +u[i, j-1]
      tv_terms(z, H, W, i, j - 1, eps2, ul, tmp);
      g = cadd(g, ul);
    }
    if (i > 0) {                            // +v[i-1, j]
      tv_terms(z, H, W, i - 1, j, eps2, tmp, vu);
      g = cadd(g, vu);
    }
    const float2 c = z[p];
    out[p] = make_float2(fmaf(-lam, g.x, c.x), fmaf(-lam, g.y, c.y));
  }
}

// Blind PIE: max |w|^2 of the probe, and empty accumulators (single block).
__global__ void k_probe_init(const float2* __restrict__ w, int n2, float2* __restrict__ acc,
                             float* __restrict__ den, float* __restrict__ scale) {
  __shared__ float red[32];
  float m = 0.f;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    m = fmaxf(m, cabs2(w[i]));
    acc[i] = make_float2(0.f, 0.f);
    den[i] = 0.f;
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(PFT_FULL_MASK, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmaxf(t, red[i]);
    *scale = t;
  }
}

// Blind PIE, end of a colour: w <- w - gamma acc / (den + delta_rel max den)
// (normalised step) or w <- w - gamma acc (scalar step of Eq. epie_probe_update),
// then the new max |w|^2 and empty accumulators (single block).
__global__ void k_probe_apply(float2* __restrict__ w, int n2, float2* __restrict__ acc, float* __restrict__ den,
                              float gamma, float delta_rel, int normalise, float* __restrict__ scale) {
  __shared__ float red[32];
  __shared__ float dmax;
  float m = 0.f;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) m = fmaxf(m, den[i]);
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(PFT_FULL_MASK, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmaxf(t, red[i]);
    dmax = t;
  }
  __syncthreads();
  const float delta = delta_rel * dmax;
  float pm = 0.f;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    const float s = normalise ? gamma / (den[i] + delta) : gamma;
    float2 v = w[i];
    v.x = fmaf(-s, acc[i].x, v.x);
    v.y = fmaf(-s, acc[i].y, v.y);
    w[i] = v;
    pm = fmaxf(pm, cabs2(v));
    acc[i] = make_float2(0.f, 0.f);
    den[i] = 0.f;
  }
  for (int o = 16; o; o >>= 1) pm = fmaxf(pm, __shfl_xor_sync(PFT_FULL_MASK, pm, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pm;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmaxf(t, red[i]);
    *scale = t;
  }
}

int grid_for(long long work) {
  long long g = (work + kThreads - 1) / kThreads;
  long long cap = 8LL * pfth::sm_count();
  return (int)std::max(1LL, std::min(g, cap));
}

}  // namespace

struct pie_ctx {
  pie_problem pb;
  int n = 0, npos = 0, H = 0, W = 0, M = 0;
  pft_plan plan;
  bool have_plan = false;
  bool have_full = false;
  // kernels per [transform][mode][log2 cluster size] with their resident-CTA capacity
  PieKernel kern[2][3][4];
  long long cap[2][3][4] = {};
  // per transform: the item-claiming coloured kernel with the most CTAs per
  // position that is built (batch dataflow sweeps), and its capacity
  PieKernel kern_claim[2];
  long long cap_claim[2] = {0, 0};
  int tuned[2][3] = {{-1, -1, -1}, {-1, -1, -1}};  // autotuned log2 cluster size, -1 = heuristic
  double tuned_ms[2] = {0.0, 0.0};                  // sweep time of the chosen variant
  float2* d_probe = nullptr;
  float probe_max2 = 0.f;
  int2* d_pos = nullptr;
  std::vector<int2> h_pos;
  float* d_amp = nullptr;      // [N][n][n]
  float* d_ampc = nullptr;     // [N][M][M]
  std::vector<int> colour, col_off, visit;
  int ncol = 0;
  int* d_sched = nullptr;
  int* d_coloff = nullptr;     // colour offsets into d_sched [ncol + 1] (persistent sweeps)
  int max_colour = 0;          // positions in the largest colour
  unsigned* d_gbar = nullptr;  // [2]: grid-barrier arrivals, error word
  int test_wait = PIE_TEST_WAIT_NONE;  // pie_ctx_test_unreachable_wait
  int* h_gstatus = nullptr;    // mapped host status word of the persistent sweeps
  int* d_gstatus = nullptr;
  // launch form of the coloured sweeps per transform (autotuned): PIE_LAUNCH_PER_COLOUR,
  // PIE_LAUNCH_PERSISTENT (one cooperative launch, grid barrier between colours) or
  // PIE_LAUNCH_DATAFLOW (one cooperative launch, per-item waits on overlapping predecessors)
  int persist[2] = {PIE_LAUNCH_PER_COLOUR, PIE_LAUNCH_PER_COLOUR};
  int flow_ci[2] = {-1, -1};   // log2 cluster size of the dataflow form (-1: as the persistent form)
  int* d_dep_off = nullptr;    // dataflow predecessors per schedule item: CSR offsets [N + 1]
  int* d_dep = nullptr;        // and schedule indices
  unsigned* d_done = nullptr;  // [N] CTAs finished per schedule item (zeroed by every sweep)
  int* d_flow_off = nullptr;   // {0, N}: the whole schedule as one "colour"
  std::vector<int> h_dep_off, h_dep;  // host copies (batches remap them to their work lists)
  std::vector<int> h_sched;            // colour-major schedule (host copy)
  float* d_inv_illum = nullptr;
  unsigned char* d_mask = nullptr;
  float2* d_prev = nullptr;
  float2* d_acc = nullptr;
  float2* d_tv = nullptr;      // TV step scratch (allocated on first use)
  float2* d_pacc = nullptr;    // blind PIE probe-step accumulators (allocated on first use)
  float* d_pden = nullptr;
  float* d_pscale = nullptr;
  float2* d_start = nullptr;   // object at the start of a regularised sweep
  double* d_red = nullptr;     // [8]
  double* h_red = nullptr;     // pinned [8]
  // captured sweeps, replayed on the caller's stream
  struct Graph {
    const void* obj;
    int transform;
    double beta;
    double gamma;  // < 0: non-blind
    bool stats;
    int mode;      // PIE_MODE_* of the sweep
    int probe_step;  // PIE_PROBE_STEP_* of a blind sweep
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  cudaStream_t cap_stream = nullptr;
};

namespace {

// Sets the shared-memory limit of a kernel and returns how many of its CTAs
// can be resident at once (clusters x cluster size for clustered kernels).
int prepare_kernel(const PieKernel& k, long long* cap) {
  PFT_CUDA_TRY(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
  if (k.cluster == 1) {
    int per_sm = 0;
    PFT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, k.threads, k.smem));
    *cap = (long long)per_sm * pfth::sm_count();
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(k.cluster * 64);
    cfg.blockDim = dim3(k.threads);
    cfg.dynamicSmemBytes = k.smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = k.cluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    PFT_CUDA_TRY(cudaOccupancyMaxActiveClusters(&nclusters, k.fn, &cfg));
    *cap = (long long)nclusters * k.cluster;
  }
  if (*cap < 1) return pfth::set_error(PFT_ERR_UNSUPPORTED, "PIE kernel does not fit on an SM");
  return PFT_OK;
}

// The order of a coloured sweep, built on the host from the scan alone:
//  - greedy colouring in visiting order (each position takes the smallest colour
//    unused by an earlier visited position whose patch overlaps its own);
//  - the colour-major schedule, visiting order within a colour;
//  - the dataflow predecessors of schedule item s: E(s) = the earlier schedule
//    items whose patches overlap item s (all of an earlier colour), minus every
//    b of E(s) that is also in E(a) for some a of E(s) (a itself waited for b
//    before it ran, so waiting for a covers b, by induction along the schedule).
// Patches are n x n with top-left corners pos[j] = (row, col) inside H x W;
// `order` is a permutation of 0..N-1 (empty: index order).
struct PieSchedule {
  std::vector<int> visit, colour, col_off, sched, dep_off, dep;
  int ncol = 0;
};

void build_schedule(const std::vector<int2>& pos, int n, int H, int W, const std::vector<int>& order,
                    PieSchedule& out, bool one_per_colour = false) {
  const int N = (int)pos.size();
  // positions bucketed by n x n cells: overlapping patches lie in neighbouring cells
  const int cw = (W + n - 1) / n + 1, ch = (H + n - 1) / n + 1;
  auto overlap = [&](int2 p, int2 q) { return std::abs(q.x - p.x) < n && std::abs(q.y - p.y) < n; };
  auto for_neighbours = [&](const std::vector<std::vector<int>>& cells, int2 p, auto&& f) {
    const int cx = p.y / n, cy = p.x / n;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int yy = cy + dy, xx = cx + dx;
        if (yy < 0 || xx < 0 || yy >= ch || xx >= cw) continue;
        for (int i : cells[(size_t)yy * cw + xx]) f(i);
      }
  };
  out.colour.assign(N, -1);
  out.visit.resize(N);
  for (int a = 0; a < N; ++a) out.visit[a] = order.empty() ? a : order[a];
  std::vector<std::vector<int>> cells((size_t)cw * ch);
  std::vector<char> used;
  int ncol = 0;
  for (int a = 0; a < N; ++a) {
    const int j = out.visit[a];
    const int2 p = pos[j];
    used.assign(ncol + 1, 0);
    for_neighbours(cells, p, [&](int i) {
      if (overlap(p, pos[i])) used[out.colour[i]] = 1;
    });
    int col = 0;
    while (col < ncol && used[col]) ++col;
    if (one_per_colour) col = ncol;  // exact sequential order: the a-th visited position is colour a
    out.colour[j] = col;
    if (col == ncol) ++ncol;
    cells[(size_t)(p.x / n) * cw + p.y / n].push_back(j);
  }
  out.ncol = ncol;
  out.col_off.assign(ncol + 1, 0);
  for (int j = 0; j < N; ++j) out.col_off[out.colour[j] + 1]++;
  for (int k = 0; k < ncol; ++k) out.col_off[k + 1] += out.col_off[k];
  out.sched.assign(N, 0);
  std::vector<int> fill(out.col_off.begin(), out.col_off.end() - 1);
  for (int j : out.visit) out.sched[fill[out.colour[j]]++] = j;
  // predecessors in schedule indices
  for (auto& cell : cells) cell.clear();
  std::vector<std::vector<int>> E(N);
  for (int s = 0; s < N; ++s) {
    const int2 p = pos[out.sched[s]];
    for_neighbours(cells, p, [&](int i) {
      if (overlap(p, pos[out.sched[i]])) E[s].push_back(i);
    });
    cells[(size_t)(p.x / n) * cw + p.y / n].push_back(s);
  }
  out.dep_off.assign(N + 1, 0);
  out.dep.clear();
  std::vector<char> mark(N, 0);  // 1: in E(s), 2: covered by another member of E(s)
  for (int s = 0; s < N; ++s) {
    for (int b : E[s]) mark[b] = 1;
    for (int a : E[s])
      for (int b : E[a])
        if (mark[b]) mark[b] = 2;
    for (int b : E[s]) {
      if (mark[b] == 1) out.dep.push_back(b);
      mark[b] = 0;
    }
    out.dep_off[s + 1] = (int)out.dep.size();
  }
}

// The context's colouring and schedule for a visiting order (empty: index order).
void colour_positions(pie_ctx* c, const std::vector<int>& order = {}, bool one_per_colour = false) {
  PieSchedule sch;
  build_schedule(c->h_pos, c->n, c->H, c->W, order, sch, one_per_colour);
  c->visit = std::move(sch.visit);
  c->colour = std::move(sch.colour);
  c->col_off = std::move(sch.col_off);
  c->ncol = sch.ncol;
  c->h_sched = std::move(sch.sched);
  c->h_dep_off = std::move(sch.dep_off);
  c->h_dep = std::move(sch.dep);
}

// The colour-major schedule, colour offsets and dataflow predecessor lists to
// the device.
int upload_schedule(pie_ctx* c, cudaStream_t st) {
  const int N = c->npos;
  PFT_CUDA_TRY(cudaMemcpyAsync(c->d_sched, c->h_sched.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  cudaFree(c->d_coloff);
  c->d_coloff = nullptr;
  PFT_CUDA_TRY(cudaMalloc(&c->d_coloff, sizeof(int) * c->col_off.size()));
  PFT_CUDA_TRY(cudaMemcpyAsync(c->d_coloff, c->col_off.data(), sizeof(int) * c->col_off.size(),
                               cudaMemcpyHostToDevice, st));
  c->max_colour = 0;
  for (int k = 0; k < c->ncol; ++k) c->max_colour = std::max(c->max_colour, c->col_off[k + 1] - c->col_off[k]);
  const std::vector<int>& off = c->h_dep_off;
  const std::vector<int>& dep = c->h_dep;
  cudaFree(c->d_dep_off);
  cudaFree(c->d_dep);
  cudaFree(c->d_done);
  cudaFree(c->d_flow_off);
  c->d_dep_off = c->d_dep = c->d_flow_off = nullptr;
  c->d_done = nullptr;
  const int flow_off[2] = {0, N};
  PFT_CUDA_TRY(cudaMalloc(&c->d_dep_off, sizeof(int) * (N + 1)));
  PFT_CUDA_TRY(cudaMalloc(&c->d_dep, sizeof(int) * std::max<size_t>(1, dep.size())));
  PFT_CUDA_TRY(cudaMalloc(&c->d_done, sizeof(unsigned) * N));
  PFT_CUDA_TRY(cudaMalloc(&c->d_flow_off, sizeof(flow_off)));
  PFT_CUDA_TRY(cudaMemcpyAsync(c->d_dep_off, off.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, st));
  if (!dep.empty())
    PFT_CUDA_TRY(cudaMemcpyAsync(c->d_dep, dep.data(), sizeof(int) * dep.size(), cudaMemcpyHostToDevice, st));
  PFT_CUDA_TRY(cudaMemcpyAsync(c->d_flow_off, flow_off, sizeof(flow_off), cudaMemcpyHostToDevice, st));
  PFT_CUDA_TRY(cudaStreamSynchronize(st));
  return PFT_OK;
}

// Launches the fused kernel for `a.count` positions. Coloured sweeps pick the
// largest cluster size whose CTAs for all positions of the colour fit on the
// GPU at once; the other modes run one CTA per position.
int launch_pie(pie_ctx* c, int transform, int mode, PieArgs a, cudaStream_t st) {
  if (a.count <= 0) return PFT_OK;
  const int t = transform == PIE_TRANSFORM_PFT ? 0 : 1;
  int ci = 0;
  if (c->tuned[t][mode] >= 0) {
    ci = c->tuned[t][mode];
  } else if (mode == MODE_COLOURED) {
    for (int q = 3; q >= 1; --q)
      if (c->kern[t][mode][q].fn && (long long)a.count * (1 << q) <= c->cap[t][mode][q]) {
        ci = q;
        break;
      }
  }
  // no size that fits the whole colour at once (or only larger clusters are
  // built, as for 256 x 256 full-FFT frames): the largest built size, whose
  // clusters loop over the colour's positions
  for (int q = 3; q >= 0 && !c->kern[t][mode][ci].fn; --q)
    if (c->kern[t][mode][q].fn) ci = q;
  const PieKernel& k = c->kern[t][mode][ci];
  if (!k.fn) return pfth::set_error(PFT_ERR_UNSUPPORTED, "no PIE kernel for this transform and mode");
  const long long clusters = std::min<long long>(a.count, std::max<long long>(1, c->cap[t][mode][ci] / k.cluster));
  const dim3 grid((unsigned)(clusters * k.cluster));
  PftConst cst = c->plan.cst;
  const float2* W = c->plan.d_W;
  const float2* tw = t == 0 ? c->plan.d_twp : pfth::twiddles(c->n);
  if (!tw) return PFT_ERR_CUDA;
  void* args_pft[] = {(void*)&a, (void*)&cst, (void*)&W, (void*)&tw};
  void* args_full[] = {(void*)&a, (void*)&tw};
  void** args = t == 0 ? args_pft : args_full;
  if (k.cluster == 1) {
    PFT_CUDA_TRY(cudaLaunchKernel(k.fn, grid, dim3(k.threads), args, k.smem, st));
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(k.threads);
    cfg.dynamicSmemBytes = k.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = k.cluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    PFT_CUDA_TRY(cudaLaunchKernelExC(&cfg, k.fn, args));
  }
  return PFT_OK;
}

// Cluster size (log2) of a persistent coloured sweep: the autotuned one, else
// the largest built (-1: none).
int persist_ci(const pie_ctx* c, int t) {
  if (c->tuned[t][MODE_COLOURED] >= 0) return c->tuned[t][MODE_COLOURED];
  for (int q = 3; q >= 0; --q)
    if (c->kern[t][MODE_COLOURED][q].fn) return q;
  return -1;
}

// One coloured sweep as a single cooperative launch of the per-colour kernel.
// The persistent form (PIE_LAUNCH_PERSISTENT): as many clusters as fit on the
// GPU at once (at most the largest colour) loop over the colours with a grid
// barrier in between. The dataflow form (PIE_LAUNCH_DATAFLOW) runs the whole
// colour-major schedule as one list, item s going to cluster s mod (clusters):
// every item waits only for its overlapping predecessors instead of a barrier
// per colour, so items of consecutive colours overlap in time. The result is
// the same as the per-colour form's: an item reads its patch after every
// earlier overlapping item has written it and before any later one does, and
// items of one colour are disjoint. All clusters are co-resident (cooperative
// launch) and each runs its items in schedule order, so every wait ends.
int launch_pie_persistent(pie_ctx* c, int transform, PieArgs a, cudaStream_t st) {
  const int t = transform == PIE_TRANSFORM_PFT ? 0 : 1;
  const bool flow = c->persist[t] == PIE_LAUNCH_DATAFLOW;
  const int ci = (flow && c->flow_ci[t] >= 0) ? c->flow_ci[t] : persist_ci(c, t);
  if (ci < 0) return pfth::set_error(PFT_ERR_UNSUPPORTED, "no PIE kernel for this transform");
  const PieKernel& k = c->kern[t][MODE_COLOURED][ci];
  if (!k.fn) return pfth::set_error(PFT_ERR_UNSUPPORTED, "no PIE kernel for this transform");
  const long long clusters = std::max<long long>(
      1, std::min<long long>(flow ? c->npos : c->max_colour, c->cap[t][MODE_COLOURED][ci] / k.cluster));
  a.list = c->d_sched;
  a.count = 0;
  a.col_off = flow ? c->d_flow_off : c->d_coloff;
  a.ncol = flow ? 1 : c->ncol;
  a.gbar = c->d_gbar;
  a.gerr = reinterpret_cast<int*>(c->d_gbar + 1);
  a.gstatus = c->d_gstatus;
  a.dep_off = flow ? c->d_dep_off : nullptr;
  a.dep = flow ? c->d_dep : nullptr;
  a.done = flow ? c->d_done : nullptr;
  a.bar_extra = c->test_wait == PIE_TEST_WAIT_GRID_BARRIER ? 1u : 0u;
  a.dep_extra = c->test_wait == PIE_TEST_WAIT_DATAFLOW ? 1u : 0u;
  PFT_CUDA_TRY(cudaMemsetAsync(c->d_gbar, 0, 2 * sizeof(unsigned), st));
  if (flow) PFT_CUDA_TRY(cudaMemsetAsync(c->d_done, 0, sizeof(unsigned) * c->npos, st));
  PftConst cst = c->plan.cst;
  const float2* W = c->plan.d_W;
  const float2* tw = t == 0 ? c->plan.d_twp : pfth::twiddles(c->n);
  if (!tw) return PFT_ERR_CUDA;
  void* args_pft[] = {(void*)&a, (void*)&cst, (void*)&W, (void*)&tw};
  void* args_full[] = {(void*)&a, (void*)&tw};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * k.cluster));
  cfg.blockDim = dim3(k.threads);
  cfg.dynamicSmemBytes = k.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = k.cluster;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = k.cluster > 1 ? 2 : 1;
  PFT_CUDA_TRY(cudaLaunchKernelExC(&cfg, k.fn, t == 0 ? args_pft : args_full));
  return PFT_OK;
}

int enqueue_sweep(pie_ctx* c, float2* obj, int transform, double beta, bool stats, cudaStream_t st,
                  double gamma = -1.0, int mode = -1, int probe_step = PIE_PROBE_STEP_NORMALISED);

__global__ void k_fill(float2* __restrict__ z, long long n, float2 v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = v;
}

// Times one sweep of every built cluster size on a scratch object, for each
// transform in the context's mode, and keeps the fastest (the autotuner).
int autotune(pie_ctx* c, cudaStream_t st) {
  const int mode = c->pb.mode == PIE_MODE_COLOURED ? MODE_COLOURED : MODE_BATCHED;
  const long long HW = (long long)c->H * c->W;
  float2* scratch = c->d_prev;
  cudaEvent_t e0, e1;
  PFT_CUDA_TRY(cudaEventCreate(&e0));
  PFT_CUDA_TRY(cudaEventCreate(&e1));
  int rc = PFT_OK;
  for (int t = 0; t < 2 && rc == PFT_OK; ++t) {
    if (t == 1 && !c->have_full) break;
    const int tr = t == 0 ? PIE_TRANSFORM_PFT : PIE_TRANSFORM_FULL;
    int best = -1;
    float best_ms = 1e30f;
    for (int q = 0; q < 4 && rc == PFT_OK; ++q) {
      if (!c->kern[t][mode][q].fn) continue;
      c->tuned[t][mode] = q;
      k_fill<<<grid_for(HW), kThreads, 0, st>>>(scratch, HW, make_float2(0.7f, 0.2f));
      rc = enqueue_sweep(c, scratch, tr, 1.0, false, st);  // warm-up
      if (rc != PFT_OK) break;
      cudaEventRecord(e0, st);
      for (int rep = 0; rep < 2 && rc == PFT_OK; ++rep) rc = enqueue_sweep(c, scratch, tr, 1.0, false, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = pfth::set_error(PFT_ERR_CUDA, "autotune sweep failed");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc == PFT_OK && ms < best_ms) {
        best_ms = ms;
        best = q;
      }
    }
    c->tuned[t][mode] = best;
    c->tuned_ms[t] = best >= 0 ? best_ms / 2.0 : 0.0;
    // coloured sweeps: the same kernel as one cooperative launch per sweep, with
    // a grid barrier per colour (at the tuned cluster size) or with per-item
    // waits (every built cluster size); the fastest form is kept
    if (rc == PFT_OK && best >= 0 && mode == MODE_COLOURED && c->d_gbar) {
      auto try_form = [&](int form, int fci) {
        c->persist[t] = form;
        c->flow_ci[t] = fci;
        k_fill<<<grid_for(HW), kThreads, 0, st>>>(scratch, HW, make_float2(0.7f, 0.2f));
        int prc = enqueue_sweep(c, scratch, tr, 1.0, false, st);
        if (prc == PFT_OK) {
          cudaEventRecord(e0, st);
          for (int rep = 0; rep < 2 && prc == PFT_OK; ++rep) prc = enqueue_sweep(c, scratch, tr, 1.0, false, st);
          cudaEventRecord(e1, st);
          if (cudaEventSynchronize(e1) != cudaSuccess) prc = PFT_ERR_CUDA;
        }
        float ms = 0.f;
        if (prc == PFT_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (prc != PFT_OK || *c->h_gstatus != PFT_OK) {
          *c->h_gstatus = PFT_OK;
          cudaGetLastError();  // a refused cooperative launch is not sticky
          if (cudaStreamSynchronize(st) != cudaSuccess) rc = pfth::set_error(PFT_ERR_CUDA, "autotune sweep failed");
          return 1e30f;
        }
        return ms;
      };
      int best_form = PIE_LAUNCH_PER_COLOUR, best_fci = -1;
      float ms = try_form(PIE_LAUNCH_PERSISTENT, -1);
      if (ms < best_ms) {
        best_ms = ms;
        best_form = PIE_LAUNCH_PERSISTENT;
      }
      for (int q = 0; q < 4 && rc == PFT_OK && c->d_done; ++q) {
        if (!c->kern[t][mode][q].fn) continue;
        ms = try_form(PIE_LAUNCH_DATAFLOW, q);
        if (ms < best_ms) {
          best_ms = ms;
          best_form = PIE_LAUNCH_DATAFLOW;
          best_fci = q;
        }
      }
      c->persist[t] = best_form;
      c->flow_ci[t] = best_fci;
      c->tuned_ms[t] = best_ms / 2.0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace

extern "C" {

int pie_ctx_destroy(pie_ctx* c) {
  if (!c) return PFT_OK;
  if (c->have_plan) {
    cudaFree(c->plan.d_W);
    cudaFree(c->plan.d_twp);
    cudaFree(c->plan.d_B);
  }
  cudaFree(c->d_probe);
  cudaFree(c->d_pos);
  cudaFree(c->d_amp);
  cudaFree(c->d_ampc);
  cudaFree(c->d_sched);
  cudaFree(c->d_coloff);
  cudaFree(c->d_dep_off);
  cudaFree(c->d_dep);
  cudaFree(c->d_done);
  cudaFree(c->d_flow_off);
  cudaFree(c->d_gbar);
  if (c->h_gstatus) cudaFreeHost(c->h_gstatus);
  cudaFree(c->d_inv_illum);
  cudaFree(c->d_mask);
  cudaFree(c->d_prev);
  cudaFree(c->d_acc);
  cudaFree(c->d_tv);
  cudaFree(c->d_start);
  cudaFree(c->d_pacc);
  cudaFree(c->d_pden);
  cudaFree(c->d_pscale);
  cudaFree(c->d_red);
  if (c->h_red) cudaFreeHost(c->h_red);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return PFT_OK;
}

int pie_ctx_create(pie_ctx** out, const pie_problem* pb, const void* probe, const int32_t* positions,
                   const float* intensities, void* stream) {
  if (!out || !pb || !probe || !positions || !intensities)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const int n = pb->n, N = pb->npos, H = pb->obj_h, W = pb->obj_w, M = pb->M;
  if (n <= 0 || N <= 0 || H < n || W < n) return pfth::set_error(PFT_ERR_INVALID_ARG, "bad problem sizes");
  if (M <= 0 || M % 2 || M > n) return pfth::set_error(PFT_ERR_INVALID_ARG, "need even 0 < M <= n");
  if (pb->mode != PIE_MODE_COLOURED && pb->mode != PIE_MODE_BATCHED)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "unknown mode %d", pb->mode);
  if (pb->path != PFT_PATH_AUTO && pb->path != PFT_PATH_FACTORISED)
    return pfth::set_error(PFT_ERR_UNSUPPORTED, "PIE is built with the factorised PFT only");
  cudaStream_t st = (cudaStream_t)stream;
  pie_ctx* c = new (std::nothrow) pie_ctx();
  if (!c) return pfth::set_error(PFT_ERR_OOM, "host allocation failed");
  c->pb = *pb;
  c->n = n; c->npos = N; c->H = H; c->W = W; c->M = M;
  int rc = PFT_OK;
#define PIE_TRY(x)                    \
  do {                                \
    rc = (x);                         \
    if (rc != PFT_OK) {               \
      pie_ctx_destroy(c);             \
      return rc;                      \
    }                                 \
  } while (0)
#define PIE_CUDA(x)                                                   \
  do {                                                                \
    cudaError_t e_ = (x);                                             \
    if (e_ != cudaSuccess) {                                          \
      rc = pfth::cuda_error(e_, #x);                                  \
      pie_ctx_destroy(c);                                             \
      return rc;                                                      \
    }                                                                 \
  } while (0)
  // positions
  c->h_pos.resize(N);
  for (int j = 0; j < N; ++j) {
    const int r = positions[2 * j], q = positions[2 * j + 1];
    if (r < 0 || q < 0 || r > H - n || q > W - n) {
      pie_ctx_destroy(c);
      return pfth::set_error(PFT_ERR_INVALID_ARG, "position %d (%d, %d) outside the object", j, r, q);
    }
    c->h_pos[j] = make_int2(r, q);
  }
  // PFT plan and kernels
  PIE_TRY(pfth::build_plan(&c->plan, n, M, pb->p, pb->eps > 0 ? pb->eps : 1e-7, 0));
  c->have_plan = true;
  {
    const int P = c->plan.p1, Q = c->plan.q1, MP = M / c->plan.p1;
    bool any = false;
    for (int mode = 0; mode < 3; ++mode)
      for (int q = 0; q < 4; ++q) {
        PieKernel k = pfth::pie_pft_kernel(P, Q, MP, mode, 1 << q);
        if (k.fn) {
          PIE_TRY(prepare_kernel(k, &c->cap[0][mode][q]));
          c->kern[0][mode][q] = k;
          any = true;
        }
        PieKernel f = pfth::pie_full_kernel(n, mode, 1 << q);
        if (f.fn) {
          PIE_TRY(prepare_kernel(f, &c->cap[1][mode][q]));
          c->kern[1][mode][q] = f;
          c->have_full = true;
        }
      }
    if (!any) {
      pie_ctx_destroy(c);
      return pfth::set_error(PFT_ERR_UNSUPPORTED, "no PIE kernel for n=%d M=%d", n, M);
    }
    for (int q = 3; q >= 2 && !c->kern_claim[0].fn; --q) {
      PieKernel k = pfth::pie_pft_kernel(P, Q, MP, MODE_COLOURED, 1 << q, true);
      if (k.fn) {
        PIE_TRY(prepare_kernel(k, &c->cap_claim[0]));
        c->kern_claim[0] = k;
      }
    }
    for (int q = 3; q >= 2 && c->have_full && !c->kern_claim[1].fn; --q) {
      PieKernel f = pfth::pie_full_kernel(n, MODE_COLOURED, 1 << q, true);
      if (f.fn) {
        PIE_TRY(prepare_kernel(f, &c->cap_claim[1]));
        c->kern_claim[1] = f;
      }
    }
  }
  if (c->have_full && !pfth::twiddles(n)) {
    pie_ctx_destroy(c);
    return PFT_ERR_CUDA;
  }
  // probe
  std::vector<float2> hp((size_t)n * n);
  PIE_CUDA(cudaMalloc(&c->d_probe, sizeof(float2) * n * n));
  PIE_CUDA(cudaMemcpyAsync(c->d_probe, probe, sizeof(float2) * n * n, cudaMemcpyDeviceToDevice, st));
  PIE_CUDA(cudaMemcpyAsync(hp.data(), probe, sizeof(float2) * n * n, cudaMemcpyDeviceToHost, st));
  PIE_CUDA(cudaStreamSynchronize(st));
  for (auto& v : hp) c->probe_max2 = std::max(c->probe_max2, v.x * v.x + v.y * v.y);
  if (!(c->probe_max2 > 0.f) || !std::isfinite(c->probe_max2)) {
    pie_ctx_destroy(c);
    return pfth::set_error(PFT_ERR_NONFINITE, "probe is zero or not finite");
  }
  PIE_CUDA(cudaMalloc(&c->d_pos, sizeof(int2) * N));
  PIE_CUDA(cudaMemcpyAsync(c->d_pos, c->h_pos.data(), sizeof(int2) * N, cudaMemcpyHostToDevice, st));
  // amplitudes (d_red[7] counts non-finite intensities)
  PIE_CUDA(cudaMalloc(&c->d_red, sizeof(double) * 8));
  PIE_CUDA(cudaMallocHost(&c->h_red, sizeof(double) * 8));
  PIE_CUDA(cudaMemsetAsync(c->d_red, 0, sizeof(double) * 8, st));
  PIE_CUDA(cudaMalloc(&c->d_amp, sizeof(float) * (size_t)N * n * n));
  PIE_CUDA(cudaMalloc(&c->d_ampc, sizeof(float) * (size_t)N * M * M));
  k_amplitudes<<<grid_for((long long)N * n * n), kThreads, 0, st>>>(intensities, c->d_amp, c->d_ampc, N, n, M,
                                                                   reinterpret_cast<unsigned*>(c->d_red + 7));
  PIE_CUDA(cudaGetLastError());
  PIE_CUDA(cudaMemcpyAsync(c->h_red + 7, c->d_red + 7, sizeof(double), cudaMemcpyDeviceToHost, st));
  PIE_CUDA(cudaStreamSynchronize(st));
  if (*reinterpret_cast<const unsigned*>(c->h_red + 7) != 0u) {
    pie_ctx_destroy(c);
    return pfth::set_error(PFT_ERR_NONFINITE, "the intensities hold a NaN or infinite value");
  }
  // colouring
  colour_positions(c);
  PIE_CUDA(cudaMalloc(&c->d_sched, sizeof(int) * N));
  PIE_TRY(upload_schedule(c, st));
  // illumination, inverse illumination, mask
  const long long HW = (long long)H * W;
  PIE_CUDA(cudaMalloc(&c->d_inv_illum, sizeof(float) * HW));
  PIE_CUDA(cudaMalloc(&c->d_mask, HW));
  PIE_CUDA(cudaMalloc(&c->d_prev, sizeof(float2) * HW));
  PIE_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  if (pb->mode == PIE_MODE_BATCHED) PIE_CUDA(cudaMalloc(&c->d_acc, sizeof(float2) * HW));
  PIE_CUDA(cudaMemsetAsync(c->d_inv_illum, 0, sizeof(float) * HW, st));
  PIE_CUDA(cudaMemsetAsync(c->d_red, 0, sizeof(double) * 8, st));
  k_illumination<<<grid_for((long long)N * n * n), kThreads, 0, st>>>(c->d_probe, c->d_pos, N, n, W, c->d_inv_illum);
  k_max<<<grid_for(HW), kThreads, 0, st>>>(c->d_inv_illum, HW, (unsigned int*)c->d_red);
  k_finish_illum<<<grid_for(HW), kThreads, 0, st>>>(c->d_inv_illum, HW, (const unsigned int*)c->d_red,
                                                    (float)(pb->delta_rel > 0 ? pb->delta_rel : 1e-3), c->d_mask);
  PIE_CUDA(cudaGetLastError());
  PIE_CUDA(cudaStreamSynchronize(st));
  PIE_CUDA(cudaMalloc(&c->d_gbar, 2 * sizeof(unsigned)));
  PIE_CUDA(cudaHostAlloc(&c->h_gstatus, sizeof(int), cudaHostAllocMapped));
  *c->h_gstatus = PFT_OK;
  PIE_CUDA(cudaHostGetDevicePointer(&c->d_gstatus, c->h_gstatus, 0));
  if (pb->autotune) PIE_TRY(autotune(c, st));
#undef PIE_TRY
#undef PIE_CUDA
  *out = c;
  return PFT_OK;
}

int pie_ctx_info_get(const pie_ctx* c, pie_ctx_info* info) {
  if (!c || !info) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  const int mode = c->pb.mode == PIE_MODE_COLOURED ? MODE_COLOURED : MODE_BATCHED;
  info->ncolours = c->ncol;
  info->p = c->plan.p1;
  info->q = c->plan.q1;
  info->r = c->plan.r1;
  info->cluster_pft = c->tuned[0][mode] >= 0 ? (1 << c->tuned[0][mode]) : 0;
  info->cluster_full = c->tuned[1][mode] >= 0 ? (1 << c->tuned[1][mode]) : 0;
  info->sweep_ms_pft = c->tuned_ms[0];
  info->sweep_ms_full = c->tuned_ms[1];
  info->persistent_pft = c->persist[0];
  info->persistent_full = c->persist[1];
  for (int t = 0; t < 2; ++t) {  // the dataflow form may run another cluster size
    if (c->persist[t] != PIE_LAUNCH_DATAFLOW || c->flow_ci[t] < 0) continue;
    (t == 0 ? info->cluster_pft : info->cluster_full) = 1 << c->flow_ci[t];
  }
  return PFT_OK;
}

int pie_scan_schedule(const int32_t* positions, int npos, int n, int obj_h, int obj_w, const int32_t* order,
                      int one_per_colour, int* ncolours, int32_t* colour, int32_t* sched, int32_t* dep_off, int32_t* dep,
                      int64_t dep_capacity, int64_t* ndep) {
  if (!positions || !ncolours || !ndep) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (npos < 1 || n < 1 || obj_h < n || obj_w < n)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "need npos >= 1 and an n x n patch inside the object");
  std::vector<int2> pos(npos);
  for (int j = 0; j < npos; ++j) {
    const int r = positions[2 * j], q = positions[2 * j + 1];
    if (r < 0 || q < 0 || r + n > obj_h || q + n > obj_w)
      return pfth::set_error(PFT_ERR_INVALID_ARG, "position %d (%d, %d) puts the patch outside the object", j, r, q);
    pos[j] = make_int2(r, q);
  }
  std::vector<int> ord;
  if (order) {
    ord.assign(order, order + npos);
    std::vector<char> seen(npos, 0);
    for (int j : ord) {
      if (j < 0 || j >= npos || seen[j]) return pfth::set_error(PFT_ERR_INVALID_ARG, "order is not a permutation");
      seen[j] = 1;
    }
  }
  PieSchedule sch;
  build_schedule(pos, n, obj_h, obj_w, ord, sch, one_per_colour != 0);
  *ncolours = sch.ncol;
  *ndep = (int64_t)sch.dep.size();
  if (dep && dep_capacity < (int64_t)sch.dep.size())
    return pfth::set_error(PFT_ERR_INVALID_ARG, "dep holds %lld entries, %lld needed", (long long)dep_capacity,
                           (long long)sch.dep.size());
  for (int j = 0; j < npos; ++j) {
    if (colour) colour[j] = sch.colour[j];
    if (sched) sched[j] = sch.sched[j];
  }
  if (dep_off)
    for (int s = 0; s <= npos; ++s) dep_off[s] = sch.dep_off[s];
  if (dep)
    for (size_t i = 0; i < sch.dep.size(); ++i) dep[i] = sch.dep[i];
  return PFT_OK;
}

int pie_ctx_colours(const pie_ctx* c, int* ncolours, int32_t* colour_of) {
  if (!c || !ncolours) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  *ncolours = c->ncol;
  if (colour_of)
    for (int j = 0; j < c->npos; ++j) colour_of[j] = c->colour[j];
  return PFT_OK;
}

}  // extern "C"

namespace {

// Enqueues one sweep on `st`: statistics buffers, the kernels of every colour
// (or the batched kernel and its update), and with `stats` the FP64 norms and
// their copy to pinned host memory.
int enqueue_sweep(pie_ctx* c, float2* obj, int transform, double beta, bool stats, cudaStream_t st,
                  double gamma, int mode, int probe_step) {
  const long long HW = (long long)c->H * c->W;
  if (mode < 0) mode = c->pb.mode;
  const bool blind = gamma >= 0.0;
  const int n2i = c->n * c->n;
  if (stats) PFT_CUDA_TRY(cudaMemcpyAsync(c->d_prev, obj, sizeof(float2) * HW, cudaMemcpyDeviceToDevice, st));
  PFT_CUDA_TRY(cudaMemsetAsync(c->d_red, 0, sizeof(double) * 8, st));
  const float n2 = (float)c->n * (float)c->n;
  PieArgs a = {};
  a.inst = nullptr;
  a.work = nullptr;
  a.obj = obj;
  a.objr = obj;
  a.obj_w = c->W;
  a.probe = c->d_probe;
  a.pos = c->d_pos;
  a.dat = transform == PIE_TRANSFORM_PFT ? c->d_ampc : c->d_amp;
  a.gprobe = nullptr;
  a.red = c->d_red;
  a.gstatus = c->d_gstatus;
  if (mode == PIE_MODE_COLOURED) {
    a.coef = (float)(beta / ((double)c->probe_max2 * n2));
    a.acc = nullptr;
    if (blind) {
      // the probe changes after every colour: the object step reads max |w|^2 from the device
      a.coef = (float)(beta / n2);
      a.pacc = c->d_pacc;
      a.pden = c->d_pden;
      a.pscale = c->d_pscale;
      k_probe_init<<<1, 1024, 0, st>>>(c->d_probe, n2i, c->d_pacc, c->d_pden, c->d_pscale);
      PFT_CUDA_TRY(cudaGetLastError());
    }
    if (!blind && c->persist[transform == PIE_TRANSFORM_PFT ? 0 : 1]) {
      int rc = launch_pie_persistent(c, transform, a, st);
      if (rc != PFT_OK) return rc;
    }
    for (int col = 0; col < c->ncol && (blind || !c->persist[transform == PIE_TRANSFORM_PFT ? 0 : 1]); ++col) {
      a.list = c->d_sched + c->col_off[col];
      a.count = c->col_off[col + 1] - c->col_off[col];
      int rc = launch_pie(c, transform, MODE_COLOURED, a, st);
      if (rc != PFT_OK) return rc;
      if (blind) {
        k_probe_apply<<<1, 1024, 0, st>>>(c->d_probe, n2i, c->d_pacc, c->d_pden, (float)gamma,
                                          (float)(c->pb.delta_rel > 0 ? c->pb.delta_rel : 1e-3),
                                          probe_step == PIE_PROBE_STEP_NORMALISED, c->d_pscale);
        PFT_CUDA_TRY(cudaGetLastError());
      }
    }
  } else {
    PFT_CUDA_TRY(cudaMemsetAsync(c->d_acc, 0, sizeof(float2) * HW, st));
    a.coef = 1.f / n2;
    a.acc = c->d_acc;
    a.list = nullptr;
    a.count = c->npos;
    int rc = launch_pie(c, transform, MODE_BATCHED, a, st);
    if (rc != PFT_OK) return rc;
    k_apply_batched<<<grid_for(HW), kThreads, 0, st>>>(obj, c->d_acc, c->d_inv_illum, (float)beta, HW);
    PFT_CUDA_TRY(cudaGetLastError());
  }
  if (stats) {
    k_diff_norms<<<grid_for(HW), kThreads, 0, st>>>(obj, c->d_prev, HW, c->d_red + 1);
    PFT_CUDA_TRY(cudaGetLastError());
    PFT_CUDA_TRY(cudaMemcpyAsync(c->h_red, c->d_red, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
  }
  return PFT_OK;
}

// Returns the executable graph of a sweep, capturing it on first use.
int sweep_graph(pie_ctx* c, float2* obj, int transform, double beta, bool stats, cudaGraphExec_t* out,
                double gamma, int mode, int probe_step) {
  for (auto& g : c->graphs)
    if (g.obj == obj && g.transform == transform && g.beta == beta && g.stats == stats && g.gamma == gamma &&
        g.mode == mode && g.probe_step == probe_step) {
      *out = g.exec;
      return PFT_OK;
    }
  cudaGraphExec_t exec = nullptr;
  const int t = transform == PIE_TRANSFORM_PFT ? 0 : 1;
  for (int attempt = 0;; ++attempt) {
    PFT_CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_sweep(c, obj, transform, beta, stats, c->cap_stream, gamma, mode, probe_step);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (rc == PFT_OK && e == cudaSuccess) {
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e == cudaSuccess) break;
    } else if (graph) {
      cudaGraphDestroy(graph);
    }
    // a cooperative launch that cannot be captured: per-colour launches instead
    if (attempt == 0 && c->persist[t] && gamma < 0.0 && mode == PIE_MODE_COLOURED) {
      cudaGetLastError();
      c->persist[t] = PIE_LAUNCH_PER_COLOUR;
      continue;
    }
    if (rc != PFT_OK) return rc;
    return pfth::cuda_error(e, "sweep graph capture");
  }
  if (c->graphs.size() >= 8) {
    cudaGraphExecDestroy(c->graphs.front().exec);
    c->graphs.erase(c->graphs.begin());
  }
  c->graphs.push_back({obj, transform, beta, gamma, stats, mode, probe_step, exec});
  *out = exec;
  return PFT_OK;
}

int iterate(pie_ctx* c, void* object, int transform, double beta, double gamma, pie_stats* stats, void* stream,
            int mode = -1, int probe_step = PIE_PROBE_STEP_NORMALISED) {
  if (!c || !object) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (mode < 0) mode = c->pb.mode;
  if (mode != PIE_MODE_COLOURED && mode != PIE_MODE_BATCHED)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "unknown mode %d", mode);
  if (mode == PIE_MODE_BATCHED && !c->d_acc)
    PFT_CUDA_TRY(cudaMalloc(&c->d_acc, sizeof(float2) * (size_t)c->H * c->W));
  if (transform != PIE_TRANSFORM_PFT && transform != PIE_TRANSFORM_FULL)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "unknown transform %d", transform);
  if (transform == PIE_TRANSFORM_FULL && !c->have_full)
    return pfth::set_error(PFT_ERR_UNSUPPORTED, "full-FFT PIE is built for n in {16, 32, 64, 128, 256}, not %d",
                           c->n);
  if (c->h_gstatus && *c->h_gstatus != PFT_OK) {
    const int e = *c->h_gstatus;
    *c->h_gstatus = PFT_OK;
    return pfth::set_error(e, e == PFT_ERR_TIMEOUT ? "a grid barrier of an earlier persistent sweep timed out"
                                                   : "an earlier sweep's kernel ran without its cluster shape");
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (gamma >= 0.0) {
    if (mode != PIE_MODE_COLOURED)
      return pfth::set_error(PFT_ERR_UNSUPPORTED, "blind PIE runs in coloured mode");
    const size_t n2 = (size_t)c->n * c->n;
    if (!c->d_pacc) PFT_CUDA_TRY(cudaMalloc(&c->d_pacc, sizeof(float2) * n2));
    if (!c->d_pden) PFT_CUDA_TRY(cudaMalloc(&c->d_pden, sizeof(float) * n2));
    if (!c->d_pscale) PFT_CUDA_TRY(cudaMalloc(&c->d_pscale, sizeof(float)));
  }
  cudaGraphExec_t exec = nullptr;
  int rc = sweep_graph(c, (float2*)object, transform, beta, stats != nullptr, &exec, gamma, mode, probe_step);
  if (rc != PFT_OK) return rc;
  PFT_CUDA_TRY(cudaGraphLaunch(exec, st));
  if (stats) {
    PFT_CUDA_TRY(cudaStreamSynchronize(st));
    if (c->h_gstatus && *c->h_gstatus != PFT_OK) {  // this sweep's own device-side failure
      const int e = *c->h_gstatus;
      *c->h_gstatus = PFT_OK;
      return pfth::set_error(e, e == PFT_ERR_TIMEOUT ? "a bounded wait of this sweep timed out"
                                                     : "this sweep's kernel ran without its cluster shape");
    }
    const double n2 = (double)c->n * (double)c->n;
    stats->phi = c->h_red[0] / ((double)c->npos * n2);
    stats->rel_change = c->h_red[2] > 0 ? std::sqrt(c->h_red[1] / c->h_red[2]) : 0.0;
    if (!std::isfinite(stats->phi) || !std::isfinite(c->h_red[1]) || !std::isfinite(c->h_red[2]))
      return pfth::set_error(PFT_ERR_NONFINITE, "non-finite objective or object change");
  }
  return PFT_OK;
}

}  // namespace

extern "C" {

int pie_iteration(pie_ctx* c, void* object, int transform, double beta, pie_stats* stats, void* stream) {
  return iterate(c, object, transform, beta, -1.0, stats, stream);
}

int pie_iteration_mode(pie_ctx* c, void* object, int transform, int mode, double beta, pie_stats* stats,
                       void* stream) {
  return iterate(c, object, transform, beta, -1.0, stats, stream, mode);
}

int pie_iteration_blind(pie_ctx* c, void* object, int transform, double beta, double gamma, int probe_step,
                        pie_stats* stats, void* stream) {
  if (!(gamma >= 0.0)) return pfth::set_error(PFT_ERR_INVALID_ARG, "need gamma >= 0");
  if (probe_step != PIE_PROBE_STEP_NORMALISED && probe_step != PIE_PROBE_STEP_SCALAR)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "unknown probe step %d", probe_step);
  return iterate(c, object, transform, beta, gamma, stats, stream, -1, probe_step);
}

int pie_ctx_probe(const pie_ctx* c, void* probe_out, void* stream) {
  if (!c || !probe_out) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  PFT_CUDA_TRY(cudaMemcpyAsync(probe_out, c->d_probe, sizeof(float2) * c->n * c->n, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
  return PFT_OK;
}

int pie_ctx_set_probe(pie_ctx* c, const void* probe, void* stream) {
  if (!c || !probe) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n2 = (size_t)c->n * c->n;
  std::vector<float2> hp(n2);
  PFT_CUDA_TRY(cudaMemcpyAsync(c->d_probe, probe, sizeof(float2) * n2, cudaMemcpyDeviceToDevice, st));
  PFT_CUDA_TRY(cudaMemcpyAsync(hp.data(), probe, sizeof(float2) * n2, cudaMemcpyDeviceToHost, st));
  PFT_CUDA_TRY(cudaStreamSynchronize(st));
  float m = 0.f;
  for (auto& v : hp) m = std::max(m, v.x * v.x + v.y * v.y);
  if (!(m > 0.f) || !std::isfinite(m)) return pfth::set_error(PFT_ERR_NONFINITE, "probe is zero or not finite");
  c->probe_max2 = m;
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);  // step scales depend on the probe
  c->graphs.clear();
  return PFT_OK;
}

int pie_tv_step(pie_ctx* c, void* object, double lambda, double eps, void* stream) {
  if (!c || !object) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (!(lambda >= 0.0) || !(eps >= 0.0)) return pfth::set_error(PFT_ERR_INVALID_ARG, "need lambda, eps >= 0");
  if (lambda == 0.0) return PFT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const long long HW = (long long)c->H * c->W;
  if (!c->d_tv) PFT_CUDA_TRY(cudaMalloc(&c->d_tv, sizeof(float2) * HW));
  PFT_CUDA_TRY(cudaMemcpyAsync(c->d_tv, object, sizeof(float2) * HW, cudaMemcpyDeviceToDevice, st));
  k_tv_step<<<grid_for(HW), kThreads, 0, st>>>(c->d_tv, (float2*)object, c->H, c->W, (float)lambda, (float)eps);
  PFT_CUDA_TRY(cudaGetLastError());
  return PFT_OK;
}

int pie_ctx_set_persistent(pie_ctx* c, int transform, int persistent) {
  if (!c) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (transform != PIE_TRANSFORM_PFT && transform != PIE_TRANSFORM_FULL)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "unknown transform %d", transform);
  const int t = transform == PIE_TRANSFORM_PFT ? 0 : 1;
  if (c->pb.mode != PIE_MODE_COLOURED)
    return pfth::set_error(PFT_ERR_UNSUPPORTED, "persistent sweeps are built for coloured mode");
  if (t == 1 && !c->have_full) return pfth::set_error(PFT_ERR_UNSUPPORTED, "full-FFT PIE is not built for this n");
  if (persistent < PIE_LAUNCH_PER_COLOUR || persistent > PIE_LAUNCH_DATAFLOW)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "unknown launch form %d", persistent);
  if (persistent && persist_ci(c, t) < 0)
    return pfth::set_error(PFT_ERR_UNSUPPORTED, "no kernel for a persistent sweep");
  if (c->persist[t] != persistent) {
    PFT_CUDA_TRY(cudaDeviceSynchronize());
    c->persist[t] = persistent;
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
  }
  return PFT_OK;
}

int pie_ctx_set_cluster(pie_ctx* c, int transform, int cluster) {
  if (!c) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (transform != PIE_TRANSFORM_PFT && transform != PIE_TRANSFORM_FULL)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "unknown transform %d", transform);
  const int t = transform == PIE_TRANSFORM_PFT ? 0 : 1;
  const int mode = c->pb.mode == PIE_MODE_COLOURED ? MODE_COLOURED : MODE_BATCHED;
  int q = -1;
  if (cluster != 0) {
    for (int i = 0; i < 4; ++i)
      if (cluster == 1 << i) q = i;
    if (q < 0) return pfth::set_error(PFT_ERR_INVALID_ARG, "cluster size %d is not 0, 1, 2, 4 or 8", cluster);
    if (!c->kern[t][mode][q].fn)
      return pfth::set_error(PFT_ERR_UNSUPPORTED, "no %d-CTA PIE kernel for this n, M and mode", cluster);
  }
  PFT_CUDA_TRY(cudaDeviceSynchronize());
  c->tuned[t][mode] = q;
  if (mode == MODE_COLOURED) c->flow_ci[t] = q;
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);  // captured sweeps hold the launch shape
  c->graphs.clear();
  return PFT_OK;
}

int pie_ctx_test_unreachable_wait(pie_ctx* c, int kind) {
  if (!c) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (kind < PIE_TEST_WAIT_NONE || kind > PIE_TEST_WAIT_DATAFLOW)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "unknown wait kind %d", kind);
  if (c->test_wait != kind) {
    PFT_CUDA_TRY(cudaDeviceSynchronize());
    c->test_wait = kind;
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);  // the hook is baked into captured sweeps
    c->graphs.clear();
  }
  return PFT_OK;
}

int pie_ctx_set_order(pie_ctx* c, const int32_t* order, int one_per_colour) {
  if (!c) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  std::vector<int> ord;
  if (order) {
    ord.assign(order, order + c->npos);
    std::vector<char> seen(c->npos, 0);
    for (int j : ord) {
      if (j < 0 || j >= c->npos || seen[j]) return pfth::set_error(PFT_ERR_INVALID_ARG, "order is not a permutation");
      seen[j] = 1;
    }
  }
  PFT_CUDA_TRY(cudaDeviceSynchronize());  // no sweep of the old schedule may still be running
  colour_positions(c, ord, one_per_colour != 0);
  int rc = upload_schedule(c, nullptr);
  if (rc != PFT_OK) return rc;
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  return PFT_OK;
}

int pie_nrmse(pie_ctx* c, const void* object, const void* truth, double* out, void* stream) {
  if (!c || !object || !truth || !out) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const long long HW = (long long)c->H * c->W;
  PFT_CUDA_TRY(cudaMemsetAsync(c->d_red + 3, 0, sizeof(double) * 4, st));
  k_align_sums<<<grid_for(HW), kThreads, 0, st>>>((const float2*)object, (const float2*)truth, c->d_mask, HW,
                                                  c->d_red + 3);
  PFT_CUDA_TRY(cudaGetLastError());
  PFT_CUDA_TRY(cudaMemcpyAsync(c->h_red + 3, c->d_red + 3, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
  PFT_CUDA_TRY(cudaStreamSynchronize(st));
  for (int q = 3; q < 7; ++q)  // std::max below would turn a NaN sum into 0
    if (!std::isfinite(c->h_red[q])) return pfth::set_error(PFT_ERR_NONFINITE, "non-finite object or truth");
  const double ip = std::hypot(c->h_red[3], c->h_red[4]);
  const double e2 = std::max(0.0, c->h_red[5] + c->h_red[6] - 2.0 * ip);
  *out = c->h_red[6] > 0 ? std::sqrt(e2 / c->h_red[6]) : 0.0;
  if (!std::isfinite(*out)) return pfth::set_error(PFT_ERR_NONFINITE, "non-finite error norm");
  return PFT_OK;
}

int warm_start_then_refine(pie_ctx* c, void* object, const pie_schedule* s, const void* truth, pie_trace* trace,
                           int* ntrace, void* stream) {
  if (!c || !object || !s) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (s->max_pft < 0 || s->max_full < 0) return pfth::set_error(PFT_ERR_INVALID_ARG, "negative sweep budget");
  if (ntrace) *ntrace = 0;
  const auto t0 = std::chrono::steady_clock::now();
  int cnt = 0;
  const struct { int tr; double beta, tol; int mx; double tv; int mode; } phases[2] = {
      {PIE_TRANSFORM_PFT, s->beta_pft, s->tol_pft, s->max_pft, s->tv_pft,
       s->pft_batched ? PIE_MODE_BATCHED : c->pb.mode},
      {PIE_TRANSFORM_FULL, s->beta_full, s->tol_full, s->max_full, s->tv_full, c->pb.mode}};
  cudaStream_t st = (cudaStream_t)stream;
  const long long HW = (long long)c->H * c->W;
  for (const auto& ph : phases) {
    if (ph.tv < 0.0) return pfth::set_error(PFT_ERR_INVALID_ARG, "negative TV weight");
    if (ph.tv > 0.0 && !c->d_start) PFT_CUDA_TRY(cudaMalloc(&c->d_start, sizeof(float2) * HW));
    for (int it = 0; it < ph.mx; ++it) {
      pie_stats stt;
      if (ph.tv > 0.0)
        PFT_CUDA_TRY(cudaMemcpyAsync(c->d_start, object, sizeof(float2) * HW, cudaMemcpyDeviceToDevice, st));
      int rc = pie_iteration_mode(c, object, ph.tr, ph.mode, ph.beta, &stt, stream);
      if (rc != PFT_OK) return rc;
      if (ph.tv > 0.0) {
        // one TV gradient step after the sweep; the stopping rule sees the regularised object
        rc = pie_tv_step(c, object, ph.tv, s->tv_eps > 0 ? s->tv_eps : 1e-3, stream);
        if (rc != PFT_OK) return rc;
        PFT_CUDA_TRY(cudaMemsetAsync(c->d_red + 1, 0, sizeof(double) * 2, st));
        k_diff_norms<<<grid_for(HW), kThreads, 0, st>>>((const float2*)object, c->d_start, HW, c->d_red + 1);
        PFT_CUDA_TRY(cudaGetLastError());
        PFT_CUDA_TRY(cudaMemcpyAsync(c->h_red + 1, c->d_red + 1, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
        PFT_CUDA_TRY(cudaStreamSynchronize(st));
        stt.rel_change = c->h_red[2] > 0 ? std::sqrt(c->h_red[1] / c->h_red[2]) : 0.0;
      }
      double e = NAN;
      if (truth) {
        rc = pie_nrmse(c, object, truth, &e, stream);
        if (rc != PFT_OK) return rc;
      }
      if (trace) {
        trace[cnt].phase = ph.tr;
        trace[cnt].phi = stt.phi;
        trace[cnt].rel_change = stt.rel_change;
        trace[cnt].nrmse = e;
        trace[cnt].seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      }
      ++cnt;
      if (ntrace) *ntrace = cnt;
      if (stt.rel_change < ph.tol) break;
    }
  }
  return PFT_OK;
}

int pie_amp_loss_grad(pie_ctx* c, const void* object, const void* probe, void* grad_obj, void* grad_probe,
                      double* loss, void* stream) {
  if (!c || !object || !probe || !grad_obj || !loss) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const long long HW = (long long)c->H * c->W;
  PFT_CUDA_TRY(cudaMemsetAsync(grad_obj, 0, sizeof(float2) * HW, st));
  if (grad_probe) PFT_CUDA_TRY(cudaMemsetAsync(grad_probe, 0, sizeof(float2) * c->n * c->n, st));
  PFT_CUDA_TRY(cudaMemsetAsync(c->d_red, 0, sizeof(double), st));
  PieArgs a = {};
  a.inst = nullptr;
  a.work = nullptr;
  a.obj = nullptr;
  a.objr = (const float2*)object;
  a.obj_w = c->W;
  a.probe = (const float2*)probe;
  a.pos = c->d_pos;
  a.list = nullptr;
  a.count = c->npos;
  a.dat = c->d_ampc;
  a.coef = 1.f;
  a.acc = (float2*)grad_obj;
  a.gprobe = (float2*)grad_probe;
  a.red = c->d_red;
  int rc = launch_pie(c, PIE_TRANSFORM_PFT, MODE_GRAD, a, st);
  if (rc != PFT_OK) return rc;
  PFT_CUDA_TRY(cudaMemcpyAsync(c->h_red, c->d_red, sizeof(double), cudaMemcpyDeviceToHost, st));
  PFT_CUDA_TRY(cudaStreamSynchronize(st));
  *loss = c->h_red[0];
  if (!std::isfinite(*loss)) return pfth::set_error(PFT_ERR_NONFINITE, "non-finite loss");
  return PFT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Many independent reconstructions swept together.
// ------------------------------------------------------------------------
struct pie_batch {
  int count = 0;
  int mode = PIE_MODE_COLOURED;
  std::vector<pie_ctx*> ctx;
  struct Class {
    int rep = 0;                    // member whose kernels and tables the class uses
    std::vector<int> members;
    std::vector<int> col_off;       // work-list offsets per colour (coloured mode)
    int2* d_work = nullptr;         // (instance, position) pairs, colour-major
    bool have_full = true;
    // dataflow form (coloured mode): the whole work list in one launch, each
    // item waiting for its instance's overlapping predecessors
    int* d_dep_off = nullptr;       // [items + 1]
    int* d_dep = nullptr;           // work-list indices
    unsigned* d_done = nullptr;     // [items]
    unsigned* d_ticket = nullptr;   // [2]: claim counter, error word
    int* d_flow_off = nullptr;      // {0, items}
    int max_width = 0;              // items in the class's largest colour
    int chain = 1;                  // longest dependency chain: the members' largest colour count
  };
  std::vector<Class> classes;
  // coloured mode: PIE_LAUNCH_PER_COLOUR (measured faster on the 64-instance
  // recipe: 119 ms against 166 ms per PFT sweep) or PIE_LAUNCH_DATAFLOW
  int launch = PIE_LAUNCH_PER_COLOUR;
  std::vector<PieInstance> h_inst;
  double* d_red = nullptr;
  double* h_red = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> events;  // [0] fork, [1 + k] join of class k
  struct Graph {
    std::vector<void*> objs;
    int transform;
    double beta;
    bool stats;
    cudaGraphExec_t exec;
    PieInstance* d_inst;  // the instance descriptors this graph reads
  };
  std::vector<Graph> graphs;
};

namespace {

// Instance descriptors for these objects and this step size (host side).
void batch_descriptors(pie_batch* b, void* const* objects, int transform, double beta) {
  const int t = transform == PIE_TRANSFORM_PFT ? 0 : 1;
  const bool coloured = b->mode == PIE_MODE_COLOURED;
  b->h_inst.resize(b->count);
  for (int i = 0; i < b->count; ++i) {
    pie_ctx* c = b->ctx[i];
    PieInstance& in = b->h_inst[i];
    const double n2 = (double)c->n * (double)c->n;
    in.obj = (float2*)objects[i];
    in.obj_w = c->W;
    in.probe = c->d_probe;
    in.pos = c->d_pos;
    in.dat = t == 0 ? c->d_ampc : c->d_amp;
    in.coef = coloured ? (float)(beta / ((double)c->probe_max2 * n2)) : (float)(1.0 / n2);
    in.acc = c->d_acc;
    in.red = b->d_red + i;
  }
}

// One dataflow launch over a shape class's work list: clusters claim items in
// schedule order (PieArgs::ticket), so the classes' launches may share the GPU
// in any proportion (no co-residency is needed for the waits to end). `width`
// clusters at most, capped by what fits on the GPU.
int launch_pie_claimed(pie_ctx* c, int transform, PieArgs a, int width, cudaStream_t st) {
  const int t = transform == PIE_TRANSFORM_PFT ? 0 : 1;
  const PieKernel& k = c->kern_claim[t];
  if (!k.fn) return pfth::set_error(PFT_ERR_UNSUPPORTED, "no item-claiming PIE kernel for this transform");
  const long long clusters = std::max<long long>(1, std::min<long long>(width, c->cap_claim[t] / k.cluster));
  PftConst cst = c->plan.cst;
  const float2* W = c->plan.d_W;
  const float2* tw = t == 0 ? c->plan.d_twp : pfth::twiddles(c->n);
  if (!tw) return PFT_ERR_CUDA;
  void* args_pft[] = {(void*)&a, (void*)&cst, (void*)&W, (void*)&tw};
  void* args_full[] = {(void*)&a, (void*)&tw};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * k.cluster));
  cfg.blockDim = dim3(k.threads);
  cfg.dynamicSmemBytes = k.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = k.cluster;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = k.cluster > 1 ? 1 : 0;
  PFT_CUDA_TRY(cudaLaunchKernelExC(&cfg, k.fn, t == 0 ? args_pft : args_full));
  return PFT_OK;
}

int batch_enqueue(pie_batch* b, const PieInstance* d_inst, void* const* objects, int transform, double beta,
                  bool stats, cudaStream_t st) {
  const int mode = b->mode == PIE_MODE_COLOURED ? MODE_COLOURED : MODE_BATCHED;
  PFT_CUDA_TRY(cudaMemsetAsync(b->d_red, 0, sizeof(double) * b->count, st));
  if (mode == MODE_BATCHED)
    for (pie_ctx* c : b->ctx)
      PFT_CUDA_TRY(cudaMemsetAsync(c->d_acc, 0, sizeof(float2) * (size_t)c->H * c->W, st));
  PFT_CUDA_TRY(cudaEventRecord(b->events[0], st));
  for (size_t k = 0; k < b->classes.size(); ++k) {
    const pie_batch::Class& cl = b->classes[k];
    cudaStream_t bs = b->branch[k];
    PFT_CUDA_TRY(cudaStreamWaitEvent(bs, b->events[0], 0));
    PieArgs a = {};
    a.inst = d_inst;
    pie_ctx* rep = b->ctx[cl.rep];
    const int t = transform == PIE_TRANSFORM_PFT ? 0 : 1;
    const bool flow = mode == MODE_COLOURED && b->launch == PIE_LAUNCH_DATAFLOW && rep->kern_claim[t].fn;
    if (flow) {
      const int items = cl.col_off.back();
      PFT_CUDA_TRY(cudaMemsetAsync(cl.d_done, 0, sizeof(unsigned) * std::max(1, items), bs));
      PFT_CUDA_TRY(cudaMemsetAsync(cl.d_ticket, 0, 2 * sizeof(unsigned), bs));
      a.work = cl.d_work;
      a.count = 0;
      a.col_off = cl.d_flow_off;
      a.ncol = 1;
      a.gbar = cl.d_ticket;
      a.gerr = reinterpret_cast<int*>(cl.d_ticket + 1);
      a.gstatus = rep->d_gstatus;
      a.dep_off = cl.d_dep_off;
      a.dep = cl.d_dep;
      a.done = cl.d_done;
      a.ticket = cl.d_ticket;
      if (items > 0) {
        // A fixed share of the GPU per class, so that the classes' persistent
        // clusters do not crowd one another out: the batch takes at least as
        // long as its longest colour chain, so a class whose chain is at least
        // half the longest gets its average parallelism (items over its chain),
        // and a class with a short chain only the clusters it needs to finish
        // within the longest chain (items over that chain).
        int chain_max = 1;
        for (const pie_batch::Class& o : b->classes) chain_max = std::max(chain_max, o.chain);
        const int span = 2 * cl.chain >= chain_max ? cl.chain : chain_max;
        const long long par = ((long long)items + span - 1) / span;
        const int width = (int)std::min<long long>(cl.max_width, std::max<long long>(1, par));
        int rc = launch_pie_claimed(rep, transform, a, width, bs);
        if (rc != PFT_OK) return rc;
      }
    }
    const int ncol = mode != MODE_COLOURED ? 1 : flow ? 0 : (int)cl.col_off.size() - 1;
    for (int col = 0; col < ncol; ++col) {
      const int off = mode == MODE_COLOURED ? cl.col_off[col] : 0;
      a.work = cl.d_work + off;
      a.count = mode == MODE_COLOURED ? cl.col_off[col + 1] - off : cl.col_off.back();
      int rc = launch_pie(b->ctx[cl.rep], transform, mode, a, bs);
      if (rc != PFT_OK) return rc;
    }
    PFT_CUDA_TRY(cudaEventRecord(b->events[1 + k], bs));
    PFT_CUDA_TRY(cudaStreamWaitEvent(st, b->events[1 + k], 0));
  }
  if (mode == MODE_BATCHED)
    for (int i = 0; i < b->count; ++i) {
      pie_ctx* c = b->ctx[i];
      const long long HW = (long long)c->H * c->W;
      k_apply_batched<<<grid_for(HW), kThreads, 0, st>>>((float2*)objects[i], c->d_acc, c->d_inv_illum,
                                                         (float)beta, HW);
      PFT_CUDA_TRY(cudaGetLastError());
    }
  if (stats)
    PFT_CUDA_TRY(cudaMemcpyAsync(b->h_red, b->d_red, sizeof(double) * b->count, cudaMemcpyDeviceToHost, st));
  return PFT_OK;
}

}  // namespace

extern "C" {

int pie_batch_destroy(pie_batch* b) {
  if (!b) return PFT_OK;
  for (auto& g : b->graphs) {
    cudaGraphExecDestroy(g.exec);
    cudaFree(g.d_inst);
  }
  for (auto& cl : b->classes) {
    cudaFree(cl.d_work);
    cudaFree(cl.d_dep_off);
    cudaFree(cl.d_dep);
    cudaFree(cl.d_done);
    cudaFree(cl.d_ticket);
    cudaFree(cl.d_flow_off);
  }
  for (auto* c : b->ctx) pie_ctx_destroy(c);
  cudaFree(b->d_red);
  if (b->h_red) cudaFreeHost(b->h_red);
  for (auto s : b->branch) cudaStreamDestroy(s);
  for (auto e : b->events) cudaEventDestroy(e);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
  return PFT_OK;
}

int pie_batch_create(pie_batch** out, int count, const pie_problem* problems, const void* const* probes,
                     const int32_t* const* positions, const float* const* intensities, void* stream) {
  if (!out || !problems || !probes || !positions || !intensities || count <= 0)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument or count <= 0");
  *out = nullptr;
  for (int i = 1; i < count; ++i)
    if (problems[i].mode != problems[0].mode)
      return pfth::set_error(PFT_ERR_INVALID_ARG, "all instances of a batch use the same mode");
  pie_batch* b = new (std::nothrow) pie_batch();
  if (!b) return pfth::set_error(PFT_ERR_OOM, "host allocation failed");
  b->count = count;
  b->mode = problems[0].mode;
  int rc = PFT_OK;
  for (int i = 0; i < count && rc == PFT_OK; ++i) {
    pie_problem pb = problems[i];
    pb.autotune = 0;  // the batch picks cluster sizes per launch
    pie_ctx* c = nullptr;
    rc = pie_ctx_create(&c, &pb, probes[i], positions[i], intensities[i], stream);
    if (rc == PFT_OK) b->ctx.push_back(c);
  }
  if (rc != PFT_OK) {
    pie_batch_destroy(b);
    return rc;
  }
  // shape classes: instances whose kernels and tables coincide
  for (int i = 0; i < count; ++i) {
    pie_ctx* c = b->ctx[i];
    int k = -1;
    for (size_t q = 0; q < b->classes.size(); ++q) {
      pie_ctx* r = b->ctx[b->classes[q].rep];
      if (r->n == c->n && r->M == c->M && r->plan.p1 == c->plan.p1 && r->plan.r1 == c->plan.r1 &&
          r->plan.xi1 == c->plan.xi1)
        k = (int)q;
    }
    if (k < 0) {
      b->classes.push_back(pie_batch::Class());
      k = (int)b->classes.size() - 1;
      b->classes[k].rep = i;
    }
    b->classes[k].members.push_back(i);
    b->classes[k].have_full = b->classes[k].have_full && c->have_full;
  }
  auto fail = [&](cudaError_t e, const char* what) {
    int code = pfth::cuda_error(e, what);
    pie_batch_destroy(b);
    return code;
  };
  for (auto& cl : b->classes) {
    int ncol = 0;
    for (int i : cl.members) ncol = std::max(ncol, b->mode == PIE_MODE_COLOURED ? b->ctx[i]->ncol : 1);
    std::vector<int2> work;
    cl.col_off.assign(1, 0);
    for (int col = 0; col < ncol; ++col) {
      for (int i : cl.members) {
        pie_ctx* c = b->ctx[i];
        for (int j = 0; j < c->npos; ++j)
          if (b->mode != PIE_MODE_COLOURED || c->colour[j] == col) work.push_back(make_int2(i, j));
      }
      cl.col_off.push_back((int)work.size());
    }
    cudaError_t e = cudaMalloc(&cl.d_work, sizeof(int2) * work.size());
    if (e != cudaSuccess) return fail(e, "cudaMalloc(work)");
    e = cudaMemcpy(cl.d_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(e, "cudaMemcpy(work)");
    if (b->mode != PIE_MODE_COLOURED) continue;
    // dataflow predecessors: instance i's k-th item in the work list is item k
    // of its own colour-major schedule, so its predecessor lists carry over
    const int items = (int)work.size();
    for (size_t q = 0; q + 1 < cl.col_off.size(); ++q)
      cl.max_width = std::max(cl.max_width, cl.col_off[q + 1] - cl.col_off[q]);
    for (int i : cl.members) cl.chain = std::max(cl.chain, b->ctx[i]->ncol);
    std::vector<std::vector<int>> widx(count);
    for (int w = 0; w < items; ++w) {
      const int i = work[w].x;
      const int k = (int)widx[i].size();
      if (b->ctx[i]->h_sched[k] != work[w].y) {
        pie_batch_destroy(b);
        return pfth::set_error(PFT_ERR_CUDA, "internal: batch work list out of schedule order");
      }
      widx[i].push_back(w);
    }
    std::vector<int> off(items + 1, 0), dep;
    for (int w = 0; w < items; ++w) {
      const int i = work[w].x;
      const pie_ctx* c = b->ctx[i];
      const int k = (int)(std::lower_bound(widx[i].begin(), widx[i].end(), w) - widx[i].begin());
      for (int d = c->h_dep_off[k]; d < c->h_dep_off[k + 1]; ++d) dep.push_back(widx[i][c->h_dep[d]]);
      off[w + 1] = (int)dep.size();
    }
    const int flow_off[2] = {0, items};
    e = cudaMalloc(&cl.d_dep_off, sizeof(int) * (items + 1));
    if (e == cudaSuccess) e = cudaMalloc(&cl.d_dep, sizeof(int) * std::max<size_t>(1, dep.size()));
    if (e == cudaSuccess) e = cudaMalloc(&cl.d_done, sizeof(unsigned) * std::max(1, items));
    if (e == cudaSuccess) e = cudaMalloc(&cl.d_ticket, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&cl.d_flow_off, sizeof(flow_off));
    if (e == cudaSuccess) e = cudaMemcpy(cl.d_dep_off, off.data(), sizeof(int) * (items + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !dep.empty())
      e = cudaMemcpy(cl.d_dep, dep.data(), sizeof(int) * dep.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cl.d_flow_off, flow_off, sizeof(flow_off), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(e, "batch dataflow lists");
  }
  cudaError_t e = cudaMalloc(&b->d_red, sizeof(double) * count);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_red, sizeof(double) * count);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  for (size_t k = 0; k < b->classes.size() && e == cudaSuccess; ++k) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->branch.push_back(s);
  }
  for (size_t k = 0; k <= b->classes.size() && e == cudaSuccess; ++k) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->events.push_back(ev);
  }
  if (e != cudaSuccess) return fail(e, "batch resources");
  *out = b;
  return PFT_OK;
}

int pie_batch_iteration(pie_batch* b, void* const* objects, int transform, double beta, double* phi,
                        void* stream) {
  if (!b || !objects) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (transform != PIE_TRANSFORM_PFT && transform != PIE_TRANSFORM_FULL)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "unknown transform %d", transform);
  for (int i = 0; i < b->count; ++i)
    if (!objects[i]) return pfth::set_error(PFT_ERR_INVALID_ARG, "object %d is NULL", i);
  if (transform == PIE_TRANSFORM_FULL)
    for (auto& cl : b->classes)
      if (!cl.have_full)
        return pfth::set_error(PFT_ERR_UNSUPPORTED, "full-FFT PIE is built for n <= 128, not %d",
                               b->ctx[cl.rep]->n);
  for (auto& cl : b->classes) {  // a wait of an earlier dataflow sweep that gave up
    pie_ctx* rep = b->ctx[cl.rep];
    if (rep->h_gstatus && *rep->h_gstatus != PFT_OK) {
      const int e = *rep->h_gstatus;
      *rep->h_gstatus = PFT_OK;
      return pfth::set_error(e, e == PFT_ERR_TIMEOUT ? "a wait of an earlier batch sweep timed out"
                                                     : "an earlier batch sweep's kernel ran without its cluster shape");
    }
  }
  std::vector<void*> objs(objects, objects + b->count);
  cudaGraphExec_t exec = nullptr;
  for (auto& g : b->graphs)
    if (g.objs == objs && g.transform == transform && g.beta == beta && g.stats == (phi != nullptr))
      exec = g.exec;
  if (!exec) {
    batch_descriptors(b, objects, transform, beta);
    PieInstance* d_inst = nullptr;
    PFT_CUDA_TRY(cudaMalloc(&d_inst, sizeof(PieInstance) * b->count));
    cudaError_t e = cudaMemcpy(d_inst, b->h_inst.data(), sizeof(PieInstance) * b->count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d_inst);
      return pfth::cuda_error(e, "cudaMemcpy(instances)");
    }
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaFree(d_inst);
      return pfth::cuda_error(e, "cudaStreamBeginCapture");
    }
    int rc = batch_enqueue(b, d_inst, objects, transform, beta, phi != nullptr, b->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (rc == PFT_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc != PFT_OK || e != cudaSuccess) {
      cudaFree(d_inst);
      return rc != PFT_OK ? rc : pfth::cuda_error(e, "sweep graph capture");
    }
    if (b->graphs.size() >= 8) {
      cudaGraphExecDestroy(b->graphs.front().exec);
      cudaFree(b->graphs.front().d_inst);
      b->graphs.erase(b->graphs.begin());
    }
    b->graphs.push_back({objs, transform, beta, phi != nullptr, exec, d_inst});
  }
  cudaStream_t st = (cudaStream_t)stream;
  PFT_CUDA_TRY(cudaGraphLaunch(exec, st));
  if (phi) {
    PFT_CUDA_TRY(cudaStreamSynchronize(st));
    for (auto& cl : b->classes) {
      pie_ctx* rep = b->ctx[cl.rep];
      if (rep->h_gstatus && *rep->h_gstatus != PFT_OK) {
        const int e = *rep->h_gstatus;
        *rep->h_gstatus = PFT_OK;
        return pfth::set_error(e, e == PFT_ERR_TIMEOUT ? "a wait of this batch sweep timed out"
                                                       : "this batch sweep's kernel ran without its cluster shape");
      }
    }
    for (int i = 0; i < b->count; ++i) {
      pie_ctx* c = b->ctx[i];
      phi[i] = b->h_red[i] / ((double)c->npos * (double)c->n * (double)c->n);
      if (!std::isfinite(phi[i])) return pfth::set_error(PFT_ERR_NONFINITE, "non-finite objective (instance %d)", i);
    }
  }
  return PFT_OK;
}

int pie_batch_classes(const pie_batch* b, int* nclasses, int* launches_per_sweep) {
  if (!b || !nclasses) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  *nclasses = (int)b->classes.size();
  if (launches_per_sweep) {
    int l = 0;
    for (auto& cl : b->classes)
      l += (b->mode == PIE_MODE_COLOURED && b->launch == PIE_LAUNCH_DATAFLOW && b->ctx[cl.rep]->kern_claim[0].fn)
               ? 1 : (int)cl.col_off.size() - 1;
    *launches_per_sweep = l;
  }
  return PFT_OK;
}

int pie_batch_set_launch(pie_batch* b, int form) {
  if (!b) return pfth::set_error(PFT_ERR_INVALID_ARG, "null argument");
  if (form != PIE_LAUNCH_PER_COLOUR && form != PIE_LAUNCH_DATAFLOW)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "a batch launches per colour or as dataflow, not form %d", form);
  if (b->mode != PIE_MODE_COLOURED)
    return pfth::set_error(PFT_ERR_UNSUPPORTED, "launch forms apply to coloured batches");
  if (b->launch != form) {
    PFT_CUDA_TRY(cudaDeviceSynchronize());
    b->launch = form;
    for (auto& g : b->graphs) {
      cudaGraphExecDestroy(g.exec);
      cudaFree(g.d_inst);
    }
    b->graphs.clear();
  }
  return PFT_OK;
}

}  // extern "C"
