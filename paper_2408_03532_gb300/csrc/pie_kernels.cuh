// Fused per-position PIE kernels (Section 2.1, Eq. pie_update with Eq. 3).
//
// One scan position j is processed by a thread-block cluster of C CTAs:
//   1. rows: CTA c forms the exit wave psi = w . Q_j z on rows [c n/C, (c+1) n/C)
//      and transforms them along axis 2 (PFT rows or FFT rows); each result is
//      written straight into the shared memory of the CTA that owns its column
//      (distributed shared memory), so the n x M (or n x n) intermediate is
//      redistributed without touching global memory;
//   2. cluster barrier;
//   3. columns: CTA c transforms its M/C (or n/C) columns along axis 1, applies
//      the modulus projection R = Psi - d . sgn(Psi) on its part of the
//      spectrum (accumulating ||R||^2 for Eq. 4), and runs the adjoint column
//      transform; results go back to the row owners;
//   4. cluster barrier;
//   5. rows: the adjoint row transform gives A^H R on CTA c's rows, and the
//      object update z -= beta conj(w) / max|w|^2 . A^H R / n^2 is applied.
// With C = 1 the cluster is one CTA and the two exchange buffers alias. Within
// a position the barriers are the hardware cluster barrier. Between positions,
// a coloured sweep launched once per colour needs no wait; the single-launch
// forms wait on a grid barrier per colour or on the completion counters of a
// position's overlapping predecessors (both bounded spin waits, below).
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include "fft_core.cuh"
#include "pft_core.cuh"

namespace pftk {

namespace cg = cooperative_groups;

enum { MODE_COLOURED = 0, MODE_BATCHED = 1, MODE_GRAD = 2 };

// One instance of a multi-instance sweep (every pointer is that instance's).
struct PieInstance {
  float2* obj;
  long long obj_w;
  const float2* probe;
  const int2* pos;
  const float* dat;
  float coef;
  float2* acc;
  double* red;
};

struct PieArgs {
  // multi-instance sweeps: work item it is (instance, position) = work[it];
  // when inst == nullptr the single-instance fields below are used
  const PieInstance* inst;
  const int2* work;
  float2* obj;              // object [H][W] (written in MODE_COLOURED)
  const float2* objr;       // object read pointer (= obj, or the gradient's input)
  long long obj_w;
  const float2* probe;      // [n][n]
  const int2* pos;          // [N] top-left (row, col)
  const int* list;          // positions to process (nullptr = 0..count-1)
  int count;
  const float* dat;         // amplitudes: [N][M][M] centred crop, or [N][n][n] FFT order
  float coef;               // update scale
  float2* acc;              // MODE_BATCHED: sum conj(w) dpsi; MODE_GRAD: grad_obj
  float2* gprobe;           // MODE_GRAD: grad_probe (may be null)
  double* red;              // red[0] += sum ||R||^2 (MODE_GRAD: the loss)
  // blind PIE (coloured mode): a second round per position accumulates the
  // probe step of Eq. epie_probe_update at the updated patch
  float2* pacc;             // sum conj(z_new) dpsi' over the colour (null = non-blind)
  float* pden;              // sum |z_new|^2 over the colour
  const float* pscale;      // max |w|^2 of the current probe (divides coef when set)
  // persistent coloured sweep (ncol > 0): one launch runs every colour; colour
  // k is list[col_off[k] .. col_off[k + 1]), with a grid barrier in between
  const int* col_off;
  int ncol;
  unsigned* gbar;           // arrival counter, zero at launch
  int* gerr;                // set when a barrier gives up (device word, zero at launch)
  int* gstatus;             // mapped host status word: PFT_ERR_TIMEOUT on a timeout
  // dataflow sweep (dep_off != nullptr, persistent with one "colour" holding the
  // whole colour-major schedule): item s waits until done[d] == C for every
  // predecessor d in dep[dep_off[s] .. dep_off[s + 1]) (the earlier items whose
  // patches overlap its own, transitively reduced), and each of its C CTAs adds
  // one to done[s] once its part of the update is written
  const int* dep_off;
  const int* dep;
  unsigned* done;           // [schedule length], zero at launch
  // dataflow sweep with claimed items (ticket != nullptr): clusters take items
  // in schedule order from *ticket (zero at launch) instead of item s going to
  // cluster s mod (clusters). An item then only waits for items already claimed
  // by running clusters, so every wait ends without the clusters being
  // co-resident (used when several sweeps share the GPU).
  unsigned* ticket;
  // test hook (pie_ctx_test_unreachable_wait): added to the target of every
  // grid barrier (bar_extra) or dataflow wait (dep_extra); zero in normal use.
  // A non-zero value makes that wait unreachable, so its bounded timeout runs.
  unsigned bar_extra;
  unsigned dep_extra;
};

template <int C>
struct Cluster {
  __device__ __forceinline__ static unsigned rank() {
    if constexpr (C == 1) return 0;
    else return cg::this_cluster().block_rank();
  }
  __device__ __forceinline__ static void sync() {
    if constexpr (C == 1) __syncthreads();
    else cg::this_cluster().sync();
  }
  template <class T>
  __device__ __forceinline__ static T* map(T* p, unsigned r) {
    if constexpr (C == 1) return p;
    else return cg::this_cluster().map_shared_rank(p, r);
  }
};

// Asynchronous exchange between the CTAs of a cluster: st.async writes a
// value into a peer's shared memory and completes `bytes` on the peer's
// mbarrier; the receiver, which announced the bytes it expects, waits on its
// own mbarrier (acquire at cluster scope) instead of a cluster-wide barrier.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t map_rank(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_async2(uint32_t raddr, float2 v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];"
               ::"r"(raddr), "f"(v.x), "f"(v.y), "r"(rbar) : "memory");
}
__device__ __forceinline__ void xbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void xbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the phase of parity `par` (2 s); a timeout sets the error
// words, and so does finding another CTA's timeout; either way the caller goes on.
__device__ __forceinline__ void xbar_wait(uint32_t bar, uint32_t par, const PieArgs& a, bool& abort) {
  if (abort) return;  // an earlier wait of this thread gave up: the sweep is already failed
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.b32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(bar), "r"(par) : "memory");
  if (ok) return;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (unsigned spin = 1;; ++spin) {  // the error word is read every 16th try only
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.b32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(bar), "r"(par) : "memory");
    if (ok) return;
    if ((spin & 15u) == 0u && a.gerr && *reinterpret_cast<volatile int*>(a.gerr)) {
      abort = true;
      return;
    }
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 2000000000ull) {
      abort = true;
      if (a.gerr) atomicExch(a.gerr, 1);
      if (a.gstatus) {
        *reinterpret_cast<volatile int*>(a.gstatus) = PFT_ERR_TIMEOUT;
        __threadfence_system();
      }
      return;
    }
  }
}

// A cluster kernel launched without its cluster shape must not address peer
// shared memory: it records an error and does nothing.
template <int C>
__device__ __forceinline__ bool cluster_shape_ok(int* gstatus) {
  if constexpr (C > 1) {
    if (cg::this_cluster().num_blocks() != (unsigned)C) {
      if (threadIdx.x == 0 && gstatus) {
        *reinterpret_cast<volatile int*>(gstatus) = PFT_ERR_CUDA;
        __threadfence_system();
      }
      return false;
    }
  }
  return true;
}

// Grid-wide barrier of a co-resident (cooperative) launch: every CTA makes its
// writes visible GPU-wide, adds one to *ctr and waits until it reaches
// `target` (CTAs x barriers so far). The wait is bounded: after 2 s, or as
// soon as another CTA has given up, it returns false (a timeout also sets the
// error words). One arrival per CTA measured faster than one per cluster
// behind two cluster barriers.
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, unsigned target, int* gerr, int* gstatus) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    int ok = 1;
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
      if (v >= target) break;
      if (*reinterpret_cast<volatile int*>(gerr)) {
        ok = 0;
        break;
      }
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 2000000000ull) {
        atomicExch(gerr, 1);
        if (gstatus) {
          *reinterpret_cast<volatile int*>(gstatus) = PFT_ERR_TIMEOUT;
          __threadfence_system();
        }
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Dataflow sweep: before reading its patch, schedule item s waits until every
// predecessor has been written by all C CTAs of the cluster that ran it. Warp 0
// polls, one predecessor per lane, with acquire loads; each wait is bounded at
// 2 s. A wait that gives up (or finds that another CTA gave up) sets the error
// words and returns without waiting: the CTA still runs every item and cluster
// barrier of its list, so the launch ends, and the host reports the timeout.
// No fence follows the polls: each lane's acquire load synchronises with its
// predecessor's release (signal_done), the CTA barrier below orders that before
// every thread's later patch reads, and those read L2 (ld.global.cg), not L1.
template <int C>
__device__ __forceinline__ void wait_deps(const PieArgs& a, int s) {
  if (threadIdx.x < 32) {
    const int b = a.dep_off[s], e = a.dep_off[s + 1];
    bool ok = *reinterpret_cast<volatile int*>(a.gerr) == 0;
    for (int i = b + (int)threadIdx.x; ok && i < e; i += 32) {
      const unsigned* f = a.done + a.dep[i];
      unsigned long long t0, t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      for (unsigned spin = 1;; ++spin) {  // the error word is read every 16th poll only
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
        if (v >= (unsigned)C + a.dep_extra) break;
        if ((spin & 15u) == 0u && *reinterpret_cast<volatile int*>(a.gerr)) {
          ok = false;
          break;
        }
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 2000000000ull) {
          atomicExch(a.gerr, 1);
          if (a.gstatus) {
            *reinterpret_cast<volatile int*>(a.gstatus) = PFT_ERR_TIMEOUT;
            __threadfence_system();
          }
          ok = false;
          break;
        }
      }
    }
  }
  __syncthreads();
}

// Dataflow sweep: this CTA's part of item s's update is written. The CTA
// barrier orders every thread's stores before thread 0's release-add, and a
// release is cumulative, so a successor whose acquire load sees the count sees
// the whole update (one release-add costs less than a fence and a relaxed add).
__device__ __forceinline__ void signal_done(const PieArgs& a, int s) {
  __syncthreads();
  if (threadIdx.x == 0)
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(a.done + s), "r"(1u) : "memory");
}

// Modulus-projection residual (Eq. 3) and its contribution to the objective.
// The objective's partial sum is FP64 for the gradient (the loss itself) and
// FP32 per thread otherwise (at most a few dozen terms; warps add in FP32
// pairwise, and everything beyond a warp is summed in FP64).
template <int MODE>
using ResAcc = typename std::conditional<MODE == MODE_GRAD, double, float>::type;

template <int MODE>
__device__ __forceinline__ float2 residual(float2 Psi, float d, ResAcc<MODE>& acc) {
  // m2 != 0 rather than m2 > 0: the same for every finite m2 >= 0, but a NaN
  // coefficient takes the general branch and stays NaN (reported by the host)
  const float m2 = cabs2(Psi);
  if (MODE == MODE_GRAD) {
    // sgn(0) = 0; the gradient of sum (|Psi| - d)^2 is 2 R
    if (m2 != 0.f) {
      const float m = sqrtf(m2);
      const float diff = m - d;
      acc += (double)diff * (double)diff;
      return cscale(Psi, 2.f * diff / m);
    }
    acc += (double)d * (double)d;
    return make_float2(0.f, 0.f);
  }
  // theta(0) = 0: a zero coefficient is replaced by d
  float2 R;
  if (m2 != 0.f) {
    R = cscale(Psi, 1.f - d * rsqrtf(m2));
  } else {
    R = make_float2(-d, 0.f);
  }
  acc += cabs2(R);
  return R;
}

// The pointers of one work item: a position of the single instance, or an
// (instance, position) pair of a multi-instance sweep.
struct PieItem {
  float2* obj;
  const float2* objr;
  long long obj_w;
  const float2* probe;
  const float* dat;      // this position's amplitudes
  float coef;
  float2* acc;
  double* red;
  long long obase;       // offset of the patch's top-left pixel
};

template <int DAT>
__device__ __forceinline__ PieItem resolve(const PieArgs& a, int it) {
  PieItem r;
  if (a.inst) {
    const int2 w = a.work[it];
    const PieInstance& in = a.inst[w.x];
    const int2 rc = in.pos[w.y];
    r.obj = in.obj;
    r.objr = in.obj;
    r.obj_w = in.obj_w;
    r.probe = in.probe;
    r.dat = in.dat + (long long)w.y * DAT;
    r.coef = in.coef;
    r.acc = in.acc;
    r.red = in.red;
    r.obase = (long long)rc.x * in.obj_w + rc.y;
  } else {
    const int j = a.list ? a.list[it] : it;
    const int2 rc = a.pos[j];
    r.obj = a.obj;
    r.objr = a.objr;
    r.obj_w = a.obj_w;
    r.probe = a.probe;
    r.dat = a.dat + (long long)j * DAT;
    r.coef = a.pscale ? a.coef / *a.pscale : a.coef;
    r.acc = a.acc;
    r.red = a.red;
    r.obase = (long long)rc.x * a.obj_w + rc.y;
  }
  return r;
}

template <int MODE>
__device__ __forceinline__ void apply_update(const PieArgs& a, const PieItem& p, long long oidx, float2 w,
                                             float2 dpsi, int pidx) {
  if (MODE == MODE_COLOURED) {
    float2 o = __ldcg(p.obj + oidx);  // L2: a persistent sweep's other CTAs wrote it
    const float2 u = cmulc(dpsi, w);  // conj(w) dpsi
    o.x = fmaf(-p.coef, u.x, o.x);
    o.y = fmaf(-p.coef, u.y, o.y);
    p.obj[oidx] = o;
  } else if (MODE == MODE_BATCHED) {
    atomicAdd(p.acc + oidx, cscale(cmulc(dpsi, w), p.coef));
  } else {
    atomicAdd(p.acc + oidx, cmulc(dpsi, w));
    if (a.gprobe) atomicAdd(a.gprobe + pidx, cmulc(dpsi, p.objr[oidx]));
  }
}

// The same with the object value at oidx already in a register (read when the
// position started: no other work item writes the patch meanwhile).
template <int MODE>
__device__ __forceinline__ void apply_update_at(const PieArgs& a, const PieItem& p, long long oidx, float2 w,
                                                float2 zold, float2 dpsi, int pidx) {
  if (MODE == MODE_COLOURED) {
    const float2 u = cmulc(dpsi, w);  // conj(w) dpsi
    p.obj[oidx] = make_float2(fmaf(-p.coef, u.x, zold.x), fmaf(-p.coef, u.y, zold.y));
  } else if (MODE == MODE_BATCHED) {
    atomicAdd(p.acc + oidx, cscale(cmulc(dpsi, w), p.coef));
  } else {
    atomicAdd(p.acc + oidx, cmulc(dpsi, w));
    if (a.gprobe) atomicAdd(a.gprobe + pidx, cmulc(dpsi, zold));
  }
}

// Blind PIE, second round: accumulate conj(z_new) dpsi' and |z_new|^2 per probe pixel.
__device__ __forceinline__ void accumulate_probe(const PieArgs& a, const PieItem& p, long long oidx, float2 dpsi,
                                                 int pidx, float inv_n2) {
  const float2 zn = p.objr[oidx];
  atomicAdd(a.pacc + pidx, cscale(cmulc(dpsi, zn), inv_n2));
  atomicAdd(a.pden + pidx, cabs2(zn));
}

// The objective's partial sums: each warp writes its share to a shared-memory
// slot (no barrier), and thread 0 adds the slots to *out after the next
// block-wide barrier, off the path between projection and adjoint.
__device__ __forceinline__ void warp_partial(double v, double* red_smem) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red_smem[threadIdx.x >> 5] = v;
}
__device__ __forceinline__ void warp_partial(float v, double* red_smem) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red_smem[threadIdx.x >> 5] = (double)v;
}
template <int NW>
__device__ __forceinline__ void flush_partials(const double* red_smem, double* out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < NW; ++i) s += red_smem[i];
    if (s != 0.0) atomicAdd(out, s);
  }
}

// Resident CTAs per SM the kernels are compiled for (a register budget): a
// coloured sweep's cluster kernels need two per SM so that every position of a
// colour is on the GPU at once; the batched and gradient sweeps run two
// (three measured the same, with more spills). Shapes with more than 8 values
// per lane or frames above 128 keep the compiler's choice.
constexpr int pie_min_blocks(int mode, int C, int n, int q) {
  return (n > 128 || q > 8) ? 1 : mode == MODE_COLOURED ? (C >= 4 ? 2 : 1) : 2;
}

// ------------------------------------------------------------- PFT variant
template <int P, int Q, int MP, int C>
struct PiePftShape {
  static constexpr int N = P * Q, M = MP * P, G = 32 / P;
  static constexpr int RN = N / C;   // rows owned by one CTA
  static constexpr int CM = M / C;   // columns owned by one CTA
  // P = 8, Q >= 16: four 8-lane groups share each column transform, one column
  // per warp. Without it a warp runs G = 4 columns and a CTA needs CM % 4 == 0,
  // so the few columns of a small-M frame sit on one warp. With Q = 16 the
  // 8-CTA cluster (two columns per CTA) is still left out: its exchange costs
  // more than the column phase it shortens.
  static constexpr bool SPLIT4 = (P == 8) && (MP == 2) && (Q >= 16);
  static constexpr bool VALID = (N % C == 0) && (M % C == 0) && CM >= 1 && (RN % G == 0) &&
                                ((SPLIT4 && Q >= 32) || CM % G == 0) && (RN % Q == 0);
  // column slice of Y, all rows: element (t, u) at t * SYT + u + u / Q
  static constexpr int SYT_BASE = N + N / Q;
  static constexpr int SYT = SYT_BASE + (((8 - SYT_BASE % 16) + 16) % 16);
  static constexpr int ZS = CM + 1;  // Z: [M][CM + 1]
  static constexpr int SG = M + 8;   // G: [RN][M + 8]
  static constexpr int OFF_W1 = 0;
  static constexpr int OFF_W2 = OFF_W1 + RMAX * M;
  static constexpr int OFF_TW = OFF_W2 + RMAX * M;
  static constexpr int OFF_Y = OFF_TW + 32;
  static constexpr int Y_SIZE = CM * SYT;
  static constexpr int G_SIZE = RN * SG;
  static constexpr int OFF_G = (C == 1) ? OFF_Y : OFF_Y + Y_SIZE;  // alias for one CTA
  static constexpr int OFF_Z = (C == 1) ? OFF_Y + (Y_SIZE > G_SIZE ? Y_SIZE : G_SIZE) : OFF_G + G_SIZE;
  static constexpr int OFF_RED = OFF_Z + M * ZS;
  static constexpr int OFF_D = OFF_RED + 16;           // amplitudes of the CTA's columns: [M][CM] floats
  static constexpr int OFF_BH = OFF_D + (M * CM + 1) / 2;  // SPLIT4: axis-1 B rows 0 .. Q/2 [Q/2 + 1][RMAX] floats
  static constexpr int BH_SIZE = SPLIT4 ? ((Q / 2 + 1) * RMAX + 1) / 2 : 0;
  static constexpr size_t SMEM = sizeof(float2) * (OFF_BH + BH_SIZE);
};

// CLAIM: the variant whose clusters claim items from PieArgs::ticket (dataflow
// sweeps of several shape classes sharing the GPU); the others assign items
// statically, without the claim's registers.
template <int P, int Q, int MP, int MODE, int C, int NT, bool CLAIM = false>
__global__ void __launch_bounds__(NT, pie_min_blocks(MODE, C, P * Q, Q)) k_pie_pft(PieArgs a, const __grid_constant__ PftConst c,
                                                const float2* __restrict__ gW, const float2* __restrict__ gtw) {
  using S = PiePftShape<P, Q, MP, C>;
  using T = Pft1D<P, Q, MP>;
  using TS = Pft1DSplit<(P <= 16 ? P : 16), Q, MP>;
  using TS4 = Pft1DSplit4<Q, MP>;
  using CL = Cluster<C>;
  constexpr int N = S::N, M = S::M, G = S::G, RN = S::RN, CM = S::CM, NW = NT / 32;
  constexpr bool SPLIT4 = S::SPLIT4;
  // every cluster size of a shape splits (or none does), so all launch forms round alike
  constexpr bool SPLIT = (P == 16) && (MP == 2);
  extern __shared__ __align__(16) float2 sm[];
  float2* sW1 = sm + S::OFF_W1;
  float2* sW2 = sm + S::OFF_W2;
  float2* stw = sm + S::OFF_TW;
  float2* sY = sm + S::OFF_Y;
  float2* sG = sm + S::OFF_G;
  float2* sZ = sm + S::OFF_Z;
  double* sred = reinterpret_cast<double*>(sm + S::OFF_RED);
  float* sD = reinterpret_cast<float*>(sm + S::OFF_D);
  float* sBh = reinterpret_cast<float*>(sm + S::OFF_BH);
  if (!cluster_shape_ok<C>(a.gstatus)) return;
  const unsigned rank = CL::rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = lane % P, g = lane / P;
  const int r0 = rank * RN;
  if constexpr (SPLIT4)  // made visible by the cluster barrier before the first item
    for (int i = threadIdx.x; i < (Q / 2 + 1) * RMAX; i += NT) sBh[i] = c.bh[0][i / RMAX][i % RMAX];
  // With one row group per warp, the probe and patch values of the warp's rows
  // stay in registers from the exit wave to the update, and the next work
  // item's are loaded as soon as the current one is done.
  constexpr bool KEEP = (RN == NW * G);
  float2 wv[Q], zv[Q];
  auto gather_static = [&](const PieItem& q) {
    for (int i = threadIdx.x; i < M * CM; i += NT) cp_async4(sD + i, q.dat + rank * CM + (i / CM) * M + (i % CM));
    cp_async_commit();
    if constexpr (KEEP) {
      const int u = r0 + warp * G + g;
      const float2* src = q.probe + u * N + Q * k;
      if (Q % 2 == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
#pragma unroll
        for (int l = 0; l < Q; l += 2) {
          const float4 t = __ldg(reinterpret_cast<const float4*>(src + l));
          wv[l] = make_float2(t.x, t.y);
          wv[l + 1] = make_float2(t.z, t.w);
        }
      } else {
#pragma unroll
        for (int l = 0; l < Q; ++l) wv[l] = __ldg(src + l);
      }
    }
  };
  auto gather_obj = [&](const PieItem& q) {
    if constexpr (KEEP) {
      const int u = r0 + warp * G + g;
      const float2* src = q.objr + q.obase + (long long)u * q.obj_w + Q * k;
      // 16-byte loads where the lane's values allow (half the L1 wavefronts):
      // all of them from a 16-byte boundary, else the inner Q - 2
      if (Q % 2 == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
#pragma unroll
        for (int l = 0; l < Q; l += 2) {
          const float4 t = __ldcg(reinterpret_cast<const float4*>(src + l));
          zv[l] = make_float2(t.x, t.y);
          zv[l + 1] = make_float2(t.z, t.w);
        }
      } else if (Q % 2 == 0) {
        zv[0] = __ldcg(src);
#pragma unroll
        for (int l = 1; l + 1 < Q; l += 2) {
          const float4 t = __ldcg(reinterpret_cast<const float4*>(src + l));
          zv[l] = make_float2(t.x, t.y);
          zv[l + 1] = make_float2(t.z, t.w);
        }
        zv[Q - 1] = __ldcg(src + Q - 1);
      } else {
#pragma unroll
        for (int l = 0; l < Q; ++l) zv[l] = __ldcg(src + l);
      }
    }
  };
  const int step = gridDim.x / C;
  const bool persistent = MODE == MODE_COLOURED && a.ncol > 0;  // every colour in this launch
  const bool flow = persistent && a.dep_off != nullptr;         // per-item waits instead
  const bool dyn = CLAIM && flow && a.ticket != nullptr;        // items claimed in schedule order
  __shared__ int s_claim;
  const int ncol = persistent ? a.ncol : 1;
  int ce = persistent ? a.col_off[1] : a.count;
  int it = (persistent ? a.col_off[0] : 0) + (int)(blockIdx.x / C);
  for (int i = threadIdx.x; i < 2 * RMAX * M; i += NT) cp_async8(sm + i, gW + i);
  fill_stage_table_async<P>(stw, gtw, P);
  cp_async_commit();
  // exchange barriers: rows -> column owners (Y) and adjoint columns -> row owners (G)
  constexpr bool XCH = (C > 1) && !CLAIM;
  __shared__ __align__(8) unsigned long long s_xbar[2];
  const uint32_t barY = smem_addr(&s_xbar[0]), barG = smem_addr(&s_xbar[1]);
  uint32_t parY = 0, parG = 0;
  bool xabort = false;
  if constexpr (XCH) {
    if (threadIdx.x == 0) {
      xbar_init(barY);
      xbar_init(barG);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  if (dyn) {
    if (rank == 0 && threadIdx.x == 0) s_claim = (int)atomicAdd(a.ticket, 1u);
    CL::sync();
    it = *CL::map(&s_claim, 0u);
  }
  if (it < ce) {
    const PieItem q = resolve<M * M>(a, it);
    gather_static(q);
    if (flow) wait_deps<C>(a, it);
    gather_obj(q);
  } else {
    cp_async_commit();
  }
  cp_async_wait_group<1>();  // the tables (the first amplitudes may still be in flight)
  CL::sync();  // every CTA of the cluster has started before any remote store
  LaneNet<P, false> net;
  net.init(k, stw);
  const int rounds = (MODE == MODE_COLOURED && a.pacc) ? 2 : 1;
  for (int col = 0; col < ncol; ++col) {
  if (col > 0) {
    if (!grid_barrier(a.gbar, (unsigned)col * gridDim.x + a.bar_extra, a.gerr, a.gstatus)) {
      cp_async_wait_all();  // the next colour's prefetch lands before the CTA leaves
      break;
    }
    if (it < ce) gather_obj(resolve<M * M>(a, it));
  }
  while (it < ce) {
    int claimed = 0;  // the next item when items are claimed
    unsigned tk = 0;
    if (dyn && rank == 0 && threadIdx.x == 0) tk = atomicAdd(a.ticket, 1u);  // the next item, claimed early
    const PieItem p = resolve<M * M>(a, it);
    const long long obase = p.obase;
    for (int round = 0; round < rounds; ++round) {
    if (KEEP && round == 1) {  // the updated patch
      gather_static(p);
      gather_obj(p);
    }
    // 1. rows (axis 2) of the exit wave -> column owners
    for (int u0 = warp * G; u0 < RN; u0 += NW * G) {
      const int u = r0 + u0 + g;
      float2 xv[Q];
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        const int v = Q * k + l;
        if constexpr (KEEP)
          xv[l] = cmul(wv[l], zv[l]);
        else
          xv[l] = cmul(__ldg(p.probe + u * N + v), __ldcg(p.objr + obase + (long long)u * p.obj_w + v));
      }
      if constexpr (XCH) {
        const uint32_t ly = smem_addr(sY);
        T::forward(xv, k, c.bh[1], sW2, net, [&](int t, float2 val) {
          const uint32_t r = (uint32_t)(t / CM);
          st_async2(map_rank(ly + 8u * (uint32_t)((t % CM) * S::SYT + u + u / Q), r), val, map_rank(barY, r));
        });
      } else {
        T::forward(xv, k, c.bh[1], sW2, net, [&](int t, float2 val) {
          float2* dst = CL::map(sY, (unsigned)(t / CM));
          dst[(t % CM) * S::SYT + u + u / Q] = val;
        });
      }
    }
    if (dyn && round == 0 && rank == 0 && threadIdx.x == 0) s_claim = (int)tk;
    if constexpr (XCH) {
      if (threadIdx.x == 0) xbar_expect(barY, (uint32_t)(8 * N * CM));  // every row of this CTA's columns
      xbar_wait(barY, parY, a, xabort);
      parY ^= 1u;
    } else {
      CL::sync();
    }
    if (dyn && round == 0) claimed = *CL::map(&s_claim, 0u);
    cp_async_wait_all();
    __syncthreads();  // the amplitudes (fetched by every thread) are visible
    // 3a. columns (axis 1) of this CTA's slice (SPLIT: one column per warp,
    // its r terms split between the two 16-lane halves)
    if constexpr (SPLIT) {
      for (int tl = warp; tl < CM; tl += NW) {
        float2 xv[Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) xv[l] = sY[tl * S::SYT + Q * k + l + k];
        TS::forward(xv, k, g, c.bh[0], sW1, net, [&](int t1, float2 val) { sZ[t1 * S::ZS + tl] = val; });
      }
    } else if constexpr (SPLIT4) {
      for (int tl = warp; tl < CM; tl += NW) {
        float2 xv[Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) xv[l] = sY[tl * S::SYT + Q * k + l + k];
        TS4::forward(xv, k, g, sBh, sW1, net, [&](int t1, float2 val) { sZ[t1 * S::ZS + tl] = val; });
      }
    } else {
      for (int cs0 = warp * G; cs0 < CM; cs0 += NW * G) {
        const int tl = cs0 + g;
        float2 xv[Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) xv[l] = sY[tl * S::SYT + Q * k + l + k];
        T::forward(xv, k, c.bh[0], sW1, net, [&](int t1, float2 val) { sZ[t1 * S::ZS + tl] = val; });
      }
    }
    // 3b. the modulus projection is applied as 3c loads the coefficients: the
    // lane group that wrote a column in 3a reads it back, so a warp barrier
    // suffices; only the group that stored an output adds its residual to the
    // objective
    __syncwarp();
    ResAcc<MODE> part = 0, unused = 0;
    const int w1 = T::first_out(k);
    auto projected = [&](int t1, int tl) {
      const int cc = (t1 - w1) / P;
      const bool own = SPLIT ? (cc & 1) == g : SPLIT4 ? cc == g : true;
      return residual<MODE>(sZ[t1 * S::ZS + tl], sD[t1 * CM + tl], own ? part : unused);
    };
    // 3c. adjoint columns -> row owners (SPLIT: half g of the warp sends half
    // of each block; SPLIT4: group g computes and sends a quarter of it)
    if constexpr (SPLIT4) {
      for (int tl = warp; tl < CM; tl += NW) {
        float2 xq[Q / 4];
        TS4::adjoint([&](int t1) { return projected(t1, tl); }, k, g, sBh, sW1, net, xq);
        const int u0 = Q * k + g * (Q / 4);
        const int tg = rank * CM + tl;
        if constexpr (XCH) {
          const uint32_t r = (uint32_t)(u0 / RN);
          const uint32_t base = map_rank(smem_addr(sG), r), rb = map_rank(barG, r);
#pragma unroll
          for (int l = 0; l < Q / 4; ++l)
            st_async2(base + 8u * (uint32_t)((u0 % RN + l) * S::SG + tg), xq[l], rb);
        } else {
          float2* dst = CL::map(sG, (unsigned)(u0 / RN));
#pragma unroll
          for (int l = 0; l < Q / 4; ++l) dst[(u0 % RN + l) * S::SG + tg] = xq[l];
        }
      }
    } else
    for (int cs0 = (SPLIT ? warp : warp * G); cs0 < CM; cs0 += (SPLIT ? NW : NW * G)) {
      const int tl = SPLIT ? cs0 : cs0 + g;
      float2 xv[Q];
      if constexpr (SPLIT)
        TS::adjoint([&](int t1) { return projected(t1, tl); }, k, g, c.bh[0], sW1, net, xv);
      else
        T::adjoint([&](int t1) { return projected(t1, tl); }, k, c.bh[0], sW1, net, xv);
      const int u0 = Q * k;
      const int tg = rank * CM + tl;
      constexpr int L0 = SPLIT ? Q / 2 : Q;  // values each lane sends
      const int lb = SPLIT ? g * (Q / 2) : 0;
      float2 xs[L0];
#pragma unroll
      for (int l = 0; l < L0; ++l) xs[l] = (SPLIT && g) ? xv[(L0 + l) % Q] : xv[l];
      if constexpr (XCH) {
        const uint32_t r = (uint32_t)(u0 / RN);
        const uint32_t base = map_rank(smem_addr(sG), r), rb = map_rank(barG, r);
#pragma unroll
        for (int l = 0; l < L0; ++l)
          st_async2(base + 8u * (uint32_t)((u0 % RN + lb + l) * S::SG + tg), xs[l], rb);
      } else {
        float2* dst = CL::map(sG, (unsigned)(u0 / RN));
#pragma unroll
        for (int l = 0; l < L0; ++l) dst[(u0 % RN + lb + l) * S::SG + tg] = xs[l];
      }
    }
    warp_partial(round == 0 ? part : ResAcc<MODE>(0), sred);
    __syncthreads();  // the warps' partial sums, read by thread 0 below
    if constexpr (XCH) {
      if (threadIdx.x == 0) xbar_expect(barG, (uint32_t)(8 * RN * M));  // every column of this CTA's rows
      xbar_wait(barG, parG, a, xabort);
      parG ^= 1u;
    } else {
      CL::sync();
    }
    if (round == 0) flush_partials<NW>(sred, p.red);
    // 5. adjoint rows and the object update
    for (int u0 = warp * G; u0 < RN; u0 += NW * G) {
      const int ul = u0 + g, u = r0 + ul;
      float2 xv[Q];
      T::adjoint([&](int t) { return sG[ul * S::SG + t]; }, k, c.bh[1], sW2, net, xv);
      if (KEEP && MODE == MODE_COLOURED && round == 0 && Q % 2 == 0) {  // 16-byte stores, as the loads
        float2* dst = p.obj + obase + (long long)u * p.obj_w + Q * k;
        float2 zn[Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          const float2 d = cmulc(xv[l], wv[l]);  // conj(w) dpsi
          zn[l] = make_float2(fmaf(-p.coef, d.x, zv[l].x), fmaf(-p.coef, d.y, zv[l].y));
        }
        if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
          for (int l = 0; l < Q; l += 2)
            *reinterpret_cast<float4*>(dst + l) = make_float4(zn[l].x, zn[l].y, zn[l + 1].x, zn[l + 1].y);
        } else {
          dst[0] = zn[0];
#pragma unroll
          for (int l = 1; l + 1 < Q; l += 2)
            *reinterpret_cast<float4*>(dst + l) = make_float4(zn[l].x, zn[l].y, zn[l + 1].x, zn[l + 1].y);
          dst[Q - 1] = zn[Q - 1];
        }
        continue;
      }
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        const int v = Q * k + l;
        const long long oidx = obase + (long long)u * p.obj_w + v;
        if (round == 0) {
          if constexpr (KEEP)
            apply_update_at<MODE>(a, p, oidx, wv[l], zv[l], xv[l], u * N + v);
          else
            apply_update<MODE>(a, p, oidx, __ldg(p.probe + u * N + v), xv[l], u * N + v);
        } else {
          accumulate_probe(a, p, oidx, xv[l], u * N + v, 1.f / (float)(N * N));
        }
      }
    }
    if (rounds == 2 && round == 0) __syncthreads();  // updated patch visible to the second round
    }  // round
    if (flow) signal_done(a, it);
    const int nxt = dyn ? claimed : it + step;
    if (nxt < ce) {  // the next item of this colour
      const PieItem q = resolve<M * M>(a, nxt);
      gather_static(q);
      if (flow) wait_deps<C>(a, nxt);
      gather_obj(q);
    }
    if constexpr (C == 1) __syncthreads();
    it = nxt;
  }
  if (col + 1 < ncol) {  // the next colour's first item: all but the object before the barrier
    ce = a.col_off[col + 2];
    it = a.col_off[col + 1] + (int)(blockIdx.x / C);
    if (it < ce)
      gather_static(resolve<M * M>(a, it));
    else
      cp_async_commit();
  }
  }  // colour
}

// ------------------------------------------------------------ FFT variant
// Lanes per row of the full-FFT kernel: the default split (min(N, 32) lanes)
// unless fewer lanes with at most 8 values each let every warp own exactly one
// row group of the CTA's N / C rows (then the probe and patch values stay in
// registers from the exit wave to the update, and each phase is one pass).
template <int N, int C, int NT>
constexpr int pie_full_lanes() {
  const int L0 = N < 32 ? N : 32, NW = NT / 32, RN = N / C;
  if (RN < NW || RN % NW != 0) return L0;
  const int G = RN / NW;
  if (32 % G != 0) return L0;
  const int L = 32 / G;
  return (L <= L0 && L >= 2 && N % L == 0 && N / L <= 8) ? L : L0;
}

template <int N, int C, int NT = 256>
struct PieFullShape {
  using F = Fft<N, pie_full_lanes<N, C, NT>()>;
  static constexpr int RN = N / C, CN = N / C;
  static constexpr bool VALID = (N % C == 0) && RN >= 1 && (RN % F::G == 0) && (CN % F::G == 0);
  static constexpr int SCS = CN + 1;  // column slice: [N][CN + 1]
  static constexpr int SRS = N + 1;   // row slice: [RN][N + 1]
  static constexpr int OFF_TW = 0;
  static constexpr int OFF_C = F::TAB;
  static constexpr int OFF_R = (C == 1) ? OFF_C : OFF_C + N * SCS;  // alias for one CTA
  static constexpr int OFF_RED = (C == 1) ? OFF_C + N * SCS : OFF_R + RN * SRS;
  static constexpr int OFF_D = OFF_RED + 16;  // amplitudes of the CTA's slot columns: [N][CN] floats
  static constexpr size_t SMEM = sizeof(float2) * (OFF_D + (N * CN + 1) / 2);
  static constexpr bool FITS = SMEM <= 232448;  // 227 KB of shared memory per CTA
};

template <int N, int MODE, int C, int NT, bool CLAIM = false>
__global__ void __launch_bounds__(NT, pie_min_blocks(MODE, C, N, 1)) k_pie_full(PieArgs a, const float2* __restrict__ gtw) {
  using S = PieFullShape<N, C, NT>;
  using F = typename S::F;
  using CL = Cluster<C>;
  constexpr int L = F::L, E = F::E, G = F::G, RN = S::RN, CN = S::CN, NW = NT / 32;
  extern __shared__ __align__(16) float2 sm[];
  float2* tw = sm + S::OFF_TW;
  float2* sC = sm + S::OFF_C;
  float2* sR = sm + S::OFF_R;
  double* sred = reinterpret_cast<double*>(sm + S::OFF_RED);
  float* sD = reinterpret_cast<float*>(sm + S::OFF_D);
  if (!cluster_shape_ok<C>(a.gstatus)) return;
  const unsigned rank = CL::rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = lane % L, g = lane / L;
  const int r0 = rank * RN, c0 = rank * CN;
  // As in the PFT variant: with one row group per warp the probe and patch
  // values stay in registers from the exit wave to the update.
  constexpr bool KEEP = (RN == NW * G);
  float2 wv[E], zv[E];
  auto gather_static = [&](const PieItem& q) {
    for (int i = threadIdx.x; i < N * CN; i += NT)
      cp_async4(sD + i, q.dat + F::freq_of_slot(i / CN) * N + F::freq_of_slot(c0 + i % CN));
    cp_async_commit();
    if constexpr (KEEP) {
      const int u = r0 + warp * G + g;
#pragma unroll
      for (int e = 0; e < E; ++e) wv[e] = __ldg(q.probe + u * N + l + L * e);
    }
  };
  auto gather_obj = [&](const PieItem& q) {
    if constexpr (KEEP) {
      const int u = r0 + warp * G + g;
#pragma unroll
      for (int e = 0; e < E; ++e) zv[e] = __ldcg(q.objr + q.obase + (long long)u * q.obj_w + l + L * e);
    }
  };
  const int step = gridDim.x / C;
  const bool persistent = MODE == MODE_COLOURED && a.ncol > 0;  // every colour in this launch
  const bool flow = persistent && a.dep_off != nullptr;         // per-item waits instead
  const bool dyn = CLAIM && flow && a.ticket != nullptr;        // items claimed in schedule order
  __shared__ int s_claim;
  const int ncol = persistent ? a.ncol : 1;
  int ce = persistent ? a.col_off[1] : a.count;
  int it = (persistent ? a.col_off[0] : 0) + (int)(blockIdx.x / C);
  F::fill_async(tw, gtw);
  cp_async_commit();
  // exchange barriers: rows -> slot-column owners (C) and adjoint columns -> row owners (R)
  constexpr bool XCH = (C > 1) && !CLAIM;
  __shared__ __align__(8) unsigned long long s_xbar[2];
  const uint32_t barC = smem_addr(&s_xbar[0]), barR = smem_addr(&s_xbar[1]);
  uint32_t parC = 0, parR = 0;
  bool xabort = false;
  if constexpr (XCH) {
    if (threadIdx.x == 0) {
      xbar_init(barC);
      xbar_init(barR);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  if (dyn) {
    if (rank == 0 && threadIdx.x == 0) s_claim = (int)atomicAdd(a.ticket, 1u);
    CL::sync();
    it = *CL::map(&s_claim, 0u);
  }
  if (it < ce) {
    const PieItem q = resolve<N * N>(a, it);
    gather_static(q);
    if (flow) wait_deps<C>(a, it);
    gather_obj(q);
  } else {
    cp_async_commit();
  }
  cp_async_wait_group<1>();  // the tables (the first amplitudes may still be in flight)
  CL::sync();
  typename F::Net net;
  F::init_net(net, l, tw);
  const int rounds = (MODE == MODE_COLOURED && a.pacc) ? 2 : 1;
  for (int col = 0; col < ncol; ++col) {
  if (col > 0) {
    if (!grid_barrier(a.gbar, (unsigned)col * gridDim.x + a.bar_extra, a.gerr, a.gstatus)) {
      cp_async_wait_all();  // the next colour's prefetch lands before the CTA leaves
      break;
    }
    if (it < ce) gather_obj(resolve<N * N>(a, it));
  }
  while (it < ce) {
    int claimed = 0;  // the next item when items are claimed
    unsigned tk = 0;
    if (dyn && rank == 0 && threadIdx.x == 0) tk = atomicAdd(a.ticket, 1u);  // the next item, claimed early
    const PieItem p = resolve<N * N>(a, it);
    const long long obase = p.obase;
    for (int round = 0; round < rounds; ++round) {
    if (KEEP && round == 1) {  // the updated patch
      gather_static(p);
      gather_obj(p);
    }
    // 1. FFT of this CTA's rows of the exit wave -> column-slot owners
    for (int u0 = warp * G; u0 < RN; u0 += NW * G) {
      const int u = r0 + u0 + g;
      float2 x[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int v = l + L * e;
        if constexpr (KEEP)
          x[e] = cmul(wv[e], zv[e]);
        else
          x[e] = cmul(__ldg(p.probe + u * N + v), __ldcg(p.objr + obase + (long long)u * p.obj_w + v));
      }
      F::fwd(x, l, tw, net);
      if constexpr (XCH) {
        const uint32_t lc = smem_addr(sC);
#pragma unroll
        for (int p = 0; p < E; ++p) {
          const int s = p * L + l;
          const uint32_t r = (uint32_t)(s / CN);
          st_async2(map_rank(lc + 8u * (uint32_t)(u * S::SCS + s % CN), r), x[p], map_rank(barC, r));
        }
      } else {
#pragma unroll
        for (int p = 0; p < E; ++p) {
          const int s = p * L + l;
          CL::map(sC, (unsigned)(s / CN))[u * S::SCS + s % CN] = x[p];
        }
      }
    }
    if (dyn && round == 0 && rank == 0 && threadIdx.x == 0) s_claim = (int)tk;
    if constexpr (XCH) {
      if (threadIdx.x == 0) xbar_expect(barC, (uint32_t)(8 * N * CN));  // every row of this CTA's slot columns
      xbar_wait(barC, parC, a, xabort);
      parC ^= 1u;
    } else {
      CL::sync();
    }
    if (dyn && round == 0) claimed = *CL::map(&s_claim, 0u);
    ResAcc<MODE> part = 0;
    if constexpr (!CLAIM) {
      // 3a-c. per warp, on its own columns and in registers: FFT of the local
      // slot column (rows in natural order -> slot order), modulus projection,
      // adjoint FFT (natural row order) -> row owners. Lane l of column b holds
      // spectrum rows p L + l, whose amplitudes are sD[(p L + l) CN + b].
      cp_async_wait_all();
      __syncthreads();  // the amplitudes (fetched by every thread) are visible
      for (int b0 = warp * G; b0 < CN; b0 += NW * G) {
        const int b = b0 + g;
        float2 x[E];
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = sC[(l + L * e) * S::SCS + b];
        F::fwd(x, l, tw, net);
#pragma unroll
        for (int p = 0; p < E; ++p) x[p] = residual<MODE>(x[p], sD[(p * L + l) * CN + b], part);
        F::adj(x, l, tw, net);
        if constexpr (XCH) {
          const uint32_t lr = smem_addr(sR);
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int u = l + L * e;
            const uint32_t r = (uint32_t)(u / RN);
            st_async2(map_rank(lr + 8u * (uint32_t)((u % RN) * S::SRS + c0 + b), r), x[e], map_rank(barR, r));
          }
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int u = l + L * e;
            CL::map(sR, (unsigned)(u / RN))[(u % RN) * S::SRS + c0 + b] = x[e];
          }
        }
      }
      warp_partial(round == 0 ? part : ResAcc<MODE>(0), sred);
      __syncthreads();  // the warps' partial sums, read by thread 0 below
    } else {  // the claiming variants keep the shared-memory round trip (registers)
      // 3a. FFT of the local slot columns (rows in natural order -> slot order)
      for (int b0 = warp * G; b0 < CN; b0 += NW * G) {
        const int b = b0 + g;
        float2 x[E];
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = sC[(l + L * e) * S::SCS + b];
        F::fwd(x, l, tw, net);
#pragma unroll
        for (int p = 0; p < E; ++p) sC[(p * L + l) * S::SCS + b] = x[p];
      }
      cp_async_wait_all();
      __syncthreads();
      // 3b. modulus projection
      for (int i = threadIdx.x; i < N * CN; i += NT) {
        float2* z = sC + (i / CN) * S::SCS + (i % CN);
        *z = residual<MODE>(*z, sD[i], part);
      }
      warp_partial(round == 0 ? part : ResAcc<MODE>(0), sred);
      __syncthreads();
      // 3c. adjoint FFT of the local columns -> row owners (natural row order)
      for (int b0 = warp * G; b0 < CN; b0 += NW * G) {
        const int b = b0 + g;
        float2 x[E];
#pragma unroll
        for (int p = 0; p < E; ++p) x[p] = sC[(p * L + l) * S::SCS + b];
        F::adj(x, l, tw, net);
        if constexpr (XCH) {
          const uint32_t lr = smem_addr(sR);
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int u = l + L * e;
            const uint32_t r = (uint32_t)(u / RN);
            st_async2(map_rank(lr + 8u * (uint32_t)((u % RN) * S::SRS + c0 + b), r), x[e], map_rank(barR, r));
          }
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int u = l + L * e;
            CL::map(sR, (unsigned)(u / RN))[(u % RN) * S::SRS + c0 + b] = x[e];
          }
        }
      }
    }
    if constexpr (XCH) {
      if (threadIdx.x == 0) xbar_expect(barR, (uint32_t)(8 * RN * N));  // every column of this CTA's rows
      xbar_wait(barR, parR, a, xabort);
      parR ^= 1u;
    } else {
      CL::sync();
    }
    if (round == 0) flush_partials<NW>(sred, p.red);
    // 5. adjoint FFT of this CTA's rows and the object update
    for (int u0 = warp * G; u0 < RN; u0 += NW * G) {
      const int ul = u0 + g, u = r0 + ul;
      float2 x[E];
#pragma unroll
      for (int p = 0; p < E; ++p) x[p] = sR[ul * S::SRS + p * L + l];
      F::adj(x, l, tw, net);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int v = l + L * e;
        const long long oidx = obase + (long long)u * p.obj_w + v;
        if (round == 0) {
          if constexpr (KEEP)
            apply_update_at<MODE>(a, p, oidx, wv[e], zv[e], x[e], u * N + v);
          else
            apply_update<MODE>(a, p, oidx, __ldg(p.probe + u * N + v), x[e], u * N + v);
        } else {
          accumulate_probe(a, p, oidx, x[e], u * N + v, 1.f / (float)(N * N));
        }
      }
    }
    if (rounds == 2 && round == 0) __syncthreads();  // updated patch visible to the second round
    }  // round
    if (flow) signal_done(a, it);
    const int nxt = dyn ? claimed : it + step;
    if (nxt < ce) {  // the next item of this colour
      const PieItem q = resolve<N * N>(a, nxt);
      gather_static(q);
      if (flow) wait_deps<C>(a, nxt);
      gather_obj(q);
    }
    if constexpr (C == 1) __syncthreads();
    it = nxt;
  }
  if (col + 1 < ncol) {  // the next colour's first item: all but the object before the barrier
    ce = a.col_off[col + 2];
    it = a.col_off[col + 1] + (int)(blockIdx.x / C);
    if (it < ce)
      gather_static(resolve<N * N>(a, it));
    else
      cp_async_commit();
  }
  }  // colour
}

// ---------------------------------------------------------------- registry
struct PieKernel {
  const void* fn = nullptr;
  size_t smem = 0;
  int cluster = 1;
  int threads = 256;
};

}  // namespace pftk

namespace pfth {
// PIE kernels for a (transform, shape, mode, cluster size); fn == nullptr if not
// built. claim: the coloured-mode variant that claims items (built for 4 and 8
// CTAs per position).
pftk::PieKernel pie_pft_kernel(int P, int Q, int MP, int mode, int C, bool claim = false);
pftk::PieKernel pie_full_kernel(int N, int mode, int C, bool claim = false);
}  // namespace pfth
