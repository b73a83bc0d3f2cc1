// Internal plan object shared by the transform and PIE translation units.
#pragma once

#include "pft_core.cuh"

struct pft_plan {
  int n1, n2, M1, M2, p1, p2, q1, q2, r1, r2;
  double xi1, xi2, eps;
  int path, precision;
  pftk::PftConst cst;     // B rows for both axes (kernel parameter space)
  float2* d_W = nullptr;  // W' of axis 1 ([RMAX][M1]) then axis 2 ([RMAX][M2]), j-major (FP32 from FP64)
  float2* d_twp = nullptr;  // [2][32] : e^{-2 pi i m / p_axis}, m < p_axis / 2 (axis 2 at +32)
  float* d_B = nullptr;     // B of axis 1 ([q1][RMAX]) then axis 2 ([q2][RMAX]) (inspection only)
  int kid = -1;             // index in the frame-kernel registry
  void* d_tc = nullptr;     // split-BF16 tensor-core table (MMA operand layout)
  void* d_tc_adj = nullptr; // its adjoint table conj(A)^T
  int* h_status = nullptr;  // device-side wait status (mapped host word)
  int* d_status = nullptr;
  bool lf = false;          // large-frame path (pft_lf.cu)
  int lf_chunk = 0;         // frames per pass of the large-frame path
  void* d_ws = nullptr;     // its workspace
};

namespace pfth {

// Frame kernels built for one pair of 1-D shapes: (P1, Q1, M1/P1) along axis 1
// (columns, length n1) and (P2, Q2, M2/P2) along axis 2 (rows, length n2).
struct FrameKernels {
  int P1, Q1, MP1, P2, Q2, MP2;
  const void* fwd;
  const void* adj;
  size_t smem;
};
int frame_kernel_count();
const FrameKernels* frame_kernels(int id);
int find_frame_kernels(int P1, int Q1, int MP1, int P2, int Q2, int MP2);

// Builds a square plan's tables; used by pft_plan_create and the PIE context.
int build_plan(pft_plan* p, int n, int M, int P, double eps, int r_force);
int build_plan2(pft_plan* p, int n1, int n2, int M1, int M2, int P1, int P2, double eps, int r1, int r2);

// Split-BF16 tensor-core path (pft_tc.cu).
bool tc_supported(int n, int M, int p);
int tc_build_tables(pft_plan* plan);
int tc_forward(const pft_plan* plan, const void* x, void* y, int64_t batch, void* stream);
int tc_build_adjoint_table(pft_plan* plan, const double* d_a);
int tc64_build_tables(pft_plan* plan);
int tc64_forward(const pft_plan* plan, const void* x, void* y, int64_t batch, void* stream);
int tc64_build_adjoint_table(pft_plan* plan);
int tc64_adjoint(const pft_plan* plan, const void* y, void* x, int64_t batch, void* stream);
int tc_adjoint(const pft_plan* plan, const void* y, void* x, int64_t batch, void* stream);

// Large frames, n in {2048, 4096, 8192} with M = 128 (pft_lf.cu).
bool lf_supported(int n, int M, int p);
int lf_build(pft_plan* plan);
int lf_forward(const pft_plan* plan, const void* x, void* y, int64_t batch, void* stream);
int lf_adjoint(const pft_plan* plan, const void* y, void* x, int64_t batch, void* stream);

}  // namespace pfth
