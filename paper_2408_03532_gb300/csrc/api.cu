// Error state, version and the host-only coefficient entry points.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "coeffs.h"
#include "common.cuh"

namespace pfth {

static thread_local char g_msg[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return set_error(PFT_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(PFT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int sm_count() {
  static int count = 0;
  if (count == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      count = 1;
  }
  return count;
}

}  // namespace pfth

extern "C" {

const char* pft_last_error(void) { return pfth::g_msg; }

int pft_version(void) { return 10000; }

int pft_design_coefficients(double eps, int r, double* xi, double* a, double* err) {
  if (!xi || !a) return pfth::set_error(PFT_ERR_INVALID_ARG, "xi and a must not be NULL");
  if (!(eps > 0.0 && eps < 1.0) || r < 1 || r > pftc::kMaxTerms)
    return pfth::set_error(PFT_ERR_INVALID_ARG, "need 0 < eps < 1 and 1 <= r <= %d", pftc::kMaxTerms);
  if (!pftc::design(eps, r, xi, a, err))
    return pfth::set_error(PFT_ERR_INVALID_ARG, "no scope found for eps=%g r=%d", eps, r);
  pfth::g_msg[0] = 0;
  return PFT_OK;
}

int pft_choose_r(double eps, double ratio, int* r) {
  if (!r) return pfth::set_error(PFT_ERR_INVALID_ARG, "r must not be NULL");
  if (!(eps > 0.0 && eps < 1.0) || !(ratio > 0.0))
    return pfth::set_error(PFT_ERR_INVALID_ARG, "need 0 < eps < 1 and ratio > 0");
  int v = pftc::choose_r(eps, ratio);
  if (v < 0) return pfth::set_error(PFT_ERR_INVALID_ARG, "no r <= %d reaches eps=%g at ratio %g",
                                    pftc::kMaxTerms, eps, ratio);
  *r = v;
  return PFT_OK;
}

}  // extern "C"
