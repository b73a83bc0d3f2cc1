// Host-side design of the PFT polynomial (Section 3.1.1 of the paper).
#pragma once

namespace pftc {

constexpr int kMaxTerms = 32;

// xi(eps, r) and a_0..a_{r-1} with w_j = i^j a_j; err = uniform error at xi.
bool design(double eps, int r, double* xi, double* a, double* err);

// Uniform error of the designed polynomial with r terms on |x| <= X.
double design_error(double X, int r);

// The choice of r in Algorithm 1: min{ r : xi(eps, r) >= ratio }, or -1.
int choose_r(double eps, double ratio);

}  // namespace pftc
