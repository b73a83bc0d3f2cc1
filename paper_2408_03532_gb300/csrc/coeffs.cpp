// Offline phase of the PFT, host side: the polynomial P(x) = sum_j w_j x^j
// approximating e^{i pi x} on |x| <= xi, and the scope xi(eps, r)
// (Section 3.1.1 of the paper; used by Algorithm 1 / Algorithm 4).
//
// e^{i pi x} = cos(pi x) + i sin(pi x) with cos even and sin odd, and the best
// approximation inherits the symmetry, w_j = i^j a_j with a_j real. This file
// designs the even part (a polynomial in x^2 for cos) and the odd part (x times
// a polynomial in x^2 for sin) each by the Remez exchange algorithm (the
// classical minimax algorithm), and measures the complex error
// |C(x) - cos(pi x) + i (S(x) - sin(pi x))| on a dense grid. xi(eps, r) is found
// by bisection on that error. Double precision throughout; the basis is scaled
// to [0, 1] so the linear systems stay well conditioned for r <= 32.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "coeffs.h"

namespace pftc {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kGrid = 4001;

// Solve A x = b (n x n, row-major) by Gaussian elimination with partial pivoting.
bool solve(std::vector<double>& A, std::vector<double>& b, int n) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      if (f == 0.0) continue;
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    double s = b[c];
    for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * b[k];
    b[c] = s / A[c * n + c];
  }
  return true;
}

// One real minimax problem on s in [0, 1] (s = x / X):
//   f(s) = cos(pi X s) with basis s^{2i}      (odd == false), or
//   f(s) = sin(pi X s) with basis s^{2i+1}    (odd == true),
// i < m. Returns the coefficients in s and the levelled error.
struct Remez {
  double X;
  int m;
  bool odd;

  double f(double s) const { return odd ? std::sin(kPi * X * s) : std::cos(kPi * X * s); }
  double basis(int i, double s) const { return std::pow(s, odd ? 2 * i + 1 : 2 * i); }
  double eval(const std::vector<double>& c, double s) const {
    // Horner in s^2
    double s2 = s * s, acc = 0.0;
    for (int i = m - 1; i >= 0; --i) acc = acc * s2 + c[i];
    return odd ? acc * s : acc;
  }
  double err(const std::vector<double>& c, double s) const { return f(s) - eval(c, s); }

  std::vector<double> run() const {
    std::vector<double> c(m, 0.0);
    if (m == 0) return c;
    // initial reference: m + 1 Chebyshev-like points in [0, 1] (in (0, 1] when odd)
    std::vector<double> ref(m + 1);
    for (int k = 0; k <= m; ++k) {
      double t = odd ? kPi * (k + 1) / (m + 1) : kPi * k / m;
      ref[k] = 0.5 * (1.0 - std::cos(t));
    }
    std::vector<double> grid(kGrid);
    for (int g = 0; g < kGrid; ++g)
      grid[g] = 0.5 * (1.0 - std::cos(kPi * g / (kGrid - 1)));
    std::vector<double> best_c(m, 0.0);
    double best_err = 1e300;
    for (int it = 0; it < 60; ++it) {
      // level: sum_i c_i phi_i(s_k) + (-1)^k E = f(s_k)
      int n = m + 1;
      std::vector<double> A(n * n), b(n);
      for (int k = 0; k < n; ++k) {
        for (int i = 0; i < m; ++i) A[k * n + i] = basis(i, ref[k]);
        A[k * n + m] = (k % 2 == 0) ? 1.0 : -1.0;
        b[k] = f(ref[k]);
      }
      if (!solve(A, b, n)) break;
      for (int i = 0; i < m; ++i) c[i] = b[i];
      double E = std::fabs(b[m]);
      double emax_grid = 0.0;
      for (int g2 = 0; g2 < kGrid; ++g2) emax_grid = std::max(emax_grid, std::fabs(err(c, grid[g2])));
      if (emax_grid < best_err) { best_err = emax_grid; best_c = c; }
      // once the error is at the rounding level the exchange only sees noise
      if (emax_grid < 1e-14) break;
      // alternating extrema of the error on the grid: one per run of equal sign
      std::vector<double> ext;
      std::vector<double> extv;
      int g = odd ? 1 : 0;
      while (g < kGrid) {
        double e = err(c, grid[g]);
        int sgn = e >= 0 ? 1 : -1;
        double best = std::fabs(e), bs = grid[g];
        int h = g + 1;
        while (h < kGrid) {
          double eh = err(c, grid[h]);
          if ((eh >= 0 ? 1 : -1) != sgn) break;
          if (std::fabs(eh) > best) { best = std::fabs(eh); bs = grid[h]; }
          ++h;
        }
        ext.push_back(bs);
        extv.push_back(sgn * best);
        g = h;
      }
      if ((int)ext.size() < n) break;  // degenerate: keep the current levelled solution
      // keep n consecutive alternating extrema containing the largest one
      int imax = 0;
      for (int k = 1; k < (int)ext.size(); ++k)
        if (std::fabs(extv[k]) > std::fabs(extv[imax])) imax = k;
      int start = std::min(std::max(imax - n / 2, 0), (int)ext.size() - n);
      // slide the window so it keeps the largest total error
      double bestsum = -1.0;
      int beststart = start;
      for (int s0 = std::max(0, imax - n + 1); s0 <= std::min(imax, (int)ext.size() - n); ++s0) {
        double sum = 0.0;
        for (int k = 0; k < n; ++k) sum += std::fabs(extv[s0 + k]);
        if (sum > bestsum) { bestsum = sum; beststart = s0; }
      }
      start = beststart;
      double emax = std::fabs(extv[imax]);
      for (int k = 0; k < n; ++k) ref[k] = ext[start + k];
      if (emax <= E * (1.0 + 1e-10)) break;
    }
    return best_c;
  }
};

struct Design {
  double xi = 0.0, err = 0.0;
  std::vector<double> a;  // w_j = i^j a_j
};

// Complex polynomial for a given X and r; fills a_j and returns the error.
double design_at(double X, int r, std::vector<double>& a) {
  int me = (r + 1) / 2, mo = r / 2;
  Remez ev{X, me, false}, od{X, mo, true};
  std::vector<double> ce = ev.run(), co = od.run();
  a.assign(r, 0.0);
  // C(x) = sum_i ce_i (x/X)^{2i};  S(x) = sum_i co_i (x/X)^{2i+1}
  // w_{2i} = ce_i / X^{2i}, w_{2i+1} = i * co_i / X^{2i+1};  a_j = w_j / i^j
  for (int i = 0; i < me; ++i) {
    double w = ce[i] / std::pow(X, 2 * i);
    a[2 * i] = (i % 2 == 0) ? w : -w;  // i^{2i} = (-1)^i
  }
  for (int i = 0; i < mo; ++i) {
    double w = co[i] / std::pow(X, 2 * i + 1);  // imaginary part of w_{2i+1}
    a[2 * i + 1] = (i % 2 == 0) ? w : -w;       // i^{2i+1} = i (-1)^i
  }
  // complex error on a dense grid of [0, X] (the modulus is even in x)
  double emax = 0.0;
  for (int g = 0; g < kGrid; ++g) {
    double s = 0.5 * (1.0 - std::cos(kPi * g / (kGrid - 1)));
    double em = std::fabs(ev.err(ce, s)), eo = (mo ? std::fabs(od.err(co, s)) : std::fabs(std::sin(kPi * X * s)));
    emax = std::max(emax, std::hypot(em, eo));
  }
  for (int g = 0; g < kGrid; ++g) {  // uniform grid as well
    double s = (double)g / (kGrid - 1);
    double em = std::fabs(ev.err(ce, s)), eo = (mo ? std::fabs(od.err(co, s)) : std::fabs(std::sin(kPi * X * s)));
    emax = std::max(emax, std::hypot(em, eo));
  }
  return emax;
}

std::mutex g_mu;
std::map<std::pair<double, int>, Design> g_cache;

}  // namespace

double design_error(double X, int r) {
  std::vector<double> a;
  return design_at(X, r, a);
}

bool design(double eps, int r, double* xi, double* a, double* err) {
  if (!(eps > 0.0 && eps < 1.0) || r < 1 || r > kMaxTerms) return false;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find({eps, r});
    if (it != g_cache.end()) {
      *xi = it->second.xi;
      if (err) *err = it->second.err;
      for (int j = 0; j < r; ++j) a[j] = it->second.a[j];
      return true;
    }
  }
  // bracket: the error grows with X
  std::vector<double> tmp;
  double lo = 1e-9, hi = 1e-9;
  if (design_at(lo, r, tmp) > eps) return false;
  while (design_at(hi, r, tmp) <= eps) {
    lo = hi;
    hi *= 2.0;
    if (hi > 64.0) return false;
  }
  for (int it = 0; it < 80 && hi / lo > 1.0 + 1e-9; ++it) {
    double mid = std::sqrt(lo * hi);
    if (design_at(mid, r, tmp) <= eps) lo = mid; else hi = mid;
  }
  Design d;
  d.xi = lo;
  d.err = design_at(lo, r, d.a);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[{eps, r}] = d;
  }
  *xi = d.xi;
  if (err) *err = d.err;
  for (int j = 0; j < r; ++j) a[j] = d.a[j];
  return true;
}

int choose_r(double eps, double ratio) {
  if (!(eps > 0.0 && eps < 1.0) || !(ratio > 0.0)) return -1;
  for (int r = 1; r <= kMaxTerms; ++r)
    if (design_error(ratio, r) <= eps) return r;
  return -1;
}

}  // namespace pftc
