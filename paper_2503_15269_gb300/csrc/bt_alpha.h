// Host-side checks and choices of the polynomial coefficients alpha of the
// a = 1 preconditioner M^-1 = (sum_j alpha_j H^j) G (Sec. 3.5).
//
// The eigenvalues of M^-1 S are q(h) (1 - h), q(h) = sum_j alpha_j h^j, over
// the eigenvalues h of H_opt, which lie in [0, 1) for every SPD
// block-tridiagonal S (Sec. 3.3).  So M^-1 is SPD for every such S exactly
// when q > 0 on [0, 1) -- with alpha_0 = 1 and q(1) > 0 required here, that
// is q > 0 on the closed [0, 1].  Every alpha_j >= 0 qualifies (Thm. 3.3's
// setting); so do the alternating Chebyshev coefficients below.
#pragma once
#include <cmath>
#include <vector>

namespace bt {

inline double poly_at(const std::vector<double>& c, double x) {
  double v = 0.0;
  for (size_t i = c.size(); i-- > 0;) v = v * x + c[i];
  return v;
}

inline void poly_trim(std::vector<double>& c, double tol) {
  while (!c.empty() && std::fabs(c.back()) <= tol) c.pop_back();
}

// Sign changes of a Sturm sequence at x (zeros skipped).
inline int sturm_changes(const std::vector<std::vector<double>>& seq, double x) {
  int ch = 0;
  double prev = 0.0;
  for (const auto& s : seq) {
    const double v = poly_at(s, x);
    if (v == 0.0) continue;
    if (prev != 0.0 && ((v > 0.0) != (prev > 0.0))) ++ch;
    prev = v;
  }
  return ch;
}

// true iff q(h) = sum_{j<m} alpha_j h^j > 0 on [0, 1]: q(0) > 0, q(1) > 0
// and no real root in (0, 1] (Sturm's theorem: the number of distinct roots
// in (0, 1] is V(0) - V(1) for the sequence q, q', -rem(...), ...).
inline bool alpha_positive_on_unit_interval(const double* alpha, int m) {
  std::vector<double> q(alpha, alpha + m);
  double scale = 0.0;
  for (double v : q) scale = std::fmax(scale, std::fabs(v));
  if (!(scale > 0.0) || !std::isfinite(scale)) return false;
  poly_trim(q, 0.0);
  if (poly_at(q, 0.0) <= 0.0 || poly_at(q, 1.0) <= 0.0) return false;
  if (q.size() <= 1) return true;
  std::vector<std::vector<double>> seq;
  seq.push_back(q);
  std::vector<double> d(q.size() - 1);
  for (size_t i = 1; i < q.size(); ++i) d[i - 1] = (double)i * q[i];
  poly_trim(d, 0.0);
  if (!d.empty()) seq.push_back(d);
  while (seq.size() >= 2 && seq.back().size() > 1) {
    std::vector<double> r = seq[seq.size() - 2];
    const std::vector<double>& b = seq.back();
    double rs = 0.0;
    for (double v : r) rs = std::fmax(rs, std::fabs(v));
    while (r.size() >= b.size()) {  // r <- r mod b
      const double f = r.back() / b.back();
      const size_t sh = r.size() - b.size();
      for (size_t i = 0; i < b.size(); ++i) r[sh + i] -= f * b[i];
      r.pop_back();
    }
    poly_trim(r, 1e-12 * rs);
    if (r.empty()) break;  // b is the gcd: the count of distinct roots stays exact
    for (double& v : r) v = -v;
    seq.push_back(r);
  }
  return sturm_changes(seq, 0.0) - sturm_changes(seq, 1.0) == 0;
}

// The Chebyshev (minimax) coefficients for rho(H_opt) <= rho: with
// x = (2h - rho)/rho, p(h) = T_m(x) / T_m((2 - rho)/rho) so that p(1) = 1,
// q(h) = (1 - p(h)) / (1 - h) (synthetic division by the root h = 1), then
// alpha = q / q(0).  T_m by the three-term recurrence in power-basis form.
inline bool alpha_chebyshev(int m, double rho, double* alpha) {
  if (m < 1 || !(rho > 0.0) || !(rho < 1.0)) return false;
  if (m == 1) {
    alpha[0] = 1.0;
    return true;
  }
  const std::vector<double> x = {-1.0, 2.0 / rho};
  std::vector<double> tp = {1.0}, t = x;
  for (int k = 1; k < m; ++k) {  // t_{k+1} = 2 x t_k - t_{k-1}
    std::vector<double> tn(t.size() + 1, 0.0);
    for (size_t i = 0; i < t.size(); ++i) {
      tn[i] += 2.0 * x[0] * t[i];
      tn[i + 1] += 2.0 * x[1] * t[i];
    }
    for (size_t i = 0; i < tp.size(); ++i) tn[i] -= tp[i];
    tp = t;
    t = tn;
  }
  const double t1 = poly_at(t, 1.0);
  // r(h) = p(h) - 1 = (h - 1) q(h): synthetic division of r by (h - 1)
  std::vector<double> r(t.size());
  for (size_t i = 0; i < t.size(); ++i) r[i] = t[i] / t1;
  r[0] -= 1.0;
  std::vector<double> q(r.size() - 1);
  double carry = 0.0;
  for (size_t k = r.size() - 1; k >= 1; --k) {
    carry = r[k] + carry;
    q[k - 1] = carry;
  }
  for (int j = 0; j < m; ++j) alpha[j] = q[j] / q[0];
  return true;
}

}  // namespace bt
