// Host-side FP64 numerics of the Leja path: the point table and the Newton
// coefficients.  Cited passages are from Deka, Moriggl, Einkemmer, "LeXInt:
// GPU-accelerated exponential integrators package" (arXiv 2310.08344).
//
//  * Leja points on [-2, 2] (Sec. 2.1, recursive definition of the Leja
//    sequence; the paper precomputes them).  Greedy maximisation of
//    prod_k |x - xi_k|, xi_0 = +2, near-ties (1e-12 relative in the
//    log-product) broken toward the larger point.
//  * Newton coefficients d_j = f[xi_0..xi_j] of f(xi) = phi_l(h (c + gamma xi))
//    (Sec. 2.1, Eq. 2), by Opitz' theorem: they form the first column of
//    f(Z) for the lower-bidiagonal matrix Z with the nodes on the diagonal.
//    phi_l is reduced to exp by prepending l zero nodes in z = h(c + gamma xi)
//    (phi_l[z_0..z_j] = exp[0,..,0, z_0..z_j]), and the sub-diagonal carries
//    h*gamma between the z-nodes so the entries come out already scaled to
//    the xi variable.  exp(Z) e_0 is formed by a shift, s Taylor sub-steps of
//    length 1/s, and the shift undone (McCurdy, Ng and Parlett 1984; Caliari
//    2007 for the use with Leja interpolation).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "lexgb_internal.h"

namespace lexgb {

namespace {

// Log-product and its derivative at x for the nodes xi[0..j).
inline void log_product_and_slope(const double* xi, int j, double x, double* lp, double* g, double* gp) {
  double s = 0.0, t = 0.0, u = 0.0;
  for (int k = 0; k < j; ++k) {
    double r = x - xi[k];
    s += std::log(std::fabs(r));
    double q = 1.0 / r;
    t += q;
    u += q * q;
  }
  if (lp) *lp = s;
  if (g) *g = t;
  if (gp) *gp = -u;
}

// Maximiser of sum_k log|x - xi_k| on the open interval (a, b) between two
// neighbouring nodes, starting from x0 inside it: the slope
// g(x) = sum_k 1/(x - xi_k) decreases strictly from +inf to -inf there, so a
// bracketed Newton iteration on g = 0 converges to the unique maximiser.
double refine_in_interval(const double* xi, int j, double a, double b, double x0) {
  double lo = a, hi = b, x = x0;
  for (int it = 0; it < 200; ++it) {
    double g, gp;
    log_product_and_slope(xi, j, x, nullptr, &g, &gp);
    if (g == 0.0) return x;
    if (g > 0.0) lo = x; else hi = x;
    double step = g / gp;
    double xn = x - step;
    if (!(xn > lo && xn < hi)) xn = lo + 0.5 * (hi - lo);
    if (std::fabs(xn - x) <= 1e-16 * std::max(1.0, std::fabs(x))) return xn;
    x = xn;
  }
  return x;
}

struct LejaTable {
  std::mutex mu;
  std::vector<double> pts;
};

LejaTable& table() {
  static LejaTable t;
  return t;
}

void compute_leja(int K, std::vector<double>& out) {
  out.assign(std::max(K, 0), 0.0);
  if (K <= 0) return;
  out[0] = 2.0;
  if (K == 1) return;
  out[1] = -2.0;  // |x - 2| is largest at the far end of [-2, 2]
  if (K == 2) return;
  // Candidate grid with arcsine density (like the Leja points themselves).
  const int M = 200000;
  std::vector<double> cand(M), val(M);
  for (int i = 0; i < M; ++i) cand[i] = 2.0 * std::cos(M_PI * (i + 0.5) / M);
  for (int i = 0; i < M; ++i) val[i] = std::fabs(cand[i] - 2.0) * std::fabs(cand[i] + 2.0);
  std::vector<double> sorted;
  sorted.reserve(K);
  sorted.push_back(-2.0);
  sorted.push_back(2.0);
  std::vector<std::pair<double, double>> refined;  // (x, log-product)
  for (int j = 2; j < K; ++j) {
    double vmax = 0.0;
    for (int i = 0; i < M; ++i) vmax = std::max(vmax, val[i]);
    // Every node interval that holds a candidate within 0.1% of the grid
    // maximum is refined exactly and the best refined point wins.  With at
    // least ~100 arcsine-spaced candidates per interval the grid value of an
    // interval's maximum is within ~1e-4 of the true one, so the interval of
    // the true maximiser is always among those refined.
    refined.clear();
    int last_iv = -1;
    for (int i = M - 1; i >= 0; --i) {  // ascending x
      if (val[i] < 0.999 * vmax) continue;
      double x = cand[i];
      int iv = int(std::upper_bound(sorted.begin(), sorted.end(), x) - sorted.begin()) - 1;
      if (iv < 0 || iv + 1 >= (int)sorted.size() || iv == last_iv) continue;
      last_iv = iv;
      double xr = refine_in_interval(out.data(), j, sorted[iv], sorted[iv + 1], x);
      double lp;
      log_product_and_slope(out.data(), j, xr, &lp, nullptr, nullptr);
      refined.emplace_back(xr, lp);
    }
    double best = -INFINITY;
    for (auto& r : refined) best = std::max(best, r.second);
    double tie = 1e-12 * std::max(1.0, std::fabs(best));
    double pick = -INFINITY;
    for (auto& r : refined)
      if (r.second >= best - tie) pick = std::max(pick, r.first);
    out[j] = pick;
    sorted.insert(std::upper_bound(sorted.begin(), sorted.end(), pick), pick);
    double nmax = 0.0;
    for (int i = 0; i < M; ++i) {
      val[i] *= std::fabs(cand[i] - pick);
      nmax = std::max(nmax, val[i]);
    }
    double inv = nmax > 0 ? 1.0 / nmax : 1.0;
    for (int i = 0; i < M; ++i) val[i] *= inv;
  }
}

}  // namespace

int leja_points(int K, double* xi) {
  if (K <= 0 || !xi) return LX_E_INVAL;
  LejaTable& t = table();
  std::lock_guard<std::mutex> lock(t.mu);
  if ((int)t.pts.size() < K) compute_leja(K, t.pts);
  std::copy(t.pts.begin(), t.pts.begin() + K, xi);
  return LX_OK;
}

int leja_coeff_count(double h, double c, double gamma, int K) {
  // |d_j| <= (h|gamma|)^j / j! * e^{max(0, h(c + 2|gamma|))}: the mean-value
  // form of the divided difference with |phi_l^{(j)}(z)| <= e^{max(z,0)}.
  // The Newton basis has norm O(1) per step only for a spectrum on the
  // focal interval (capacity 1); where the spectrum reaches off the real
  // axis (advection-dominated grids) it grows geometrically, so the bound is
  // taken with twice h|gamma|: coefficients beyond the first J with
  // (2 h|gamma|)^J / J! * e^{...} below 1e-40 are negligible for any
  // tolerance; the loop cap is J.
  double hg = 2.0 * std::fabs(h * gamma);
  double zplus = std::max(0.0, h * (c + 2.0 * std::fabs(gamma)));
  double logb = zplus;
  int J = 1;
  for (; J < K; ++J) {
    logb += std::log(hg) - std::log((double)J);
    if (J >= 32 && logb < std::log(1e-40)) break;
  }
  return std::min(K, J + 8);
}

int leja_coeffs_ws(int l, double h, double c, double gamma, const double* xi, int K, double* d, double* ws) {
  if (l < 0 || K <= 0 || !xi || !d || !(gamma != 0.0) || !std::isfinite(h * c) || !std::isfinite(h * gamma))
    return LX_E_INVAL;
  const int n = l + K;
  // Z: diagonal (0 x l, z_0..z_{K-1}); sub-diagonal 1 on the first l links,
  // h*gamma afterwards.  Shift by mu (mid-range of the diagonal).
  // workspace: diag, sub, v, term, nxt, acc (6 n doubles)
  double* diag = ws;
  double* sub = ws + n;
  double* v = ws + 2 * n;
  double* term = ws + 3 * n;
  double* nxt = ws + 4 * n;
  double* acc = ws + 5 * n;
  for (int i = 0; i < n; ++i) sub[i] = 0.0;
  double zmin = 0.0, zmax = 0.0;
  for (int i = 0; i < l; ++i) diag[i] = 0.0;
  for (int j = 0; j < K; ++j) {
    double z = h * (c + gamma * xi[j]);
    diag[l + j] = z;
    zmin = std::min(zmin, z);
    zmax = std::max(zmax, z);
  }
  for (int i = 1; i < n; ++i) sub[i] = (i <= l) ? 1.0 : h * gamma;
  const double mu = 0.5 * (zmin + zmax);
  double norm1 = 0.0;
  for (int i = 0; i < n; ++i) {
    diag[i] -= mu;
    norm1 = std::max(norm1, std::fabs(diag[i]) + (i + 1 < n ? std::fabs(sub[i + 1]) : 0.0));
  }
  const double theta = 2.0;  // sub-step norm: ~22 Taylor terms reach 1e-18
  int s = std::max(1, (int)std::ceil(norm1 / theta));
  const double inv_s = 1.0 / s;
  // e^{mu} is applied a 1/s slice per sub-step, so v stays at the size of
  // exp(t Z) e_0 for every t and never overflows.
  const double emu_step = std::exp(mu * inv_s);
  for (int i = 0; i < n; ++i) v[i] = 0.0;
  v[0] = 1.0;
  for (int step = 0; step < s; ++step) {
    for (int i = 0; i < n; ++i) term[i] = acc[i] = v[i];
    for (int k = 1; k < 60; ++k) {
      double tmax = 0.0, amax = 0.0;
      const double f = inv_s / k;
      nxt[0] = diag[0] * term[0] * f;
      for (int i = 1; i < n; ++i) nxt[i] = (diag[i] * term[i] + sub[i] * term[i - 1]) * f;
      for (int i = 0; i < n; ++i) {
        acc[i] += nxt[i];
        tmax = std::max(tmax, std::fabs(nxt[i]));
        amax = std::max(amax, std::fabs(acc[i]));
      }
      std::swap(term, nxt);
      if (tmax <= 1e-18 * amax) break;
    }
    for (int i = 0; i < n; ++i) acc[i] *= emu_step;
    std::swap(v, acc);
  }
  for (int j = 0; j < K; ++j) d[j] = v[l + j];
  // The first coefficient is phi_l(z_0); at z_0 = 0 (xi_0 = 2 on the interval
  // [c - 2 gamma, 0]) it is exactly 1/l!.
  if (h * (c + gamma * xi[0]) == 0.0) {
    double f = 1.0;
    for (int k = 2; k <= l; ++k) f *= k;
    d[0] = 1.0 / f;
  }
  for (int j = 0; j < K; ++j)
    if (!std::isfinite(d[j])) return LX_E_NONFINITE;
  return LX_OK;
}

int leja_coeffs(int l, double h, double c, double gamma, const double* xi, int K, double* d) {
  if (l < 0 || K <= 0) return LX_E_INVAL;
  std::vector<double> ws(6 * (size_t)(l + K));
  return leja_coeffs_ws(l, h, c, gamma, xi, K, d, ws.data());
}

}  // namespace lexgb

extern "C" {

lx_status lx_leja_points(int K, double* xi_out) { return (lx_status)lexgb::leja_points(K, xi_out); }

lx_status lx_leja_coeffs(int l, double h, double c, double gamma, const double* xi, int K, double* d_out) {
  return (lx_status)lexgb::leja_coeffs(l, h, c, gamma, xi, K, d_out);
}

int lx_leja_coeff_count(double h, double c, double gamma, int K) { return lexgb::leja_coeff_count(h, c, gamma, K); }

// The focal interval from a spectral-radius estimate (Sec. 2.2, Listing 7's
// time loop): the eigenvalue bound lambda = -1.05 rho sets the interval
// [lambda, 0] = [c - 2 gamma, c + 2 gamma], i.e. c = lambda / 2 and
// gamma = -lambda / 4.
lx_status lx_spectral_interval(double rho, double* c, double* gamma) {
  if (!c || !gamma || !std::isfinite(rho) || !(rho > 0.0)) return LX_E_INVAL;
  const double lambda = -1.05 * rho;
  *c = lambda / 2.0;
  *gamma = -lambda / 4.0;
  return LX_OK;
}

}  // extern "C"
