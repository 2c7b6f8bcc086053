// Kernel design for the planner (Sec. 3.2, App. A): the map error function l(x) of the
// modified ES kernel (Eq. semicircle2, Eq. maperror), its supremum over the retained part of
// the image |x| <= 1 / (2 sigma) -- the kernel's accuracy epsilon -- and the two-parameter
// search for the (beta, mu) that minimise it.  The paper prints the optimum for
// alpha in {4, 7, 8, 12, 16}; the search extends the planner's table to the other supports.
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "host_math.h"

namespace wg {

namespace {

// Double-exponential (tanh-sinh) quadrature on [-1, 1]: nodes s_i = tanh(pi/2 sinh t_i),
// t_i = i h; 1 - s_i^2 is formed as 1 / cosh^2(pi/2 sinh t_i), which stays exact next to the
// end points where the modified ES kernel has its (1 - s^2)^mu branch point.
struct DeNodes {
  std::vector<double> s, oms2, w;
};

DeNodes make_de_nodes(int level, double tmax) {
  DeNodes q;
  const double h = std::ldexp(1.0, -level);
  const int m = (int)std::ceil(tmax / h);
  for (int i = -m; i <= m; ++i) {
    const double t = i * h;
    const double a = 0.5 * M_PI * std::sinh(t);
    const double ch = std::cosh(a);
    const double oms2 = 1.0 / (ch * ch);
    const double w = h * 0.5 * M_PI * std::cosh(t) * oms2;
    if (w < 1e-300) continue;
    q.s.push_back(std::tanh(a));
    q.oms2.push_back(oms2);
    q.w.push_back(w);
  }
  return q;
}

const DeNodes& psi_nodes() {
  static const DeNodes q = make_de_nodes(7, 4.0);
  return q;
}
const DeNodes& nu_nodes() {
  static const DeNodes q = make_de_nodes(6, 3.5);
  return q;
}

// phi at x (cells) from (1 - (2x/alpha)^2), given directly where it is known exactly
inline double phi_of_oms2(int alpha, double beta, double mu, double oms2) {
  return std::exp(alpha * beta * (std::pow(oms2, mu) - 1.0));
}

}  // namespace

double es_psi(int alpha, double beta, double mu, double k) {
  // psi(k) = int_{-alpha/2}^{alpha/2} phi(t) cos(2 pi k t) dt with t = alpha s / 2
  const DeNodes& q = psi_nodes();
  long double acc = 0.0L;
  for (size_t i = 0; i < q.s.size(); ++i)
    acc += (long double)q.w[i] * phi_of_oms2(alpha, beta, mu, q.oms2[i]) *
           std::cos(M_PI * alpha * k * q.s[i]);
  return 0.5 * alpha * (double)acc;
}

double es_map_error(int alpha, double beta, double mu, double x) {
  // Eq. (maperror): l(x)^2 = int_0^1 |1 - sum_a phi(a - nu) e^{2 pi i (a - nu) x} / psi(x)|^2
  // d nu, a over the grid points, nu the visibility's fractional position.  The set of a with
  // |a - nu| < alpha / 2 changes where nu - alpha / 2 is an integer: at nu = 0 for even alpha,
  // nu = 1/2 for odd alpha, so the integral is taken piecewise between those points.
  const double ps = es_psi(alpha, beta, mu, x);
  const DeNodes& q = nu_nodes();
  const double half = 0.5 * alpha;
  std::array<double, 3> cuts = {0.0, 0.5, 1.0};
  const int npieces = (alpha % 2 == 0) ? 1 : 2;
  long double tot = 0.0L;
  for (int p = 0; p < npieces; ++p) {
    const double a0 = npieces == 1 ? 0.0 : cuts[p], a1 = npieces == 1 ? 1.0 : cuts[p + 1];
    const double mid = 0.5 * (a0 + a1), hw = 0.5 * (a1 - a0);
    const int jlo = (int)std::ceil(mid - half), jhi = (int)std::floor(mid + half);
    for (size_t i = 0; i < q.s.size(); ++i) {
      const double nu = mid + hw * q.s[i];
      double sr = 0.0, si = 0.0;
      for (int j = jlo; j <= jhi; ++j) {
        const double d = j - nu;                 // |d| < alpha / 2 inside the piece
        const double r = 2.0 * d / alpha;
        const double f = phi_of_oms2(alpha, beta, mu, std::max(0.0, 1.0 - r * r));
        const double ang = 2.0 * M_PI * d * x;
        sr += f * std::cos(ang);
        si += f * std::sin(ang);
      }
      const double er = 1.0 - sr / ps, ei = -si / ps;
      tot += (long double)(hw * q.w[i]) * (er * er + ei * ei);
    }
  }
  return std::sqrt((double)tot);
}

double es_kernel_eps(int alpha, double beta, double mu, double sigma) {
  // sup of l(x) over 0 <= x <= 1 / (2 sigma) (l is even): a scan, then a golden-section
  // refinement around every local maximum of the scan (end samples included) -- the search
  // below would otherwise shape the kernel so that a lobe's peak falls between scan points.
  // The lobes of l narrow towards the edge of the range (to ~0.5 % of it for alpha = 14 at
  // sigma = 1.15), so the scan takes 144 steps over the first 90 % and 144 over the last 10 %.
  const double xmax = 0.5 / sigma;
  std::vector<double> xs, v;
  const int n1 = 144, n2 = 144;
  for (int i = 0; i < n1; ++i) xs.push_back(0.9 * xmax * i / n1);
  for (int i = 0; i <= n2; ++i) xs.push_back(xmax * (0.9 + 0.1 * i / n2));
  for (double x : xs) v.push_back(es_map_error(alpha, beta, mu, x));
  const int n = (int)xs.size() - 1;
  double best = *std::max_element(v.begin(), v.end());
  const double g = 0.5 * (std::sqrt(5.0) - 1.0);
  for (int i = 0; i <= n; ++i) {
    const bool peak = (i == 0 || v[i] >= v[i - 1]) && (i == n || v[i] >= v[i + 1]);
    if (!peak) continue;
    // the lobe's top lies within a step of the sample -- on the inner side only for an end
    // sample, where the peak may sit just inside the interval
    double a = xs[std::max(0, i - 1)], b = xs[std::min(n, i + 1)];
    double c = b - g * (b - a), d = a + g * (b - a);
    double fc = es_map_error(alpha, beta, mu, c), fd = es_map_error(alpha, beta, mu, d);
    for (int it = 0; it < 12; ++it) {
      if (fc > fd) { b = d; d = c; fd = fc; c = b - g * (b - a); fc = es_map_error(alpha, beta, mu, c); }
      else { a = c; c = d; fc = fd; d = a + g * (b - a); fd = es_map_error(alpha, beta, mu, d); }
    }
    best = std::max(best, std::max(fc, fd));
  }
  return best;
}

namespace {

// One Nelder-Mead run on f from a simplex of steps (0.04 beta0, 0.02) around (beta0, mu0);
// returns the best vertex and its value.
template <typename F>
std::array<double, 3> nelder_mead(F&& f, double beta0, double mu0) {
  std::array<std::array<double, 2>, 3> x = {{{beta0, mu0}, {beta0 * 1.04, mu0}, {beta0, mu0 + 0.02}}};
  std::array<double, 3> fx;
  for (int i = 0; i < 3; ++i) fx[i] = f(x[i][0], x[i][1]);
  for (int it = 0; it < 160; ++it) {
    int o[3] = {0, 1, 2};
    std::sort(o, o + 3, [&](int p, int q) { return fx[p] < fx[q]; });
    const int lo = o[0], md = o[1], hi = o[2];
    const double size = std::fabs(x[hi][0] - x[lo][0]) + std::fabs(x[hi][1] - x[lo][1]) +
                        std::fabs(x[md][0] - x[lo][0]) + std::fabs(x[md][1] - x[lo][1]);
    if (size < 2e-6 || fx[hi] - fx[lo] < 1e-6) break;
    const double cx = 0.5 * (x[lo][0] + x[md][0]), cy = 0.5 * (x[lo][1] + x[md][1]);
    const double rx = cx + (cx - x[hi][0]), ry = cy + (cy - x[hi][1]);
    const double fr = f(rx, ry);
    if (fr < fx[lo]) {
      const double ex = cx + 2.0 * (cx - x[hi][0]), ey = cy + 2.0 * (cy - x[hi][1]);
      const double fe = f(ex, ey);
      if (fe < fr) { x[hi] = {ex, ey}; fx[hi] = fe; }
      else { x[hi] = {rx, ry}; fx[hi] = fr; }
    } else if (fr < fx[md]) {
      x[hi] = {rx, ry}; fx[hi] = fr;
    } else {
      const bool outside = fr < fx[hi];
      const double kx = outside ? cx + 0.5 * (rx - cx) : cx + 0.5 * (x[hi][0] - cx);
      const double ky = outside ? cy + 0.5 * (ry - cy) : cy + 0.5 * (x[hi][1] - cy);
      const double fk = f(kx, ky);
      if (fk < std::min(fr, fx[hi])) {
        x[hi] = {kx, ky}; fx[hi] = fk;
      } else {   // shrink towards the best point
        for (int i : {md, hi}) {
          x[i] = {x[lo][0] + 0.5 * (x[i][0] - x[lo][0]), x[lo][1] + 0.5 * (x[i][1] - x[lo][1])};
          fx[i] = f(x[i][0], x[i][1]);
        }
      }
    }
  }
  int b = 0;
  for (int i = 1; i < 3; ++i)
    if (fx[i] < fx[b]) b = i;
  return {x[b][0], x[b][1], fx[b]};
}

}  // namespace

KernelRow kernel_search(int alpha, double sigma, double beta0, double mu0) {
  // Sec. 3.2: minimise the supremum norm of the map error over (beta, mu) -- Nelder-Mead on
  // log(epsilon) from (beta0, mu0), with beta > 0 and mu in (0.2, 1.5).  The supremum is a
  // maximum over the map error's lobes, so the objective has kinks where two lobes are equal
  // and a simplex can stall on one: the run is restarted from its best point, with a fresh
  // simplex, until a restart gains less than 0.1 %.
  auto f = [&](double b, double m) {
    if (!(b > 0.05) || !(m > 0.2) || !(m < 1.5)) return 1e3;
    return std::log(es_kernel_eps(alpha, b, m, sigma));
  };
  std::array<double, 3> best = nelder_mead(f, beta0, mu0);
  for (int restart = 0; restart < 6; ++restart) {
    std::array<double, 3> r = nelder_mead(f, best[0], best[1]);
    const bool gain = r[2] < best[2] - 1e-3;
    if (r[2] < best[2]) best = r;
    if (!gain) break;
  }
  KernelRow r;
  r.alpha = alpha; r.sigma = sigma; r.beta = best[0]; r.mu = best[1]; r.eps = std::exp(best[2]);
  return r;
}

}  // namespace wg
