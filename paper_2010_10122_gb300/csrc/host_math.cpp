// Host-side kernel mathematics and planner (FP64).  See host_math.h.
#include "host_math.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>

namespace wg {

const std::vector<KernelRow>& kernel_table() {
  // App. A, "Optimal parameters for alpha = 4 / 7 / 8 / 12 / 16": sigma, epsilon, beta, mu as
  // printed (the alpha = 12 table has no sigma = 1.85 row).
  static const std::vector<KernelRow> rows = {
      // alpha = 4
      {4, 1.15, 0.025654879, 1.3873426689, 0.5436851297},
      {4, 1.2, 0.013809249, 1.3008419165, 0.5902137484},
      {4, 1.25, 0.0085840685, 1.3274088935, 0.5953499486},
      {4, 1.3, 0.0057322498, 1.3617063353, 0.5965631622},
      {4, 1.35, 0.0042494419, 1.384549988, 0.5990241291},
      {4, 1.4, 0.0033459552, 1.4405325088, 0.5924776015},
      {4, 1.45, 0.0028187359, 1.4635220066, 0.5929442711},
      {4, 1.5, 0.0023843943, 1.5539689162, 0.5772217314},
      {4, 1.55, 0.0020343796, 1.5991008653, 0.5721765215},
      {4, 1.6, 0.0017143851, 1.6581546365, 0.5644747137},
      {4, 1.65, 0.0014730848, 1.7135331415, 0.5572788589},
      {4, 1.7, 0.0012554492, 1.7464330378, 0.5548742415},
      {4, 1.75, 0.0010610904, 1.7887326906, 0.5509877716},
      {4, 1.8, 0.00090885567, 1.8122309426, 0.5502273972},
      {4, 1.85, 0.0007757401, 1.8304451327, 0.550396716},
      {4, 1.9, 0.0006740398, 1.8484487383, 0.5502376937},
      {4, 1.95, 0.00058655391, 1.8742215688, 0.5489738941},
      {4, 2.0, 0.00051911189, 1.90694363, 0.5468009434},
      // alpha = 7
      {7, 1.15, 0.00078476028, 1.5248706519, 0.5288306317},
      {7, 1.2, 0.00027127166, 1.5739348793, 0.5287992619},
      {7, 1.25, 0.00012594628, 1.6245240723, 0.527921777},
      {7, 1.3, 7.0214545e-05, 1.6835745981, 0.5257484101},
      {7, 1.35, 4.1972457e-05, 1.7343424414, 0.5239793844},
      {7, 1.4, 2.378019e-05, 1.7845017738, 0.5224266045},
      {7, 1.45, 1.3863408e-05, 1.8180597789, 0.5221834768},
      {7, 1.5, 9.1605353e-06, 1.868082272, 0.5206277502},
      {7, 1.55, 6.479159e-06, 1.9188980015, 0.5183134674},
      {7, 1.6, 4.6544571e-06, 1.9536166143, 0.5178695891},
      {7, 1.65, 3.5489761e-06, 1.9786267068, 0.5178430252},
      {7, 1.7, 2.7030348e-06, 2.0027666534, 0.5178577604},
      {7, 1.75, 2.0533894e-06, 2.0289949199, 0.5176300336},
      {7, 1.8, 1.6069122e-06, 2.0596412946, 0.5167551932},
      {7, 1.85, 1.2936794e-06, 2.0720606842, 0.5178747891},
      {7, 1.9, 1.0768664e-06, 2.090898174, 0.5181009847},
      {7, 1.95, 9.0890421e-07, 2.1086185697, 0.5184537843},
      {7, 2.0, 7.7488775e-07, 2.1278284187, 0.5186377792},
      // alpha = 8
      {8, 1.15, 0.00026818611, 1.568124649, 0.5223052481},
      {8, 1.2, 7.8028732e-05, 1.620926145, 0.5219287175},
      {8, 1.25, 2.7460918e-05, 1.6851585171, 0.519925059},
      {8, 1.3, 1.3421658e-05, 1.7442373315, 0.5182155619},
      {8, 1.35, 7.5158217e-06, 1.7876782642, 0.5176319503},
      {8, 1.4, 4.2472384e-06, 1.8294321912, 0.5171860211},
      {8, 1.45, 2.5794802e-06, 1.871691821, 0.5161733611},
      {8, 1.5, 1.6131994e-06, 1.9213040541, 0.5145350888},
      {8, 1.55, 1.0974814e-06, 1.9637229131, 0.5134005827},
      {8, 1.6, 7.531955e-07, 2.0002761373, 0.5128849282},
      {8, 1.65, 5.5097346e-07, 2.0275645736, 0.5127082324},
      {8, 1.7, 4.0136726e-07, 2.0498410409, 0.5130237662},
      {8, 1.75, 2.906467e-07, 2.073158517, 0.5131757153},
      {8, 1.8, 2.1834922e-07, 2.0907418726, 0.5136046561},
      {8, 1.85, 1.6329905e-07, 2.1164552354, 0.5133333878},
      {8, 1.9, 1.2828598e-07, 2.126157016, 0.5143004427},
      {8, 1.95, 1.0171134e-07, 2.1363206613, 0.515235491},
      {8, 2.0, 8.1881369e-08, 2.1397013368, 0.5166895497},
      // alpha = 12
      {12, 1.15, 2.7535895e-06, 1.6661837519, 0.5098172147},
      {12, 1.2, 5.2570038e-07, 1.7294557459, 0.5089239596},
      {12, 1.25, 1.378658e-07, 1.7698182384, 0.5099240718},
      {12, 1.3, 4.4329167e-08, 1.8092042442, 0.510607427},
      {12, 1.35, 1.7038991e-08, 1.8619112597, 0.5093832337},
      {12, 1.4, 6.5438748e-09, 1.9069147481, 0.5089479889},
      {12, 1.45, 2.9874764e-09, 1.9318398074, 0.5098082325},
      {12, 1.5, 1.4920459e-09, 1.9628483155, 0.5100985753},
      {12, 1.55, 8.0989276e-10, 2.0129847811, 0.5085327805},
      {12, 1.6, 4.1660575e-10, 2.0517921747, 0.5079102398},
      {12, 1.65, 2.3539727e-10, 2.06983884, 0.5085131064},
      {12, 1.7, 1.3497289e-10, 2.0887365361, 0.5090417146},
      {12, 1.75, 8.3256938e-11, 2.106955733, 0.5095920671},
      {12, 1.8, 5.8834619e-11, 2.1359415217, 0.5091887069},
      {12, 1.9, 2.6412908e-11, 2.2006369514, 0.5075889699},
      {12, 1.95, 1.7189689e-11, 2.2146741638, 0.5080017404},
      {12, 2.0, 1.2174796e-11, 2.2431392199, 0.5075191177},
      // alpha = 16
      {16, 1.3, 1.1509596e-10, 1.7892839755, 0.5122877693},
      {16, 1.35, 3.2440049e-11, 1.8914441282, 0.5063521839},
      {16, 1.4, 8.4329616e-12, 1.9296369098, 0.5065170208},
      {16, 1.45, 3.1161739e-12, 1.9674735425, 0.5063244338},
      {16, 1.5, 1.2100308e-12, 2.0130787701, 0.5055587965},
      {16, 1.55, 4.6082202e-13, 2.0438032614, 0.5056309683},
      {16, 1.6, 1.7883238e-13, 2.0329561822, 0.5089045671},
      {16, 1.65, 9.2853815e-14, 2.0494514743, 0.5103582604},
      {16, 1.7, 5.6614567e-14, 2.0925119791, 0.5083767402},
      {16, 1.75, 2.875391e-14, 2.1461524027, 0.5062037834},
      {16, 1.8, 1.6578982e-14, 2.1490040175, 0.508272183},
      {16, 1.85, 1.1782751e-14, 2.1811826814, 0.5072570059},
      {16, 1.9, 8.9196865e-15, 2.1981176583, 0.5075840871},
      {16, 1.95, 6.6530006e-15, 2.234001135, 0.5060133105},
      {16, 2.0, 5.0563492e-15, 2.2621631913, 0.5056924675},
  };
  return rows;
}

const std::vector<KernelRow>& kernel_table_design() {
  static const std::vector<KernelRow> rows = {
#include "kernel_table_design.inc"
  };
  return rows;
}

double es_phi(int alpha, double beta, double mu, double x) {
  double s = 2.0 * x / alpha;
  if (std::fabs(s) > 1.0) return 0.0;
  return std::exp(alpha * beta * (std::pow(1.0 - s * s, mu) - 1.0));
}

double PolyKernel::eval_piece(int i, double z) const {
  const double* ci = &c[(size_t)i * (deg + 1)];
  double r = ci[deg];
  for (int d = deg - 1; d >= 0; --d) r = r * z + ci[d];
  return r;
}

double PolyKernel::eval(double x) const {
  double t = x + 0.5 * alpha;  // position from the left support edge, in cells
  if (t < 0.0 || t > alpha) return 0.0;
  int i = std::min((int)std::floor(t), alpha - 1);
  double z = 2.0 * (t - i) - 1.0;
  return eval_piece(i, z);
}

PolyKernel make_poly_kernel(int alpha, double beta, double mu, int deg) {
  // Sec. 4.2: each of the alpha unit pieces is interpolated at the deg + 1 roots of the
  // Chebyshev polynomial T_{deg+1}.  The interpolant is formed as a Chebyshev series
  // (discrete orthogonality at the roots) and converted to monomials in z with the
  // three-term recurrence T_{n+1} = 2 z T_n - T_{n-1}, accumulated in long double.
  PolyKernel K;
  K.alpha = alpha; K.deg = deg; K.beta = beta; K.mu = mu;
  const int np = deg + 1;
  K.c.assign((size_t)alpha * np, 0.0);
  std::vector<double> zq(np), fq(np);
  for (int q = 0; q < np; ++q) zq[q] = std::cos(M_PI * (q + 0.5) / np);
  // monomial coefficients of T_0 .. T_deg
  std::vector<std::vector<long double>> T(np, std::vector<long double>(np, 0.0L));
  T[0][0] = 1.0L;
  if (np > 1) T[1][1] = 1.0L;
  for (int n = 1; n + 1 < np; ++n)
    for (int d = 0; d < np; ++d) {
      long double v = -T[n - 1][d];
      if (d > 0) v += 2.0L * T[n][d - 1];
      T[n + 1][d] = v;
    }
  for (int i = 0; i < alpha; ++i) {
    for (int q = 0; q < np; ++q) {
      double x = -0.5 * alpha + i + 0.5 * (zq[q] + 1.0);
      fq[q] = es_phi(alpha, beta, mu, x);
    }
    std::vector<long double> mono(np, 0.0L);
    for (int n = 0; n < np; ++n) {
      long double a = 0.0L;
      for (int q = 0; q < np; ++q) a += (long double)fq[q] * std::cos(M_PI * n * (q + 0.5) / np);
      a *= 2.0L / np;
      if (n == 0) a *= 0.5L;
      for (int d = 0; d < np; ++d) mono[d] += a * T[n][d];
    }
    for (int d = 0; d < np; ++d) K.c[(size_t)i * np + d] = (double)mono[d];
  }
  return K;
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  // Newton iteration on P_n from the Chebyshev-like initial guesses.
  x.assign(n, 0.0); w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      // p1 = P_n(z), p0 = P_{n-1}(z)
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1; p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

double psi_poly(const PolyKernel& K, double k) {
  // int_{-alpha/2}^{alpha/2} phi(x) cos(2 pi k x) dx, piece by piece; on a piece the
  // integrand is a polynomial of degree deg times a cosine with at most half a turn,
  // so 32 Gauss-Legendre nodes integrate it to rounding level.
  static thread_local std::vector<double> gx, gw;
  if (gx.empty()) gauss_legendre(32, gx, gw);
  long double sum = 0.0L;
  for (int i = 0; i < K.alpha; ++i) {
    double x0 = -0.5 * K.alpha + i + 0.5;  // piece centre
    for (size_t q = 0; q < gx.size(); ++q) {
      double z = gx[q];
      double x = x0 + 0.5 * z;
      sum += (long double)(0.5 * gw[q]) * K.eval_piece(i, z) * std::cos(2.0 * M_PI * k * x);
    }
  }
  return (double)sum;
}

std::vector<double> psi_cheb_coeffs(const PolyKernel& K, int m) {
  // psi is even, so expand g(y) = psi(k) with y = 8 k^2 - 1 in [-1, 1] for |k| <= 1/2:
  // Chebyshev interpolation at the m roots of T_m.
  std::vector<double> c(m, 0.0), g(m);
  for (int q = 0; q < m; ++q) {
    double y = std::cos(M_PI * (q + 0.5) / m);
    double k = std::sqrt((y + 1.0) / 8.0);
    g[q] = psi_poly(K, k);
  }
  for (int n = 0; n < m; ++n) {
    long double a = 0.0L;
    for (int q = 0; q < m; ++q) a += (long double)g[q] * std::cos(M_PI * n * (q + 0.5) / m);
    a *= 2.0L / m;
    if (n == 0) a *= 0.5L;
    c[n] = (double)a;
  }
  return c;
}

double psi_cheb_eval(const std::vector<double>& c, double k) {
  double y = 8.0 * k * k - 1.0;
  double b1 = 0.0, b2 = 0.0;
  for (int n = (int)c.size() - 1; n >= 1; --n) {
    double b0 = 2.0 * y * b1 - b2 + c[n];
    b2 = b1; b1 = b0;
  }
  return y * b1 - b2 + c[0];
}

static bool seven_smooth(int64_t n) {
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

int64_t good_size(int64_t n, int64_t mult) {
  int64_t q = std::max<int64_t>(1, (n + mult - 1) / mult);
  while (!seven_smooth(q)) ++q;
  return q * mult;
}

bool df64_line_plan(int64_t n, Df64LinePlan* lp) {
  if (n < 2 || n > kDf64MaxSide) return false;
  int k = 0;
  int64_t m = n;
  int p2 = 0;
  while (m % 2 == 0) { m /= 2; ++p2; }
  if (p2 == 1) {
    lp->radix[k++] = 2;
  } else {
    int e8 = p2 / 3, rem = p2 % 3;
    if (rem == 1) --e8;                  // 2^(3q+1) = 8^(q-1) * 4 * 4 (q >= 1 since p2 >= 4)
    for (int i = 0; i < e8; ++i) lp->radix[k++] = 8;
    if (rem == 1) { lp->radix[k++] = 4; lp->radix[k++] = 4; }
    if (rem == 2) lp->radix[k++] = 4;
  }
  for (int p : {5, 3, 7, 11})
    while (m % p == 0 && k < 24) { lp->radix[k++] = p; m /= p; }
  if (m != 1) return false;
  lp->nst = k;
  lp->threads = (int)std::max<int64_t>(64, (n / 8 + 31) / 32 * 32);
  return lp->threads <= 832;
}

int df64_line_split(int64_t n) {
  Df64LinePlan lp;
  if (n <= kDf64MaxSide) {
    // above 2048 points a line runs as two halves on a cluster of 2 CTAs when the half needs
    // only the common radices 8, 4, 5, 3 (measured on GB300, ms per plane, one CTA -> two:
    // 3456 0.736 -> 0.709, 4096 1.30 -> 1.00, 6400 3.41 -> 3.03; gridding error at alpha 16,
    // sigma 1.6 over 256 pixels and three plans 4.4-5.4e-13 -> 3.1-3.4e-13); a half that needs
    // the generic radices 7, 11 or a radix 2 keeps one CTA per line (2816: 0.79 -> 0.87)
    if (n > 2048 && n % 2 == 0 && df64_line_plan(n / 2, &lp)) {
      bool common = true;
      for (int i = 0; i < lp.nst; ++i)
        if (lp.radix[i] == 2 || lp.radix[i] == 7 || lp.radix[i] == 11) common = false;
      if (common) return 2;
    }
    return df64_line_plan(n, &lp) ? 1 : 0;
  }
  if (n > kDf64MaxSplitSide) return 0;
  for (int s : {2, 4})
    if (n % s == 0 && n / s <= kDf64MaxSide) return df64_line_plan(n / s, &lp) ? s : 0;
  return 0;
}

bool df64_side_ok(int64_t n) { return df64_line_split(n) != 0; }

// The FP32 plane FFT's sides: 1, 2, 4 or 8 CTAs per line with at most kF32MaxPart points per
// CTA, each part with prime factors 2, 3, 5, 7, 11 only.
bool f32_side_ok(int64_t n) {
  if (n < 2 || n > kF32MaxSide) return false;
  auto smooth = [](int64_t m) {
    if (m < 2) return false;
    for (int p : {2, 3, 5, 7, 11})
      while (m % p == 0) m /= p;
    return m == 1;
  };
  for (int s : {1, 2, 4, 8})
    if (n % s == 0 && n / s <= kF32MaxPart && smooth(n / s)) return true;
  return false;
}

double rounding_gain(const PolyKernel& K, const std::vector<double>& psi_c, int64_t nx,
                     int64_t ny, double psx, double psy, int64_t nu, int64_t nv, int do_w,
                     double nshift, double dw) {
  // int phi^2 over the support, Gauss-Legendre per piece (the integrand is a polynomial)
  static thread_local std::vector<double> gx, gw;
  if (gx.empty()) gauss_legendre(32, gx, gw);
  long double phi2 = 0.0L;
  for (int i = 0; i < K.alpha; ++i)
    for (size_t q = 0; q < gx.size(); ++q) {
      double v = K.eval_piece(i, gx[q]);
      phi2 += (long double)(0.5 * gw[q]) * v * v;
    }
  // rms of the correction over a midpoint lattice of pixels
  const int su = (int)std::min<int64_t>(nx, 64), sv = (int)std::min<int64_t>(ny, 64);
  std::vector<double> jx(su), jy(sv), iu(su), iv(sv);
  for (int a = 0; a < su; ++a) {
    jx[a] = -0.5 * nx + (a + 0.5) * (double)nx / su;
    iu[a] = 1.0 / psi_cheb_eval(psi_c, jx[a] / nu);
  }
  for (int b = 0; b < sv; ++b) {
    jy[b] = -0.5 * ny + (b + 0.5) * (double)ny / sv;
    iv[b] = 1.0 / psi_cheb_eval(psi_c, jy[b] / nv);
  }
  long double acc = 0.0L;
  for (int a = 0; a < su; ++a)
    for (int b = 0; b < sv; ++b) {
      double l = jx[a] * psx, m = jy[b] * psy;
      double r2 = l * l + m * m;
      double n = std::sqrt(std::max(0.0, 1.0 - r2));
      double c = iu[a] * iv[b] / n;
      if (do_w) {
        double nm1 = -r2 / (1.0 + n);
        c /= psi_cheb_eval(psi_c, (nm1 - nshift) * dw);
      }
      acc += (long double)c * c;
    }
  double rms = std::sqrt((double)(acc / ((long double)su * sv)));
  return rms * std::pow((double)phi2, do_w ? 1.5 : 1.0);
}

double plane_rounding(int kind, int prec, int64_t nu, int64_t nv) {
  // unit roundoff of the plane arithmetic; the caller multiplies by the rounding gain
  double u = kind == kFftDf64 ? 0x1p-47 : (prec ? 0x1p-53 : 0x1p-24);   // kFftF32: FP32
  return u * std::log2((double)nu * (double)nv);
}

// Coefficient of the rounding term at rounding gain G.  Measured on GB300 (2048^2 image, 1e6
// visibilities, alpha 16, double-float planes): the degrid error added (4.0 - 6.1)e-15 x G over
// sigma 1.5 - 2.0 (G 880 - 2.7), i.e. c = 0.024 - 0.037; the gridded image's error over the
// whole image (a stratified pixel sample weighting the edge band, where the correction
// amplifies the rounding most) varies from plan to plan (the summation order inside a bin
// differs) and reached c = 0.043 at G 290, 0.081 at G 880 and 0.062 at G 1600.  The spread
// widens with G, so the coefficient does: 0.065 (1 + G / 2000).
double rounding_coefficient(double gain) { return 0.065 * (1.0 + gain / 2000.0); }

// Measured plane-transform times on GB300, written by calibrate_fft.py: batched cuFFT 2-D C2C
// and Z2Z, the library's double-float FFT and its FP32 FFT (0 where not measured or not
// supported), full (unpruned) transforms.
struct FftRow {
  int64_t n;
  double ms32, ms64, msdf, msf32;
};
static const FftRow kFftTable[] = {
#include "fft_table.inc"
};
static const size_t kFftRows = sizeof(kFftTable) / sizeof(kFftTable[0]);

static double row_ms(const FftRow& r, int kind, int prec) {
  if (kind == kFftDf64) return r.msdf;
  if (kind == kFftF32) return r.msf32;
  return prec ? r.ms64 : r.ms32;
}

// Milliseconds of one n x n plane transform of the given kind: the table value, else an
// n^2 log n extrapolation from the largest measured size.
static double fft_ms_square(int64_t n, int kind, int prec) {
  for (size_t i = 0; i < kFftRows; ++i)
    if (kFftTable[i].n == n && row_ms(kFftTable[i], kind, prec) > 0) return row_ms(kFftTable[i], kind, prec);
  for (size_t i = kFftRows; i-- > 0;) {
    const FftRow& L = kFftTable[i];
    double ref = row_ms(L, kind, prec);
    if (ref <= 0) continue;
    double a = (double)n * n * std::log2((double)n * n), b = (double)L.n * L.n * std::log2((double)L.n * L.n);
    return ref * a / b * 1.3;   // unmeasured sizes are priced a little higher
  }
  // the library's FP32 FFT at a size beyond the table: priced above cuFFT's C2C
  if (kind == kFftF32) return 2.0 * fft_ms_square(n, kFftCufft2d, prec);
  return std::numeric_limits<double>::infinity();
}

// One nu x nv plane of the given kind: per-cell cost averaged over the two axis lengths; the
// pruned kinds transform only the image lines in one of their two passes.  Z2Z: half the work
// scales with the image fraction.  Double-float FFT: its pruned column pass (the slower pass
// per line) and the pruned loads / stores of its row pass leave 0.15 + 0.85 x the image
// fraction of the full transform (measured on GB300: 0.542 ms for a 3456^2 plane with a 2048^2
// image, against 0.828 ms for the full transform).
static double fft_ms(int64_t nu, int64_t nv, int kind, int prec, int64_t nx, int64_t ny) {
  double cu = fft_ms_square(nu, kind, prec) / ((double)nu * nu);
  double cv = fft_ms_square(nv, kind, prec) / ((double)nv * nv);
  double full = 0.5 * (cu + cv) * (double)nu * nv;
  // image fraction of a side, the geometric mean over the two (square planes: nx / nu); a single
  // side's fraction would favour a plane longer in that direction
  const double frac = std::min(1.0, std::sqrt((double)nx / (double)nu * (double)ny / (double)nv));
  if (kind == kFftPrunedZ2Z) return full * (0.5 + 0.5 * frac) * 1.07;   // 1-D plans: 7 % overhead
  if (kind == kFftDf64) return full * (0.15 + 0.85 * frac);
  // FP32 FFT (memory-bound): the pruned passes move (1 + f)^2 / 4 of the full transform's
  // bytes (column pass: f^2 loaded, f stored; row pass: f loaded, 1 stored; f = image fraction)
  if (kind == kFftF32) return full * (1.0 + frac) * (1.0 + frac) / 4.0;
  return full;
}

static bool kind_supports(int kind, int64_t n) {
  if (kind == kFftDf64) return df64_side_ok(n);
  if (kind == kFftF32) return f32_side_ok(n);
  return true;
}

// Grid-size candidates >= nmin: the next measured sizes (multiples of `mult`), or FFT-friendly
// sizes beyond the table.
static std::vector<int64_t> size_candidates(int64_t nmin, int64_t mult, int kind) {
  std::vector<int64_t> c;
  for (size_t i = 0; i < kFftRows && c.size() < 10; ++i)
    if (kFftTable[i].n >= nmin && kFftTable[i].n % mult == 0 && kind_supports(kind, kFftTable[i].n))
      c.push_back(kFftTable[i].n);
  if (c.empty() && kind != kFftDf64) c.push_back(good_size(nmin, mult));
  return c;
}

// GB300 cost model (seconds), Sec. 4.1: per w-plane the FFT (measured) plus plane traffic
// per cell and the w-screen phase per image pixel; per visibility the (de)gridding work,
// alpha planes x alpha rows x the lanes of the visibility's group (G = 4, 8 or 16 >= alpha;
// the FP64 gridding kernel spreads its lanes over the alpha^2 cells instead, so FP64 counts
// the mean of G and alpha).  The per-cell / per-pixel / per-visibility constants are measured
// stage times of this library on GB300 (2048^2 image, 1e6 visibilities, alpha = G = 8 in FP32
// and 16 in FP64) divided by the units processed.
static double plan_cost(int prec, int kind, int64_t nu, int64_t nv, int64_t nw, int alpha,
                        int64_t nvis, int64_t nx, int64_t ny) {
  double cells = (double)nu * nv;
  double k_cell = prec ? 3.0e-12 : 2.5e-12;   // s per plane cell (screen / (de)grid traffic)
  // s per image pixel per plane (screen phase and accumulation): FP64 in pair arithmetic with an
  // FP64 anchor every 16 planes (double-float planes), FP64 otherwise; FP32
  double k_pix = prec ? (kind == kFftDf64 ? 6.0e-12 : 1.2e-11) : 1.8e-12;
  // s per visibility per alpha^2 x lanes; FP64 plans with the double-float FFT (de)grid in pair
  // arithmetic on the FP32 pipes, about twice as fast as FP64 arithmetic
  double k_vis = prec ? (kind == kFftDf64 ? 5.0e-12 : 1.05e-11) : 3.6e-12;
  const int G = alpha <= 4 ? 4 : (alpha <= 8 ? 8 : 16);
  const double lanes = prec ? 0.5 * (G + alpha) : (double)G;
  return nw * (1e-3 * fft_ms(nu, nv, kind, prec, nx, ny) + cells * k_cell + (double)(nx * ny) * k_pix) +
         (double)nvis * alpha * alpha * lanes * k_vis;
}

// Cheapest (nu, nv) for one plane among the candidates (FFT + traffic per cell); false if the
// FFT kind supports none.
static bool choose_grid(int64_t nmin_u, int64_t nmin_v, int prec, int kind, int64_t mult,
                        int64_t nx, int64_t ny, int64_t* nu, int64_t* nv) {
  double k_cell = prec ? 3.0e-12 : 2.5e-12;
  double best = std::numeric_limits<double>::infinity();
  for (int64_t a : size_candidates(nmin_u, mult, kind))
    for (int64_t b : size_candidates(nmin_v, mult, kind)) {
      double c = 1e-3 * fft_ms(a, b, kind, prec, nx, ny) + k_cell * (double)a * b;
      if (c < best) { best = c; *nu = a; *nv = b; }
    }
  return std::isfinite(best);
}

int choose_plan(const PlanInput& in, PlanParams& out, char* err, int errlen) {
  auto fail = [&](const char* msg) {
    std::snprintf(err, errlen, "%s", msg);
    return 1;
  };
  if (in.nx < 32 || in.ny < 32 || (in.nx & 1) || (in.ny & 1))
    return fail("npix_x and npix_y must be even and at least 32");
  if (!(in.psx > 0) || !(in.psy > 0)) return fail("pixel sizes must be positive");
  if (!(in.eps > 2e-13)) return fail("epsilon must be larger than 2e-13");
  if (in.prec == 0 && in.eps < 1e-5) return fail("single precision requires epsilon >= 1e-5");
  if (in.fft_impl < 0 || in.fft_impl > 4) return fail("fft_impl must be 0, 1, 2, 3 or 4");
  if (in.prec == 0 && (in.fft_impl == kFftDf64 || in.fft_impl == kFftPrunedZ2Z))
    return fail("fft_impl 2 and 3 need WG_F64");
  if (in.prec == 1 && in.fft_impl == kFftF32) return fail("fft_impl 4 needs WG_F32");
  // most negative n - 1 over the image: the corner pixel (-nx/2, -ny/2) (Sec. 2, sets L, M)
  double lmax = 0.5 * in.nx * in.psx, mmax = 0.5 * in.ny * in.psy;
  double r2 = lmax * lmax + mmax * mmax;
  if (r2 >= 1.0) return fail("field of view exceeds the unit disc (l^2 + m^2 >= 1)");
  double nm1_min = -r2 / (1.0 + std::sqrt(1.0 - r2));
  if (in.tile != 0 && in.tile != 16 && in.tile != 32) return fail("tile must be 16 or 32");

  // FFT kinds to consider: FP32 plans use cuFFT C2C (the library's FP32 FFT only on request:
  // measured slower than cuFFT at the sizes the planner picks, and its pruned time is modelled,
  // not measured); FP64 plans the pruned Z2Z transform or the double-float FFT, whichever is
  // cheaper among those whose rounding fits epsilon
  std::vector<int> kinds;
  if (in.fft_impl != 0) kinds.push_back(in.fft_impl);
  else if (in.prec == 0) kinds.push_back(kFftCufft2d);
  else { kinds.push_back(kFftPrunedZ2Z); kinds.push_back(kFftDf64); }

  double safety = in.eps_safety > 0 ? in.eps_safety : kDefaultEpsSafety;
  bool found = false, size_ok = false;
  PlanParams best;
  best.cost = std::numeric_limits<double>::infinity();
  // kernels: the App. A table (alpha 4, 7, 8, 12, 16) and the searched ones for the other
  // supports (kernel_design.cpp)
  std::vector<KernelRow> T = kernel_table();
  for (const auto& r : kernel_table_design()) T.push_back(r);
  for (int alpha = 4; alpha <= kMaxAlpha; ++alpha) {
    if (in.force_alpha > 0 && alpha != in.force_alpha) continue;
    // uv tile side: 32 cells; 16 for FP64 kernels wider than 8 (16-lane groups), whose
    // (tile + alpha - 1)^2 staging area would otherwise crowd shared memory
    int tile = in.tile > 0 ? in.tile : ((in.prec == 1 && alpha > 8) ? 16 : 32);
    if (alpha - 1 > tile) continue;
    std::vector<const KernelRow*> rows;
    for (const auto& r : T) {
      if (r.alpha != alpha) continue;
      if (in.force_sigma > 0 && std::fabs(r.sigma - in.force_sigma) > 1e-9) continue;
      if (r.eps <= in.eps * safety) rows.push_back(&r);
    }
    std::sort(rows.begin(), rows.end(),
              [](const KernelRow* a, const KernelRow* b) { return a->sigma < b->sigma; });
    for (int kind : kinds) {
      // Sec. 4.1: for each alpha the smallest sigma whose kernel meets epsilon -- here the
      // kernel term together with the plane rounding of this FFT kind (unless sigma is forced)
      for (const KernelRow* pick : rows) {
        PlanParams p;
        p.alpha = alpha; p.sigma = pick->sigma; p.beta = pick->beta; p.mu = pick->mu;
        p.eps_kernel = pick->eps;
        p.tile = tile;
        p.fft_kind = kind;
        // Sec. 2: N >= ceil(sigma n); among the FFT-friendly multiples of the tile above it
        // the one with the cheapest measured plane transform
        int64_t minn = std::max<int64_t>(2 * alpha, 16);
        if (!choose_grid(std::max<int64_t>((int64_t)std::ceil(p.sigma * in.nx), minn),
                         std::max<int64_t>((int64_t)std::ceil(p.sigma * in.ny), minn), in.prec,
                         kind, tile, in.nx, in.ny, &p.nu, &p.nv))
          break;   // larger sigma only needs larger grids
        size_ok = true;
        p.ntu = p.nu / tile; p.ntv = p.nv / tile;
        p.nm1_min = nm1_min;
        if (in.do_w) {
          double span;  // extent of the n - 1 values the w-kernel must resolve
          if (in.w_shift) {
            p.nshift = 0.5 * nm1_min;   // centre of [nm1_min, 0]
            span = 0.5 * std::fabs(nm1_min);
          } else {
            p.nshift = 0.0;
            span = std::fabs(nm1_min);
          }
          // Sec. 2: Delta w = 1 / (2 sigma max |n - 1|) (Nyquist), with the maximum taken over
          // the n - 1 values relative to the reference nshift
          p.dw = 1.0 / (2.0 * p.sigma * span);
          double wmin = in.wmin, wmax = std::max(in.wmax, in.wmin);
          // Eq. (wcirc): first plane half a kernel width below the smallest w
          p.w0 = wmin - 0.5 * p.dw * (alpha - 1);
          // N_w = (max w - min w) / Delta w + alpha, rounded up, plus one plane of slack for
          // rounding in the per-visibility plane index
          p.nw = (int64_t)std::ceil((wmax - wmin) / p.dw) + alpha + 1;
        } else {
          p.nshift = 0.0; p.dw = 1.0; p.w0 = 0.0; p.nw = 1;
        }
        if (p.nw > 4095) break;  // plane index must fit 12 bits (FP32 phase split)
        PolyKernel K = make_poly_kernel(alpha, p.beta, p.mu, alpha + 3);
        std::vector<double> pc = psi_cheb_coeffs(K, kPsiChebTerms);
        p.gain = rounding_gain(K, pc, in.nx, in.ny, in.psx, in.psy, p.nu, p.nv, in.do_w,
                               p.nshift, p.dw);
        double e_k = p.eps_kernel / safety;
        double e_r = rounding_coefficient(p.gain) * plane_rounding(kind, in.prec, p.nu, p.nv) * p.gain;
        p.err_model = std::sqrt(e_k * e_k + e_r * e_r);
        if (in.force_sigma <= 0 && p.err_model > in.eps) continue;
        p.cost = plan_cost(in.prec, kind, p.nu, p.nv, p.nw, alpha, in.nvis, in.nx, in.ny);
        if (p.cost < best.cost) { best = p; found = true; }
        break;
      }
    }
  }
  if (!found) {
    if (!size_ok && in.fft_impl == kFftDf64)
      return fail("the double-float FFT supports grid sides up to 25600 only");
    if (!size_ok && in.fft_impl == kFftF32)
      return fail("the FP32 plane FFT supports grid sides up to 32768 only");
    return fail("no kernel in the table meets the requested epsilon");
  }
  out = best;
  return 0;
}

}  // namespace wg
