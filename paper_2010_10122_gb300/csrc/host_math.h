// Host-side kernel mathematics and planner of the w-gridder (FP64, no device code).
#pragma once
#include <cstdint>
#include <vector>

namespace wg {

constexpr double kSpeedOfLight = 299792458.0;
constexpr int kMaxAlpha = 16;
constexpr int kMaxDeg = kMaxAlpha + 3;          // Sec. 4.2: pieces of degree alpha + 3
constexpr int kPsiChebTerms = 28;               // psi(k) as sum_n c_n T_n(8 k^2 - 1), |k| <= 1/2
// Kernels are chosen with table epsilon <= safety * requested epsilon.  The table epsilon is
// the 1-D map error (App. A, Eq. maperror); the 2-D / 3-D gridding error combines the u, v and
// w errors and was measured up to 1.17 times the table value (alpha = 4), so 0.8 by default.
constexpr double kDefaultEpsSafety = 0.8;

struct KernelRow {
  int alpha;
  double sigma, eps, beta, mu;
};

// App. A: optimal modified-ES parameters for alpha in {4, 7, 8, 12, 16}.
const std::vector<KernelRow>& kernel_table();
// The same optimisation run by kernel_search for the other supports (alpha 5, 6, 9, 10, 11,
// 13, 14, 15; sigma 1.15 ... 2.0), generated into kernel_table_design.inc.
const std::vector<KernelRow>& kernel_table_design();

// Kernel design (kernel_design.cpp), for the exact modified ES kernel:
// psi(k) by tanh-sinh quadrature; the map error function l(x) of Eq. (maperror) by
// piecewise tanh-sinh quadrature over the fractional position nu; its supremum over
// |x| <= 1 / (2 sigma) (the kernel's epsilon, App. A); and the (beta, mu) minimising it from a
// starting point (Nelder-Mead on log epsilon).
double es_psi(int alpha, double beta, double mu, double k);
double es_map_error(int alpha, double beta, double mu, double x);
double es_kernel_eps(int alpha, double beta, double mu, double sigma);
KernelRow kernel_search(int alpha, double sigma, double beta0, double mu0);

// Eq. (semicircle2): exp(alpha beta [(1 - (2x/alpha)^2)^mu - 1]) on [-alpha/2, alpha/2].
double es_phi(int alpha, double beta, double mu, double x);

// Piecewise polynomial of Sec. 4.2.  Piece i covers x in [-alpha/2 + i, -alpha/2 + i + 1];
// with local coordinate z in [-1, 1] (x = -alpha/2 + i + (z + 1)/2) it is
// sum_d c[i * (deg + 1) + d] z^d, interpolating phi at the deg + 1 Chebyshev roots.
struct PolyKernel {
  int alpha = 0, deg = 0;
  double beta = 0, mu = 0;
  std::vector<double> c;  // alpha * (deg + 1) monomial coefficients
  double eval(double x) const;  // 0 outside [-alpha/2, alpha/2]
  double eval_piece(int i, double z) const;
};
PolyKernel make_poly_kernel(int alpha, double beta, double mu, int deg);

// psi(k) = int phi_poly(x) exp(2 pi i k x) dx (real: phi is even); Gauss-Legendre per piece.
double psi_poly(const PolyKernel& K, double k);

// Coefficients c_0..c_{m-1} with psi(k) ~= sum_n c_n T_n(8 k^2 - 1) for |k| <= 1/2.
std::vector<double> psi_cheb_coeffs(const PolyKernel& K, int m);
double psi_cheb_eval(const std::vector<double>& c, double k);

// Gauss-Legendre nodes / weights on [-1, 1].
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// Smallest multiple of `mult` that is >= n and whose quotient by `mult` has no prime
// factor above 7 (FFT-friendly sizes for cuFFT).
int64_t good_size(int64_t n, int64_t mult);

// Plane FFT implementations.
enum FftKind { kFftCufft2d = 1, kFftDf64 = 2, kFftPrunedZ2Z = 3, kFftF32 = 4 };
// The library's FP32 plane FFT: up to kF32MaxPart points per CTA (two buffers of complex64 in
// shared memory); longer lines run on a cluster of 2, 4 or 8 CTAs.
constexpr int kF32MaxPart = 12800;
// sides at most 46340: a plane holds fewer than 2^31 elements (32-bit offsets within a plane)
constexpr int kF32MaxSide = 46340;
bool f32_side_ok(int64_t n);
// The double-float FFT keeps two buffers of n complex df64 values in shared memory per CTA
// (200 KB at most): sides up to 6400 whose prime factors are 2, 3, 5, 7 and 11 run one line
// per CTA (above 2048 points as two halves on a cluster of 2 CTAs when the half needs only the
// radices 8, 4, 5, 3); sides up to 25600 that are 2 or 4 times such a side run each line on a
// cluster of 2 or 4 CTAs.
constexpr int64_t kDf64MaxSide = 6400;
constexpr int64_t kDf64MaxSplitSide = 4 * kDf64MaxSide;
// Radix plan and CTA size of one double-float line transform: radices 8 and 4 for the power
// of two (2 only for n = 2 * odd), then 5, 3, 7, 11; n / 8 threads rounded up to a warp
// multiple (at least 64).
struct Df64LinePlan {
  int nst = 0, threads = 0;
  int radix[24];
};
bool df64_line_plan(int64_t n, Df64LinePlan* plan);
// CTAs per line of the double-float FFT for side n: 1, or the smallest S in {2, 4} with n / S
// a supported single-CTA side; 0 if n is not supported
int df64_line_split(int64_t n);
bool df64_side_ok(int64_t n);

// Gain of plane rounding into the result.  A plane value perturbed by a relative (normwise)
// rounding delta reaches the degridded visibilities / gridded image through the kernel
// footprint and the correction 1 / (n psi_u psi_v psi_w) of Eqs. R1 / Rad1; for an image with
// uniformly spread flux the relative error of the result is delta * G with
//   G = rms over the image of 1 / (n psi_u psi_v psi_w)  *  (int phi^2 dx)^(d / 2),
// d = 3 with w-stacking (2 without): the rms per cell of an unnormalised FFT of I * corr is
// ||I * corr||, and the footprint sums alpha cells per axis with weights phi.  Evaluated on a
// lattice of at most 64 x 64 pixel samples.
double rounding_gain(const PolyKernel& K, const std::vector<double>& psi_c, int64_t nx,
                     int64_t ny, double psx, double psy, int64_t nu, int64_t nv, int do_w,
                     double nshift, double dw);

// Relative normwise rounding of one plane transform (and the arithmetic around it) of the
// given kind and precision on an nu x nv grid: c * u * log2(nu nv), with u the unit roundoff
// (FP32 2^-24, FP64 2^-53, double-float 2^-47) and c fitted on GB300 measurements.
double plane_rounding(int kind, int prec, int64_t nu, int64_t nv);   // u log2(nu nv)
double rounding_coefficient(double gain);                              // c(G) of the rounding term

struct PlanInput {
  int64_t nx, ny;
  double psx, psy;
  double eps;
  int prec;          // 0 f32, 1 f64
  int do_w, w_shift;
  double eps_safety;
  int force_alpha;
  double force_sigma;
  int tile;
  double umax, vmax, wmin, wmax;  // wavelengths (|u|, |v| maxima, |w| range)
  int64_t nvis;
  int fft_impl = 0;  // requested plane FFT: 0 automatic, else an FftKind
};

struct PlanParams {
  int alpha = 0;
  double sigma = 0, beta = 0, mu = 0, eps_kernel = 0;
  int64_t nu = 0, nv = 0, nw = 0;
  double dw = 0, w0 = 0;
  double nm1_min = 0;   // most negative n - 1 over the image (corner pixel)
  double nshift = 0;    // reference subtracted from n - 1
  int tile = 0;
  int64_t ntu = 0, ntv = 0;
  double cost = 0;
  int fft_kind = kFftCufft2d;
  double gain = 0;       // rounding_gain of the plan
  double err_model = 0;  // predicted eps_rms: kernel term (+) plane rounding term
};

// Returns 0 on success; on failure fills err (WG_ERR_ARG class problems).
int choose_plan(const PlanInput& in, PlanParams& out, char* err, int errlen);

}  // namespace wg
