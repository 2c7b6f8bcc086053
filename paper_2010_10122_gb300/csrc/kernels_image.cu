// Image-side kernels of the w-gridder: per-pixel correction and w-screen phase table
// (Eqs. R1, Rad1), the w-screen + zero padding into the uv planes (Eq. R2), and the
// conjugate-screen accumulation over planes with the final correction (Eq. Rad1).
//
// Plane layout: plane p of a batch is nu x nv complex, C order; image pixel (jx, jy) sits at
// cell ((jx - nx/2) mod nu, (jy - ny/2) mod nv), so that a plain forward / inverse 2-D DFT
// of the plane evaluates sum_t e^{-/+ 2 pi i (a t_x / nu + b t_y / nv)} with t = j - n/2.
#include "df64.cuh"
#include "wgrid_internal.h"

namespace wg {

// w-screen phase of plane j (global plane index) in cycles, reduced to [-1, 1].
// table: A = frac(w0 (n - 1 - nshift)), B = dw (n - 1 - nshift) with |B| <= 1/(2 sigma).
// FP32: B = Bhi + Blo, Bhi on a 2^-13 lattice, so j * Bhi (j < 4096) is exact in float and
// its integer part can be dropped exactly; the residual j * Blo is below 1/4 in size.
__device__ __forceinline__ float screen_cycles(const Z4<float>& t, int j) {
  float th = (float)j * t.w;          // exact
  th -= rintf(th);                    // exact
  return t.v + th + (float)j * t.pad;
}
__device__ __forceinline__ double screen_cycles(const Z4<double>& t, int j) {
  double c = fma((double)j, t.w, t.v);
  return c - rint(c);
}
__device__ __forceinline__ void sincos2pi(float c, float* s, float* co) { sincospif(2.0f * c, s, co); }
__device__ __forceinline__ void sincos2pi(double c, double* s, double* co) { sincospi(2.0 * c, s, co); }

// ---------------------------------------------------------------------------------------
// prep (once per plan): per pixel, corr = 1 / (n psi_u psi_v psi_w) (Eqs. R1, Rad1, with Psi
// the product of psi over the three directions, Sec. 2) and the screen phase parameters.
// ---------------------------------------------------------------------------------------
template <typename R>
__global__ void k_prep(const __grid_constant__ ImgParams P, Z4<R>* __restrict__ table) {
  const Geom& g = P.g;
  int jy = blockIdx.x * blockDim.x + threadIdx.x;
  int jx = blockIdx.y;
  if (jy >= g.ny) return;
  double l = (double)(jx - g.nx / 2) * g.psx;
  double m = (double)(jy - g.ny / 2) * g.psy;
  double r2 = __dadd_rn(__dmul_rn(l, l), __dmul_rn(m, m));
  double n = sqrt(1.0 - r2);
  double nm1 = -r2 / (1.0 + n);
  double corr = P.cinv_u[jx] * P.cinv_v[jy] / n;
  double A = 0.0, B = 0.0;
  if (g.do_w) {
    double xw = nm1 - g.nshift;
    double kw = xw * g.dw;                 // psi_w argument, |kw| <= 1/(2 sigma)
    double y = 8.0 * kw * kw - 1.0;        // Clenshaw for sum c_n T_n(y)
    double b1 = 0.0, b2 = 0.0;
#pragma unroll
    for (int i = kPsiChebTerms - 1; i >= 1; --i) {
      double b0 = fma(2.0 * y, b1, P.psi_c[i] - b2);
      b2 = b1; b1 = b0;
    }
    double psiw = fma(y, b1, P.psi_c[0] - b2);
    corr /= psiw;
    double a = g.w0 * xw;
    A = a - rint(a);
    B = g.dw * xw;
  }
  int64_t pix = (int64_t)jx * g.ny + jy;
  Z4<R> t;
  t.u = (R)corr;
  t.v = (R)A;
  if (sizeof(R) == 4) {
    double bhi = rint(B * 8192.0) / 8192.0;
    t.w = (R)bhi;
    t.pad = (R)(B - bhi);
  } else {
    t.w = (R)B;
    t.pad = (R)0;
  }
  table[pix] = t;
}

template <typename R>
cudaError_t launch_prep(const ImgParams& P, Z4<R>* table, cudaStream_t s) {
  dim3 grid((P.g.ny + 255) / 256, P.g.nx);
  k_prep<R><<<grid, 256, 0, s>>>(P, table);
  return cudaGetLastError();
}

// image index of plane cell x (or -1 in the zero padding)
__device__ __forceinline__ int cell_to_pixel(int x, int n, int N) {
  if (x < n / 2) return x + n / 2;
  if (x >= N - n / 2) return x - (N - n / 2);
  return -1;
}

// Screen values v e^{2 pi i cycles(j)} for consecutive planes j = j0, j0 + 1, ... (v = 1 for the
// plain screen, the corrected pixel value for the screened image).  FP32: each plane from its
// exactly reduced phase with sincospif.  FP64: sincospi at an anchor plane every kAnchor planes
// and a complex rotation by e^{2 pi i B} in between (4 FMAs per plane instead of an FP64
// sincospi; the rotation's rounding grows by ~1e-16 per plane and is reset at each anchor).
constexpr int kAnchor = 16;
template <typename R> struct ScreenIter;
template <> struct ScreenIter<float> {
  Z4<float> t; int j; float v, c, s;
  __device__ void start(const Z4<float>& tt, int j0, float vv = 1.0f) { t = tt; j = j0; v = vv; eval(); }
  __device__ void eval() {
    float cyc = screen_cycles(t, j);
    sincos2pi(cyc, &s, &c);
    c *= v; s *= v;
  }
  __device__ void next() { ++j; eval(); }
};
template <> struct ScreenIter<double> {
  Z4<double> t; int j, k; double v, c, s, rc, rs;
  __device__ void start(const Z4<double>& tt, int j0, double vv = 1.0) {
    t = tt; j = j0; k = 0; v = vv;
    double b = t.w - rint(t.w);
    sincos2pi(b, &rs, &rc);
    anchor();
  }
  __device__ void anchor() {
    sincos2pi(screen_cycles(t, j), &s, &c);
    c *= v; s *= v;
  }
  __device__ void next() {
    ++j;
    if (++k == kAnchor) {
      k = 0;
      anchor();
    } else {
      double nc = fma(c, rc, -s * rs);
      s = fma(s, rc, c * rs);
      c = nc;
    }
  }
};

// ---------------------------------------------------------------------------------------
// screen: planes[p] = I * corr * exp(+2 pi i c_j (n - 1 - nshift)) at the image cells, 0
// elsewhere (Eqs. R1, R2 with the sign of Eq. rime), for global planes j = b0 .. b0 + nb - 1.
// image_only: one thread per image pixel, the padding cells are not written (the plane FFT
// treats them as zeros without reading them); otherwise one thread per plane cell.
// ---------------------------------------------------------------------------------------
template <typename R>
__global__ void k_screen(const Geom g, const R* __restrict__ dirty,
                         const Z4<R>* __restrict__ table, typename C2<R>::T* __restrict__ planes,
                         int b0, int nb, int image_only) {
  using CT = typename C2<R>::T;
  const int64_t ncell = (int64_t)g.nu * g.nv;
  int jx, jy;
  int64_t cell;
  if (image_only) {
    jy = blockIdx.x * blockDim.x + threadIdx.x;
    jx = blockIdx.y;
    if (jy >= g.ny) return;
    const int x = jx < g.nx / 2 ? g.nu - g.nx / 2 + jx : jx - g.nx / 2;
    const int y = jy < g.ny / 2 ? g.nv - g.ny / 2 + jy : jy - g.ny / 2;
    cell = (int64_t)x * g.nv + y;
  } else {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    const int x = blockIdx.y;
    if (y >= g.nv) return;
    cell = (int64_t)x * g.nv + y;
    jx = cell_to_pixel(x, g.nx, g.nu); jy = cell_to_pixel(y, g.ny, g.nv);
    if (jx < 0 || jy < 0) {
      CT zero; zero.x = (R)0; zero.y = (R)0;
      for (int p = 0; p < nb; ++p) planes[p * ncell + cell] = zero;
      return;
    }
  }
  const int64_t pix = (int64_t)jx * g.ny + jy;
  const Z4<R> t = table[pix];
  const R val = dirty[pix] * t.u;   // I~ = I / (n Psi), Eq. R1
  if (!g.do_w) {
    CT v; v.x = val; v.y = (R)0;
    planes[cell] = v;
    return;
  }
  ScreenIter<R> it;
  it.start(t, b0, val);
  for (int p = 0; p < nb; ++p) {
    CT v; v.x = it.c; v.y = it.s;
    planes[p * ncell + cell] = v;
    it.next();
  }
}

template <typename R>
cudaError_t launch_screen(const Geom& g, const R* dirty, const Z4<R>* table,
                          typename C2<R>::T* planes, int b0, int nb, bool image_only,
                          cudaStream_t s) {
  if (image_only) {
    dim3 grid((g.ny + 255) / 256, g.nx);
    k_screen<R><<<grid, 256, 0, s>>>(g, dirty, table, planes, b0, nb, 1);
  } else {
    dim3 grid((g.nv + 255) / 256, g.nu);
    k_screen<R><<<grid, 256, 0, s>>>(g, dirty, table, planes, b0, nb, 0);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// accumulate: acc += sum_p Re(conj(screen_p) H_p) over the batch (Eq. Rad1); on the last
// batch dirty = acc * corr (the division by n Psi of Eq. Rad1), real part kept.
// ---------------------------------------------------------------------------------------
template <typename R>
__global__ void k_accumulate(const Geom g, const Z4<R>* __restrict__ table,
                             const typename C2<R>::T* __restrict__ planes, int b0, int nb,
                             double* __restrict__ acc, int first, int last,
                             R* __restrict__ dirty) {
  using CT = typename C2<R>::T;
  int jy = blockIdx.x * blockDim.x + threadIdx.x;
  int jx = blockIdx.y;
  if (jy >= g.ny) return;
  int x = jx < g.nx / 2 ? g.nu - g.nx / 2 + jx : jx - g.nx / 2;
  int y = jy < g.ny / 2 ? g.nv - g.ny / 2 + jy : jy - g.ny / 2;
  const int64_t ncell = (int64_t)g.nu * g.nv;
  const int64_t cell = (int64_t)x * g.nv + y;
  const int64_t pix = (int64_t)jx * g.ny + jy;
  Z4<R> t = table[pix];
  R sum = (R)0;
  if (!g.do_w) {
    sum = planes[cell].x;
  } else {
    ScreenIter<R> it;
    it.start(t, b0);
    for (int p = 0; p < nb; ++p) {
      CT h = planes[p * ncell + cell];
      sum += it.c * h.x + it.s * h.y;   // Re(exp(-2 pi i cyc) h)
      it.next();
    }
  }
  double a = first ? (double)sum : acc[pix] + (double)sum;
  if (last) dirty[pix] = (R)(a * (double)t.u);
  else acc[pix] = a;
}

template <typename R>
cudaError_t launch_accumulate(const Geom& g, const Z4<R>* table, const typename C2<R>::T* planes,
                              int b0, int nb, double* acc, bool first, bool last, R* dirty,
                              cudaStream_t s) {
  dim3 grid((g.ny + 255) / 256, g.nx);
  k_accumulate<R><<<grid, 256, 0, s>>>(g, table, planes, b0, nb, acc, first ? 1 : 0,
                                       last ? 1 : 0, dirty);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// double-float image side (FP64 plans with the double-float FFT): the planes hold float pairs
// (float4 per cell: re hi, re lo, im hi, im lo) on the image side as well, so the screen and
// the accumulation run in pair arithmetic on the FP32 pipes instead of FP64 (GB300 issues FP64
// FMAs at 1/64 of the FP32 rate).  The per-plane screen factor e^{2 pi i cycles(j)} is anchored
// by an FP64 sincospi every kAnchor planes and rotated by e^{2 pi i B} in pair arithmetic in
// between (relative error ~1e-14 per step).  Errors made here are image-domain errors: the
// transform multiplies them by psi and the correction divides it out again, so unlike the
// plane FFT's rounding they are not amplified by the 1 / psi correction.
// ---------------------------------------------------------------------------------------
struct ScreenIterDD {
  Z4<double> t; int j, k; cdd cur, rot; double v;
  __device__ void start(const Z4<double>& tt, int j0, double vv) {
    t = tt; j = j0; k = 0; v = vv;
    double rs, rc;
    sincos2pi(t.w - rint(t.w), &rs, &rc);
    rot.r = split_double(rc); rot.i = split_double(rs);
    anchor();
  }
  __device__ void anchor() {
    double s, c;
    sincos2pi(screen_cycles(t, j), &s, &c);
    cur.r = split_double(c * v); cur.i = split_double(s * v);
  }
  __device__ void next() {
    ++j;
    if (++k == kAnchor) { k = 0; anchor(); }
    else cur = c_mul(cur, rot);
  }
};

// planes[p] = I * corr * e^{+2 pi i c_j (n - 1 - nshift)} at the image cells as float pairs
// (the double-float FFT treats the other cells as zeros without reading them)
__global__ void k_screen_dd(const Geom g, const double* __restrict__ dirty,
                            const Z4<double>* __restrict__ table, float4* __restrict__ planes,
                            int b0, int nb) {
  const int64_t ncell = (int64_t)g.nu * g.nv;
  const int jy = blockIdx.x * blockDim.x + threadIdx.x;
  const int jx = blockIdx.y;
  if (jy >= g.ny) return;
  const int x = jx < g.nx / 2 ? g.nu - g.nx / 2 + jx : jx - g.nx / 2;
  const int y = jy < g.ny / 2 ? g.nv - g.ny / 2 + jy : jy - g.ny / 2;
  const int64_t cell = (int64_t)x * g.nv + y;
  const int64_t pix = (int64_t)jx * g.ny + jy;
  const Z4<double> t = table[pix];
  const double val = dirty[pix] * t.u;   // I~ = I / (n Psi), Eq. R1
  if (!g.do_w) {
    const dd a = split_double(val);
    planes[cell] = make_float4(a.h, a.l, 0.f, 0.f);
    return;
  }
  ScreenIterDD it;
  it.start(t, b0, val);
  for (int p = 0; p < nb; ++p) {
    planes[p * ncell + cell] = store_cdd(it.cur);
    it.next();
  }
}

cudaError_t launch_screen_dd(const Geom& g, const double* dirty, const Z4<double>* table,
                             float4* planes, int b0, int nb, cudaStream_t s) {
  dim3 grid((g.ny + 255) / 256, g.nx);
  k_screen_dd<<<grid, 256, 0, s>>>(g, dirty, table, planes, b0, nb);
  return cudaGetLastError();
}

// acc += sum_p Re(conj(screen_p) H_p) over the batch in pair arithmetic (Eq. Rad1), the
// batch's sum added to the FP64 accumulator; on the last batch dirty = acc * corr
__global__ void k_accumulate_dd(const Geom g, const Z4<double>* __restrict__ table,
                                const float4* __restrict__ planes, int b0, int nb,
                                double* __restrict__ acc, int first, int last,
                                double* __restrict__ dirty) {
  const int jy = blockIdx.x * blockDim.x + threadIdx.x;
  const int jx = blockIdx.y;
  if (jy >= g.ny) return;
  const int x = jx < g.nx / 2 ? g.nu - g.nx / 2 + jx : jx - g.nx / 2;
  const int y = jy < g.ny / 2 ? g.nv - g.ny / 2 + jy : jy - g.ny / 2;
  const int64_t ncell = (int64_t)g.nu * g.nv;
  const int64_t cell = (int64_t)x * g.nv + y;
  const int64_t pix = (int64_t)jx * g.ny + jy;
  const Z4<double> t = table[pix];
  dd sum = dd_make(0.f, 0.f);
  if (!g.do_w) {
    const float4 h = planes[cell];
    sum = dd_make(h.x, h.y);
  } else {
    ScreenIterDD it;
    it.start(t, b0, 1.0);
    for (int p = 0; p < nb; ++p) {
      const cdd h = load_cdd(planes[p * ncell + cell]);
      // Re(exp(-2 pi i cyc) h) = cos h.re + sin h.im
      sum = dd_add(sum, dd_dot2(it.cur.r, h.r, it.cur.i, h.i, 1.0f));
      it.next();
    }
  }
  const double a = first ? join_double(sum) : acc[pix] + join_double(sum);
  if (last) dirty[pix] = a * t.u;
  else acc[pix] = a;
}

cudaError_t launch_accumulate_dd(const Geom& g, const Z4<double>* table, const float4* planes,
                                 int b0, int nb, double* acc, bool first, bool last,
                                 double* dirty, cudaStream_t s) {
  dim3 grid((g.ny + 255) / 256, g.nx);
  k_accumulate_dd<<<grid, 256, 0, s>>>(g, table, planes, b0, nb, acc, first ? 1 : 0,
                                       last ? 1 : 0, dirty);
  return cudaGetLastError();
}

#define WG_INST(R)                                                                          \
  template cudaError_t launch_prep<R>(const ImgParams&, Z4<R>*, cudaStream_t);              \
  template cudaError_t launch_screen<R>(const Geom&, const R*, const Z4<R>*, C2<R>::T*, int, \
                                        int, bool, cudaStream_t);                           \
  template cudaError_t launch_accumulate<R>(const Geom&, const Z4<R>*, const C2<R>::T*, int, \
                                            int, double*, bool, bool, R*, cudaStream_t);
WG_INST(float)
WG_INST(double)
#undef WG_INST

}  // namespace wg
