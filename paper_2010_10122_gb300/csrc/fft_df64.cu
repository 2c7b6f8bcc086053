// 2-D complex FFT of FP64 planes computed in double-float ("df64") arithmetic on the FP32 pipes.
//
// GB300 executes FP64 FMAs at ~1/58 of its FP32 rate, which makes cuFFT's double-precision
// transforms the dominant cost of the FP64 (eps ~ 1e-12) mode.  Here every value is carried as
// an unevaluated sum hi + lo of two floats (48-bit significand); additions use the two-sum and
// products the fma-based two-product error-free transformations, so a radix-8 butterfly costs a
// few hundred FP32 operations instead of FP64 ones.  Normwise accuracy of a length-3200
// transform is ~5e-15 relative (vs ~3e-16 for FP64), well below what eps >= 1e-12 needs.
//
// Algorithm: each 1-D transform is a mixed-radix (8, 4, 2, 5, 3 and a generic radix for 7 / 11)
// Stockham autosort FFT run by one CTA in shared memory with ping-pong buffers; the 2-D plane
// transform is a pass over rows (contiguous) followed by a pass over columns (several adjacent
// columns per CTA, so the strided global accesses move whole sectors).  Planes stay complex128
// in global memory: the row pass splits doubles into df64 on load and stores df64, the column
// pass loads df64 and joins back to doubles on store.  Transforms are unnormalised, forward =
// e^{-2 pi i}, like cuFFT's.
#include <cmath>
#include <cstring>

#include "wgrid_internal.h"

namespace wg {

struct dd {
  float h, l;
};
struct cdd {
  dd r, i;
};

__device__ __forceinline__ dd dd_make(float h, float l) { dd x; x.h = h; x.l = l; return x; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ dd two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd_make(s, e);
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return dd_make(s, e);
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.h, b.h);
  float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return fast_two_sum(s.h, e);
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd_make(-a.h, -a.l); }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ cdd c_add(cdd a, cdd b) { cdd c; c.r = dd_add(a.r, b.r); c.i = dd_add(a.i, b.i); return c; }
__device__ __forceinline__ cdd c_sub(cdd a, cdd b) { cdd c; c.r = dd_sub(a.r, b.r); c.i = dd_sub(a.i, b.i); return c; }
__device__ __forceinline__ cdd c_mul(cdd a, cdd b) {
  cdd c;
  c.r = dd_sub(dd_mul(a.r, b.r), dd_mul(a.i, b.i));
  c.i = dd_add(dd_mul(a.r, b.i), dd_mul(a.i, b.r));
  return c;
}
__device__ __forceinline__ cdd c_scale(cdd a, dd s) { cdd c; c.r = dd_mul(a.r, s); c.i = dd_mul(a.i, s); return c; }
// multiply by -i (fwd = true) or +i
__device__ __forceinline__ cdd c_mul_mi(cdd a, bool fwd) {
  cdd c;
  if (fwd) { c.r = a.i; c.i = dd_neg(a.r); }
  else { c.r = dd_neg(a.i); c.i = a.r; }
  return c;
}

__device__ __forceinline__ cdd load_cdd(const float4& v) {
  cdd c; c.r = dd_make(v.x, v.y); c.i = dd_make(v.z, v.w); return c;
}
__device__ __forceinline__ float4 store_cdd(const cdd& c) { return make_float4(c.r.h, c.r.l, c.i.h, c.i.l); }

__device__ __forceinline__ dd split_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return dd_make(h, l);
}
__device__ __forceinline__ double join_double(dd x) { return (double)x.h + (double)x.l; }

// df64 constants of the small DFT kernels
struct DftConst {
  dd c31;            // sin(2 pi / 3)
  dd c51, c52;       // cos(2 pi / 5), cos(4 pi / 5)
  dd s51, s52;       // sin(2 pi / 5), sin(4 pi / 5)
  dd r2;             // sqrt(2) / 2
};

constexpr int kMaxStages = 24;
struct FftLine {
  int n;                     // transform length
  int nst;                   // number of radix stages
  int radix[kMaxStages];
  const float4* tw;          // e^{-2 pi i t / n}, t = 0 .. n - 1, df64
  DftConst k;
};

// W^(t) for the transform direction: table entry (forward) or its conjugate (inverse)
__device__ __forceinline__ cdd twiddle(const float4* __restrict__ tw, int t, bool fwd) {
  float4 v = __ldg(&tw[t]);
  cdd w = load_cdd(v);
  if (!fwd) w.i = dd_neg(w.i);
  return w;
}

__device__ __forceinline__ void dft2(cdd* x) {
  cdd a = c_add(x[0], x[1]), b = c_sub(x[0], x[1]);
  x[0] = a; x[1] = b;
}
__device__ __forceinline__ void dft4(cdd* x, bool fwd) {
  cdd t0 = c_add(x[0], x[2]), t1 = c_sub(x[0], x[2]);
  cdd t2 = c_add(x[1], x[3]), t3 = c_mul_mi(c_sub(x[1], x[3]), fwd);
  x[0] = c_add(t0, t2); x[2] = c_sub(t0, t2);
  x[1] = c_add(t1, t3); x[3] = c_sub(t1, t3);
}
__device__ __forceinline__ void dft8(cdd* x, bool fwd, const DftConst& k) {
  cdd e[4] = {x[0], x[2], x[4], x[6]}, o[4] = {x[1], x[3], x[5], x[7]};
  dft4(e, fwd);
  dft4(o, fwd);
  // o_k *= W8^k, W8 = e^{-/+ 2 pi i / 8}
  {
    // k = 1: (1 -/+ i) / sqrt2
    cdd a = o[1], r;
    if (fwd) { r.r = dd_add(a.r, a.i); r.i = dd_sub(a.i, a.r); }
    else { r.r = dd_sub(a.r, a.i); r.i = dd_add(a.i, a.r); }
    o[1] = c_scale(r, k.r2);
    o[2] = c_mul_mi(o[2], fwd);
    // k = 3: (-1 -/+ i) / sqrt2
    a = o[3];
    if (fwd) { r.r = dd_sub(a.i, a.r); r.i = dd_neg(dd_add(a.r, a.i)); }
    else { r.r = dd_neg(dd_add(a.r, a.i)); r.i = dd_sub(a.r, a.i); }
    o[3] = c_scale(r, k.r2);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    x[q] = c_add(e[q], o[q]);
    x[q + 4] = c_sub(e[q], o[q]);
  }
}
__device__ __forceinline__ void dft3(cdd* x, bool fwd, const DftConst& k) {
  cdd t1 = c_add(x[1], x[2]);
  cdd y0 = c_add(x[0], t1);
  dd half = dd_make(0.5f, 0.f);
  cdd t2 = c_sub(x[0], c_scale(t1, half));
  cdd t3 = c_mul_mi(c_scale(c_sub(x[1], x[2]), k.c31), fwd);   // -/+ i s (x1 - x2)
  x[0] = y0;
  x[1] = c_add(t2, t3);
  x[2] = c_sub(t2, t3);
}
__device__ __forceinline__ void dft5(cdd* x, bool fwd, const DftConst& k) {
  cdd t1 = c_add(x[1], x[4]), t2 = c_add(x[2], x[3]);
  cdd t3 = c_sub(x[1], x[4]), t4 = c_sub(x[2], x[3]);
  cdd y0 = c_add(x[0], c_add(t1, t2));
  cdd a1 = c_add(x[0], c_add(c_scale(t1, k.c51), c_scale(t2, k.c52)));
  cdd a2 = c_add(x[0], c_add(c_scale(t1, k.c52), c_scale(t2, k.c51)));
  cdd b1 = c_add(c_scale(t3, k.s51), c_scale(t4, k.s52));
  cdd b2 = c_sub(c_scale(t3, k.s52), c_scale(t4, k.s51));
  cdd ib1 = c_mul_mi(b1, fwd), ib2 = c_mul_mi(b2, fwd);   // -/+ i b
  x[0] = y0;
  x[1] = c_add(a1, ib1);
  x[4] = c_sub(a1, ib1);
  x[2] = c_add(a2, ib2);
  x[3] = c_sub(a2, ib2);
}
// generic radix r (7, 11): y_q = sum_k x_k W_n^{k q n / r}
template <int R>
__device__ __forceinline__ void dft_generic(cdd* x, bool fwd, const float4* __restrict__ tw, int n) {
  cdd y[R];
  const int step = n / R;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    cdd acc = x[0];
#pragma unroll
    for (int kk = 1; kk < R; ++kk) acc = c_add(acc, c_mul(x[kk], twiddle(tw, ((kk * q) % R) * step, fwd)));
    y[q] = acc;
  }
#pragma unroll
  for (int q = 0; q < R; ++q) x[q] = y[q];
}

// One radix-R Stockham stage over `lines` lines of length n held in shared memory.
template <int R>
__device__ __forceinline__ void stage(const float4* __restrict__ src, float4* __restrict__ dst,
                                      int n, int lines, int Ns, bool fwd, const FftLine& L) {
  const int M = n / R;
  const int tstep = n / (Ns * R);
  for (int b = threadIdx.x; b < lines * M; b += blockDim.x) {
    const int line = b / M, j = b - line * M;
    const float4* s = src + line * n;
    float4* d = dst + line * n;
    const int jm = j % Ns;
    cdd x[R];
#pragma unroll
    for (int kk = 0; kk < R; ++kk) x[kk] = load_cdd(s[j + kk * M]);
    if (Ns > 1) {
#pragma unroll
      for (int kk = 1; kk < R; ++kk) x[kk] = c_mul(x[kk], twiddle(L.tw, (jm * kk * tstep) % n, fwd));
    }
    if (R == 2) dft2(x);
    else if (R == 4) dft4(x, fwd);
    else if (R == 8) dft8(x, fwd, L.k);
    else if (R == 3) dft3(x, fwd, L.k);
    else if (R == 5) dft5(x, fwd, L.k);
    else dft_generic<R>(x, fwd, L.tw, n);
    const int idx = (j / Ns) * Ns * R + jm;
#pragma unroll
    for (int q = 0; q < R; ++q) d[idx + q * Ns] = store_cdd(x[q]);
  }
}

// Transform `lines` lines of one plane: line c, element i at global offset
// base + (line0 + c) * line_stride + i * elem_stride (complex elements).
// mode 0: load doubles, store df64; mode 1: load df64, store doubles.
__global__ void __launch_bounds__(256)
k_fft_lines(const __grid_constant__ FftLine L, void* __restrict__ data, int64_t plane_elems,
            int lines_per_plane, int lines, int64_t line_stride, int64_t elem_stride, int mode,
            int fwd) {
  extern __shared__ __align__(16) float4 fsm[];
  const int n = L.n;
  float4* bufA = fsm;
  float4* bufB = fsm + (size_t)lines * n;
  const int blocks_per_plane = lines_per_plane / lines;
  const int plane = blockIdx.x / blocks_per_plane;
  const int line0 = (blockIdx.x - plane * blocks_per_plane) * lines;
  const int64_t base = (int64_t)plane * plane_elems + (int64_t)line0 * line_stride;
  const int total = lines * n;
  // load: consecutive threads walk the contiguous direction (coalesced global access)
  if (mode == 0) {
    const double2* in = reinterpret_cast<const double2*>(data);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      int c, i;
      if (elem_stride == 1) { c = e / n; i = e - c * n; }
      else { i = e / lines; c = e - i * lines; }
      double2 v = in[base + c * line_stride + i * elem_stride];
      cdd x; x.r = split_double(v.x); x.i = split_double(v.y);
      bufA[c * n + i] = store_cdd(x);
    }
  } else {
    const float4* in = reinterpret_cast<const float4*>(data);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      int c, i;
      if (elem_stride == 1) { c = e / n; i = e - c * n; }
      else { i = e / lines; c = e - i * lines; }
      bufA[c * n + i] = in[base + c * line_stride + i * elem_stride];
    }
  }
  __syncthreads();
  float4* src = bufA;
  float4* dst = bufB;
  int Ns = 1;
  const bool f = fwd != 0;
  for (int s = 0; s < L.nst; ++s) {
    const int R = L.radix[s];
    switch (R) {
      case 2: stage<2>(src, dst, n, lines, Ns, f, L); break;
      case 3: stage<3>(src, dst, n, lines, Ns, f, L); break;
      case 4: stage<4>(src, dst, n, lines, Ns, f, L); break;
      case 5: stage<5>(src, dst, n, lines, Ns, f, L); break;
      case 7: stage<7>(src, dst, n, lines, Ns, f, L); break;
      case 8: stage<8>(src, dst, n, lines, Ns, f, L); break;
      default: stage<11>(src, dst, n, lines, Ns, f, L); break;
    }
    Ns *= R;
    __syncthreads();
    float4* t = src; src = dst; dst = t;
  }
  if (mode == 0) {
    float4* out = reinterpret_cast<float4*>(data);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      int c, i;
      if (elem_stride == 1) { c = e / n; i = e - c * n; }
      else { i = e / lines; c = e - i * lines; }
      out[base + c * line_stride + i * elem_stride] = src[c * n + i];
    }
  } else {
    double2* out = reinterpret_cast<double2*>(data);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      int c, i;
      if (elem_stride == 1) { c = e / n; i = e - c * n; }
      else { i = e / lines; c = e - i * lines; }
      cdd x = load_cdd(src[c * n + i]);
      double2 v; v.x = join_double(x.r); v.y = join_double(x.i);
      out[base + c * line_stride + i * elem_stride] = v;
    }
  }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
static bool factor_radices(int n, int* r, int* nst) {
  int k = 0;
  int m = n;
  for (int p : {8, 4, 2, 5, 3, 7, 11}) {
    while (m % p == 0 && k < kMaxStages) { r[k++] = p; m /= p; }
  }
  *nst = k;
  return m == 1;
}

static dd host_dd(long double v) {
  float h = (float)v;
  float l = (float)(v - (long double)h);
  dd x; x.h = h; x.l = l;
  return x;
}

struct Df64Fft {
  int nu = 0, nv = 0;
  FftLine lu, lv;
  float4* tw_u = nullptr;
  float4* tw_v = nullptr;
  int lines_u = 1, lines_v = 1;   // lines per CTA in the column / row pass
};

static constexpr size_t kFftSmem = 200 * 1024;

bool df64_fft_supported(int64_t nu, int64_t nv) {
  int r[kMaxStages], k;
  if (nu > (int64_t)(kFftSmem / (2 * sizeof(float4))) || nv > (int64_t)(kFftSmem / (2 * sizeof(float4))))
    return false;
  return factor_radices((int)nu, r, &k) && factor_radices((int)nv, r, &k);
}

static cudaError_t make_line(int n, FftLine* L, float4** tw) {
  std::memset(L, 0, sizeof(*L));
  L->n = n;
  if (!factor_radices(n, L->radix, &L->nst)) return cudaErrorInvalidValue;
  std::vector<float4> h(n);
  const long double two_pi = 6.283185307179586476925286766559L;
  for (int t = 0; t < n; ++t) {
    long double a = two_pi * (long double)t / (long double)n;
    dd c = host_dd(cosl(a)), s = host_dd(-sinl(a));
    h[t] = make_float4(c.h, c.l, s.h, s.l);
  }
  cudaError_t e = cudaMalloc((void**)tw, sizeof(float4) * n);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(*tw, h.data(), sizeof(float4) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  L->tw = *tw;
  const long double pi = 3.141592653589793238462643383279L;
  L->k.c31 = host_dd(sinl(2 * pi / 3));
  L->k.c51 = host_dd(cosl(2 * pi / 5));
  L->k.c52 = host_dd(cosl(4 * pi / 5));
  L->k.s51 = host_dd(sinl(2 * pi / 5));
  L->k.s52 = host_dd(sinl(4 * pi / 5));
  L->k.r2 = host_dd(sqrtl(2.0L) / 2);
  return cudaSuccess;
}

static int lines_per_cta(int n, int lines_total) {
  int c = (int)(kFftSmem / (2 * sizeof(float4) * (size_t)n));
  c = std::max(1, std::min(c, 8));
  while (c > 1 && lines_total % c != 0) --c;
  return c;
}

cudaError_t df64_fft_create(int64_t nu, int64_t nv, Df64Fft** out) {
  *out = nullptr;
  Df64Fft* f = new Df64Fft();
  f->nu = (int)nu; f->nv = (int)nv;
  cudaError_t e = make_line((int)nu, &f->lu, &f->tw_u);
  if (e == cudaSuccess) e = make_line((int)nv, &f->lv, &f->tw_v);
  if (e != cudaSuccess) {
    if (f->tw_u) cudaFree(f->tw_u);
    if (f->tw_v) cudaFree(f->tw_v);
    delete f;
    return e;
  }
  f->lines_v = lines_per_cta(f->nv, f->nu);   // row pass: rows of length nv
  f->lines_u = lines_per_cta(f->nu, f->nv);   // column pass: columns of length nu
  *out = f;
  return cudaSuccess;
}

void df64_fft_destroy(Df64Fft* f) {
  if (f == nullptr) return;
  if (f->tw_u) cudaFree(f->tw_u);
  if (f->tw_v) cudaFree(f->tw_v);
  delete f;
}

// In-place transform of `batch` nu x nv complex128 planes; sign -1 forward, +1 inverse.
cudaError_t df64_fft_exec(Df64Fft* f, double2* data, int64_t batch, int sign, cudaStream_t s) {
  const int64_t plane = (int64_t)f->nu * f->nv;
  const int fwd = sign < 0 ? 1 : 0;
  // rows (length nv, contiguous): doubles -> df64
  {
    size_t smem = 2 * sizeof(float4) * (size_t)f->lines_v * f->nv;
    cudaError_t e = cudaFuncSetAttribute(k_fft_lines, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFftSmem);
    if (e != cudaSuccess) return e;
    int64_t blocks = batch * (f->nu / f->lines_v);
    k_fft_lines<<<(unsigned)blocks, 256, smem, s>>>(f->lv, data, plane, f->nu, f->lines_v,
                                                     (int64_t)f->nv, 1, 0, fwd);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // columns (length nu, stride nv): df64 -> doubles
  {
    size_t smem = 2 * sizeof(float4) * (size_t)f->lines_u * f->nu;
    int64_t blocks = batch * (f->nv / f->lines_u);
    k_fft_lines<<<(unsigned)blocks, 256, smem, s>>>(f->lu, data, plane, f->nv, f->lines_u, 1,
                                                     (int64_t)f->nv, 1, fwd);
    return cudaGetLastError();
  }
}

}  // namespace wg
