// 2-D complex FFT of FP64 planes computed in double-float ("df64") arithmetic on the FP32 pipes.
//
// GB300 executes FP64 FMAs at 1/64 of its FP32 rate, which makes cuFFT's double-precision
// transforms the dominant cost of the FP64 (eps ~ 1e-12) mode.  Here every value is carried as
// an unevaluated sum hi + lo of two floats (48-bit significand); additions use the two-sum and
// products the fma-based two-product error-free transformations, so a radix-8 butterfly costs a
// few hundred FP32 operations instead of FP64 ones.  Normwise accuracy of a 3200 x 3200
// transform is ~5e-15 relative (vs ~2e-16 for FP64); the planner accounts for it (its
// rounding is amplified by the 1 / psi correction, see plane_rounding / rounding_gain).
//
// Algorithm: each 1-D transform is a mixed-radix (8 and 4 for the power of two, 5, 3, the
// symmetric 7 and 11, 2 only for n = 2 * odd) Stockham autosort FFT run by one CTA per
// line with about n / 8 threads (one radix-8 butterfly each) over two n-element shared-memory
// buffers (ping-pong); up to n = 3584 two CTAs share an SM.  A pass that reads float pairs in
// full runs persistent CTAs instead, which copy their next line into the free buffer (cp.async)
// while storing the current one.  Lines above 6400 points, and lines above 2048 whose half needs
// only the radices 8, 4, 5, 3, run on a thread-block cluster of 2 or 4 CTAs
// (k_fft_lines_cluster).  The 2-D plane transform is a pass over rows (contiguous) and a
// pass over columns.  On the image side planes are complex128 (the pass that reads them splits
// doubles into float pairs on load, the pass that writes them joins the pairs back); on the uv
// side they are complex128 or, for the (de)gridding kernels in pair arithmetic, float pairs.
// Transforms are unnormalised, forward = e^{-2 pi i}, like cuFFT's.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "df64.cuh"
#include "host_math.h"
#include "wgrid_internal.h"

namespace wg {

// df64 constants of the small DFT kernels
struct DftConst {
  dd c31;            // sin(2 pi / 3)
  dd c51, c52;       // cos(2 pi / 5), cos(4 pi / 5)
  dd s51, s52;       // sin(2 pi / 5), sin(4 pi / 5)
  dd r2;             // sqrt(2) / 2
  dd c7[3], s7[3];   // cos, sin (2 pi k / 7), k = 1 .. 3
  dd c11[5], s11[5]; // cos, sin (2 pi k / 11), k = 1 .. 5
};

constexpr int kMaxStages = 24;
struct FftLine {
  int n;                     // transform length held by one CTA (half the line when split)
  int nst;                   // number of radix stages
  int threads;               // CTA size of the line kernel (about n / 8)
  int radix[kMaxStages];
  const float4* tw;          // e^{-2 pi i t / n}, t = 0 .. n - 1, df64
  // split lines (length S n, S = split = 2 or 4, too long for one CTA's shared memory): CTA h
  // (h < S) of a line transforms y_h[j] = e^{-/+ 2 pi i j h / (S n)} sum_{r < S} x[j + r n]
  // e^{-/+ 2 pi i r h / S}, one radix-S decimation-in-frequency step applied while loading,
  // and its n outputs are the line's outputs S k + h.  split = 1: one CTA per line.
  int split;
  const float4* tw2;         // e^{-2 pi i t / (S n)}, t = 0 .. S n - 1, df64 (split lines only)
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
// odd radix R (7, 11): with a_k = x_k + x_{R-k} and b_k = x_k - x_{R-k} (k = 1 .. P = (R - 1) / 2),
//   y_q = x_0 + sum_k a_k cos(2 pi k q / R) -/+ i sum_k b_k sin(2 pi k q / R),
// and y_{R-q} the same with the other sign of the sine sum (forward: minus for y_q); the sums
// are chains of dd_fma against the pair constants (4 P^2 of them instead of the (R - 1)^2
// complex products of a plain DFT)
template <int R>
__device__ __forceinline__ void dft_odd(cdd* x, bool fwd, const dd* cs, const dd* sn) {
  constexpr int P = (R - 1) / 2;
  cdd a[P], b[P];
#pragma unroll
  for (int k = 1; k <= P; ++k) {
    a[k - 1] = c_add(x[k], x[R - k]);
    b[k - 1] = c_sub(x[k], x[R - k]);
  }
  cdd y0 = x[0];
#pragma unroll
  for (int k = 0; k < P; ++k) y0 = c_add(y0, a[k]);
#pragma unroll
  for (int q = 1; q <= P; ++q) {
    cdd re = x[0], im;
    im.r = dd_make(0.f, 0.f);
    im.i = im.r;
#pragma unroll
    for (int k = 1; k <= P; ++k) {
      const int m = (k * q) % R;
      const int mm = m <= P ? m : R - m;
      const dd c = cs[mm - 1];
      const dd sv = m <= P ? sn[mm - 1] : dd_neg(sn[mm - 1]);
      re.r = dd_fma(a[k - 1].r, c, re.r);
      re.i = dd_fma(a[k - 1].i, c, re.i);
      im.r = dd_fma(b[k - 1].r, sv, im.r);
      im.i = dd_fma(b[k - 1].i, sv, im.i);
    }
    const cdd mi = c_mul_mi(im, true);   // -i im
    x[q] = fwd ? c_add(re, mi) : c_sub(re, mi);
    x[R - q] = fwd ? c_sub(re, mi) : c_add(re, mi);
  }
  x[0] = y0;
}

template <int R>
__device__ __forceinline__ void butterfly(cdd* x, bool fwd, const FftLine& L) {
  if constexpr (R == 2) dft2(x);
  else if constexpr (R == 3) dft3(x, fwd, L.k);
  else if constexpr (R == 4) dft4(x, fwd);
  else if constexpr (R == 5) dft5(x, fwd, L.k);
  else if constexpr (R == 8) dft8(x, fwd, L.k);
  else if constexpr (R == 7) dft_odd<7>(x, fwd, L.k.c7, L.k.s7);
  else dft_odd<11>(x, fwd, L.k.c11, L.k.s11);
}


// One radix-R Stockham stage of a length-n line: butterfly j (j = tid, tid + T, ...) reads
// src[j + kk M], twiddles, transforms and writes dst[(j / Ns) Ns R + j mod Ns + q Ns].
// Shared-memory position of line element e: the low three bits of e are XORed with the next
// three (swz = 7, lines whose length is a multiple of 8), so that the stride-R writes of the
// first stages spread over the banks; a permutation within aligned groups of 8 elements.
__device__ __forceinline__ int swizzle(int e, int swz) { return e ^ ((e >> 3) & swz); }

template <int R>
__device__ __forceinline__ void stage(const float4* __restrict__ src, float4* __restrict__ dst,
                                      int n, int Ns, bool fwd, const FftLine& L, int swz) {
  const int M = n / R;
  const int tstep = n / (Ns * R);
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const int jq = j / Ns, jm = j - jq * Ns;
    cdd x[R];
#pragma unroll
    for (int kk = 0; kk < R; ++kk) x[kk] = load_cdd(src[swizzle(j + kk * M, swz)]);
    if (Ns > 1) {
      // jm * kk * tstep < Ns * R * tstep = n: no reduction needed
#pragma unroll
      for (int kk = 1; kk < R; ++kk) x[kk] = c_mul(x[kk], twiddle(L.tw, jm * kk * tstep, fwd));
    }
    butterfly<R>(x, fwd, L);
    const int idx = jq * Ns * R + jm;
#pragma unroll
    for (int q = 0; q < R; ++q) dst[swizzle(idx + q * Ns, swz)] = store_cdd(x[q]);
  }
}

constexpr int kLoadBatch = 4;   // doubles a thread loads at once (mode 0)

// 16-byte asynchronous global -> shared copies (cp.async): a line's load is issued before the
// previous line's store, so the two overlap
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Transform lines g = blockIdx.x, blockIdx.x + gridDim.x, ... < nlines (a persistent CTA): line
// g is line g mod lines_per_plane of plane g / lines_per_plane, element i at global offset
// plane * plane_elems + line * line_stride + i * elem_stride (complex elements).  The plane's
// lines from `split` on are shifted by `skip` (a pass over the first and last rows of a plane
// only, skipping the middle).  mode 0: load doubles, store df64; mode 1: load df64, store
// doubles; mode 2: load and store df64.  Elements lhalf .. n - lhalf - 1 are known zeros and not
// loaded, elements shalf .. n - shalf - 1 are not stored (lhalf = shalf = n: everything).  Two
// n-element shared-memory buffers (ping-pong); with kAsync, after the last stage the buffer the
// stages no longer read receives the next line (asynchronous copies) while the result is stored
// (a line loaded through registers, kAsync false, gains nothing from it: those launches run one
// line per CTA).  kAll
// adds the rare radices 2, 7 and 11, kept out of the common instance so that its register
// allocation is not burdened with them.
template <int TMAX, int MINB, bool kAll, bool kAsync, bool kSplit>
__global__ void __launch_bounds__(TMAX, MINB)
k_fft_lines(const __grid_constant__ FftLine L, void* __restrict__ data, int64_t plane_elems,
            int lines_per_plane, int64_t line_stride, int64_t elem_stride, int mode, int fwd,
            int split, int skip, int lhalf, int shalf, int64_t nlines) {
  extern __shared__ __align__(16) float4 fsm[];
  const int n = L.n;
  const int S = kSplit ? L.split : 1;      // CTAs per line
  const int nfull = S * n;                 // elements of the whole line
  const int T = blockDim.x;
  const int swz = (n & 7) == 0 ? 7 : 0;
  float4* src = fsm;
  float4* dst = fsm + n;
  auto line_base = [&](int64_t gl) -> int64_t {
    gl /= S;                               // S CTAs per line, h = gl mod S
    const int64_t plane = gl / lines_per_plane;
    int line = (int)(gl - plane * lines_per_plane);
    if (line >= split) line += skip;
    return plane * plane_elems + (int64_t)line * line_stride;
  };
  // line gl into buffer b, each thread its elements i = tid, tid + T, ...; known zeros are
  // written directly.  kAsync (pairs, modes 1 and 2): asynchronous copies, completed by the
  // thread's cp_async_wait_all.  Otherwise loaded kLoadBatch at a time through registers, doubles
  // (mode 0) split into float pairs on the way.
  // element i of the whole line as a df64 complex value (0 in the known-zero range)
  auto load_elem = [&](const float4* g4, int64_t base, int i) -> cdd {
    if (i >= lhalf && i < nfull - lhalf) {
      cdd z; z.r = dd_make(0.f, 0.f); z.i = z.r;
      return z;
    }
    const float4 v = g4[base + (int64_t)i * elem_stride];
    if (mode == 0) {
      const double2 d = make_double2(__hiloint2double(__float_as_int(v.y), __float_as_int(v.x)),
                                     __hiloint2double(__float_as_int(v.w), __float_as_int(v.z)));
      cdd x; x.r = split_double(d.x); x.i = split_double(d.y);
      return x;
    }
    return load_cdd(v);
  };
  auto issue = [&](int64_t gl, float4* b) {
    const int64_t base = line_base(gl);
    const float4* g4 = reinterpret_cast<const float4*>(data);
    if constexpr (kSplit) {   // the decimation step of this CTA's part (see FftLine)
      const int h = (int)(gl % S);
      const bool f = fwd != 0;
#pragma unroll 2
      for (int j = threadIdx.x; j < n; j += T) {
        // output h of the radix-S DFT only (h is the same for the whole CTA)
        cdd y;
        if (S == 2) {
          const cdd x0 = load_elem(g4, base, j), x1 = load_elem(g4, base, j + n);
          y = h == 0 ? c_add(x0, x1) : c_sub(x0, x1);
        } else {
          cdd x4[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) x4[r] = load_elem(g4, base, j + r * n);
          if ((h & 1) == 0) {
            const cdd t0 = c_add(x4[0], x4[2]), t2 = c_add(x4[1], x4[3]);
            y = h == 0 ? c_add(t0, t2) : c_sub(t0, t2);
          } else {
            const cdd t1 = c_sub(x4[0], x4[2]), t3 = c_mul_mi(c_sub(x4[1], x4[3]), f);
            y = h == 1 ? c_add(t1, t3) : c_sub(t1, t3);
          }
        }
        if (h > 0) y = c_mul(y, twiddle(L.tw2, j * h, f));
        b[swizzle(j, swz)] = store_cdd(y);
      }
      return;
    }
    if (kAsync) {
      for (int i = threadIdx.x; i < n; i += T) {
        float4* d = b + swizzle(i, swz);
        if (i < lhalf || i >= n - lhalf) cp_async16(d, g4 + base + i * elem_stride);
        else *d = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      cp_async_commit();
      return;
    }
    for (int i0 = threadIdx.x; i0 < n; i0 += kLoadBatch * T) {
      float4 v[kLoadBatch];
#pragma unroll
      for (int k = 0; k < kLoadBatch; ++k) {
        const int i = i0 + k * T;
        if (i < n) v[k] = (i < lhalf || i >= n - lhalf) ? g4[base + i * elem_stride]
                                                        : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < kLoadBatch; ++k) {
        const int i = i0 + k * T;
        if (i < n) {
          if (mode == 0) {
            const double2 d = make_double2(__hiloint2double(__float_as_int(v[k].y), __float_as_int(v[k].x)),
                                           __hiloint2double(__float_as_int(v[k].w), __float_as_int(v[k].z)));
            cdd x; x.r = split_double(d.x); x.i = split_double(d.y);
            b[swizzle(i, swz)] = store_cdd(x);
          } else {
            b[swizzle(i, swz)] = v[k];
          }
        }
      }
    }
  };
  const bool f = fwd != 0;
  // the radix stages in the two buffers; the result ends in src
  auto run_stages = [&]() {
    int Ns = 1;
    for (int s = 0; s < L.nst; ++s) {
      const int R = L.radix[s];
      switch (R) {
        case 3: stage<3>(src, dst, n, Ns, f, L, swz); break;
        case 4: stage<4>(src, dst, n, Ns, f, L, swz); break;
        case 5: stage<5>(src, dst, n, Ns, f, L, swz); break;
        case 8: stage<8>(src, dst, n, Ns, f, L, swz); break;
        default:
          if (kAll) {
            if (R == 2) stage<2>(src, dst, n, Ns, f, L, swz);
            else if (R == 7) stage<7>(src, dst, n, Ns, f, L, swz);
            else stage<11>(src, dst, n, Ns, f, L, swz);
          }
          break;
      }
      __syncthreads();
      float4* t = src; src = dst; dst = t;
      Ns *= R;
    }
  };
  // result element i of this CTA is element i (or, split, 2 i + h) of the line
  auto store_line = [&](int64_t gl) {
    const int64_t base = line_base(gl);
    const int h = (int)(gl % S), st = S;
    if (mode != 1) {
      float4* out = reinterpret_cast<float4*>(data) + base;
      for (int i = threadIdx.x; i < n; i += T) {
        const int o = st * i + h;
        if (o < shalf || o >= nfull - shalf) out[(int64_t)o * elem_stride] = src[swizzle(i, swz)];
      }
    } else {
      double2* out = reinterpret_cast<double2*>(data) + base;
      for (int i = threadIdx.x; i < n; i += T) {
        const int o = st * i + h;
        if (o >= shalf && o < nfull - shalf) continue;   // not needed downstream
        cdd x = load_cdd(src[swizzle(i, swz)]);
        double2 v; v.x = join_double(x.r); v.y = join_double(x.i);
        out[(int64_t)o * elem_stride] = v;
      }
    }
  };
  int64_t gl = blockIdx.x;
  if (gl >= nlines) return;
  if constexpr (!kAsync) {   // one line (or half line) per CTA
    issue(gl, src);
    __syncthreads();
    run_stages();
    store_line(gl);
    return;
  }
  issue(gl, src);
  cp_async_wait_all();
  __syncthreads();
  for (;;) {
    run_stages();
    // the result is in src; dst is no longer read: the next line's copies go there while the
    // result is stored
    const int64_t gn = gl + gridDim.x;
    const bool more = gn < nlines;
    if (more) issue(gn, dst);
    store_line(gl);
    if (!more) break;
    cp_async_wait_all();
    __syncthreads();   // the next line is in place everywhere, and src is no longer read
    float4* t = src; src = dst; dst = t;
    gl = gn;
  }
}

// Split lines on a thread-block cluster of S = L.split CTAs (2 or 4): CTA h copies points
// [h n, h n + n) of its line into shared memory with asynchronous 16-byte copies (all of them
// in flight at once; known zeros written directly, doubles split into float pairs in place),
// the cluster exchanges the parts through distributed shared memory for the radix-S
// decimation-in-frequency step (CTA h forms only its own y_h, see FftLine), and each CTA then
// transforms its n points like a one-CTA line and stores the line's outputs S k + h.  The
// register-path split of k_fft_lines reads all S n points of the line in every CTA with few
// loads in flight; it remains the fallback when a cluster cannot be launched.
template <int TMAX, int MINB, bool kAll>
__global__ void __launch_bounds__(TMAX, MINB)
k_fft_lines_cluster(const __grid_constant__ FftLine L, void* __restrict__ data, int64_t plane_elems,
                    int lines_per_plane, int64_t line_stride, int64_t elem_stride, int mode,
                    int fwd, int split, int skip, int lhalf, int shalf) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) float4 fsm[];
  cg::cluster_group cl = cg::this_cluster();
  const int n = L.n, S = L.split, nfull = S * n, T = blockDim.x;
  const int swz = (n & 7) == 0 ? 7 : 0;
  const bool f = fwd != 0;
  const int h = (int)cl.block_rank();           // cluster dims (S, 1, 1): blockIdx.x mod S
  const int64_t lid = blockIdx.x / (unsigned)S;
  const int64_t plane = lid / lines_per_plane;
  int line = (int)(lid - plane * lines_per_plane);
  if (line >= split) line += skip;
  const int64_t base = plane * plane_elems + (int64_t)line * line_stride;
  float4* A = fsm;
  float4* B = fsm + n;
  const float4* g4 = reinterpret_cast<const float4*>(data);
  const int i0 = h * n;
  for (int j = threadIdx.x; j < n; j += T) {
    const int i = i0 + j;
    float4* d = A + swizzle(j, swz);
    if (i < lhalf || i >= nfull - lhalf) cp_async16(d, g4 + base + (int64_t)i * elem_stride);
    else *d = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  cp_async_commit();
  cp_async_wait_all();
  if (mode == 0) {   // doubles in: each split into a float pair in place (the same 16 bytes)
    for (int j = threadIdx.x; j < n; j += T) {
      const int i = i0 + j;
      if (i >= lhalf && i < nfull - lhalf) continue;
      float4* d = A + swizzle(j, swz);
      const float4 v = *d;
      const double2 dv = make_double2(__hiloint2double(__float_as_int(v.y), __float_as_int(v.x)),
                                      __hiloint2double(__float_as_int(v.w), __float_as_int(v.z)));
      cdd x; x.r = split_double(dv.x); x.i = split_double(dv.y);
      *d = store_cdd(x);
    }
  }
  cl.sync();         // every part is in place
  const float4* P[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) P[r] = cl.map_shared_rank(A, (unsigned)(r < S ? r : 0));
  for (int j = threadIdx.x; j < n; j += T) {
    const int off = swizzle(j, swz);
    cdd y;
    if (S == 2) {
      const cdd x0 = load_cdd(P[0][off]), x1 = load_cdd(P[1][off]);
      y = h == 0 ? c_add(x0, x1) : c_sub(x0, x1);
    } else {
      cdd x4[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) x4[r] = load_cdd(P[r][off]);
      if ((h & 1) == 0) {
        const cdd t0 = c_add(x4[0], x4[2]), t2 = c_add(x4[1], x4[3]);
        y = h == 0 ? c_add(t0, t2) : c_sub(t0, t2);
      } else {
        const cdd t1 = c_sub(x4[0], x4[2]), t3 = c_mul_mi(c_sub(x4[1], x4[3]), f);
        y = h == 1 ? c_add(t1, t3) : c_sub(t1, t3);
      }
    }
    if (h > 0) y = c_mul(y, twiddle(L.tw2, j * h, f));
    B[off] = store_cdd(y);
  }
  cl.sync();         // the other CTAs have read this CTA's part: A is free for the stages
  float4* src = B;
  float4* dst = A;
  int Ns = 1;
  for (int st = 0; st < L.nst; ++st) {
    const int R = L.radix[st];
    switch (R) {
      case 3: stage<3>(src, dst, n, Ns, f, L, swz); break;
      case 4: stage<4>(src, dst, n, Ns, f, L, swz); break;
      case 5: stage<5>(src, dst, n, Ns, f, L, swz); break;
      case 8: stage<8>(src, dst, n, Ns, f, L, swz); break;
      default:
        if (kAll) {
          if (R == 2) stage<2>(src, dst, n, Ns, f, L, swz);
          else if (R == 7) stage<7>(src, dst, n, Ns, f, L, swz);
          else stage<11>(src, dst, n, Ns, f, L, swz);
        }
        break;
    }
    __syncthreads();
    float4* t = src; src = dst; dst = t;
    Ns *= R;
  }
  // result element i of this CTA is element S i + h of the line
  if (mode != 1) {
    float4* out = reinterpret_cast<float4*>(data) + base;
    for (int i = threadIdx.x; i < n; i += T) {
      const int o = S * i + h;
      if (o < shalf || o >= nfull - shalf) out[(int64_t)o * elem_stride] = src[swizzle(i, swz)];
    }
  } else {
    double2* out = reinterpret_cast<double2*>(data) + base;
    for (int i = threadIdx.x; i < n; i += T) {
      const int o = S * i + h;
      if (o >= shalf && o < nfull - shalf) continue;   // not needed downstream
      const cdd x = load_cdd(src[swizzle(i, swz)]);
      double2 v; v.x = join_double(x.r); v.y = join_double(x.i);
      out[(int64_t)o * elem_stride] = v;
    }
  }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
static dd host_dd(long double v) {
  float h = (float)v;
  float l = (float)(v - (long double)h);
  dd x; x.h = h; x.l = l;
  return x;
}

struct Df64Fft {
  int nu = 0, nv = 0;
  FftLine lu, lv;
  float4* tw_u = nullptr;   // line twiddles, then (split lines) the decimation twiddles
  float4* tw_v = nullptr;
};

// Two buffers of n df64 complex values in shared memory per CTA (two CTAs per SM up to n =
// 3584); split lines (df64_line_split) run on clusters of two or four CTAs.
static constexpr int64_t kMaxSide = kDf64MaxSide;

bool df64_fft_supported(int64_t nu, int64_t nv) { return df64_side_ok(nu) && df64_side_ok(nv); }

// e^{-2 pi i t / len} for t = 0 .. count - 1 as df64 (float4: re hi, re lo, im hi, im lo)
static void twiddles(int len, int count, float4* h) {
  const long double two_pi = 6.283185307179586476925286766559L;
  for (int t = 0; t < count; ++t) {
    long double a = two_pi * (long double)t / (long double)len;
    dd c = host_dd(cosl(a)), s = host_dd(-sinl(a));
    h[t] = make_float4(c.h, c.l, s.h, s.l);
  }
}

static cudaError_t make_line(int nline, FftLine* L, float4** tw) {
  std::memset(L, 0, sizeof(*L));
  const int S = df64_line_split(nline);
  if (S == 0) return cudaErrorInvalidValue;
  const int n = nline / S;
  L->n = n;
  L->split = S;
  Df64LinePlan lp;
  if (!df64_line_plan(n, &lp) || lp.nst > kMaxStages) return cudaErrorInvalidValue;
  L->nst = lp.nst;
  L->threads = lp.threads;
  for (int i = 0; i < lp.nst; ++i) L->radix[i] = lp.radix[i];
  const bool split = S > 1;
  const int ntab = split ? n + nline : n;
  std::vector<float4> h(ntab);
  twiddles(n, n, h.data());
  if (split) twiddles(nline, nline, h.data() + n);
  cudaError_t e = cudaMalloc((void**)tw, sizeof(float4) * ntab);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(*tw, h.data(), sizeof(float4) * ntab, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  L->tw = *tw;
  L->tw2 = split ? *tw + n : nullptr;
  const long double pi = 3.141592653589793238462643383279L;
  L->k.c31 = host_dd(sinl(2 * pi / 3));
  L->k.c51 = host_dd(cosl(2 * pi / 5));
  L->k.c52 = host_dd(cosl(4 * pi / 5));
  L->k.s51 = host_dd(sinl(2 * pi / 5));
  L->k.s52 = host_dd(sinl(4 * pi / 5));
  L->k.r2 = host_dd(sqrtl(2.0L) / 2);
  for (int q = 1; q <= 3; ++q) {
    L->k.c7[q - 1] = host_dd(cosl(2 * pi * q / 7));
    L->k.s7[q - 1] = host_dd(sinl(2 * pi * q / 7));
  }
  for (int q = 1; q <= 5; ++q) {
    L->k.c11[q - 1] = host_dd(cosl(2 * pi * q / 11));
    L->k.s11[q - 1] = host_dd(sinl(2 * pi * q / 11));
  }
  return cudaSuccess;
}

cudaError_t df64_fft_create(int64_t nu, int64_t nv, Df64Fft** out) {
  *out = nullptr;
  if (!df64_fft_supported(nu, nv)) return cudaErrorInvalidValue;
  Df64Fft* f = new Df64Fft();
  f->nu = (int)nu; f->nv = (int)nv;
  cudaError_t e = make_line((int)nu, &f->lu, &f->tw_u);
  if (e == cudaSuccess) e = make_line((int)nv, &f->lv, &f->tw_v);
  const int smax = (int)(2 * kMaxSide * sizeof(float4));
#define WG_SMEM_ATTR(TM, MB, A, Y, P)                                                           \
  if (e == cudaSuccess)                                                                          \
    e = cudaFuncSetAttribute(k_fft_lines<TM, MB, A, Y, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax)
  WG_SMEM_ATTR(448, 2, false, false, false); WG_SMEM_ATTR(448, 2, false, true, false);
  WG_SMEM_ATTR(448, 2, true, false, false);  WG_SMEM_ATTR(448, 2, true, true, false);
  WG_SMEM_ATTR(832, 1, false, false, false); WG_SMEM_ATTR(832, 1, false, true, false);
  WG_SMEM_ATTR(832, 1, true, false, false);  WG_SMEM_ATTR(832, 1, true, true, false);
  WG_SMEM_ATTR(448, 2, false, false, true);  WG_SMEM_ATTR(448, 2, true, false, true);
  WG_SMEM_ATTR(832, 1, false, false, true);  WG_SMEM_ATTR(832, 1, true, false, true);
#undef WG_SMEM_ATTR
#define WG_SMEM_ATTR_C(TM, MB, A)                                                                \
  if (e == cudaSuccess)                                                                          \
    e = cudaFuncSetAttribute(k_fft_lines_cluster<TM, MB, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax)
  WG_SMEM_ATTR_C(448, 2, false); WG_SMEM_ATTR_C(448, 2, true);
  WG_SMEM_ATTR_C(832, 1, false); WG_SMEM_ATTR_C(832, 1, true);
#undef WG_SMEM_ATTR_C
  if (e != cudaSuccess) {
    if (f->tw_u) cudaFree(f->tw_u);
    if (f->tw_v) cudaFree(f->tw_v);
    delete f;
    return e;
  }
  *out = f;
  return cudaSuccess;
}

void df64_fft_destroy(Df64Fft* f) {
  if (f == nullptr) return;
  if (f->tw_u) cudaFree(f->tw_u);
  if (f->tw_v) cudaFree(f->tw_v);
  delete f;
}

static cudaError_t launch_lines(const FftLine& L, double2* data, int64_t batch, int64_t plane,
                                int lines_per_plane, int64_t line_stride, int64_t elem_stride,
                                int mode, int fwd, int split, int skip, int lhalf, int shalf,
                                cudaStream_t s) {
  if (lines_per_plane == 0 || batch == 0) return cudaSuccess;
  const size_t smem = 2 * sizeof(float4) * (size_t)L.n;
  // split lines: L.split CTAs per line
  const int64_t nlines = batch * lines_per_plane * L.split;
  // persistent CTAs: as many as fit the GPU at once (two per SM up to 448 threads, else one)
  int dev = 0, sms = 0;
  cudaError_t ea = cudaGetDevice(&dev);
  if (ea == cudaSuccess) ea = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (ea != cudaSuccess) return ea;
  // pairs in, every element loaded: persistent CTAs with asynchronous loads (inverse row pass
  // 40.8 -> 38.5 ms per bench grid call); doubles in (converted on load) or pruned loads: one
  // line per CTA (the persistent form measured 1.2 ms slower on the forward row pass)
  const bool async = mode != 0 && 2 * (int64_t)lhalf >= L.n && L.split == 1;
  const int64_t blocks =
      async ? std::min<int64_t>(nlines, (int64_t)sms * (L.threads <= 448 ? 2 : 1)) : nlines;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  bool common = true;   // radices 8, 4, 5, 3 only
  for (int i = 0; i < L.nst; ++i)
    if (L.radix[i] == 2 || L.radix[i] == 7 || L.radix[i] == 11) common = false;
  if (L.split > 1) {
    // a cluster of L.split CTAs per line (k_fft_lines_cluster); the register-path split below if
    // the cluster cannot be launched
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)nlines);
    cfg.blockDim = dim3((unsigned)L.threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    std::memset(attr, 0, sizeof(attr));
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)L.split;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (nlines > 0x7fffffffLL) return cudaErrorInvalidValue;
    cudaError_t ec;
#define WG_CLUSTER(TM, MB, A)                                                                   \
    ec = cudaLaunchKernelEx(&cfg, k_fft_lines_cluster<TM, MB, A>, L, data, plane,               \
                            lines_per_plane, line_stride, elem_stride, mode, fwd, split, skip,  \
                            lhalf, shalf)
    if (L.threads <= 448) { if (common) WG_CLUSTER(448, 2, false); else WG_CLUSTER(448, 2, true); }
    else { if (common) WG_CLUSTER(832, 1, false); else WG_CLUSTER(832, 1, true); }
#undef WG_CLUSTER
    if (ec == cudaSuccess) return cudaSuccess;
    cudaGetLastError();   // the launch was refused (no kernel ran): the register-path split
  }
#define WG_LINES1(TM, MB, A, Y, P)                                                              \
  k_fft_lines<TM, MB, A, Y, P><<<(unsigned)blocks, L.threads, smem, s>>>(                       \
      L, data, plane, lines_per_plane, line_stride, elem_stride, mode, fwd, split, skip, lhalf, \
      shalf, nlines)
#define WG_LINES(TM, MB, A)                                                                     \
  if (L.split > 1) WG_LINES1(TM, MB, A, false, true);                                           \
  else if (async) WG_LINES1(TM, MB, A, true, false);                                            \
  else WG_LINES1(TM, MB, A, false, false)
  if (L.threads <= 448) {
    if (common) { WG_LINES(448, 2, false); } else { WG_LINES(448, 2, true); }
  } else {
    if (common) { WG_LINES(832, 1, false); } else { WG_LINES(832, 1, true); }
  }
#undef WG_LINES1
#undef WG_LINES
  return cudaGetLastError();
}

// In-place transform of `batch` nu x nv complex128 planes; sign -1 forward, +1 inverse.
// df64_planes: the planes on the grid side are double-float pairs (float4 per complex value:
// re hi, re lo, im hi, im lo) instead of doubles -- the forward transform's output and the
// inverse transform's input; image_pairs: the image side (forward input, inverse output) is
// pairs as well.
// keep_rows = keep_cols = 0: the full 2-D transform.  Otherwise only the image block -- the first
// and last keep_rows/2 rows and keep_cols/2 columns of a plane -- matters, and the column pass
// (strided, the slower pass per line) runs over the image columns only:
//  forward: the image block holds the only nonzero input: the column pass over the image
//    columns loads only their image rows, then the row pass over all rows loads only the image
//    columns (the rest is zero and never read, so the caller need not write it);
//  inverse: only the image block is read afterwards: the row pass over all rows stores only the
//    image columns, then the column pass over those columns stores only the image rows (other
//    cells are left undefined).
cudaError_t df64_fft_exec(Df64Fft* f, double2* data, int64_t batch, int sign, cudaStream_t s,
                          int64_t keep_rows, int64_t keep_cols, bool df64_planes, bool image_pairs) {
  const int64_t plane = (int64_t)f->nu * f->nv;
  const int fwd = sign < 0 ? 1 : 0;
  const bool prune = keep_rows > 0 && keep_cols > 0;
  if (prune && ((keep_rows & 1) || (keep_cols & 1) || keep_rows > f->nu || keep_cols > f->nv))
    return cudaErrorInvalidValue;
  // pass modes: 0 loads doubles and stores pairs, 1 loads pairs and stores doubles, 2 pairs
  // in and out; the grid side is the forward output / inverse input, the image side the other
  const int img_in = image_pairs ? 2 : 0, img_out = image_pairs ? 2 : 1;
  const int uv_in = df64_planes ? 2 : 0, uv_out = df64_planes ? 2 : 1;
  cudaError_t e;
  if (!prune) {
    // rows (length nv, contiguous), then columns (length nu, stride nv)
    e = launch_lines(f->lv, data, batch, plane, f->nu, f->nv, 1, fwd ? img_in : uv_in, fwd,
                     f->nu, 0, f->nv, f->nv, s);
    if (e != cudaSuccess) return e;
    return launch_lines(f->lu, data, batch, plane, f->nv, 1, f->nv, fwd ? uv_out : img_out, fwd,
                        f->nv, 0, f->nu, f->nu, s);
  }
  const int rh = (int)(keep_rows / 2);   // image half-extent along u (rows)
  const int ch = (int)(keep_cols / 2);   // along v (columns)
  const int ncols = 2 * ch, cskip = f->nv - ncols;   // image columns: [0, ch) and [nv - ch, nv)
  if (fwd) {
    // image columns (length nu, stride nv), image rows loaded; then all rows (length nv),
    // image columns loaded
    e = launch_lines(f->lu, data, batch, plane, ncols, 1, f->nv, img_in, fwd, ch, cskip, rh,
                     f->nu, s);
    if (e != cudaSuccess) return e;
    return launch_lines(f->lv, data, batch, plane, f->nu, f->nv, 1, uv_out, fwd, f->nu, 0, ch,
                        f->nv, s);
  }
  // inverse: all rows, image columns stored; then the image columns, image rows stored
  e = launch_lines(f->lv, data, batch, plane, f->nu, f->nv, 1, uv_in, fwd, f->nu, 0, f->nv, ch, s);
  if (e != cudaSuccess) return e;
  return launch_lines(f->lu, data, batch, plane, ncols, 1, f->nv, img_out, fwd, ch, cskip, f->nu,
                      rh, s);
}

}  // namespace wg
