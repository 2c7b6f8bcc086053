// 2-D complex FFT of FP32 planes on the library's own line kernels, with the image-block pruning
// of the double-float FFT (fft_df64.cu): forward, the strided column pass runs over the image
// columns only and loads only their image rows, then the row pass over all rows loads only the
// image columns; inverse, the row pass stores only the image columns and the column pass over
// those stores only the image rows.  The screen therefore writes only the image cells and the
// accumulation reads only them.
//
// Memory access.  A CTA of the strided (column) pass transforms C adjacent columns at once, so
// that every row it touches is one contiguous C x 8-byte segment (C = 4: a whole 32-byte sector)
// instead of one 8-byte element per row.  The lines sit in shared memory as [point][column].  A
// line longer than fits one CTA is split over S = 2, 4 or 8 CTAs of a thread-block cluster: CTA
// h loads points [h n, h n + n) of the line (n = N / S) from HBM once, the cluster exchanges them
// through distributed shared memory for one radix-S decimation-in-frequency step,
//     y_h[j] = W_N^{j h} sum_r x[j + r n] W_S^{r h},
// and CTA h then transforms y_h on its own (its outputs are the line's points S k + h).  Row
// passes (C = 1) gather the outputs back through distributed shared memory so that every CTA
// stores one contiguous run of the line.
//
// Each n-point transform is a mixed-radix Stockham autosort FFT in shared memory (ping-pong
// buffers): radix 8 and 4 for the power of two (2 only for n = 2 x odd), then 5, 3, 7, 11; the
// odd radices use the symmetric form (sum and difference of x_k and x_{R-k} against cosines and
// sines), half the multiplies of a plain DFT.  Twiddles come from tables rounded from long
// double.  Transforms are unnormalised, forward = e^{-2 pi i}, like cuFFT's.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host_math.h"
#include "wgrid_internal.h"

namespace cg = cooperative_groups;

namespace wg {

namespace {

constexpr int kF32MaxStages = 24;

struct OddRadix {           // cos and sin of 2 pi k / R, k = 1 .. (R - 1) / 2
  float c[5], s[5];
};

struct F32Lines {
  int N;                    // line length
  int n;                    // points per CTA: N / S
  int S;                    // CTAs per line (a thread-block cluster when > 1)
  int C;                    // adjacent lines per CTA (strided passes), 1 for rows
  int T;                    // threads per CTA (a multiple of 32 and of C)
  int nst;
  int radix[kF32MaxStages];
  unsigned dmagic[kF32MaxStages];   // floor(2^32 / Ns) + 1 for the stage's Ns > 1: j / Ns =
                                    // umulhi(j, dmagic) for j, Ns < 2^16
  const float2* tw;         // e^{-2 pi i t / n}, t < n
  const float2* twN;        // e^{-2 pi i t / N}, t < N (split lines)
  OddRadix r3, r5, r7, r11;
  float r2;                 // sqrt(2) / 2
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i
__device__ __forceinline__ float2 cmul_mi(float2 a, bool fwd) {
  return fwd ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}
// w * a (forward) or conj(w) * a (inverse), w from the forward table
__device__ __forceinline__ float2 twmul(float2 a, float2 w, bool fwd) {
  return fwd ? make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x))
             : make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}

__device__ __forceinline__ void fdft2(float2* x) {
  const float2 a = cadd(x[0], x[1]), b = csub(x[0], x[1]);
  x[0] = a; x[1] = b;
}
__device__ __forceinline__ void fdft4(float2* x, bool fwd) {
  const float2 t0 = cadd(x[0], x[2]), t1 = csub(x[0], x[2]);
  const float2 t2 = cadd(x[1], x[3]), t3 = cmul_mi(csub(x[1], x[3]), fwd);
  x[0] = cadd(t0, t2); x[2] = csub(t0, t2);
  x[1] = cadd(t1, t3); x[3] = csub(t1, t3);
}
__device__ __forceinline__ void fdft8(float2* x, bool fwd, float r2) {
  float2 e[4] = {x[0], x[2], x[4], x[6]}, o[4] = {x[1], x[3], x[5], x[7]};
  fdft4(e, fwd);
  fdft4(o, fwd);
  // o_k *= W8^k
  {
    float2 a = o[1], r;
    if (fwd) { r.x = a.x + a.y; r.y = a.y - a.x; }   // (1 - i) a
    else { r.x = a.x - a.y; r.y = a.y + a.x; }       // (1 + i) a
    o[1] = cscale(r, r2);
    o[2] = cmul_mi(o[2], fwd);
    a = o[3];
    if (fwd) { r.x = a.y - a.x; r.y = -(a.x + a.y); }  // (-1 - i) a
    else { r.x = -(a.x + a.y); r.y = a.x - a.y; }       // (-1 + i) a
    o[3] = cscale(r, r2);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    x[q] = cadd(e[q], o[q]);
    x[q + 4] = csub(e[q], o[q]);
  }
}
// odd radix R: with a_k = x_k + x_{R-k}, b_k = x_k - x_{R-k} (k = 1 .. P = (R - 1) / 2),
//   y_q = x_0 + sum_k a_k cos(2 pi k q / R) -/+ i sum_k b_k sin(2 pi k q / R),
//   y_{R-q} the same with the other sign of the sine sum (forward: minus for y_q).
template <int R>
__device__ __forceinline__ void fdft_odd(float2* x, bool fwd, const OddRadix& K) {
  constexpr int P = (R - 1) / 2;
  float2 a[P], b[P];
#pragma unroll
  for (int k = 1; k <= P; ++k) {
    a[k - 1] = cadd(x[k], x[R - k]);
    b[k - 1] = csub(x[k], x[R - k]);
  }
  float2 y0 = x[0];
#pragma unroll
  for (int k = 0; k < P; ++k) y0 = cadd(y0, a[k]);
#pragma unroll
  for (int q = 1; q <= P; ++q) {
    float2 re = x[0], im = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 1; k <= P; ++k) {
      const int m = (k * q) % R;
      const int mm = m <= P ? m : R - m;
      const float cs = K.c[mm - 1];
      const float sn = m <= P ? K.s[mm - 1] : -K.s[mm - 1];
      re.x = fmaf(a[k - 1].x, cs, re.x);
      re.y = fmaf(a[k - 1].y, cs, re.y);
      im.x = fmaf(b[k - 1].x, sn, im.x);
      im.y = fmaf(b[k - 1].y, sn, im.y);
    }
    const float2 mi = make_float2(im.y, -im.x);   // -i * im
    x[q] = fwd ? cadd(re, mi) : csub(re, mi);
    x[R - q] = fwd ? csub(re, mi) : cadd(re, mi);
  }
  x[0] = y0;
}

template <int R>
__device__ __forceinline__ void fbutterfly(float2* x, bool fwd, const F32Lines& L) {
  if constexpr (R == 2) fdft2(x);
  else if constexpr (R == 4) fdft4(x, fwd);
  else if constexpr (R == 8) fdft8(x, fwd, L.r2);
  else if constexpr (R == 3) fdft_odd<3>(x, fwd, L.r3);
  else if constexpr (R == 5) fdft_odd<5>(x, fwd, L.r5);
  else if constexpr (R == 7) fdft_odd<7>(x, fwd, L.r7);
  else fdft_odd<11>(x, fwd, L.r11);
}

// shared-memory slot of line point e (n a multiple of 8: the low three bits XORed with the next
// three, which spreads the stride-R accesses of the early stages over the banks)
__device__ __forceinline__ int fswz(int e, int swz) { return e ^ ((e >> 3) & swz); }

// one radix-R Stockham stage over the C lines of the CTA: butterfly j of line c reads src[j +
// kk M], writes dst[(j / Ns) Ns R + j mod Ns + q Ns]; consecutive threads take consecutive lines
// and then consecutive j, so a warp's accesses are contiguous runs
template <int R, int C, bool FWD>
__device__ __forceinline__ void fstage(const float2* __restrict__ src, float2* __restrict__ dst,
                                       int n, int Ns, unsigned dmagic, const F32Lines& L, int swz,
                                       int c) {
  const int M = n / R;
  const int tstep = n / (Ns * R);
  const int total = M * C;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int j = C == 1 ? b : b / C;
    const int jq = Ns == 1 ? j : (int)__umulhi((unsigned)j, dmagic);
    const int jm = j - jq * Ns;
    float2 x[R];
#pragma unroll
    for (int kk = 0; kk < R; ++kk) x[kk] = src[fswz(j + kk * M, swz) * C + c];
    if (Ns > 1) {
      const int t1 = jm * tstep;
#pragma unroll
      for (int kk = 1; kk < R; ++kk) x[kk] = twmul(x[kk], __ldg(&L.tw[kk * t1]), FWD);
    }
    fbutterfly<R>(x, FWD, L);
    const int o = jq * Ns * R + jm;
#pragma unroll
    for (int q = 0; q < R; ++q) dst[fswz(o + q * Ns, swz) * C + c] = x[q];
  }
}

// Transforms lines of `data` in place.  CTA blockIdx.x: part h = blockIdx.x mod S of line group
// blockIdx.x / S; group g of plane p holds lines q = g C + c (c < C, q < nlines), line q being
// line q (q < split_at) or q + skip of the plane, element i at p * plane_elems + line *
// line_stride + i * elem_stride.  Elements lhalf .. N - lhalf - 1 of a line are known zeros (not
// loaded); only outputs o < shalf or o >= N - shalf are stored.
template <int C, int TMAX, int MINB, bool FWD>
__global__ void __launch_bounds__(TMAX, MINB)
k_fft_lines_f32(const __grid_constant__ F32Lines L, float2* __restrict__ data, int64_t plane_elems,
                int groups, int nlines, int line_stride, int elem_stride, int split_at, int skip,
                int lhalf, int shalf) {
  extern __shared__ __align__(16) float2 fsm2[];
  const int n = L.n, S = L.S, N = L.N;
  const int T = blockDim.x;
  const int swz = (n & 7) == 0 ? 7 : 0;
  constexpr bool fwd = FWD;
  const int h = S > 1 ? (int)(blockIdx.x % (unsigned)S) : 0;   // rank in the cluster (S, 1, 1)
  const unsigned lg = blockIdx.x / (unsigned)S;
  const unsigned plane = lg / (unsigned)groups;
  const int grp = (int)(lg - plane * (unsigned)groups);
  float2* A = fsm2;
  float2* B = fsm2 + (size_t)n * C;
  const int c = C == 1 ? 0 : (int)(threadIdx.x % C);   // T is a multiple of C: fixed per thread
  const int q = grp * C + c;
  const bool valid = q < nlines;
  const int line = q < split_at ? q : q + skip;
  // one plane holds fewer than 2^31 elements: offsets within it are 32-bit
  float2* __restrict__ pl = data + (int64_t)plane * plane_elems + line * line_stride;
  const int i0 = h * n;

  // this CTA's part of the line(s): points [h n, h n + n)
  for (int e = threadIdx.x; e < n * C; e += T) {
    const int j = C == 1 ? e : e / C;
    const int i = i0 + j;
    float2 v = make_float2(0.f, 0.f);
    if (valid && (i < lhalf || i >= N - lhalf)) v = pl[i * elem_stride];
    A[fswz(j, swz) * C + c] = v;
  }
  float2* src = A;
  float2* dst = B;
  if (S > 1) {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const float2* part[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) part[r] = r < S ? cl.map_shared_rank(A, r) : A;
    for (int e = threadIdx.x; e < n * C; e += T) {
      const int j = C == 1 ? e : e / C;
      const int off = fswz(j, swz) * C + c;
      float2 y;
      if (S == 2) {
        const float2 x0 = part[0][off], x1 = part[1][off];
        y = h == 0 ? cadd(x0, x1) : csub(x0, x1);
      } else if (S == 4) {
        float2 x[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) x[r] = part[r][off];
        fdft4(x, fwd);
        y = x[0];
#pragma unroll
        for (int r = 1; r < 4; ++r) if (h == r) y = x[r];
      } else {
        float2 x[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) x[r] = part[r][off];
        fdft8(x, fwd, L.r2);
        y = x[0];
#pragma unroll
        for (int r = 1; r < 8; ++r) if (h == r) y = x[r];
      }
      if (h > 0) y = twmul(y, __ldg(&L.twN[j * h]), fwd);
      B[off] = y;
    }
    cl.sync();          // every part of A has been read: A is free for the stages
    src = B;
    dst = A;
  } else {
    __syncthreads();
  }

  int Ns = 1;
  for (int st = 0; st < L.nst; ++st) {
    const int R = L.radix[st];
    const unsigned dm = L.dmagic[st];
    switch (R) {
      case 2: fstage<2, C, FWD>(src, dst, n, Ns, dm, L, swz, c); break;
      case 3: fstage<3, C, FWD>(src, dst, n, Ns, dm, L, swz, c); break;
      case 4: fstage<4, C, FWD>(src, dst, n, Ns, dm, L, swz, c); break;
      case 5: fstage<5, C, FWD>(src, dst, n, Ns, dm, L, swz, c); break;
      case 7: fstage<7, C, FWD>(src, dst, n, Ns, dm, L, swz, c); break;
      case 8: fstage<8, C, FWD>(src, dst, n, Ns, dm, L, swz, c); break;
      default: fstage<11, C, FWD>(src, dst, n, Ns, dm, L, swz, c); break;
    }
    __syncthreads();
    float2* t = src; src = dst; dst = t;
    Ns *= R;
  }

  if (C == 1 && S > 1) {
    // output o = k S + r sits at position k of part r: gather through the cluster so that this
    // CTA stores the contiguous run [h n, h n + n)
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    for (int e = threadIdx.x; e < n; e += T) {
      const int o = i0 + e;
      const int k = o / S, r = o - k * S;
      if (valid && (o < shalf || o >= N - shalf))
        pl[o * elem_stride] = cl.map_shared_rank(src, (unsigned)r)[fswz(k, swz)];
    }
    cl.sync();          // the other parts have read this CTA's results
  } else {
    for (int e = threadIdx.x; e < n * C; e += T) {
      const int k = C == 1 ? e : e / C;
      const int o = k * S + h;
      if (valid && (o < shalf || o >= N - shalf))
        pl[o * elem_stride] = src[fswz(k, swz) * C + c];
    }
  }
}

bool smooth_part(int n) {
  if (n < 2) return false;
  int m = n;
  for (int p : {2, 3, 5, 7, 11})
    while (m % p == 0) m /= p;
  return m == 1;
}

// radix plan for one CTA's n points
bool f32_radix_plan(int n, F32Lines* L) {
  if (!smooth_part(n)) return false;
  int k = 0, m = n, p2 = 0;
  while (m % 2 == 0) { m /= 2; ++p2; }
  if (p2 == 1) {
    L->radix[k++] = 2;
  } else if (p2 > 0) {
    int e8 = p2 / 3, rem = p2 % 3;
    if (rem == 1) --e8;
    for (int i = 0; i < e8; ++i) L->radix[k++] = 8;
    if (rem == 1) { L->radix[k++] = 4; L->radix[k++] = 4; }
    if (rem == 2) L->radix[k++] = 4;
  }
  for (int p : {5, 3, 7, 11})
    while (m % p == 0 && k < kF32MaxStages) { L->radix[k++] = p; m /= p; }
  if (m != 1) return false;
  L->nst = k;
  uint64_t ns = 1;
  for (int st = 0; st < k; ++st) {
    L->dmagic[st] = ns > 1 ? (unsigned)((1ull << 32) / ns + 1) : 0u;
    ns *= (uint64_t)L->radix[st];
  }
  return true;
}

// Shape of the line kernels (wg_fft_f32_tune): adjacent lines per CTA of the strided pass,
// points per CTA at most (both buffers: 16 bytes per point), points per thread and stage.
struct F32Tune {            // defaults: the fastest of a sweep on GB300 (2816- and 11264-point sides)
  int cols = 4;
  int max_points = kF32MaxPart;
  int per_thread = 16;
};
F32Tune g_tune;

// Split and shape of the lines of length N with up to C lines per CTA: the fewest CTAs per line
// (1, 2, 4, 8) whose part fits max_points (fewer lines per CTA if no split fits).
bool f32_line_shape(int N, int C, const F32Tune& tu, F32Lines* L) {
  for (int cc = C; cc >= 1; cc /= 2)
    for (int s : {1, 2, 4, 8}) {
      if (N % s != 0) continue;
      const int n = N / s;
      if (n < 2 || (int64_t)n * cc > tu.max_points) continue;
      F32Lines t;
      std::memset(&t, 0, sizeof(t));
      if (!f32_radix_plan(n, &t)) continue;
      t.N = N; t.n = n; t.S = s; t.C = cc;
      const int want = (n * cc + tu.per_thread - 1) / tu.per_thread;
      t.T = std::max(64, std::min(1024, (want + 31) / 32 * 32));
      *L = t;
      return true;
    }
  return false;
}

void host_twiddles(int len, int count, float2* h) {
  const long double two_pi = 6.283185307179586476925286766559L;
  for (int t = 0; t < count; ++t) {
    const long double a = two_pi * (long double)t / (long double)len;
    h[t] = make_float2((float)cosl(a), (float)-sinl(a));
  }
}

void odd_constants(int R, OddRadix* K) {
  const long double two_pi = 6.283185307179586476925286766559L;
  std::memset(K, 0, sizeof(*K));
  for (int k = 1; k <= (R - 1) / 2; ++k) {
    K->c[k - 1] = (float)cosl(two_pi * k / R);
    K->s[k - 1] = (float)sinl(two_pi * k / R);
  }
}

}  // namespace

int f32_line_split(int64_t n) {
  if (n < 2 || n > kF32MaxSide) return 0;
  F32Tune tu;
  tu.max_points = kF32MaxPart;
  F32Lines L;
  return f32_line_shape((int)n, 1, tu, &L) ? L.S : 0;
}

bool f32_fft_supported(int64_t nu, int64_t nv) {
  return f32_line_split(nu) != 0 && f32_line_split(nv) != 0;
}

int f32_fft_tune(int cols, int max_points, int per_thread) {
  F32Tune t;
  if (cols != 0) t.cols = cols;
  if (max_points != 0) t.max_points = max_points;
  if (per_thread != 0) t.per_thread = per_thread;
  if (t.cols != 1 && t.cols != 2 && t.cols != 4 && t.cols != 8) return -1;
  if (t.max_points < 64 || t.max_points > kF32MaxPart) return -1;
  if (t.per_thread < 2 || t.per_thread > 64) return -1;
  g_tune = t;
  return 0;
}

struct F32Fft {
  int nu = 0, nv = 0;
  F32Lines cols, rows;      // lines along u (the strided column pass), along v (the row pass)
  float2* tw_c = nullptr;
  float2* tw_r = nullptr;
};

static cudaError_t make_f32_lines(int N, int C, const F32Tune& tu, F32Lines* L, float2** tw) {
  std::memset(L, 0, sizeof(*L));
  if (!f32_line_shape(N, C, tu, L)) {
    // a side the tuned part size cannot take: the largest part the kernels allow
    F32Tune big = tu;
    big.max_points = kF32MaxPart;
    if (!f32_line_shape(N, C, big, L)) return cudaErrorInvalidValue;
  }
  const int n = L->n, S = L->S;
  const int ntab = S > 1 ? n + N : n;
  std::vector<float2> h(ntab);
  host_twiddles(n, n, h.data());
  if (S > 1) host_twiddles(N, N, h.data() + n);
  cudaError_t e = cudaMalloc((void**)tw, sizeof(float2) * ntab);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(*tw, h.data(), sizeof(float2) * ntab, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  L->tw = *tw;
  L->twN = S > 1 ? *tw + n : nullptr;
  odd_constants(3, &L->r3);
  odd_constants(5, &L->r5);
  odd_constants(7, &L->r7);
  odd_constants(11, &L->r11);
  L->r2 = (float)(sqrtl(2.0L) / 2);
  return cudaSuccess;
}

// (lines per CTA, threads at most, CTAs per SM the registers must allow, direction)
#define WG_F32_VARIANTS(X)                                                                   \
  X(1, 512, 2, true) X(1, 1024, 1, true) X(2, 512, 2, true) X(2, 1024, 1, true)              \
  X(4, 512, 2, true) X(4, 1024, 1, true) X(8, 512, 2, true) X(8, 1024, 1, true)              \
  X(1, 512, 2, false) X(1, 1024, 1, false) X(2, 512, 2, false) X(2, 1024, 1, false)          \
  X(4, 512, 2, false) X(4, 1024, 1, false) X(8, 512, 2, false) X(8, 1024, 1, false)

cudaError_t f32_fft_create(int64_t nu, int64_t nv, F32Fft** out) {
  *out = nullptr;
  if (!f32_fft_supported(nu, nv)) return cudaErrorInvalidValue;
  F32Fft* f = new F32Fft();
  f->nu = (int)nu; f->nv = (int)nv;
  const F32Tune tu = g_tune;
  cudaError_t e = make_f32_lines((int)nu, tu.cols, tu, &f->cols, &f->tw_c);
  if (e == cudaSuccess) e = make_f32_lines((int)nv, 1, tu, &f->rows, &f->tw_r);
  const int smax = (int)(2 * (size_t)kF32MaxPart * sizeof(float2));
#define WG_ATTR(CC, TM, MB, FW)                                                               \
  if (e == cudaSuccess)                                                                       \
    e = cudaFuncSetAttribute(k_fft_lines_f32<CC, TM, MB, FW>,                                 \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  WG_F32_VARIANTS(WG_ATTR)
#undef WG_ATTR
  if (e != cudaSuccess) {
    if (f->tw_c) cudaFree(f->tw_c);
    if (f->tw_r) cudaFree(f->tw_r);
    delete f;
    return e;
  }
  *out = f;
  return cudaSuccess;
}

void f32_fft_destroy(F32Fft* f) {
  if (f == nullptr) return;
  if (f->tw_c) cudaFree(f->tw_c);
  if (f->tw_r) cudaFree(f->tw_r);
  delete f;
}

static cudaError_t launch_f32_lines(const F32Lines& L, float2* data, int64_t batch, int64_t plane,
                                    int nlines, int64_t line_stride, int64_t elem_stride, int fwd,
                                    int split_at, int skip, int lhalf, int shalf, cudaStream_t s) {
  if (nlines == 0 || batch == 0) return cudaSuccess;
  const size_t smem = 2 * sizeof(float2) * (size_t)L.n * L.C;
  const int groups = (nlines + L.C - 1) / L.C;
  const int64_t nblocks = batch * groups * L.S;
  if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)nblocks);
  cfg.blockDim = dim3((unsigned)L.T);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  std::memset(attr, 0, sizeof(attr));
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)L.S;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = L.S > 1 ? 1 : 0;
#define WG_LAUNCH(CC, TM, MB, FW)                                                               \
  return cudaLaunchKernelEx(&cfg, k_fft_lines_f32<CC, TM, MB, FW>, L, data, plane, groups,     \
                            nlines, (int)line_stride, (int)elem_stride, split_at, skip, lhalf, \
                            shalf)
#define WG_PICK(CC)                                                                             \
  {                                                                                             \
    if (L.T <= 512) { if (fwd) WG_LAUNCH(CC, 512, 2, true); else WG_LAUNCH(CC, 512, 2, false); } \
    else { if (fwd) WG_LAUNCH(CC, 1024, 1, true); else WG_LAUNCH(CC, 1024, 1, false); }          \
  }
  switch (L.C) {
    case 1: WG_PICK(1)
    case 2: WG_PICK(2)
    case 4: WG_PICK(4)
    default: WG_PICK(8)
  }
#undef WG_PICK
#undef WG_LAUNCH
  return cudaErrorInvalidValue;
}

// In-place transform of `batch` nu x nv complex64 planes, sign -1 forward, +1 inverse; keep_rows
// = keep_cols = 0: the full 2-D transform, else pruned to the image block as described above.
cudaError_t f32_fft_exec(F32Fft* f, float2* data, int64_t batch, int sign, cudaStream_t s,
                         int64_t keep_rows, int64_t keep_cols) {
  const int64_t plane = (int64_t)f->nu * f->nv;
  const int fwd = sign < 0 ? 1 : 0;
  const bool prune = keep_rows > 0 && keep_cols > 0;
  if (prune && ((keep_rows & 1) || (keep_cols & 1) || keep_rows > f->nu || keep_cols > f->nv))
    return cudaErrorInvalidValue;
  cudaError_t e;
  if (!prune) {
    e = launch_f32_lines(f->rows, data, batch, plane, f->nu, f->nv, 1, fwd, f->nu, 0, f->nv, f->nv, s);
    if (e != cudaSuccess) return e;
    return launch_f32_lines(f->cols, data, batch, plane, f->nv, 1, f->nv, fwd, f->nv, 0, f->nu, f->nu, s);
  }
  const int rh = (int)(keep_rows / 2), ch = (int)(keep_cols / 2);
  const int ncols = 2 * ch, cskip = f->nv - ncols;
  if (fwd) {
    e = launch_f32_lines(f->cols, data, batch, plane, ncols, 1, f->nv, fwd, ch, cskip, rh, f->nu, s);
    if (e != cudaSuccess) return e;
    return launch_f32_lines(f->rows, data, batch, plane, f->nu, f->nv, 1, fwd, f->nu, 0, ch, f->nv, s);
  }
  e = launch_f32_lines(f->rows, data, batch, plane, f->nu, f->nv, 1, fwd, f->nu, 0, f->nv, ch, s);
  if (e != cudaSuccess) return e;
  return launch_f32_lines(f->cols, data, batch, plane, ncols, 1, f->nv, fwd, ch, cskip, f->nu, rh, s);
}

}  // namespace wg
