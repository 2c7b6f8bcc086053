// 2-D complex FFT of FP32 planes on the library's own line kernels, with the image-block pruning
// of the double-float FFT (fft_df64.cu): forward, the strided column pass runs over the image
// columns only and loads only their image rows, then the row pass over all rows loads only the
// image columns; inverse, the row pass stores only the image columns and the column pass over
// those stores only the image rows.  The screen therefore writes only the image cells and the
// accumulation reads only them (two passes over HBM per plane instead of the three or more of a
// full 2-D transform of the zero-padded plane).
//
// Each 1-D transform is a mixed-radix (8 and 4 for the power of two, 2 only for n = 2 * odd,
// then 5, 3, and a generic radix for 7 / 11) Stockham autosort FFT in shared memory (two
// buffers, ping-pong), n / 8 threads per line half.  Lines longer than kF32MaxPart run on S = 2
// or 4 CTAs: CTA h transforms y_h[j] = e^{-/+ 2 pi i j h / n} sum_r x[j + r n / S]
// e^{-/+ 2 pi i r h / S} (one radix-S decimation-in-frequency step folded into its loads) and
// stores the line's outputs S k + h.  Twiddles come from FP64-accurate tables.  Transforms are
// unnormalised, forward = e^{-2 pi i}, like cuFFT's.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host_math.h"
#include "wgrid_internal.h"

namespace wg {

namespace {

constexpr int kF32MaxStages = 24;

struct F32Line {
  int n;                    // points held by one CTA
  int split;                // CTAs per line (1, 2, 4)
  int nst, threads;
  int radix[kF32MaxStages];
  const float2* tw;         // e^{-2 pi i t / n}, t < n
  const float2* tw2;        // e^{-2 pi i t / (S n)}, t < S n (split lines)
  float c31, c51, c52, s51, s52, r2;
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i
__device__ __forceinline__ float2 cmul_mi(float2 a, bool fwd) {
  return fwd ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}
__device__ __forceinline__ float2 twid(const float2* __restrict__ tw, int t, bool fwd) {
  const float2 w = __ldg(&tw[t]);
  return fwd ? w : make_float2(w.x, -w.y);
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
__device__ __forceinline__ void fdft8(float2* x, bool fwd, const F32Line& L) {
  float2 e[4] = {x[0], x[2], x[4], x[6]}, o[4] = {x[1], x[3], x[5], x[7]};
  fdft4(e, fwd);
  fdft4(o, fwd);
  // o_k *= W8^k
  {
    float2 a = o[1], r;
    if (fwd) { r.x = a.x + a.y; r.y = a.y - a.x; }   // (1 - i) a
    else { r.x = a.x - a.y; r.y = a.y + a.x; }       // (1 + i) a
    o[1] = cscale(r, L.r2);
    o[2] = cmul_mi(o[2], fwd);
    a = o[3];
    if (fwd) { r.x = a.y - a.x; r.y = -(a.x + a.y); }  // (-1 - i) a
    else { r.x = -(a.x + a.y); r.y = a.x - a.y; }       // (-1 + i) a
    o[3] = cscale(r, L.r2);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    x[q] = cadd(e[q], o[q]);
    x[q + 4] = csub(e[q], o[q]);
  }
}
__device__ __forceinline__ void fdft3(float2* x, bool fwd, const F32Line& L) {
  const float2 t1 = cadd(x[1], x[2]);
  const float2 y0 = cadd(x[0], t1);
  const float2 t2 = csub(x[0], cscale(t1, 0.5f));
  const float2 t3 = cmul_mi(cscale(csub(x[1], x[2]), L.c31), fwd);
  x[0] = y0;
  x[1] = cadd(t2, t3);
  x[2] = csub(t2, t3);
}
__device__ __forceinline__ void fdft5(float2* x, bool fwd, const F32Line& L) {
  const float2 t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
  const float2 t3 = csub(x[1], x[4]), t4 = csub(x[2], x[3]);
  const float2 y0 = cadd(x[0], cadd(t1, t2));
  const float2 a1 = cadd(x[0], cadd(cscale(t1, L.c51), cscale(t2, L.c52)));
  const float2 a2 = cadd(x[0], cadd(cscale(t1, L.c52), cscale(t2, L.c51)));
  const float2 b1 = cadd(cscale(t3, L.s51), cscale(t4, L.s52));
  const float2 b2 = csub(cscale(t3, L.s52), cscale(t4, L.s51));
  const float2 ib1 = cmul_mi(b1, fwd), ib2 = cmul_mi(b2, fwd);
  x[0] = y0;
  x[1] = cadd(a1, ib1);
  x[4] = csub(a1, ib1);
  x[2] = cadd(a2, ib2);
  x[3] = csub(a2, ib2);
}
// generic radix R (7, 11): y_q = sum_k x_k W_n^{k q n / R}
template <int R>
__device__ __forceinline__ void fdft_generic(float2* x, bool fwd, const float2* __restrict__ tw, int n) {
  float2 y[R];
  const int step = n / R;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    float2 acc = x[0];
#pragma unroll
    for (int kk = 1; kk < R; ++kk) acc = cadd(acc, cmul(x[kk], twid(tw, ((kk * q) % R) * step, fwd)));
    y[q] = acc;
  }
#pragma unroll
  for (int q = 0; q < R; ++q) x[q] = y[q];
}

template <int R>
__device__ __forceinline__ void fbutterfly(float2* x, bool fwd, const F32Line& L) {
  if (R == 2) fdft2(x);
  else if (R == 3) fdft3(x, fwd, L);
  else if (R == 4) fdft4(x, fwd);
  else if (R == 5) fdft5(x, fwd, L);
  else if (R == 8) fdft8(x, fwd, L);
  else fdft_generic<R>(x, fwd, L.tw, L.n);
}

// shared-memory position of line element e (low three bits XORed with the next three, lines
// that are a multiple of 8 long): spreads the stride-R accesses of the first stages over banks
__device__ __forceinline__ int fswz(int e, int swz) { return e ^ ((e >> 3) & swz); }

// one radix-R Stockham stage: butterfly j reads src[j + kk M], writes dst[(j / Ns) Ns R +
// j mod Ns + q Ns]
template <int R>
__device__ __forceinline__ void fstage(const float2* __restrict__ src, float2* __restrict__ dst,
                                       int n, int Ns, bool fwd, const F32Line& L, int swz) {
  const int M = n / R;
  const int tstep = n / (Ns * R);
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const int jq = j / Ns, jm = j - jq * Ns;
    float2 x[R];
#pragma unroll
    for (int kk = 0; kk < R; ++kk) x[kk] = src[fswz(j + kk * M, swz)];
    if (Ns > 1) {
#pragma unroll
      for (int kk = 1; kk < R; ++kk) x[kk] = cmul(x[kk], twid(L.tw, jm * kk * tstep, fwd));
    }
    fbutterfly<R>(x, fwd, L);
    const int idx = jq * Ns * R + jm;
#pragma unroll
    for (int q = 0; q < R; ++q) dst[fswz(idx + q * Ns, swz)] = x[q];
  }
}

// Transform lines gl = blockIdx.x (one line, or one line part when split, per CTA): line gl / S
// is line (gl / S) mod lines_per_plane of plane (gl / S) / lines_per_plane, element i at
// plane * plane_elems + line * line_stride + i * elem_stride; lines from `split_at` on are
// shifted by `skip`.  Elements lhalf .. N - lhalf - 1 of the whole line (N = S n) are known zeros
// and not loaded; only elements < shalf or >= N - shalf are stored.  kAll adds the rare
// radices 2, 7, 11.
template <int TMAX, int MINB, bool kAll, bool kSplit>
__global__ void __launch_bounds__(TMAX, MINB)
k_fft_lines_f32(const __grid_constant__ F32Line L, float2* __restrict__ data, int64_t plane_elems,
                int lines_per_plane, int64_t line_stride, int64_t elem_stride, int fwd,
                int split_at, int skip, int lhalf, int shalf, int64_t nlines) {
  extern __shared__ __align__(16) float2 fsm2[];
  const int n = L.n;
  const int S = kSplit ? L.split : 1;
  const int nfull = S * n;
  const int T = blockDim.x;
  const int swz = (n & 7) == 0 ? 7 : 0;
  const int64_t gl = blockIdx.x;
  if (gl >= nlines) return;
  float2* src = fsm2;
  float2* dst = fsm2 + n;
  const int64_t lid = gl / S;
  const int h = (int)(gl - lid * S);
  const int64_t plane = lid / lines_per_plane;
  int line = (int)(lid - plane * lines_per_plane);
  if (line >= split_at) line += skip;
  const int64_t base = plane * plane_elems + (int64_t)line * line_stride;
  const bool f = fwd != 0;
  auto elem = [&](int i) -> float2 {
    if (i >= lhalf && i < nfull - lhalf) return make_float2(0.f, 0.f);
    return data[base + (int64_t)i * elem_stride];
  };
  if constexpr (kSplit) {
#pragma unroll 2
    for (int j = threadIdx.x; j < n; j += T) {
      float2 x4[4];
      if (S == 2) {
        x4[0] = elem(j);
        x4[1] = elem(j + n);
        fdft2(x4);
      } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) x4[r] = elem(j + r * n);
        fdft4(x4, f);
      }
      float2 y = x4[h];
      if (h > 0) y = cmul(y, twid(L.tw2, j * h, f));
      src[fswz(j, swz)] = y;
    }
  } else {
#pragma unroll 4
    for (int i = threadIdx.x; i < n; i += T) src[fswz(i, swz)] = elem(i);
  }
  __syncthreads();
  int Ns = 1;
  for (int s = 0; s < L.nst; ++s) {
    const int R = L.radix[s];
    switch (R) {
      case 3: fstage<3>(src, dst, n, Ns, f, L, swz); break;
      case 4: fstage<4>(src, dst, n, Ns, f, L, swz); break;
      case 5: fstage<5>(src, dst, n, Ns, f, L, swz); break;
      case 8: fstage<8>(src, dst, n, Ns, f, L, swz); break;
      default:
        if (kAll) {
          if (R == 2) fstage<2>(src, dst, n, Ns, f, L, swz);
          else if (R == 7) fstage<7>(src, dst, n, Ns, f, L, swz);
          else fstage<11>(src, dst, n, Ns, f, L, swz);
        }
        break;
    }
    __syncthreads();
    float2* t = src; src = dst; dst = t;
    Ns *= R;
  }
#pragma unroll 4
  for (int i = threadIdx.x; i < n; i += T) {
    const int o = S * i + h;
    if (o < shalf || o >= nfull - shalf) data[base + (int64_t)o * elem_stride] = src[fswz(i, swz)];
  }
}

// radix plan for one CTA's n points (same rules as the double-float FFT) and its CTA size
bool f32_line_plan(int n, F32Line* L) {
  if (n < 2 || n > kF32MaxPart) return false;
  int k = 0, m = n, p2 = 0;
  while (m % 2 == 0) { m /= 2; ++p2; }
  if (p2 == 1) {
    L->radix[k++] = 2;
  } else if (p2 > 0) {
    int e8 = p2 / 3, rem = p2 % 3;
    if (rem == 1) --e8;
    if (rem == 1 && e8 < 0) return false;   // p2 = 1 handled above
    for (int i = 0; i < e8; ++i) L->radix[k++] = 8;
    if (rem == 1) { L->radix[k++] = 4; L->radix[k++] = 4; }
    if (rem == 2) L->radix[k++] = 4;
  }
  for (int p : {5, 3, 7, 11})
    while (m % p == 0 && k < kF32MaxStages) { L->radix[k++] = p; m /= p; }
  if (m != 1) return false;
  L->nst = k;
  L->threads = std::max(64, std::min(1024, (n / 8 + 31) / 32 * 32));
  return true;
}

void host_twiddles(int len, int count, float2* h) {
  const long double two_pi = 6.283185307179586476925286766559L;
  for (int t = 0; t < count; ++t) {
    const long double a = two_pi * (long double)t / (long double)len;
    h[t] = make_float2((float)cosl(a), (float)-sinl(a));
  }
}

}  // namespace

int f32_line_split(int64_t n) {
  F32Line L;
  // first choice: the fewest CTAs per line with at most kF32SplitAbove points each (two CTAs
  // per SM fit up to that size); else the fewest with at most kF32MaxPart
  for (int64_t limit : {(int64_t)kF32SplitAbove, (int64_t)kF32MaxPart})
    for (int s : {1, 2, 4}) {
      if (n % s != 0 || n / s > limit) continue;
      std::memset(&L, 0, sizeof(L));
      if (f32_line_plan((int)(n / s), &L)) return s;
    }
  return 0;
}

bool f32_fft_supported(int64_t nu, int64_t nv) {
  return f32_line_split(nu) != 0 && f32_line_split(nv) != 0;
}

struct F32Fft {
  int nu = 0, nv = 0;
  F32Line lu, lv;
  float2* tw_u = nullptr;
  float2* tw_v = nullptr;
};

static cudaError_t make_f32_line(int nline, F32Line* L, float2** tw) {
  std::memset(L, 0, sizeof(*L));
  const int S = f32_line_split(nline);
  if (S == 0) return cudaErrorInvalidValue;
  const int n = nline / S;
  if (!f32_line_plan(n, L)) return cudaErrorInvalidValue;
  L->n = n;
  L->split = S;
  const int ntab = S > 1 ? n + nline : n;
  std::vector<float2> h(ntab);
  host_twiddles(n, n, h.data());
  if (S > 1) host_twiddles(nline, nline, h.data() + n);
  cudaError_t e = cudaMalloc((void**)tw, sizeof(float2) * ntab);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(*tw, h.data(), sizeof(float2) * ntab, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  L->tw = *tw;
  L->tw2 = S > 1 ? *tw + n : nullptr;
  const long double pi = 3.141592653589793238462643383279L;
  L->c31 = (float)sinl(2 * pi / 3);
  L->c51 = (float)cosl(2 * pi / 5);
  L->c52 = (float)cosl(4 * pi / 5);
  L->s51 = (float)sinl(2 * pi / 5);
  L->s52 = (float)sinl(4 * pi / 5);
  L->r2 = (float)(sqrtl(2.0L) / 2);
  return cudaSuccess;
}

#define WG_F32_VARIANTS(X)                                                                   \
  X(512, 2, false, false) X(512, 1, true, false) X(512, 2, false, true) X(512, 1, true, true) \
  X(1024, 1, false, false) X(1024, 1, true, false) X(1024, 1, false, true) X(1024, 1, true, true)

cudaError_t f32_fft_create(int64_t nu, int64_t nv, F32Fft** out) {
  *out = nullptr;
  if (!f32_fft_supported(nu, nv)) return cudaErrorInvalidValue;
  F32Fft* f = new F32Fft();
  f->nu = (int)nu; f->nv = (int)nv;
  cudaError_t e = make_f32_line((int)nu, &f->lu, &f->tw_u);
  if (e == cudaSuccess) e = make_f32_line((int)nv, &f->lv, &f->tw_v);
  const int smax = (int)(2 * kF32MaxPart * sizeof(float2));
#define WG_ATTR(TM, MB, A, P)                                                                 \
  if (e == cudaSuccess)                                                                       \
    e = cudaFuncSetAttribute(k_fft_lines_f32<TM, MB, A, P>,                                   \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  WG_F32_VARIANTS(WG_ATTR)
#undef WG_ATTR
  if (e != cudaSuccess) {
    if (f->tw_u) cudaFree(f->tw_u);
    if (f->tw_v) cudaFree(f->tw_v);
    delete f;
    return e;
  }
  *out = f;
  return cudaSuccess;
}

void f32_fft_destroy(F32Fft* f) {
  if (f == nullptr) return;
  if (f->tw_u) cudaFree(f->tw_u);
  if (f->tw_v) cudaFree(f->tw_v);
  delete f;
}

static cudaError_t launch_f32_lines(const F32Line& L, float2* data, int64_t batch, int64_t plane,
                                    int lines_per_plane, int64_t line_stride, int64_t elem_stride,
                                    int fwd, int split_at, int skip, int lhalf, int shalf,
                                    cudaStream_t s) {
  if (lines_per_plane == 0 || batch == 0) return cudaSuccess;
  const size_t smem = 2 * sizeof(float2) * (size_t)L.n;
  const int64_t nlines = batch * lines_per_plane * L.split;
  if (nlines > 0x7fffffffLL) return cudaErrorInvalidValue;
  bool common = true;   // radices 8, 4, 5, 3 only
  for (int i = 0; i < L.nst; ++i)
    if (L.radix[i] == 2 || L.radix[i] == 7 || L.radix[i] == 11) common = false;
  const bool small = L.threads <= 512;
#define WG_LAUNCH(TM, MB, A, P)                                                                  \
  k_fft_lines_f32<TM, MB, A, P><<<(unsigned)nlines, L.threads, smem, s>>>(                     \
      L, data, plane, lines_per_plane, line_stride, elem_stride, fwd, split_at, skip, lhalf,   \
      shalf, nlines)
#define WG_PICK(TM, MB, MBALL)                                                                   \
  if (L.split > 1) { if (common) WG_LAUNCH(TM, MB, false, true); else WG_LAUNCH(TM, MBALL, true, true); } \
  else { if (common) WG_LAUNCH(TM, MB, false, false); else WG_LAUNCH(TM, MBALL, true, false); }
  // the rare radices (generic 7 / 11 DFTs) get more registers: one CTA per SM
  if (small) { WG_PICK(512, 2, 1) } else { WG_PICK(1024, 1, 1) }
#undef WG_PICK
#undef WG_LAUNCH
  return cudaGetLastError();
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
    e = launch_f32_lines(f->lv, data, batch, plane, f->nu, f->nv, 1, fwd, f->nu, 0, f->nv, f->nv, s);
    if (e != cudaSuccess) return e;
    return launch_f32_lines(f->lu, data, batch, plane, f->nv, 1, f->nv, fwd, f->nv, 0, f->nu, f->nu, s);
  }
  const int rh = (int)(keep_rows / 2), ch = (int)(keep_cols / 2);
  const int ncols = 2 * ch, cskip = f->nv - ncols;
  if (fwd) {
    e = launch_f32_lines(f->lu, data, batch, plane, ncols, 1, f->nv, fwd, ch, cskip, rh, f->nu, s);
    if (e != cudaSuccess) return e;
    return launch_f32_lines(f->lv, data, batch, plane, f->nu, f->nv, 1, fwd, f->nu, 0, ch, f->nv, s);
  }
  e = launch_f32_lines(f->lv, data, batch, plane, f->nu, f->nv, 1, fwd, f->nu, 0, f->nv, ch, s);
  if (e != cudaSuccess) return e;
  return launch_f32_lines(f->lu, data, batch, plane, ncols, 1, f->nv, fwd, ch, cskip, f->nu, rh, s);
}

}  // namespace wg
