// Internal declarations of the GB300 w-gridder: plan layout, kernel parameter blocks and
// kernel launchers.  Not part of the public ABI (see include/wgrid.h).
#pragma once
#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "host_math.h"
#include "wgrid.h"

namespace wg {

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

// Per-visibility record of the on-device index, in tile-sorted order (structure of arrays).
//   idx:  k | (folded << 31)           (k = row * nchan + chan)
//   meta: du | dv << 8 | c0 << 16      (first cell inside the source tile, first w-plane)
//   z:    Horner coordinates zu, zv, zw in [-1, 1) of the first kernel piece (Sec. 4.2)
//   ph:   exp(2 pi i w_k nshift) (only when the w reference is shifted)
template <typename R> struct alignas(4 * sizeof(R)) Z4 { R u, v, w, pad; };

constexpr uint32_t kFoldBit = 0x80000000u;

// Geometry shared by all device kernels of a plan (passed by value).
struct Geom {
  int64_t nrows, nchan, nvis;
  int nx, ny;
  int nu, nv, nw;
  int tile, ntu, ntv;
  int alpha, deg;
  int do_w;
  int alpha_w;          // alpha when w-gridding, 1 otherwise (a single plane, weight 1)
  double psx, psy;
  double w0, dw, nshift;
  double w0_dw;         // w0 / dw
  int grid_variant;     // 0 automatic, 1 shared atomics, 2 plane-owner warps, 3 row-band owners
  int df64_planes;      // FP64 plans with the double-float FFT: the uv planes hold double-float
                        // pairs (float4 per cell) and (de)gridding runs in pair arithmetic
};

// Kernel polynomial coefficients, layout [d][G] so lane j reads c[d * kMaxG + j].
constexpr int kMaxG = 16;
template <typename R> struct Coef { R c[(kMaxDeg + 1) * kMaxG]; };

// psi_w Chebyshev coefficients (in y = 8 k^2 - 1) and per-axis correction tables.
struct ImgParams {
  Geom g;
  double psi_c[kPsiChebTerms];
  const double* cinv_u;  // (nx) 1 / psi_u((jx - nx/2) / nu)
  const double* cinv_v;  // (ny)
};

template <typename R>
struct IndexView {
  const uint32_t* off;     // (ntiles * nw + 1) start of bucket (tile, c0)
  const uint32_t* idx;
  const uint32_t* meta;
  const Z4<R>* z;
  const typename C2<R>::T* ph;  // may be null
  // optional per-visibility kernel values (u, v, w pieces, each padded to kMaxG), evaluated once
  // per call instead of on every (tile, sub-batch) visit; null = evaluate by Horner
  const R* wts;
};

struct PlanImpl;

// Record `msg` as this thread's wg_last_error() message and return `code`.
int report_error(int code, const char* msg);

// ---- double-float FFT (fft_df64.cu) -----------------------------------------------------
struct Df64Fft;
bool df64_fft_supported(int64_t nu, int64_t nv);
cudaError_t df64_fft_create(int64_t nu, int64_t nv, Df64Fft** out);
void df64_fft_destroy(Df64Fft* f);
cudaError_t df64_fft_exec(Df64Fft* f, double2* data, int64_t batch, int sign, cudaStream_t s,
                          int64_t keep_rows = 0, int64_t keep_cols = 0, bool df64_planes = false,
                          bool image_pairs = false);

// ---- FP32 plane FFT (fft_f32.cu) -------------------------------------------------------
struct F32Fft;
int f32_line_split(int64_t n);   // CTAs per row line for side n (0: not supported)
bool f32_fft_supported(int64_t nu, int64_t nv);
// shape of the line kernels for transforms created afterwards (0 keeps a default); -1: invalid
int f32_fft_tune(int cols, int max_points, int per_thread);
cudaError_t f32_fft_create(int64_t nu, int64_t nv, F32Fft** out);
void f32_fft_destroy(F32Fft* f);
cudaError_t f32_fft_exec(F32Fft* f, float2* data, int64_t batch, int sign, cudaStream_t s,
                         int64_t keep_rows = 0, int64_t keep_cols = 0);

// ---- index kernels (kernels_index.cu) ------------------------------------------------
cudaError_t launch_extent(const double* uvw, int64_t nrows, unsigned long long* ext4,
                          cudaStream_t s);
cudaError_t launch_bin_count(const Geom& g, const double* uvw, const double* chan4,
                             const uint8_t* mask, uint32_t* hist, uint32_t* key,
                             uint32_t* rank, int* err, cudaStream_t s);
cudaError_t launch_scan(uint32_t* data, int64_t n, uint32_t* scratch, cudaStream_t s);
size_t scan_scratch_elems(int64_t n);
template <typename R>
cudaError_t launch_bin_scatter(const Geom& g, const double* uvw, const double* chan4,
                               const uint32_t* key, const uint32_t* rank, const uint32_t* off,
                               uint32_t* idx, uint32_t* meta, Z4<R>* z,
                               typename C2<R>::T* ph, cudaStream_t s);

// records of a compact index (idx only) recomputed per call: meta, z and (if ph) the w-reference
// phase of index positions 0 .. nvis_idx - 1
template <typename R>
cudaError_t launch_expand(const Geom& g, const double* uvw, const double* chan4,
                          const uint32_t* idx, int64_t nvis_idx, uint32_t* meta, Z4<R>* z,
                          typename C2<R>::T* ph, cudaStream_t s);

// ---- image-side kernels (kernels_image.cu) -------------------------------------------
// table: per pixel (corr, A, Bhi, Blo) for f32, (corr, A, B, 0) for f64; corr = 1/(n Psi).
template <typename R>
cudaError_t launch_prep(const ImgParams& P, Z4<R>* table, cudaStream_t s);
template <typename R>
cudaError_t launch_screen(const Geom& g, const R* dirty, const Z4<R>* table,
                          typename C2<R>::T* planes, int b0, int nb, bool image_only,
                          cudaStream_t s);
template <typename R>
cudaError_t launch_accumulate(const Geom& g, const Z4<R>* table,
                              const typename C2<R>::T* planes, int b0, int nb, double* acc,
                              bool first, bool last, R* dirty, cudaStream_t s);

// the same for FP64 plans whose planes hold double-float pairs on the image side as well
// (float4 per cell), in pair arithmetic
cudaError_t launch_screen_dd(const Geom& g, const double* dirty, const Z4<double>* table,
                             float4* planes, int b0, int nb, cudaStream_t s);
cudaError_t launch_accumulate_dd(const Geom& g, const Z4<double>* table, const float4* planes,
                                 int b0, int nb, double* acc, bool first, bool last,
                                 double* dirty, cudaStream_t s);

// ---- (de)gridding kernels (kernels_grid.cu) ------------------------------------------
// kernel values of every indexed visibility: wts[pos * 3 kMaxG + d kMaxG + j]
template <typename R>
cudaError_t launch_weights(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                           int64_t nvis_idx, R* wts, cudaStream_t s);
// planes per degrid CTA (shared-memory budget); plane batches are multiples of it
template <typename R>
int degrid_subbatch(const Geom& g);
// partial sums: slot (sub-batch id - first sub-batch id of the visibility) x visibility position
template <typename R>
cudaError_t launch_degrid(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                          const typename C2<R>::T* planes, int b0, int nb, int bs,
                          typename C2<R>::T* partial, int64_t nvis_idx, cudaStream_t s);
template <typename R>
cudaError_t launch_degrid_finalize(const Geom& g, const IndexView<R>& ix,
                                   const typename C2<R>::T* partial, int64_t nvis_idx, int bs,
                                   const R* wgt, typename C2<R>::T* vis, cudaStream_t s);
// For double-float planes (g.df64_planes) `vis` is the output of launch_grid_vis_dd and `wgt`
// is not used.
template <typename R>
cudaError_t launch_grid(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                        const typename C2<R>::T* vis, const R* wgt,
                        typename C2<R>::T* planes, int b0, int nb, cudaStream_t s);
// weighted, folded, phase-rotated visibility data per index position as double-float pairs
cudaError_t launch_grid_vis_dd(const IndexView<double>& ix, const double2* vis, const double* wgt,
                               int64_t nvis_idx, float4* out, cudaStream_t s);

}  // namespace wg
