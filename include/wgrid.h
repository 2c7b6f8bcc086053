/*
 * wgrid.h — C ABI of the GB300 w-gridding library (libwgrid.so).
 *
 * The library applies the wide-field radio-interferometric response operator
 *
 *     (R I)_k ~= (R0 I)_k = sum_{l,m} exp(-2 pi i [u_k l + v_k m - w_k (n_lm - 1)]) I_lm / n_lm
 *
 * (Arras et al., "Efficient wide-field radio interferometry response", Sec. 2, Eq. rime,
 * approximated by w-gridding, Eqs. nfft / R1-R3) and its exact adjoint R^dagger (Eqs.
 * adjnfft / Rad1-Rad2).  "degrid" is R (dirty image -> visibilities, the paper's
 * dirty2ms, App. B); "grid" is R^dagger (visibilities -> dirty image, ms2dirty).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array pointers are DEVICE pointers (cudaMalloc'd or managed), C order, contiguous,
 *    unless an argument says otherwise.  The caller owns every buffer; outputs are
 *    overwritten completely (masked visibilities get 0).
 *  - uvw:   (nrows, 3) float64, baseline coordinates in metres (Sec. 2).
 *    freq:  (nchan,)   float64, channel frequencies in Hz (> 0).
 *    Visibility k is (row, chan), k = row * nchan + chan; u_k = u~_row * freq_chan / c with
 *    c = 299792458 m/s (Sec. 2, effective coordinates).
 *  - dirty: (npix_x, npix_y) real, pixel (jx, jy) at l = (jx - npix_x/2) * pixsize_x,
 *    m = (jy - npix_y/2) * pixsize_y (Sec. 2, sets L and M); x pairs with u.
 *  - vis:   (nrows, nchan) complex, interleaved (re, im).
 *  - Precision (App. B: the data type selects the precision): WG_F32 uses float / complex64
 *    buffers, FP32 uv planes, FP32 (de)gridding and FP32 plane FFTs; WG_F64 uses double /
 *    complex128 buffers and an FP64-accurate pipeline, whose uv planes, plane FFTs and
 *    (de)gridding sums run either in FP64 (fft_impl 1 or 3) or, with the library's
 *    double-float FFT (fft_impl 2, the usual automatic choice), in double-float pair
 *    arithmetic on the FP32 pipes (a pair of floats, ~48-bit significand, unit roundoff
 *    2^-47); the planner sizes sigma so that this rounding stays inside epsilon.  Both modes
 *    form coordinates, plane indices and the per-visibility w-reference phase in FP64 and
 *    accumulate the gridded image in FP64.  The per-plane w-screen phase is FP64 in WG_F64;
 *    WG_F32 reduces it exactly in FP32 (a 13-bit split of Delta w (n - 1)) before sincospif.
 *  - wgt:   optional (nrows, nchan) real weights of the buffer precision; multiplies the
 *    degrid output and the grid input (App. B).  NULL = all ones.
 *  - mask:  optional (nrows, nchan) uint8; visibilities with mask == 0 are not processed
 *    (App. B).  It is fixed when the plan is made.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).  All device work
 *    of a call is ordered on it; calls return when the work is enqueued, except where an
 *    entry point says it synchronises.
 *  - Return value: WG_OK (0) or a WG_ERR_* code; wg_last_error() gives a message for the
 *    calling thread.  A failing call leaves outputs unspecified and the plan usable.
 */
#ifndef WGRID_H
#define WGRID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum wg_status {
  WG_OK = 0,
  WG_ERR_ARG = 1,     /* invalid argument (sizes, epsilon range, null pointer, FoV > unit disc) */
  WG_ERR_OOM = 2,     /* device allocation failed or exceeds the workspace cap */
  WG_ERR_CUDA = 3,    /* a CUDA runtime call failed (message has the CUDA error string) */
  WG_ERR_CUFFT = 4,   /* a cuFFT call failed */
  WG_ERR_TIMEOUT = 5, /* a bounded host wait on device work ran out (wg_wait) */
  WG_ERR_INTERNAL = 6 /* a device-side consistency check failed (e.g. plane index out of range) */
};

enum wg_precision { WG_F32 = 0, WG_F64 = 1 };

/* Opaque plan: geometry, kernel choice and the on-device visibility index for one set of
 * (uvw, freq, mask, image geometry, epsilon, precision).  Reusable for any number of
 * degrid / grid calls.  The plan's device data is read-only after creation and every
 * wg_degrid / wg_grid call allocates its own workspace, so those calls on one plan may run
 * concurrently on different streams (host threads included).  wg_plan_destroy waits for all
 * work on the plan's device before it frees the plan. */
typedef struct wg_plan wg_plan;

/* Options for wg_plan_create (zero-initialise, then set what you need). */
typedef struct wg_options {
  int do_wstacking;        /* 1: full w-gridding (Sec. 2); 0: w assumed zero (App. B) */
  int w_shift;             /* 1: grid w against (n - n_s) with n_s the mid-point of n over
                              the image (halves the plane count, see notes); 0: the paper's
                              Delta w = 1 / (2 sigma max|n - 1|) (Sec. 2). Default used by
                              wg_default_options: 1 */
  double eps_safety;       /* kernels are chosen with table epsilon <= epsilon * eps_safety
                              (default 0.8: the table value is a 1-D error, the gridding
                              combines the u, v and w errors) */
  size_t max_workspace;    /* cap on the per-call device workspace in bytes; 0 = automatic
                              (a fraction of the free device memory) */
  int force_alpha;         /* >0: only consider kernels with this support (tests) */
  double force_sigma;      /* >0: only consider this oversampling factor (tests) */
  int tile;                /* uv tile side in cells (16 or 32; 0 = automatic) */
  int grid_variant;        /* gridding accumulation: 0 = automatic (shared-memory atomics for
                              WG_F32, plane-owner warps for WG_F64), 1 = shared-memory atomics, 2 =
                              plane-owner warps (deterministic), 3 = row-band owner warps
                              (WG_F32, alpha <= 8, 32-cell tiles: each warp owns 4 rows of the
                              tile in every plane; deterministic; other plans fall back to 1);
                              WG_F64 plans with the double-float FFT always use plane-owner
                              warps (their planes are double-float pairs, written by that
                              kernel only) */
  int fft_impl;            /* plane FFTs: 0 = automatic (WG_F32: cuFFT C2C; WG_F64: the
                              cheaper of 2 and 3 whose predicted error fits epsilon),
                              1 = cuFFT 2-D, 2 = the library's double-float FFT (WG_F64 only,
                              grid sides up to 6400 with prime factors 2, 3, 5, 7, 11, and
                              sides up to 25600 that are 2 or 4 times such a side (each line
                              then runs on a thread-block cluster of 2 or 4 CTAs, as do lines
                              above 2048 points whose half needs only the radices 8, 4, 5,
                              3); its ~5e-15 rounding is amplified by the
                              1 / psi correction, so the planner may raise sigma for it; the
                              uv planes are then kept as double-float pairs and (de)gridded in
                              pair arithmetic),
                              3 = pruned cuFFT Z2Z (WG_F64 only: 1-D passes that skip the
                              plane rows outside the image),
                              4 = the library's FP32 FFT (WG_F32 only, never chosen
                              automatically: pruned to the image block, but measured about 2x
                              slower than cuFFT C2C per plane; sides up to 46340 that are 1, 2,
                              4 or 8 times a part of at most 12800 points with prime factors 2,
                              3, 5, 7, 11) */
  int compact_index;       /* 1: the plan keeps a compact index -- 4 bytes per visibility (its
                              position, in processing order) and a copy of uvw (24 bytes per
                              row) -- and every call recomputes the visibilities' cell offsets,
                              kernel coordinates and w-reference phases into its workspace
                              (Sec. 4.3 keeps a compact index the same way), and a WG_F64 plan
                              keeps no kernel-value table either (evaluated per call); 0
                              (default): the plan keeps those records (32 bytes per visibility
                              in WG_F32, 56 in WG_F64) */
} wg_options;

/* Per-call statistics (optional output).  Stage times are CUDA-event times measured on the
 * call's stream; filling them synchronises the stream at the end of the call. */
typedef struct wg_stats {
  double ms_total;     /* whole call */
  double ms_prep;      /* per-call preparation: the records of a compact index and per-call
                          kernel values (FP64), when the plan does not keep them */
  double ms_screen;    /* w-screen + zero padding into the planes (Eq. R2) */
  double ms_fft;       /* cuFFT plane transforms (separately timed stage) */
  double ms_grid;      /* (de)gridding kernels (Eqs. R3 / Rad2) */
  double ms_accum;     /* conjugate screen + accumulation over planes + correction (Eq. Rad1) */
  int64_t n_batches;   /* plane batches processed */
  int64_t n_planes;    /* w-planes processed */
  size_t workspace_bytes; /* device workspace used by the call */
  int64_t n_kernels;   /* library kernels launched by the call, the double-float FFT's passes
                          included (cuFFT's own not counted) */
  int64_t n_fft_calls; /* plane-FFT executions (one per batch of planes) */
} wg_stats;

/* Plan parameters chosen by the planner (Sec. 4.1, App. A). */
typedef struct wg_plan_info {
  int alpha;           /* kernel support (cells) */
  double sigma;        /* oversampling factor of the chosen kernel */
  double beta, mu;     /* modified-ES kernel parameters (Eq. semicircle2) */
  double eps_kernel;   /* the kernel's table accuracy (App. A) */
  int64_t nu, nv;      /* uv grid size (cells) */
  int64_t nw;          /* number of w-planes */
  double dw, w0;       /* plane spacing and position of plane 0 (wavelengths) */
  double nshift;       /* reference n_s - 1 subtracted from n - 1 (0 for the paper's scheme) */
  int tile;            /* uv tile side */
  int64_t ntiles;      /* tiles in the uv grid */
  int64_t nvis;        /* visibilities in the plan (unmasked) */
  int64_t batch;       /* w-planes per batch */
  size_t index_bytes;  /* device bytes held by the plan (visibility index, per-pixel table, and
                          for FP64 plans with a full index the kernel-value table, 384 bytes per
                          visibility, when it fits a quarter of the free memory) */
  size_t workspace_bytes; /* device bytes a degrid / grid call allocates */
  double umax, vmax, wmin, wmax; /* |u|, |v| maxima and |w| range in wavelengths */
  int fft_impl;        /* plane FFT used: 1 cuFFT 2-D, 2 double-float, 3 pruned cuFFT Z2Z,
                          4 the library's FP32 FFT */
  double rounding_gain; /* factor by which relative plane rounding reaches the result: rms of
                           1 / (n psi_u psi_v psi_w) over the image x (int phi^2)^(3/2) */
  double err_model;    /* predicted eps_rms: kernel term eps_kernel / eps_safety and plane
                          rounding term (unit roundoff x c log2(nu nv) x rounding_gain, c = 0.065 (1 +
                          rounding_gain / 2000)),
                          added in quadrature; the planner keeps it <= epsilon unless sigma
                          is forced */
} wg_plan_info;

/* Fill *opt with defaults (do_wstacking = 1, w_shift = 1, eps_safety = 0.8, rest 0). */
void wg_default_options(wg_options* opt);

/*
 * wg_plan_create — plan the w-gridding of one observation (Sec. 2 and 4.1):
 * reads the uvw extent on the device, chooses (alpha, sigma, beta, mu) from the kernel
 * table of App. A with a cost model (Sec. 4.1), fixes the grid (Sec. 2: N = ceil(sigma n)),
 * Delta w, w_0 and N_w (Sec. 2, Eq. wcirc), builds the piecewise-polynomial kernel
 * (Sec. 4.2) and bins the visibilities into uv tiles and w-planes on the device
 * (the GPU counterpart of the index of Sec. 4.3).  Synchronises `stream`.
 *   uvw, freq, mask: device pointers as above (mask may be NULL); not retained.
 *   npix_x, npix_y: image size, even and >= 32 (App. B).
 *   epsilon: requested accuracy, > 2e-13 (App. B); WG_F32 requires epsilon >= 1e-5.
 *   opt: may be NULL (defaults).
 *   out: receives the plan; release with wg_plan_destroy.
 * Errors: WG_ERR_ARG (sizes, epsilon, pixel outside the unit disc, freq <= 0, no kernel
 * meets epsilon), WG_ERR_OOM, WG_ERR_CUDA, WG_ERR_CUFFT.
 */
int wg_plan_create(const double* uvw, const double* freq, int64_t nrows, int64_t nchan,
                   int64_t npix_x, int64_t npix_y, double pixsize_x, double pixsize_y,
                   double epsilon, int precision, const uint8_t* mask,
                   const wg_options* opt, void* stream, wg_plan** out);

/* Release a plan and its device memory.  Synchronises the plan's device first (every stream
 * on it, so calls still in flight on any stream finish before their index memory is freed). */
int wg_plan_destroy(wg_plan* plan);

/* Copy the plan parameters into *info (host call, no device work). */
int wg_plan_get_info(const wg_plan* plan, wg_plan_info* info);

/*
 * wg_degrid — vis = R(dirty) (Eqs. R1-R3; the paper's dirty2ms):
 * per batch of w-planes: w-screen and zero-pad the corrected image (Eqs. R1, R2), 2-D FFT
 * (cuFFT), degrid every visibility from the planes it touches (Eq. R3), accumulate.
 *   dirty: (npix_x, npix_y) float (WG_F32) or double (WG_F64), device.
 *   wgt:   optional weights, device, or NULL.
 *   vis:   (nrows, nchan) complex output, device.
 *   stats: optional; filling it synchronises the stream.
 * Allocates its workspace stream-ordered (cudaMallocAsync) and frees it before returning.
 */
int wg_degrid(wg_plan* plan, const void* dirty, const void* wgt, void* vis, void* stream,
              wg_stats* stats);

/*
 * wg_degrid_noalloc — the same result as wg_degrid, computed without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that cannot allocate device
 * memory while they run, e.g. code whose device memory is owned by another allocator (a
 * framework's caching allocator or a fixed arena, where a cudaMalloc could fail, fragment the
 * arena or synchronise the device) and real-time loops that must not allocate between
 * set-up and shutdown.  Such a caller creates the plan once at set-up (wg_plan_create does
 * allocate) with options.max_workspace <= WG_NOALLOC_SCRATCH_BYTES, then calls this entry
 * point as often as it likes.
 *   The per-call workspace (uv planes and the cuFFT work area) lives in one
 * file-scope device array of WG_NOALLOC_SCRATCH_BYTES (64 MiB) that every GPU which loads the
 * library holds until the process exits.  Nothing in it has to start at zero.  This call makes
 * no cudaMalloc / cudaFree or other allocating call; the plan's cuFFT handles run on the
 * scratch through cufftSetWorkArea.
 *   The array's device address is looked up (cudaGetSymbolAddress, once per device) by
 * wg_plan_create, for plans whose per-call workspace fits the array, with the plan's device
 * current.  Under CUDA's lazy module loading that lookup is when the runtime loads the module
 * that holds the array and allocates its 64 MiB, so create such plans during set-up, where
 * allocation is allowed, and before any stream capture.  The plan's device must be current.
 *   All calls share the one array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU (other streams, other threads, other plans) race and corrupt each
 * other's results; order them on one stream or synchronise between them.
 * Arguments as for wg_degrid (no stats).  Errors: WG_ERR_ARG when the plan's per-call
 * workspace (wg_plan_info.workspace_bytes) exceeds WG_NOALLOC_SCRATCH_BYTES, for NULL
 * arguments or a different current device; WG_ERR_CUDA, WG_ERR_CUFFT as for wg_degrid.
 */
#define WG_NOALLOC_SCRATCH_BYTES (64ull << 20)
int wg_degrid_noalloc(wg_plan* plan, const void* dirty, const void* wgt, void* vis, void* stream);

/*
 * wg_grid — dirty = R^dagger(vis) (Eqs. Rad1, Rad2; the paper's ms2dirty): per batch of
 * w-planes: grid the visibilities onto the planes (Eq. Rad2), inverse 2-D FFT (cuFFT),
 * multiply by the conjugate w-screen and accumulate over planes; finally divide by
 * n * Psi and keep the real part (Eq. Rad1).
 *   vis:   (nrows, nchan) complex input, device.  wgt: optional, device, or NULL.
 *   dirty: (npix_x, npix_y) real output, device.
 */
int wg_grid(wg_plan* plan, const void* vis, const void* wgt, void* dirty, void* stream,
            wg_stats* stats);

/*
 * One-shot forms with the paper's argument order (App. B): plan, run, destroy.
 * do_wstacking as in App. B.  Synchronise `stream` (plan creation does).
 */
int wg_dirty2ms(const double* uvw, const double* freq, int64_t nrows, int64_t nchan,
                const void* dirty, const void* wgt, int64_t npix_x, int64_t npix_y,
                double pixsize_x, double pixsize_y, double epsilon, int precision,
                int do_wstacking, const uint8_t* mask, void* vis, void* stream);
int wg_ms2dirty(const double* uvw, const double* freq, int64_t nrows, int64_t nchan,
                const void* vis, const void* wgt, int64_t npix_x, int64_t npix_y,
                double pixsize_x, double pixsize_y, double epsilon, int precision,
                int do_wstacking, const uint8_t* mask, void* dirty, void* stream);

/* The per-call workspaces come from a stream-ordered memory pool per device that keeps freed
 * memory cached for the next call (no release threshold).  wg_pool_trim releases the current
 * device's cached memory beyond keep_bytes back to the driver (cudaMemPoolTrimTo; memory of
 * calls still in flight is not touched).  For long-running callers that mix plans of many sizes
 * (a server), so that cached workspace does not crowd out new plans.  Errors: WG_ERR_CUDA. */
int wg_pool_trim(size_t keep_bytes);

/* Bounded host wait: returns WG_OK once all work enqueued on `stream` (void* cudaStream_t,
 * NULL = legacy default stream) so far has finished, WG_ERR_TIMEOUT if it has not finished
 * after timeout_ms milliseconds (the work keeps running; call again or give up on it), or
 * WG_ERR_CUDA if the stream reports an error.  timeout_ms < 0 waits without bound.  Polls
 * cudaStreamQuery with short sleeps; launches nothing. */
int wg_wait(void* stream, double timeout_ms);

/* Message of the last failing call on this thread ("" if none). Never NULL. */
const char* wg_last_error(void);

/* ------------------------------------------------------------------------------------
 * Host-only helpers (no device work; callable without a GPU).  They expose the planner
 * and kernel mathematics so they can be checked on their own.
 * ------------------------------------------------------------------------------------ */

/* Number of rows of the built-in kernel table (App. A, alpha in {4, 7, 8, 12, 16}). */
int wg_kernel_table_size(void);
/* Row i of the table: alpha, sigma, epsilon, beta, mu.  Returns WG_ERR_ARG if out of range. */
int wg_kernel_table_row(int i, int* alpha, double* sigma, double* eps, double* beta, double* mu);

/* Modified ES kernel phi(x) of Eq. (semicircle2), direct evaluation, for n points. */
int wg_kernel_phi(int alpha, double beta, double mu, const double* x, double* out, int64_t n);
/* The piecewise polynomial of Sec. 4.2 (alpha pieces of degree alpha+3, Chebyshev-node
 * interpolation) evaluated by Horner at n points x in grid cells (0 outside the support). */
int wg_kernel_poly(int alpha, double beta, double mu, const double* x, double* out, int64_t n);
/* psi(k) = int phi(x) exp(2 pi i k x) dx of the piecewise polynomial (Gauss-Legendre per
 * piece), k in cycles per cell, for n points. */
int wg_kernel_psi(int alpha, double beta, double mu, const double* k, double* out, int64_t n);

/* Kernels found by the same optimisation for the supports the paper does not print
 * (alpha 5, 6, 9, 10, 11, 13, 14, 15; sigma 1.15 to 2.0 in steps of 0.05); the planner uses
 * them beside the App. A table.  Row i: alpha, sigma, epsilon, beta, mu (WG_ERR_ARG if out of
 * range). */
int wg_kernel_design_size(void);
int wg_kernel_design_row(int i, int* alpha, double* sigma, double* eps, double* beta, double* mu);
/* Accuracy of the exact modified ES kernel (alpha, beta, mu) at oversampling sigma: the
 * supremum of the map error function l(x) of Eq. (maperror) over |x| <= 1 / (2 sigma) (Sec. 3.2,
 * App. A), with psi and the integral over the fractional position by tanh-sinh quadrature. */
int wg_kernel_eps(int alpha, double beta, double mu, double sigma, double* eps);
/* The kernel search of Sec. 3.2: (beta, mu) minimising wg_kernel_eps for (alpha, sigma),
 * Nelder-Mead on log epsilon from (beta0, mu0).  alpha in 2..16, sigma in [1.05, 2.5]. */
int wg_kernel_search(int alpha, double sigma, double beta0, double mu0, double* beta, double* mu,
                     double* eps);

/* Planner dry run: the parameters wg_plan_create would choose for the given image, epsilon,
 * precision, options and uvw extent (|u|max, |v|max, |w|min, |w|max in wavelengths) and
 * visibility count.  Fills alpha, sigma, beta, mu, eps_kernel, nu, nv, nw, dw, w0, nshift,
 * tile, ntiles of *info. */
int wg_plan_params(int64_t npix_x, int64_t npix_y, double pixsize_x, double pixsize_y,
                   double epsilon, int precision, const wg_options* opt, double umax,
                   double vmax, double wmin, double wmax, int64_t nvis, wg_plan_info* info);

/* Planner calibration: time the batched 2-D FFT of `batch` n x n planes on the current device,
 * `reps` executions after one warm-up, and return the mean time per plane in milliseconds.
 * impl 1 = cuFFT (C2C for WG_F32, Z2Z for WG_F64), 2 = the library's double-float FFT
 * (WG_F64 only), 4 = the library's FP32 FFT (WG_F32 only).  Allocates and frees its own device memory; synchronises the device.
 * Errors: WG_ERR_ARG (also for an unsupported size), WG_ERR_OOM, WG_ERR_CUFFT, WG_ERR_CUDA. */
int wg_fft_time(int64_t n, int precision, int64_t batch, int reps, int impl, double* ms_per_plane);

/* In-place unnormalised 2-D FFT of `batch` contiguous nu x nv complex planes (device pointer,
 * complex64 for WG_F32, complex128 for WG_F64), sign -1 = forward (e^{-2 pi i}), +1 = inverse,
 * with the same implementations the plans use (impl as for wg_fft_time).  Plans and frees its
 * transform on each call (a utility, not a hot path); synchronises `stream`. */
int wg_fft2d(void* data, int64_t nu, int64_t nv, int64_t batch, int precision, int impl, int sign,
             void* stream);

/* Shape of the library's FP32 plane FFT (impl 4) for the transforms and plans created after the
 * call, process-wide: `cols` adjacent columns per CTA in the strided pass (1, 2, 4 or 8; each
 * row segment a CTA reads is cols x 8 bytes), at most `max_points` line points per CTA (64 ..
 * 12800; 16 bytes of shared memory each; longer lines run on a cluster of 2, 4 or 8 CTAs) and
 * `per_thread` points per thread and stage (2 .. 64).  0 keeps an argument's default (4, 12800,
 * 16).  A calibration knob: results do not depend on it.  Not thread-safe against concurrent
 * plan creation.  Errors: WG_ERR_ARG for a value out of range (nothing changes). */
int wg_fft_f32_tune(int cols, int max_points, int per_thread);

/* Arithmetic peak of the current device: FP32 (precision WG_F32) or FP64 (WG_F64) fused
 * multiply-add throughput in flop/s (an FMA counts 2), the best of five timed launches of
 * independent FMA chains on every SM (CUDA events, after a warm-up launch).  The roofline
 * denominator of the library's ALU-bound kernels.  Allocates and frees a small output buffer;
 * synchronises the device.  Errors: WG_ERR_ARG, WG_ERR_OOM, WG_ERR_CUDA. */
int wg_fma_peak(int precision, double* flops_per_s);

/* Library version string. */
const char* wg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WGRID_H */
