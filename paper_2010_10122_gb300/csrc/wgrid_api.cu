// C ABI of the GB300 w-gridder (include/wgrid.h): plans, degrid / grid pipelines, one-shot
// calls and host-only helpers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <memory>
#include <string>
#include <thread>

#include "wgrid_internal.h"

using namespace wg;

// ---------------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------------
static thread_local std::string g_last_error;

static int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

// for the other translation units of the library (wgrid_internal.h)
int wg::report_error(int code, const char* msg) { return set_error(code, "%s", msg); }

#define WG_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return set_error(WG_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                       __FILE__, __LINE__);                                              \
  } while (0)

#define WG_CUFFT(call)                                                                   \
  do {                                                                                   \
    cufftResult r_ = (call);                                                             \
    if (r_ != CUFFT_SUCCESS)                                                             \
      return set_error(WG_ERR_CUFFT, "%s failed: cufftResult %d", #call, (int)r_);       \
  } while (0)

#define WG_TRY(call)              \
  do {                            \
    int rc_ = (call);             \
    if (rc_ != WG_OK) return rc_; \
  } while (0)

// ---------------------------------------------------------------------------------------
// stream-ordered device memory from a library pool (kept cached between calls)
// ---------------------------------------------------------------------------------------
static cudaMemPool_t device_pool(int dev) {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (pools[dev] == nullptr) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t thr = std::numeric_limits<uint64_t>::max();
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    pools[dev] = p;
  }
  return pools[dev];
}

static int pool_alloc(void** ptr, size_t bytes, int dev, cudaStream_t s) {
  *ptr = nullptr;
  if (bytes == 0) return WG_OK;
  cudaMemPool_t pool = device_pool(dev);
  if (pool == nullptr) return set_error(WG_ERR_CUDA, "cudaMemPoolCreate failed");
  cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes, pool, s);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(WG_ERR_OOM, "device allocation of %zu bytes failed", bytes);
  }
  if (e != cudaSuccess)
    return set_error(WG_ERR_CUDA, "cudaMallocFromPoolAsync: %s", cudaGetErrorString(e));
  return WG_OK;
}

static void pool_free(void* ptr, cudaStream_t s) {
  if (ptr != nullptr) cudaFreeAsync(ptr, s);
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------------------
// allocation-free degrid: the per-call workspace lives in a file-scope device array
// ---------------------------------------------------------------------------------------
static_assert(WG_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch size must keep 256-byte alignment");
static __device__ __align__(256) unsigned char g_noalloc_scratch[WG_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on device `dev` (which must be current).  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device and cached.
static int noalloc_scratch(int dev, unsigned char** out) {
  static std::mutex mu;
  static std::vector<unsigned char*> addr;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
  if (addr[dev] == nullptr) {
    void* a = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
    if (e != cudaSuccess || a == nullptr)
      return set_error(WG_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    addr[dev] = static_cast<unsigned char*>(a);
  }
  *out = addr[dev];
  return WG_OK;
}


// ---------------------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------------------
struct wg_plan {
  PlanParams pp;
  Geom g;
  int prec = 0;
  wg_options opt;
  int device = 0;
  int64_t nrows = 0, nchan = 0, nvis_total = 0, nvis = 0;
  double umax = 0, vmax = 0, wmin = 0, wmax = 0;
  // device data owned by the plan
  double* chan4 = nullptr;
  double* cinv_u = nullptr;
  double* cinv_v = nullptr;
  uint32_t* off = nullptr;
  uint32_t* idx = nullptr;
  uint32_t* meta = nullptr;
  void* z = nullptr;
  void* ph = nullptr;
  void* table = nullptr;   // per pixel: 1 / (n Psi) and the w-screen phase parameters
  // compact index: the plan keeps only idx (and a copy of uvw); every call recomputes the
  // records (meta, z, ph) into its workspace
  bool compact = false;
  bool use_ph = false;      // the records carry e^{2 pi i w nshift} (w reference shifted)
  double* uvw_dev = nullptr;
  size_t index_bytes = 0;
  Coef<float> coef_f;
  Coef<double> coef_d;
  double psi_c[kPsiChebTerms];
  // batching and FFT
  int64_t batch = 1;
  cufftHandle fft_full = 0, fft_rem = 0;
  bool has_full = false, has_rem = false;
  Df64Fft* dfft = nullptr;   // double-float plane FFT (WG_F64) instead of cuFFT
  F32Fft* ffft = nullptr;    // the library's FP32 plane FFT (WG_F32) instead of cuFFT
  // pruned cuFFT transform: 1-D row plan (rows of one image block) and column plan (all
  // columns of one plane); rows outside the image are skipped
  bool pruned = false;
  cufftHandle fft_row = 0, fft_col = 0;
  bool has_row = false, has_col = false;
  int degrid_bs = 1;         // planes per degrid CTA; batches are multiples of it
  bool use_wts = false;      // per-call kernel-value table (FP64, when it fits the workspace)
  void* wts_plan = nullptr;  // plan-resident kernel-value table (FP64, when it is small)
  int nslot = 1;             // degrid partial-sum slots per visibility
  size_t fft_ws = 0;
  size_t ws_bytes = 0;
  std::mutex fft_mu;
  // device address of the library's static scratch array (wg_degrid_noalloc), looked up when
  // the plan is made if its per-call workspace fits the array; null otherwise
  unsigned char* noalloc_ws = nullptr;
};

static size_t cplx_bytes(int prec) { return prec ? 16 : 8; }

void wg_default_options(wg_options* opt) {
  if (opt == nullptr) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->do_wstacking = 1;
  opt->w_shift = 1;
  opt->eps_safety = kDefaultEpsSafety;
}

static int free_plan_device(wg_plan* p) {
  void* ptrs[] = {p->chan4, p->cinv_u, p->cinv_v, p->off, p->idx, p->meta, p->z, p->ph, p->table,
                  p->wts_plan, p->uvw_dev};
  for (void* q : ptrs)
    if (q != nullptr) cudaFree(q);
  if (p->has_full) cufftDestroy(p->fft_full);
  if (p->has_rem) cufftDestroy(p->fft_rem);
  p->has_full = p->has_rem = false;
  df64_fft_destroy(p->dfft);
  p->dfft = nullptr;
  f32_fft_destroy(p->ffft);
  p->ffft = nullptr;
  if (p->has_row) cufftDestroy(p->fft_row);
  if (p->has_col) cufftDestroy(p->fft_col);
  p->has_row = p->has_col = false;
  return WG_OK;
}

template <typename T>
static int dev_alloc(T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) return WG_OK;
  cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(WG_ERR_OOM, "cudaMalloc of %zu bytes failed", count * sizeof(T));
  }
  if (e != cudaSuccess) return set_error(WG_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(e));
  return WG_OK;
}

static int make_fft(cufftHandle* h, int prec, int64_t nu, int64_t nv, int64_t batch,
                    size_t* ws) {
  WG_CUFFT(cufftCreate(h));
  cufftResult r = cufftSetAutoAllocation(*h, 0);
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(*h);
    return set_error(WG_ERR_CUFFT, "cufftSetAutoAllocation: %d", (int)r);
  }
  long long n[2] = {(long long)nu, (long long)nv};
  r = cufftMakePlanMany64(*h, 2, n, nullptr, 1, 0, nullptr, 1, 0, prec ? CUFFT_Z2Z : CUFFT_C2C,
                          (long long)batch, ws);
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(*h);
    if (r == CUFFT_ALLOC_FAILED) return set_error(WG_ERR_OOM, "cuFFT plan allocation failed");
    return set_error(WG_ERR_CUFFT, "cufftMakePlanMany64 (%lld x %lld x %lld): %d", n[0], n[1],
                     (long long)batch, (int)r);
  }
  return WG_OK;
}

// 1-D batched transform of length n: element stride `stride`, transforms `dist` apart
static int make_fft1d(cufftHandle* h, int prec, int64_t n, int64_t stride, int64_t dist,
                      int64_t batch, size_t* ws) {
  WG_CUFFT(cufftCreate(h));
  cufftResult r = cufftSetAutoAllocation(*h, 0);
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(*h);
    return set_error(WG_ERR_CUFFT, "cufftSetAutoAllocation: %d", (int)r);
  }
  long long nn[1] = {(long long)n}, emb[1] = {(long long)n};
  r = cufftMakePlanMany64(*h, 1, nn, emb, (long long)stride, (long long)dist, emb,
                          (long long)stride, (long long)dist, prec ? CUFFT_Z2Z : CUFFT_C2C,
                          (long long)batch, ws);
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(*h);
    if (r == CUFFT_ALLOC_FAILED) return set_error(WG_ERR_OOM, "cuFFT plan allocation failed");
    return set_error(WG_ERR_CUFFT, "cufftMakePlanMany64 1-D (%lld): %d", nn[0], (int)r);
  }
  return WG_OK;
}

// per-call workspace layout
struct Workspace {
  size_t planes = 0, fft = 0, acc = 0, wts = 0, visd = 0, total = 0;   // acc: grid accumulator / degrid partials
  size_t rec = 0;   // compact index: the recomputed records (meta, z, ph) of every position
  size_t rec_meta = 0, rec_z = 0;   // offsets of z and ph inside the record region
};

static size_t z_bytes(int prec) { return prec ? sizeof(Z4<double>) : sizeof(Z4<float>); }

static Workspace workspace_layout(const wg_plan* p, int64_t batch, size_t fft_ws) {
  Workspace w;
  w.planes = align_up((size_t)batch * p->pp.nu * p->pp.nv * cplx_bytes(p->prec), 256);
  w.fft = align_up(fft_ws, 256);
  size_t grid_acc = (size_t)p->g.nx * p->g.ny * 8;
  size_t partials = (size_t)p->nslot * std::max<int64_t>(1, p->nvis) * cplx_bytes(p->prec);
  w.acc = align_up(std::max(grid_acc, partials), 256);
  w.wts = p->use_wts ? align_up((size_t)std::max<int64_t>(1, p->nvis) * 3 * kMaxG * 8, 256) : 0;
  // double-float planes: the gridding's prepared visibility data, a pair per part and position
  w.visd = p->g.df64_planes ? align_up((size_t)std::max<int64_t>(1, p->nvis) * 16, 256) : 0;
  if (p->compact) {
    const size_t n = (size_t)std::max<int64_t>(1, p->nvis);
    w.rec_meta = align_up(n * 4, 256);
    w.rec_z = align_up(n * z_bytes(p->prec), 256);
    w.rec = w.rec_meta + w.rec_z + (p->use_ph ? align_up(n * cplx_bytes(p->prec), 256) : 0);
  }
  w.total = w.planes + w.fft + w.acc + w.wts + w.visd + w.rec;
  return w;
}

static int build_index(wg_plan* p, const double* uvw, const uint8_t* mask, cudaStream_t s) {
  const Geom& g = p->g;
  const int64_t nkeys = (int64_t)g.ntu * g.ntv * g.nw;
  if (nkeys + 1 > (int64_t)std::numeric_limits<uint32_t>::max())
    return set_error(WG_ERR_ARG, "too many (tile, plane) buckets: %lld", (long long)nkeys);
  if (p->nvis_total >= (int64_t)kFoldBit)
    return set_error(WG_ERR_ARG, "at most 2^31 - 1 visibilities per plan");
  WG_TRY(dev_alloc(&p->off, (size_t)nkeys + 1));
  uint32_t *key = nullptr, *rank = nullptr, *scratch = nullptr;
  int* err = nullptr;
  int rc = WG_OK;
  size_t nscr = scan_scratch_elems(nkeys + 1);
  do {
    if ((rc = pool_alloc((void**)&key, sizeof(uint32_t) * std::max<int64_t>(1, p->nvis_total),
                         p->device, s)) != WG_OK) break;
    if ((rc = pool_alloc((void**)&rank, sizeof(uint32_t) * std::max<int64_t>(1, p->nvis_total),
                         p->device, s)) != WG_OK) break;
    if ((rc = pool_alloc((void**)&scratch, sizeof(uint32_t) * nscr, p->device, s)) != WG_OK) break;
    if ((rc = pool_alloc((void**)&err, sizeof(int), p->device, s)) != WG_OK) break;
    cudaError_t e = cudaMemsetAsync(p->off, 0, sizeof(uint32_t) * (nkeys + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_bin_count(g, uvw, p->chan4, mask, p->off, key, rank, err, s);
    if (e == cudaSuccess) e = launch_scan(p->off, nkeys + 1, scratch, s);
    uint32_t nvalid = 0;
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nvalid, p->off + nkeys, sizeof(uint32_t),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "index build: %s", cudaGetErrorString(e)); break; }
    if (herr != 0) { rc = set_error(WG_ERR_INTERNAL, "w-plane index out of range in index build"); break; }
    p->nvis = nvalid;
    size_t zsz = z_bytes(p->prec);
    size_t phsz = cplx_bytes(p->prec);
    size_t n = std::max<int64_t>(1, p->nvis);
    const bool use_ph = g.do_w && g.nshift != 0.0;
    p->use_ph = use_ph;
    if ((rc = dev_alloc(&p->idx, n)) != WG_OK) break;
    if (p->compact) {
      // a copy of uvw to recompute the records from; idx alone is scattered
      const size_t nr = (size_t)std::max<int64_t>(1, p->nrows) * 3;
      if ((rc = dev_alloc(&p->uvw_dev, nr)) != WG_OK) break;
      if (p->nrows > 0 &&
          (e = cudaMemcpyAsync(p->uvw_dev, uvw, sizeof(double) * 3 * p->nrows,
                               cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
        rc = set_error(WG_ERR_CUDA, "uvw copy: %s", cudaGetErrorString(e));
        break;
      }
      if (p->prec)
        e = launch_bin_scatter<double>(g, uvw, p->chan4, key, rank, p->off, p->idx, nullptr,
                                       nullptr, nullptr, s);
      else
        e = launch_bin_scatter<float>(g, uvw, p->chan4, key, rank, p->off, p->idx, nullptr,
                                      nullptr, nullptr, s);
      if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "index scatter: %s", cudaGetErrorString(e)); break; }
      p->index_bytes = sizeof(uint32_t) * (nkeys + 1) + n * 4 + nr * sizeof(double);
      break;
    }
    if ((rc = dev_alloc(&p->meta, n)) != WG_OK) break;
    if ((rc = dev_alloc((unsigned char**)&p->z, n * zsz)) != WG_OK) break;
    if (use_ph && (rc = dev_alloc((unsigned char**)&p->ph, n * phsz)) != WG_OK) break;
    if (p->prec)
      e = launch_bin_scatter<double>(g, uvw, p->chan4, key, rank, p->off, p->idx, p->meta,
                                     (Z4<double>*)p->z, (double2*)p->ph, s);
    else
      e = launch_bin_scatter<float>(g, uvw, p->chan4, key, rank, p->off, p->idx, p->meta,
                                    (Z4<float>*)p->z, (float2*)p->ph, s);
    if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "index scatter: %s", cudaGetErrorString(e)); break; }
    p->index_bytes = sizeof(uint32_t) * (nkeys + 1) + n * (8 + zsz + (use_ph ? phsz : 0));
  } while (0);
  pool_free(key, s); pool_free(rank, s); pool_free(scratch, s); pool_free(err, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (rc == WG_OK && e2 != cudaSuccess)
    rc = set_error(WG_ERR_CUDA, "index build: %s", cudaGetErrorString(e2));
  return rc;
}

static PlanInput plan_input(int64_t npix_x, int64_t npix_y, double psx, double psy, double eps,
                            int prec, const wg_options& o, double umax, double vmax,
                            double wmin, double wmax, int64_t nvis) {
  PlanInput in;
  in.nx = npix_x; in.ny = npix_y; in.psx = psx; in.psy = psy; in.eps = eps; in.prec = prec;
  in.do_w = o.do_wstacking; in.w_shift = o.w_shift; in.eps_safety = o.eps_safety;
  in.force_alpha = o.force_alpha; in.force_sigma = o.force_sigma; in.tile = o.tile;
  in.umax = umax; in.vmax = vmax; in.wmin = wmin; in.wmax = wmax; in.nvis = nvis;
  in.fft_impl = o.fft_impl;
  return in;
}

static void fill_coefs(wg_plan* p) {
  PolyKernel K = make_poly_kernel(p->pp.alpha, p->pp.beta, p->pp.mu, p->pp.alpha + 3);
  std::memset(&p->coef_f, 0, sizeof(p->coef_f));
  std::memset(&p->coef_d, 0, sizeof(p->coef_d));
  for (int i = 0; i < K.alpha; ++i)
    for (int d = 0; d <= K.deg; ++d) {
      double c = K.c[(size_t)i * (K.deg + 1) + d];
      p->coef_d.c[d * kMaxG + i] = c;
      p->coef_f.c[d * kMaxG + i] = (float)c;
    }
  std::vector<double> pc = psi_cheb_coeffs(K, kPsiChebTerms);
  for (int i = 0; i < kPsiChebTerms; ++i) p->psi_c[i] = pc[i];
}

int wg_plan_create(const double* uvw, const double* freq, int64_t nrows, int64_t nchan,
                   int64_t npix_x, int64_t npix_y, double pixsize_x, double pixsize_y,
                   double epsilon, int precision, const uint8_t* mask, const wg_options* opt,
                   void* stream, wg_plan** out) {
  if (out == nullptr) return set_error(WG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (precision != WG_F32 && precision != WG_F64) return set_error(WG_ERR_ARG, "bad precision");
  if (nrows < 0 || nchan < 1) return set_error(WG_ERR_ARG, "nrows must be >= 0 and nchan >= 1");
  if ((nrows > 0 && uvw == nullptr) || freq == nullptr) return set_error(WG_ERR_ARG, "uvw / freq is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<wg_plan> p(new wg_plan());
  if (opt) p->opt = *opt; else wg_default_options(&p->opt);
  if (p->opt.eps_safety <= 0) p->opt.eps_safety = kDefaultEpsSafety;
  if (p->opt.compact_index < 0 || p->opt.compact_index > 1)
    return set_error(WG_ERR_ARG, "compact_index must be 0 or 1");
  p->compact = p->opt.compact_index == 1;
  p->prec = precision;
  p->nrows = nrows; p->nchan = nchan; p->nvis_total = nrows * nchan;
  WG_CUDA(cudaGetDevice(&p->device));

  // channel frequencies and the uvw extent (device reduction)
  std::vector<double> f(nchan);
  WG_CUDA(cudaMemcpyAsync(f.data(), freq, sizeof(double) * nchan, cudaMemcpyDeviceToHost, s));
  unsigned long long* ext = nullptr;
  unsigned long long hext[4] = {0ull, 0ull, (unsigned long long)0x7fefffffffffffffull, 0ull};
  WG_TRY(pool_alloc((void**)&ext, sizeof(hext), p->device, s));
  WG_CUDA(cudaMemcpyAsync(ext, hext, sizeof(hext), cudaMemcpyHostToDevice, s));
  if (nrows > 0) WG_CUDA(launch_extent(uvw, nrows, ext, s));
  WG_CUDA(cudaMemcpyAsync(hext, ext, sizeof(hext), cudaMemcpyDeviceToHost, s));
  pool_free(ext, s);
  WG_CUDA(cudaStreamSynchronize(s));
  double fmin = std::numeric_limits<double>::max(), fmax = 0.0;
  for (double v : f) {
    if (!(v > 0.0) || !std::isfinite(v)) return set_error(WG_ERR_ARG, "frequencies must be positive");
    fmin = std::min(fmin, v); fmax = std::max(fmax, v);
  }
  double ext_d[4];
  for (int i = 0; i < 4; ++i) std::memcpy(&ext_d[i], &hext[i], sizeof(double));
  if (nrows == 0) ext_d[2] = 0.0;
  if (!std::isfinite(ext_d[0]) || !std::isfinite(ext_d[1]) || !std::isfinite(ext_d[3]))
    return set_error(WG_ERR_ARG, "uvw contains non-finite values");
  p->umax = ext_d[0] * fmax / kSpeedOfLight;
  p->vmax = ext_d[1] * fmax / kSpeedOfLight;
  p->wmin = p->opt.do_wstacking ? ext_d[2] * fmin / kSpeedOfLight : 0.0;
  p->wmax = p->opt.do_wstacking ? ext_d[3] * fmax / kSpeedOfLight : 0.0;
  if (p->umax * pixsize_x > 1e6 || p->vmax * pixsize_y > 1e6)
    return set_error(WG_ERR_ARG, "uv coordinates too large for the pixel size (|u| dl > 1e6)");

  char err[256];
  PlanInput in = plan_input(npix_x, npix_y, pixsize_x, pixsize_y, epsilon, precision, p->opt,
                            p->umax, p->vmax, p->wmin, p->wmax, p->nvis_total);
  if (choose_plan(in, p->pp, err, sizeof(err)) != 0) return set_error(WG_ERR_ARG, "%s", err);
  const PlanParams& pp = p->pp;
  Geom& g = p->g;
  g.nrows = nrows; g.nchan = nchan; g.nvis = p->nvis_total;
  g.nx = (int)npix_x; g.ny = (int)npix_y;
  g.nu = (int)pp.nu; g.nv = (int)pp.nv; g.nw = (int)pp.nw;
  g.tile = pp.tile; g.ntu = (int)pp.ntu; g.ntv = (int)pp.ntv;
  g.alpha = pp.alpha; g.deg = pp.alpha + 3;
  g.do_w = p->opt.do_wstacking ? 1 : 0;
  g.alpha_w = g.do_w ? pp.alpha : 1;
  g.psx = pixsize_x; g.psy = pixsize_y;
  g.w0 = pp.w0; g.dw = pp.dw; g.nshift = pp.nshift;
  g.w0_dw = pp.w0 / pp.dw;
  g.grid_variant = p->opt.grid_variant;
  if (g.grid_variant < 0 || g.grid_variant > 3) return set_error(WG_ERR_ARG, "grid_variant must be 0, 1, 2 or 3");
  fill_coefs(p.get());

  int rc = WG_OK;
  auto fail = [&](int code) { free_plan_device(p.get()); return code; };
  // per-channel scales and the per-axis correction 1 / psi
  {
    std::vector<double> c4(4 * nchan);
    for (int64_t ch = 0; ch < nchan; ++ch) {
      double s_ = f[ch] / kSpeedOfLight;
      c4[4 * ch + 0] = s_ * pixsize_x * pp.nu;
      c4[4 * ch + 1] = s_ * pixsize_y * pp.nv;
      c4[4 * ch + 2] = s_ / pp.dw;
      c4[4 * ch + 3] = s_;
    }
    std::vector<double> cu(npix_x), cv(npix_y);
    std::vector<double> pc(p->psi_c, p->psi_c + kPsiChebTerms);
    for (int64_t j = 0; j < npix_x; ++j)
      cu[j] = 1.0 / psi_cheb_eval(pc, (double)(j - npix_x / 2) / pp.nu);
    for (int64_t j = 0; j < npix_y; ++j)
      cv[j] = 1.0 / psi_cheb_eval(pc, (double)(j - npix_y / 2) / pp.nv);
    if ((rc = dev_alloc(&p->chan4, c4.size())) != WG_OK) return fail(rc);
    if ((rc = dev_alloc(&p->cinv_u, cu.size())) != WG_OK) return fail(rc);
    if ((rc = dev_alloc(&p->cinv_v, cv.size())) != WG_OK) return fail(rc);
    cudaError_t e = cudaMemcpy(p->chan4, c4.data(), sizeof(double) * c4.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->cinv_u, cu.data(), sizeof(double) * cu.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->cinv_v, cv.data(), sizeof(double) * cv.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(set_error(WG_ERR_CUDA, "upload: %s", cudaGetErrorString(e)));
  }
  if ((rc = build_index(p.get(), uvw, mask, s)) != WG_OK) return fail(rc);
  // per-pixel correction 1 / (n Psi) and screen phase parameters (Eqs. R1, R2, Rad1): depend
  // only on the geometry, so they are computed once and kept with the plan
  {
    size_t tb = (size_t)npix_x * npix_y * 4 * (precision ? 8 : 4);
    if ((rc = dev_alloc((unsigned char**)&p->table, tb)) != WG_OK) return fail(rc);
    ImgParams ip;
    ip.g = g;
    std::memcpy(ip.psi_c, p->psi_c, sizeof(ip.psi_c));
    ip.cinv_u = p->cinv_u; ip.cinv_v = p->cinv_v;
    cudaError_t e = precision ? launch_prep<double>(ip, (Z4<double>*)p->table, s)
                              : launch_prep<float>(ip, (Z4<float>*)p->table, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(set_error(WG_ERR_CUDA, "prep: %s", cudaGetErrorString(e)));
    p->index_bytes += tb;
  }

  // plane FFTs: the kind the planner chose (FP64: pruned cuFFT Z2Z or the double-float FFT,
  // whichever is cheaper with its rounding inside epsilon)
  const bool use_df64 = pp.fft_kind == kFftDf64;
  // with the double-float FFT the uv planes stay double-float pairs between the (de)gridding
  // kernels and the transform, and the (de)gridding arithmetic runs in pair arithmetic too
  g.df64_planes = use_df64 && precision == WG_F64 ? 1 : 0;
  if (use_df64 && !df64_fft_supported(pp.nu, pp.nv))
    return fail(set_error(WG_ERR_INTERNAL, "double-float FFT does not support %lld x %lld",
                          (long long)pp.nu, (long long)pp.nv));
  // batch of planes: as many as the workspace budget allows
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(set_error(WG_ERR_CUDA, "cudaMemGetInfo"));
  size_t budget = p->opt.max_workspace;
  if (budget == 0) budget = std::min<size_t>(free_b / 2, (size_t)96 << 30);
  const size_t plane_b = (size_t)pp.nu * pp.nv * cplx_bytes(precision);
  int64_t B = std::max<int64_t>(1, std::min<int64_t>(pp.nw, (int64_t)(budget / (2 * plane_b))));
  p->degrid_bs = precision ? degrid_subbatch<double>(g) : degrid_subbatch<float>(g);
  p->nslot = (g.alpha_w - 1 + p->degrid_bs - 1) / p->degrid_bs + 1;
  // degrid sub-batches must be aligned to multiples of degrid_bs across batches
  auto align_batch = [&](int64_t b) {
    return b >= p->degrid_bs ? b / p->degrid_bs * p->degrid_bs : b;
  };
  if (B < pp.nw) B = align_batch(B);
  if (B < p->degrid_bs && B < pp.nw) p->degrid_bs = (int)B;   // tiny budgets: one sub-batch per batch
  // FP64: Horner on every tile / sub-batch visit would put the (de)gridding on the FP64 pipe
  // (and double its work), so each visibility's kernel values are evaluated once: with the plan
  // (they depend only on the plan's coordinates), else once per call.
  // With an automatic workspace the per-call table may take up to a quarter of the free memory
  // on top of the plane budget (1e8 visibilities: 38 GB); under a caller's cap it must fit a
  // quarter of the cap
  const size_t wts_bytes = (size_t)std::max<int64_t>(1, p->nvis) * 3 * kMaxG * 8;
  // (a compact plan keeps no per-visibility data beyond its index, so no resident table).  A
  // per-call table would take the same memory for the call's duration (and the workspace pool
  // keeps it cached), so a full plan keeps the table whenever it fits a quarter of the free
  // memory: computed once instead of on every call (1e8 visibilities: 38 GB, ~0.2 s per call)
  const bool wts_resident = precision == WG_F64 && p->nvis > 0 && !p->compact &&
                            wts_bytes <= free_b / 4;
  p->use_wts = precision == WG_F64 && !wts_resident &&
               wts_bytes <= (p->opt.max_workspace == 0 ? free_b / 4 : budget / 4);
  const size_t wts_extra = (p->opt.max_workspace == 0 && p->use_wts) ? align_up(wts_bytes, 256) : 0;
  budget += wts_extra;
  p->nslot = (g.alpha_w - 1 + p->degrid_bs - 1) / p->degrid_bs + 1;
  if (pp.fft_kind == kFftF32) {
    if (precision != WG_F32 || !f32_fft_supported(pp.nu, pp.nv))
      return fail(set_error(WG_ERR_INTERNAL, "FP32 plane FFT does not support %lld x %lld",
                            (long long)pp.nu, (long long)pp.nv));
    cudaError_t e = f32_fft_create(pp.nu, pp.nv, &p->ffft);
    if (e != cudaSuccess) return fail(set_error(WG_ERR_CUDA, "FP32 FFT setup: %s", cudaGetErrorString(e)));
    p->fft_ws = 0;
    while (B > 1 && workspace_layout(p.get(), B, 0).total > budget)
      B = std::max<int64_t>(1, align_batch(B * 3 / 4));
    p->batch = B;
  } else if (use_df64) {
    cudaError_t e = df64_fft_create(pp.nu, pp.nv, &p->dfft);
    if (e != cudaSuccess) return fail(set_error(WG_ERR_CUDA, "double-float FFT setup: %s", cudaGetErrorString(e)));
    p->fft_ws = 0;
    while (B > 1 && workspace_layout(p.get(), B, 0).total > budget)
      B = std::max<int64_t>(1, align_batch(B * 3 / 4));
    p->batch = B;
  } else if (pp.fft_kind == kFftPrunedZ2Z) {
    // FP64 cuFFT is compute-bound on GB300: transform only the rows that hold the image
    // (degrid: rows are the first pass; grid: the last pass, on the rows the image needs)
    p->pruned = true;
    size_t ws_r = 0, ws_c = 0;
    if ((rc = make_fft1d(&p->fft_row, precision, pp.nv, 1, pp.nv, npix_x / 2, &ws_r)) != WG_OK) return fail(rc);
    p->has_row = true;
    if ((rc = make_fft1d(&p->fft_col, precision, pp.nu, pp.nv, 1, pp.nv, &ws_c)) != WG_OK) return fail(rc);
    p->has_col = true;
    p->fft_ws = std::max(ws_r, ws_c);
    while (B > 1 && workspace_layout(p.get(), B, p->fft_ws).total > budget)
      B = std::max<int64_t>(1, align_batch(B * 3 / 4));
    p->batch = B;
  } else {
    for (;;) {
      size_t ws = 0;
      if ((rc = make_fft(&p->fft_full, precision, pp.nu, pp.nv, B, &ws)) != WG_OK) {
        if (rc == WG_ERR_OOM && B > 1) { B = std::max<int64_t>(1, align_batch(B / 2)); continue; }
        return fail(rc);
      }
      p->has_full = true;
      Workspace w = workspace_layout(p.get(), B, ws);
      if (w.total <= budget || B == 1) { p->fft_ws = ws; break; }
      cufftDestroy(p->fft_full); p->has_full = false;
      B = std::max<int64_t>(1, align_batch(B * 3 / 4));
    }
    p->batch = B;
    int64_t rem = pp.nw % B;
    if (rem != 0) {
      size_t ws = 0;
      if ((rc = make_fft(&p->fft_rem, precision, pp.nu, pp.nv, rem, &ws)) != WG_OK) return fail(rc);
      p->has_rem = true;
      p->fft_ws = std::max(p->fft_ws, ws);
    }
  }
  if (wts_resident) {
    if ((rc = dev_alloc((unsigned char**)&p->wts_plan, wts_bytes)) != WG_OK) return fail(rc);
    IndexView<double> ixd{p->off, p->idx, p->meta, (const Z4<double>*)p->z,
                          (const double2*)p->ph, nullptr};
    void* zt = nullptr;   // compact index: the Horner coordinates, recomputed for this once
    uint32_t* mt = nullptr;
    if (p->compact) {
      if ((rc = pool_alloc(&zt, (size_t)p->nvis * sizeof(Z4<double>), p->device, s)) != WG_OK) return fail(rc);
      if ((rc = pool_alloc((void**)&mt, (size_t)p->nvis * 4, p->device, s)) != WG_OK) { pool_free(zt, s); return fail(rc); }
      cudaError_t ee = launch_expand<double>(g, p->uvw_dev, p->chan4, p->idx, p->nvis, mt,
                                             (Z4<double>*)zt, nullptr, s);
      if (ee != cudaSuccess) { pool_free(zt, s); pool_free(mt, s); return fail(set_error(WG_ERR_CUDA, "expand: %s", cudaGetErrorString(ee))); }
      ixd.z = (const Z4<double>*)zt;
      ixd.meta = mt;
    }
    cudaError_t e = launch_weights<double>(g, p->coef_d, ixd, p->nvis, (double*)p->wts_plan, s);
    pool_free(zt, s);
    pool_free(mt, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(set_error(WG_ERR_CUDA, "kernel values: %s", cudaGetErrorString(e)));
    p->index_bytes += wts_bytes;
  }
  p->ws_bytes = workspace_layout(p.get(), B, p->fft_ws).total;
  if (p->opt.max_workspace != 0 && p->ws_bytes > p->opt.max_workspace)
    return fail(set_error(WG_ERR_OOM, "one w-plane needs %zu bytes of workspace, above the cap %zu",
                          p->ws_bytes, (size_t)p->opt.max_workspace));
  // plans that wg_degrid_noalloc can run: look up the static scratch array now, while the
  // plan's device is current and allocation is allowed (under lazy module loading this is when
  // the CUDA runtime allocates the array), so that the calls themselves allocate nothing
  if (p->ws_bytes <= (size_t)WG_NOALLOC_SCRATCH_BYTES &&
      (rc = noalloc_scratch(p->device, &p->noalloc_ws)) != WG_OK)
    return fail(rc);
  *out = p.release();
  return WG_OK;
}

int wg_plan_destroy(wg_plan* plan) {
  if (plan == nullptr) return WG_OK;
  // calls on the plan may be in flight on any stream of its device: wait for all of them
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != plan->device) cudaSetDevice(plan->device);
  cudaDeviceSynchronize();
  free_plan_device(plan);
  if (cur >= 0 && cur != plan->device) cudaSetDevice(cur);
  delete plan;
  return WG_OK;
}

int wg_plan_get_info(const wg_plan* p, wg_plan_info* info) {
  if (p == nullptr || info == nullptr) return set_error(WG_ERR_ARG, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->alpha = p->pp.alpha; info->sigma = p->pp.sigma; info->beta = p->pp.beta;
  info->mu = p->pp.mu; info->eps_kernel = p->pp.eps_kernel;
  info->nu = p->pp.nu; info->nv = p->pp.nv; info->nw = p->pp.nw;
  info->dw = p->pp.dw; info->w0 = p->pp.w0; info->nshift = p->pp.nshift;
  info->tile = p->pp.tile; info->ntiles = p->pp.ntu * p->pp.ntv;
  info->nvis = p->nvis; info->batch = p->batch;
  info->index_bytes = p->index_bytes; info->workspace_bytes = p->ws_bytes;
  info->umax = p->umax; info->vmax = p->vmax; info->wmin = p->wmin; info->wmax = p->wmax;
  info->fft_impl = p->pp.fft_kind; info->rounding_gain = p->pp.gain;
  info->err_model = p->pp.err_model;
  return WG_OK;
}

// ---------------------------------------------------------------------------------------
// per-stage timing
// ---------------------------------------------------------------------------------------
struct StageTimer {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<std::pair<int, cudaEvent_t>> marks;  // (stage entered, event)
  cudaEvent_t t0 = nullptr;
  void start(bool enable, cudaStream_t st) {
    on = enable; s = st;
    if (!on) return;
    cudaEventCreate(&t0);
    cudaEventRecord(t0, s);
  }
  // record the end of a stage
  void mark(int stage) {
    if (!on) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    marks.emplace_back(stage, e);
  }
  void finish(wg_stats* st) {
    if (!on) return;
    cudaEventSynchronize(marks.empty() ? t0 : marks.back().second);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    cudaEvent_t prev = t0;
    for (auto& m : marks) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, prev, m.second);
      acc[m.first] += ms;
      prev = m.second;
    }
    float tot = 0.f;
    if (!marks.empty()) cudaEventElapsedTime(&tot, t0, marks.back().second);
    st->ms_total = tot;
    st->ms_prep = acc[0]; st->ms_screen = acc[1]; st->ms_fft = acc[2];
    st->ms_grid = acc[3]; st->ms_accum = acc[4];
    for (auto& m : marks) cudaEventDestroy(m.second);
    cudaEventDestroy(t0);
  }
};
enum { ST_PREP = 0, ST_SCREEN = 1, ST_FFT = 2, ST_GRID = 3, ST_ACCUM = 4, ST_OTHER = 5 };

static int run_fft(wg_plan* p, int64_t nb, void* data, void* work, int dir, cudaStream_t s) {
  if (p->ffft != nullptr) {
    // pruned to the image block like the double-float FFT: the screen writes only the image
    // cells and the accumulation reads only them
    cudaError_t e = f32_fft_exec(p->ffft, (float2*)data, nb, dir == CUFFT_FORWARD ? -1 : 1, s,
                                 p->g.nx, p->g.ny);
    if (e != cudaSuccess) return set_error(WG_ERR_CUDA, "FP32 FFT: %s", cudaGetErrorString(e));
    return WG_OK;
  }
  if (p->dfft != nullptr) {
    // the image occupies the first and last nx/2 rows and ny/2 columns of a plane: degrid's
    // input is zero elsewhere (and not written by the screen) and grid reads only that block
    cudaError_t e = df64_fft_exec(p->dfft, (double2*)data, nb, dir == CUFFT_FORWARD ? -1 : 1, s,
                                  p->g.nx, p->g.ny, p->g.df64_planes != 0, p->g.df64_planes != 0);
    if (e != cudaSuccess) return set_error(WG_ERR_CUDA, "double-float FFT: %s", cudaGetErrorString(e));
    return WG_OK;
  }
  std::lock_guard<std::mutex> lk(p->fft_mu);
  if (p->pruned) {
    const int64_t nu = p->pp.nu, nv = p->pp.nv, half = p->g.nx / 2;
    const int64_t plane = nu * nv;
    auto* base = (cufftDoubleComplex*)data;
    WG_CUFFT(cufftSetStream(p->fft_row, s));
    WG_CUFFT(cufftSetWorkArea(p->fft_row, work));
    WG_CUFFT(cufftSetStream(p->fft_col, s));
    WG_CUFFT(cufftSetWorkArea(p->fft_col, work));
    auto rows = [&](cufftDoubleComplex* pl) -> int {
      WG_CUFFT(cufftExecZ2Z(p->fft_row, pl, pl, dir));                              // rows [0, nx/2)
      WG_CUFFT(cufftExecZ2Z(p->fft_row, pl + (nu - half) * nv, pl + (nu - half) * nv, dir));  // last nx/2
      return WG_OK;
    };
    for (int64_t b = 0; b < nb; ++b) {
      cufftDoubleComplex* pl = base + b * plane;
      if (dir == CUFFT_FORWARD) {   // degrid: image rows hold the only nonzero data
        WG_TRY(rows(pl));
        WG_CUFFT(cufftExecZ2Z(p->fft_col, pl, pl, dir));
      } else {                      // grid: the image reads only its own rows
        WG_CUFFT(cufftExecZ2Z(p->fft_col, pl, pl, dir));
        WG_TRY(rows(pl));
      }
    }
    return WG_OK;
  }
  cufftHandle h = (nb == p->batch) ? p->fft_full : p->fft_rem;
  if (nb != p->batch && !p->has_rem) return set_error(WG_ERR_INTERNAL, "no FFT plan for %lld planes", (long long)nb);
  WG_CUFFT(cufftSetStream(h, s));
  WG_CUFFT(cufftSetWorkArea(h, work));
  if (p->prec)
    WG_CUFFT(cufftExecZ2Z(h, (cufftDoubleComplex*)data, (cufftDoubleComplex*)data, dir));
  else
    WG_CUFFT(cufftExecC2C(h, (cufftComplex*)data, (cufftComplex*)data, dir));
  return WG_OK;
}

template <typename R>
static int degrid_impl(wg_plan* p, const R* dirty, const R* wgt, typename C2<R>::T* vis,
                       cudaStream_t s, wg_stats* stats, unsigned char* external_ws = nullptr) {
  StageTimer tm;
  tm.start(stats != nullptr, s);
  const Geom& g = p->g;
  if (p->nvis_total > 0)
    WG_CUDA(cudaMemsetAsync(vis, 0, sizeof(typename C2<R>::T) * p->nvis_total, s));
  if (p->nvis == 0) {
    tm.mark(ST_OTHER);
    if (stats) { std::memset(stats, 0, sizeof(*stats)); tm.finish(stats); }
    return WG_OK;
  }
  Workspace w = workspace_layout(p, p->batch, p->fft_ws);
  unsigned char* ws = external_ws;
  if (ws == nullptr) WG_TRY(pool_alloc((void**)&ws, w.total, p->device, s));
  auto* planes = (typename C2<R>::T*)ws;
  void* fftw = ws + w.planes;
  auto* partial = (typename C2<R>::T*)(ws + w.planes + w.fft);
  R* wts_call = w.wts ? (R*)(ws + w.planes + w.fft + w.acc) : nullptr;   // filled per call
  R* wts = p->wts_plan ? (R*)p->wts_plan : wts_call;
  const auto* table = (const Z4<R>*)p->table;
  int rc = WG_OK;
  IndexView<R> ix{p->off, p->idx, p->meta, (const Z4<R>*)p->z, (const typename C2<R>::T*)p->ph, wts};
  const Coef<R>& coef = *reinterpret_cast<const Coef<R>*>(sizeof(R) == 4 ? (const void*)&p->coef_f
                                                                         : (const void*)&p->coef_d);
  int64_t nbatches = 0;
  do {
    cudaError_t e = cudaSuccess;
    if (p->compact) {   // the records of the compact index, recomputed into the workspace
      unsigned char* rb = ws + (w.total - w.rec);
      ix.meta = (const uint32_t*)rb;
      ix.z = (const Z4<R>*)(rb + w.rec_meta);
      ix.ph = p->use_ph ? (const typename C2<R>::T*)(rb + w.rec_meta + w.rec_z) : nullptr;
      e = launch_expand<R>(g, p->uvw_dev, p->chan4, p->idx, p->nvis, (uint32_t*)ix.meta,
                           (Z4<R>*)ix.z, (typename C2<R>::T*)ix.ph, s);
      if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "expand: %s", cudaGetErrorString(e)); break; }
    }
    if (wts_call != nullptr) {
      e = launch_weights<R>(g, coef, ix, p->nvis, wts_call, s);
      if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "weights: %s", cudaGetErrorString(e)); break; }
    }
    if (p->compact || wts_call != nullptr) tm.mark(ST_PREP);
    for (int64_t b0 = 0; b0 < g.nw; b0 += p->batch) {
      int nb = (int)std::min<int64_t>(p->batch, g.nw - b0);
      // with the double-float FFT the screen writes only the image cells (see df64_fft_exec);
      // with double-float planes it writes them as pairs, in pair arithmetic
      if constexpr (sizeof(R) == 8) {
        if (g.df64_planes)
          e = launch_screen_dd(g, (const double*)dirty, (const Z4<double>*)table, (float4*)planes,
                               (int)b0, nb, s);
        else
          e = launch_screen<R>(g, dirty, table, planes, (int)b0, nb, p->dfft != nullptr, s);
      } else {
        e = launch_screen<R>(g, dirty, table, planes, (int)b0, nb, p->ffft != nullptr, s);
      }
      if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "screen: %s", cudaGetErrorString(e)); break; }
      tm.mark(ST_SCREEN);
      if ((rc = run_fft(p, nb, planes, fftw, CUFFT_FORWARD, s)) != WG_OK) break;
      tm.mark(ST_FFT);
      e = launch_degrid<R>(g, coef, ix, planes, (int)b0, nb, p->degrid_bs, partial, p->nvis, s);
      if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "degrid: %s", cudaGetErrorString(e)); break; }
      tm.mark(ST_GRID);
      ++nbatches;
    }
    if (rc != WG_OK) break;
    e = launch_degrid_finalize<R>(g, ix, partial, p->nvis, p->degrid_bs, wgt, vis, s);
    if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "degrid finalize: %s", cudaGetErrorString(e)); break; }
    tm.mark(ST_GRID);
  } while (0);
  if (external_ws == nullptr) pool_free(ws, s);
  if (rc != WG_OK) return rc;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    tm.finish(stats);
    stats->n_batches = nbatches; stats->n_planes = g.nw; stats->workspace_bytes = w.total;
    // screen + degrid per batch, finalize, weights; the double-float FFT's two passes per batch
    stats->n_kernels = 2 * nbatches + 1 + (wts_call != nullptr) +
                       (p->dfft != nullptr || p->ffft != nullptr ? 2 * nbatches : 0) + (p->compact ? 1 : 0);
    stats->n_fft_calls = nbatches;
  }
  return WG_OK;
}

template <typename R>
static int grid_impl(wg_plan* p, const typename C2<R>::T* vis, const R* wgt, R* dirty,
                     cudaStream_t s, wg_stats* stats) {
  StageTimer tm;
  tm.start(stats != nullptr, s);
  const Geom& g = p->g;
  if (p->nvis == 0) {
    WG_CUDA(cudaMemsetAsync(dirty, 0, sizeof(R) * g.nx * g.ny, s));
    tm.mark(ST_OTHER);
    if (stats) { std::memset(stats, 0, sizeof(*stats)); tm.finish(stats); }
    return WG_OK;
  }
  Workspace w = workspace_layout(p, p->batch, p->fft_ws);
  unsigned char* ws = nullptr;
  WG_TRY(pool_alloc((void**)&ws, w.total, p->device, s));
  auto* planes = (typename C2<R>::T*)ws;
  void* fftw = ws + w.planes;
  const auto* table = (const Z4<R>*)p->table;
  auto* acc = (double*)(ws + w.planes + w.fft);
  R* wts_call = w.wts ? (R*)(ws + w.planes + w.fft + w.acc) : nullptr;   // filled per call
  R* wts = p->wts_plan ? (R*)p->wts_plan : wts_call;
  int rc = WG_OK;
  IndexView<R> ix{p->off, p->idx, p->meta, (const Z4<R>*)p->z, (const typename C2<R>::T*)p->ph, wts};
  const Coef<R>& coef = *reinterpret_cast<const Coef<R>*>(sizeof(R) == 4 ? (const void*)&p->coef_f
                                                                         : (const void*)&p->coef_d);
  int64_t nbatches = 0;
  do {
    cudaError_t e = cudaSuccess;
    if (p->compact) {   // the records of the compact index, recomputed into the workspace
      unsigned char* rb = ws + (w.total - w.rec);
      ix.meta = (const uint32_t*)rb;
      ix.z = (const Z4<R>*)(rb + w.rec_meta);
      ix.ph = p->use_ph ? (const typename C2<R>::T*)(rb + w.rec_meta + w.rec_z) : nullptr;
      e = launch_expand<R>(g, p->uvw_dev, p->chan4, p->idx, p->nvis, (uint32_t*)ix.meta,
                           (Z4<R>*)ix.z, (typename C2<R>::T*)ix.ph, s);
      if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "expand: %s", cudaGetErrorString(e)); break; }
    }
    if (wts_call != nullptr) {
      e = launch_weights<R>(g, coef, ix, p->nvis, wts_call, s);
      if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "weights: %s", cudaGetErrorString(e)); break; }
    }
    if (p->compact || wts_call != nullptr) tm.mark(ST_PREP);
    // double-float planes: weights, fold and w-reference phase applied once, as pairs, and the
    // gridding kernel reads those instead of vis / wgt
    const typename C2<R>::T* vgrid = vis;
    if constexpr (sizeof(R) == 8) {
      if (g.df64_planes) {
        auto* visd = (float4*)(ws + w.planes + w.fft + w.acc + w.wts);
        e = launch_grid_vis_dd(ix, vis, wgt, p->nvis, visd, s);
        if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "grid data: %s", cudaGetErrorString(e)); break; }
        vgrid = (const typename C2<R>::T*)visd;
      }
    }
    for (int64_t b0 = 0; b0 < g.nw; b0 += p->batch) {
      int nb = (int)std::min<int64_t>(p->batch, g.nw - b0);
      e = launch_grid<R>(g, coef, ix, vgrid, wgt, planes, (int)b0, nb, s);
      if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "grid: %s", cudaGetErrorString(e)); break; }
      tm.mark(ST_GRID);
      if ((rc = run_fft(p, nb, planes, fftw, CUFFT_INVERSE, s)) != WG_OK) break;
      tm.mark(ST_FFT);
      if constexpr (sizeof(R) == 8) {
        if (g.df64_planes)
          e = launch_accumulate_dd(g, (const Z4<double>*)table, (const float4*)planes, (int)b0, nb,
                                   acc, b0 == 0, b0 + nb >= g.nw, (double*)dirty, s);
        else
          e = launch_accumulate<R>(g, table, planes, (int)b0, nb, acc, b0 == 0, b0 + nb >= g.nw,
                                   dirty, s);
      } else {
        e = launch_accumulate<R>(g, table, planes, (int)b0, nb, acc, b0 == 0, b0 + nb >= g.nw,
                                 dirty, s);
      }
      if (e != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "accumulate: %s", cudaGetErrorString(e)); break; }
      tm.mark(ST_ACCUM);
      ++nbatches;
    }
  } while (0);
  pool_free(ws, s);
  if (rc != WG_OK) return rc;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    tm.finish(stats);
    stats->n_batches = nbatches; stats->n_planes = g.nw; stats->workspace_bytes = w.total;
    // grid + accumulate per batch, weights; the double-float FFT's two passes per batch
    stats->n_kernels = 2 * nbatches + (wts_call != nullptr) +
                       (p->dfft != nullptr || p->ffft != nullptr ? 2 * nbatches : 0) +
                       (g.df64_planes ? 1 : 0) + (p->compact ? 1 : 0);
    stats->n_fft_calls = nbatches;
  }
  return WG_OK;
}

int wg_degrid(wg_plan* plan, const void* dirty, const void* wgt, void* vis, void* stream,
              wg_stats* stats) {
  if (plan == nullptr || dirty == nullptr || (vis == nullptr && plan->nvis_total > 0))
    return set_error(WG_ERR_ARG, "NULL plan / dirty / vis");
  cudaStream_t s = (cudaStream_t)stream;
  if (plan->prec)
    return degrid_impl<double>(plan, (const double*)dirty, (const double*)wgt, (double2*)vis, s, stats);
  return degrid_impl<float>(plan, (const float*)dirty, (const float*)wgt, (float2*)vis, s, stats);
}

int wg_degrid_noalloc(wg_plan* plan, const void* dirty, const void* wgt, void* vis,
                      void* stream) {
  if (plan == nullptr || dirty == nullptr || (vis == nullptr && plan->nvis_total > 0))
    return set_error(WG_ERR_ARG, "NULL plan / dirty / vis");
  if (plan->ws_bytes > (size_t)WG_NOALLOC_SCRATCH_BYTES)
    return set_error(WG_ERR_ARG,
                     "plan needs %zu bytes of per-call workspace, more than the %llu-byte static "
                     "scratch; create it with max_workspace <= WG_NOALLOC_SCRATCH_BYTES",
                     plan->ws_bytes, (unsigned long long)WG_NOALLOC_SCRATCH_BYTES);
  int dev = -1;
  WG_CUDA(cudaGetDevice(&dev));
  if (dev != plan->device)
    return set_error(WG_ERR_ARG, "current device %d is not the plan's device %d", dev, plan->device);
  unsigned char* ws = plan->noalloc_ws;   // looked up by wg_plan_create
  if (ws == nullptr) return set_error(WG_ERR_INTERNAL, "static scratch address missing");
  cudaStream_t s = (cudaStream_t)stream;
  if (plan->prec)
    return degrid_impl<double>(plan, (const double*)dirty, (const double*)wgt, (double2*)vis, s,
                               nullptr, ws);
  return degrid_impl<float>(plan, (const float*)dirty, (const float*)wgt, (float2*)vis, s,
                            nullptr, ws);
}

int wg_grid(wg_plan* plan, const void* vis, const void* wgt, void* dirty, void* stream,
            wg_stats* stats) {
  if (plan == nullptr || dirty == nullptr || (vis == nullptr && plan->nvis_total > 0))
    return set_error(WG_ERR_ARG, "NULL plan / vis / dirty");
  cudaStream_t s = (cudaStream_t)stream;
  if (plan->prec)
    return grid_impl<double>(plan, (const double2*)vis, (const double*)wgt, (double*)dirty, s, stats);
  return grid_impl<float>(plan, (const float2*)vis, (const float*)wgt, (float*)dirty, s, stats);
}

int wg_dirty2ms(const double* uvw, const double* freq, int64_t nrows, int64_t nchan,
                const void* dirty, const void* wgt, int64_t npix_x, int64_t npix_y,
                double pixsize_x, double pixsize_y, double epsilon, int precision,
                int do_wstacking, const uint8_t* mask, void* vis, void* stream) {
  wg_options o;
  wg_default_options(&o);
  o.do_wstacking = do_wstacking;
  wg_plan* p = nullptr;
  WG_TRY(wg_plan_create(uvw, freq, nrows, nchan, npix_x, npix_y, pixsize_x, pixsize_y, epsilon,
                        precision, mask, &o, stream, &p));
  int rc = wg_degrid(p, dirty, wgt, vis, stream, nullptr);
  std::string keep = g_last_error;
  wg_plan_destroy(p);
  g_last_error = keep;
  return rc;
}

int wg_ms2dirty(const double* uvw, const double* freq, int64_t nrows, int64_t nchan,
                const void* vis, const void* wgt, int64_t npix_x, int64_t npix_y,
                double pixsize_x, double pixsize_y, double epsilon, int precision,
                int do_wstacking, const uint8_t* mask, void* dirty, void* stream) {
  wg_options o;
  wg_default_options(&o);
  o.do_wstacking = do_wstacking;
  wg_plan* p = nullptr;
  WG_TRY(wg_plan_create(uvw, freq, nrows, nchan, npix_x, npix_y, pixsize_x, pixsize_y, epsilon,
                        precision, mask, &o, stream, &p));
  int rc = wg_grid(p, vis, wgt, dirty, stream, nullptr);
  std::string keep = g_last_error;
  wg_plan_destroy(p);
  g_last_error = keep;
  return rc;
}

const char* wg_last_error(void) { return g_last_error.c_str(); }

int wg_pool_trim(size_t keep_bytes) {
  int dev = 0;
  WG_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool = device_pool(dev);
  if (pool == nullptr) return set_error(WG_ERR_CUDA, "cudaMemPoolCreate failed");
  WG_CUDA(cudaMemPoolTrimTo(pool, keep_bytes));
  return WG_OK;
}

int wg_wait(void* stream, double timeout_ms) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!(timeout_ms >= 0.0)) {   // negative (or NaN): unbounded
    WG_CUDA(cudaStreamSynchronize(s));
    return WG_OK;
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) return WG_OK;
    if (e != cudaErrorNotReady)
      return set_error(WG_ERR_CUDA, "cudaStreamQuery: %s", cudaGetErrorString(e));
    const double ms = std::chrono::duration<double, std::milli>(
                          std::chrono::steady_clock::now() - t0).count();
    if (ms >= timeout_ms)
      return set_error(WG_ERR_TIMEOUT, "stream work not finished after %.1f ms", ms);
    std::this_thread::sleep_for(std::chrono::microseconds(ms < 1.0 ? 20 : 200));
  }
}

// ---------------------------------------------------------------------------------------
// host-only helpers
// ---------------------------------------------------------------------------------------
int wg_kernel_table_size(void) { return (int)kernel_table().size(); }

int wg_kernel_table_row(int i, int* alpha, double* sigma, double* eps, double* beta, double* mu) {
  const auto& T = kernel_table();
  if (i < 0 || i >= (int)T.size()) return set_error(WG_ERR_ARG, "row %d out of range", i);
  if (alpha) *alpha = T[i].alpha;
  if (sigma) *sigma = T[i].sigma;
  if (eps) *eps = T[i].eps;
  if (beta) *beta = T[i].beta;
  if (mu) *mu = T[i].mu;
  return WG_OK;
}

int wg_kernel_phi(int alpha, double beta, double mu, const double* x, double* out, int64_t n) {
  if (alpha < 1 || alpha > kMaxAlpha || !x || !out) return set_error(WG_ERR_ARG, "bad arguments");
  for (int64_t i = 0; i < n; ++i) out[i] = es_phi(alpha, beta, mu, x[i]);
  return WG_OK;
}

int wg_kernel_poly(int alpha, double beta, double mu, const double* x, double* out, int64_t n) {
  if (alpha < 1 || alpha > kMaxAlpha || !x || !out) return set_error(WG_ERR_ARG, "bad arguments");
  PolyKernel K = make_poly_kernel(alpha, beta, mu, alpha + 3);
  for (int64_t i = 0; i < n; ++i) out[i] = K.eval(x[i]);
  return WG_OK;
}

int wg_kernel_psi(int alpha, double beta, double mu, const double* k, double* out, int64_t n) {
  if (alpha < 1 || alpha > kMaxAlpha || !k || !out) return set_error(WG_ERR_ARG, "bad arguments");
  PolyKernel K = make_poly_kernel(alpha, beta, mu, alpha + 3);
  for (int64_t i = 0; i < n; ++i) out[i] = psi_poly(K, k[i]);
  return WG_OK;
}

int wg_kernel_design_size(void) { return (int)kernel_table_design().size(); }

int wg_kernel_design_row(int i, int* alpha, double* sigma, double* eps, double* beta, double* mu) {
  const auto& T = kernel_table_design();
  if (i < 0 || i >= (int)T.size()) return set_error(WG_ERR_ARG, "row out of range");
  if (alpha) *alpha = T[i].alpha;
  if (sigma) *sigma = T[i].sigma;
  if (eps) *eps = T[i].eps;
  if (beta) *beta = T[i].beta;
  if (mu) *mu = T[i].mu;
  return WG_OK;
}

int wg_kernel_eps(int alpha, double beta, double mu, double sigma, double* eps) {
  if (alpha < 2 || alpha > kMaxAlpha || !(beta > 0) || !(mu > 0) || !(sigma > 1.0) || !eps)
    return set_error(WG_ERR_ARG, "bad arguments");
  *eps = es_kernel_eps(alpha, beta, mu, sigma);
  return WG_OK;
}

int wg_kernel_search(int alpha, double sigma, double beta0, double mu0, double* beta, double* mu,
                     double* eps) {
  if (alpha < 2 || alpha > kMaxAlpha || !(sigma >= 1.05 && sigma <= 2.5) || !(beta0 > 0) ||
      !(mu0 > 0.2 && mu0 < 1.5) || !beta || !mu || !eps)
    return set_error(WG_ERR_ARG, "bad arguments");
  KernelRow r = kernel_search(alpha, sigma, beta0, mu0);
  *beta = r.beta; *mu = r.mu; *eps = r.eps;
  return WG_OK;
}

int wg_plan_params(int64_t npix_x, int64_t npix_y, double pixsize_x, double pixsize_y,
                   double epsilon, int precision, const wg_options* opt, double umax,
                   double vmax, double wmin, double wmax, int64_t nvis, wg_plan_info* info) {
  if (info == nullptr) return set_error(WG_ERR_ARG, "info is NULL");
  wg_options o;
  if (opt) o = *opt; else wg_default_options(&o);
  if (o.eps_safety <= 0) o.eps_safety = kDefaultEpsSafety;
  PlanInput in = plan_input(npix_x, npix_y, pixsize_x, pixsize_y, epsilon, precision, o, umax,
                            vmax, wmin, wmax, nvis);
  PlanParams pp;
  char err[256];
  if (choose_plan(in, pp, err, sizeof(err)) != 0) return set_error(WG_ERR_ARG, "%s", err);
  std::memset(info, 0, sizeof(*info));
  info->alpha = pp.alpha; info->sigma = pp.sigma; info->beta = pp.beta; info->mu = pp.mu;
  info->eps_kernel = pp.eps_kernel; info->nu = pp.nu; info->nv = pp.nv; info->nw = pp.nw;
  info->dw = pp.dw; info->w0 = pp.w0; info->nshift = pp.nshift; info->tile = pp.tile;
  info->ntiles = pp.ntu * pp.ntv; info->nvis = nvis;
  info->umax = umax; info->vmax = vmax; info->wmin = wmin; info->wmax = wmax;
  info->fft_impl = pp.fft_kind; info->rounding_gain = pp.gain; info->err_model = pp.err_model;
  return WG_OK;
}

// One in-place batched 2-D transform object for the utilities below.
struct FftUtil {
  cufftHandle h = 0;
  bool has_h = false;
  Df64Fft* d = nullptr;
  F32Fft* f = nullptr;
  void* work = nullptr;
  ~FftUtil() {
    if (has_h) cufftDestroy(h);
    df64_fft_destroy(d);
    f32_fft_destroy(f);
    if (work) cudaFree(work);
  }
};

static int fft_util_make(FftUtil& u, int64_t nu, int64_t nv, int64_t batch, int precision, int impl) {
  if (impl == 2) {
    if (precision != WG_F64 || !df64_fft_supported(nu, nv))
      return set_error(WG_ERR_ARG, "double-float FFT needs WG_F64 and sides with factors 2, 3, 5, 7, 11 "
                                   "up to 6400, or 2 or 4 times such a side up to 25600");
    cudaError_t e = df64_fft_create(nu, nv, &u.d);
    if (e != cudaSuccess) return set_error(WG_ERR_CUDA, "double-float FFT setup: %s", cudaGetErrorString(e));
    return WG_OK;
  }
  if (impl == 4) {
    if (precision != WG_F32 || !f32_fft_supported(nu, nv))
      return set_error(WG_ERR_ARG, "the FP32 plane FFT needs WG_F32 and sides that are 1, 2, 4 or 8 "
                                   "times a part of at most 12800 points with factors 2, 3, 5, 7, 11");
    cudaError_t e = f32_fft_create(nu, nv, &u.f);
    if (e != cudaSuccess) return set_error(WG_ERR_CUDA, "FP32 FFT setup: %s", cudaGetErrorString(e));
    return WG_OK;
  }
  if (impl != 1) return set_error(WG_ERR_ARG, "impl must be 1 (cuFFT), 2 (double-float) or 4 (FP32)");
  size_t ws = 0;
  WG_TRY(make_fft(&u.h, precision, nu, nv, batch, &ws));
  u.has_h = true;
  if (ws > 0) WG_TRY(dev_alloc((unsigned char**)&u.work, ws));
  WG_CUFFT(cufftSetWorkArea(u.h, u.work));
  return WG_OK;
}

static int fft_util_exec(FftUtil& u, void* data, int64_t batch, int precision, int sign, cudaStream_t s) {
  if (u.f != nullptr) {
    cudaError_t e = f32_fft_exec(u.f, (float2*)data, batch, sign, s);
    if (e != cudaSuccess) return set_error(WG_ERR_CUDA, "FP32 FFT: %s", cudaGetErrorString(e));
    return WG_OK;
  }
  if (u.d != nullptr) {
    cudaError_t e = df64_fft_exec(u.d, (double2*)data, batch, sign, s);
    if (e != cudaSuccess) return set_error(WG_ERR_CUDA, "double-float FFT: %s", cudaGetErrorString(e));
    return WG_OK;
  }
  WG_CUFFT(cufftSetStream(u.h, s));
  int dir = sign < 0 ? CUFFT_FORWARD : CUFFT_INVERSE;
  if (precision)
    WG_CUFFT(cufftExecZ2Z(u.h, (cufftDoubleComplex*)data, (cufftDoubleComplex*)data, dir));
  else
    WG_CUFFT(cufftExecC2C(u.h, (cufftComplex*)data, (cufftComplex*)data, dir));
  return WG_OK;
}

int wg_fft2d(void* data, int64_t nu, int64_t nv, int64_t batch, int precision, int impl, int sign,
             void* stream) {
  if (data == nullptr || nu < 2 || nv < 2 || batch < 1 || (precision != WG_F32 && precision != WG_F64))
    return set_error(WG_ERR_ARG, "bad arguments");
  FftUtil u;
  WG_TRY(fft_util_make(u, nu, nv, batch, precision, impl));
  cudaStream_t s = (cudaStream_t)stream;
  WG_TRY(fft_util_exec(u, data, batch, precision, sign, s));
  WG_CUDA(cudaStreamSynchronize(s));
  return WG_OK;
}

int wg_fft_f32_tune(int cols, int max_points, int per_thread) {
  if (f32_fft_tune(cols, max_points, per_thread) != 0)
    return set_error(WG_ERR_ARG, "wg_fft_f32_tune: cols 1, 2, 4 or 8; max_points 64 .. 12800; "
                                 "per_thread 2 .. 64 (0 keeps a default)");
  return WG_OK;
}

int wg_fft_time(int64_t n, int precision, int64_t batch, int reps, int impl, double* ms_per_plane) {
  if (n < 2 || batch < 1 || reps < 1 || ms_per_plane == nullptr ||
      (precision != WG_F32 && precision != WG_F64))
    return set_error(WG_ERR_ARG, "bad arguments");
  size_t bytes = (size_t)n * n * batch * cplx_bytes(precision);
  FftUtil u;
  WG_TRY(fft_util_make(u, n, n, batch, precision, impl));
  void* data = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = WG_OK;
  do {
    if ((rc = dev_alloc((unsigned char**)&data, bytes)) != WG_OK) break;
    if (cudaMemset(data, 0, bytes) != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "memset"); break; }
    cudaEventCreate(&e0); cudaEventCreate(&e1);
    float ms = 0.f;
    for (int r = 0; r <= reps && rc == WG_OK; ++r) {
      if (r == 1) cudaEventRecord(e0, 0);
      rc = fft_util_exec(u, data, batch, precision, -1, 0);
    }
    if (rc != WG_OK) break;
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = set_error(WG_ERR_CUDA, "sync"); break; }
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_per_plane = ms / (double)(reps * batch);
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (data) cudaFree(data);
  return rc;
}

const char* wg_version(void) { return "wgrid-gb300 0.1 (sm_103a)"; }
