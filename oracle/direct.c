/*
 * Direct-sum oracle for the wide-field interferometric response (test
 * infrastructure only: the product path never links, loads or calls this file).
 *
 * What it computes, in plain FP64 with no approximation of the operator:
 *
 *   degrid  (R0 I)_k  = sum_{l in L} sum_{m in M}
 *                         exp(-2 pi i [u_k l + v_k m - w_k (n_lm - 1)]) I_lm / n_lm
 *           the discretised measurement equation, Sec. 2, Eq. (rime) (Eq. 2 of the
 *           paper), with the pixel sets L = {(-n_l/2 + j) dl}, M = {(-n_m/2 + j) dm}
 *           and n = sqrt(1 - l^2 - m^2) (Sec. 2, below Eq. 1);
 *
 *   grid    (R0^dagger d)_lm = Re sum_k exp(+2 pi i [u_k l + v_k m - w_k (n_lm - 1)]) d_k / n_lm
 *           the direct adjoint used as the accuracy reference in Sec. 5.2; the real
 *           part is taken because R maps a real image to complex data (Sec. 5.1,
 *           Eq. adjointness).
 *
 * Effective coordinates: u = u~ * f / c (and likewise v, w), Sec. 2 (u := u~ (x) 1/lambda).
 * Visibility k is (row, chan) with k = row * nchan + chan (C order of the (nrows, nchan)
 * data array of the paper's interface, App. B).
 *
 * Interface options of App. B that change the operator:
 *   wgt   (optional, real) multiplies the degridded output, and the grid input;
 *   mask  (optional, uint8) visibilities with mask == 0 are not processed: their degrid
 *         output is 0 and they contribute nothing to the grid output;
 *   do_wstacking == 0: "the w values are assumed to be zero" (w := 0; the 1/n factor of
 *         Eq. rime stays).
 *
 * Numerics: the phase u l + v m - w (n - 1) is formed in double-double (each product
 * split exactly with fma), reduced modulo one cycle, and only then turned into an angle;
 * sums over terms are Neumaier-compensated.  n - 1 is computed as
 * -(l^2 + m^2) / (1 + sqrt(1 - l^2 - m^2)) so that it carries full relative precision.
 *
 * Threads: POSIX threads over output elements; each output element is one plain sum.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define SPEED_OF_LIGHT 299792458.0

typedef struct { double hi, lo; } dd_t;

/* exact product a*b = p + e (fma-based TwoProduct) */
static inline dd_t two_prod(double a, double b) {
  dd_t r;
  r.hi = a * b;
  r.lo = fma(a, b, -r.hi);
  return r;
}

/* exact sum a+b = s + e (Knuth TwoSum) */
static inline dd_t two_sum(double a, double b) {
  dd_t r;
  r.hi = a + b;
  double bb = r.hi - a;
  r.lo = (a - (r.hi - bb)) + (b - bb);
  return r;
}

static inline dd_t dd_add(dd_t x, dd_t y) {
  dd_t s = two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return two_sum(s.hi, s.lo);
}

/* fractional part of a double-double number of cycles, in [-0.5, 0.5] */
static inline double dd_frac(dd_t x) {
  double r = nearbyint(x.hi);
  return (x.hi - r) + x.lo;
}

/* Neumaier compensated accumulator */
typedef struct { double s, c; } acc_t;
static inline void acc_add(acc_t* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

typedef struct {
  /* geometry */
  const double* uvw; const double* freq; int64_t nrows, nchan;
  int64_t nx, ny; double psx, psy; int do_w;
  const double* wgt; const uint8_t* mask;
  /* per-pixel precomputation */
  double* l; double* m; double* nm1; double* ninv;
  /* degrid */
  const double* dirty; double* vis_out; const int64_t* vsel; int64_t nvsel;
  /* grid */
  const double* vis_in; double* dirty_out; const int64_t* psel; int64_t npsel;
  /* work split */
  int64_t begin, end;
} job_t;

static void vis_coords(const job_t* J, int64_t k, double* u, double* v, double* w) {
  int64_t row = k / J->nchan, ch = k % J->nchan;
  double s = J->freq[ch] / SPEED_OF_LIGHT;
  *u = J->uvw[3 * row + 0] * s;
  *v = J->uvw[3 * row + 1] * s;
  *w = J->do_w ? J->uvw[3 * row + 2] * s : 0.0;
}

/* phase in cycles: u l + v m - w (n - 1), reduced to [-0.5, 0.5] */
static inline double phase_cycles(double u, double v, double w, double l, double m, double nm1) {
  dd_t a = two_prod(u, l);
  dd_t b = two_prod(v, m);
  dd_t c = two_prod(-w, nm1);
  return dd_frac(dd_add(dd_add(a, b), c));
}

static void* degrid_worker(void* arg) {
  job_t* J = (job_t*)arg;
  int64_t npix = J->nx * J->ny;
  for (int64_t t = J->begin; t < J->end; ++t) {
    int64_t k = J->vsel ? J->vsel[t] : t;
    double* out = J->vis_out + 2 * t;
    if (J->mask && J->mask[k] == 0) { out[0] = 0.0; out[1] = 0.0; continue; }
    double u, v, w;
    vis_coords(J, k, &u, &v, &w);
    acc_t re = {0, 0}, im = {0, 0};
    for (int64_t p = 0; p < npix; ++p) {
      double val = J->dirty[p];
      if (val == 0.0) continue;
      int64_t jx = p / J->ny, jy = p % J->ny;
      double f = phase_cycles(u, v, w, J->l[jx], J->m[jy], J->nm1[p]);
      double s, c;
      sincos(2.0 * M_PI * f, &s, &c);
      double a = val * J->ninv[p];
      /* exp(-2 pi i f) = cos - i sin */
      acc_add(&re, a * c);
      acc_add(&im, -a * s);
    }
    double g = J->wgt ? J->wgt[k] : 1.0;
    out[0] = g * (re.s + re.c);
    out[1] = g * (im.s + im.c);
  }
  return NULL;
}

static void* grid_worker(void* arg) {
  job_t* J = (job_t*)arg;
  int64_t nvis = J->nrows * J->nchan;
  for (int64_t t = J->begin; t < J->end; ++t) {
    int64_t p = J->psel ? J->psel[t] : t;
    int64_t jx = p / J->ny, jy = p % J->ny;
    double l = J->l[jx], m = J->m[jy], nm1 = J->nm1[p];
    acc_t re = {0, 0};
    for (int64_t k = 0; k < nvis; ++k) {
      if (J->mask && J->mask[k] == 0) continue;
      double g = J->wgt ? J->wgt[k] : 1.0;
      double dr = g * J->vis_in[2 * k], di = g * J->vis_in[2 * k + 1];
      if (dr == 0.0 && di == 0.0) continue;
      double u, v, w;
      vis_coords(J, k, &u, &v, &w);
      double f = phase_cycles(u, v, w, l, m, nm1);
      double s, c;
      sincos(2.0 * M_PI * f, &s, &c);
      /* Re(exp(+2 pi i f) d) = c dr - s di */
      acc_add(&re, c * dr - s * di);
    }
    J->dirty_out[t] = (re.s + re.c) * J->ninv[p];
  }
  return NULL;
}

/* returns 0 on success, -1 if a pixel lies outside the unit disc (l^2 + m^2 > 1) */
static int pixel_setup(job_t* J) {
  J->l = (double*)malloc(sizeof(double) * J->nx);
  J->m = (double*)malloc(sizeof(double) * J->ny);
  J->nm1 = (double*)malloc(sizeof(double) * J->nx * J->ny);
  J->ninv = (double*)malloc(sizeof(double) * J->nx * J->ny);
  for (int64_t j = 0; j < J->nx; ++j) J->l[j] = (double)(j - J->nx / 2) * J->psx;
  for (int64_t j = 0; j < J->ny; ++j) J->m[j] = (double)(j - J->ny / 2) * J->psy;
  for (int64_t jx = 0; jx < J->nx; ++jx)
    for (int64_t jy = 0; jy < J->ny; ++jy) {
      double r2 = J->l[jx] * J->l[jx] + J->m[jy] * J->m[jy];
      if (r2 > 1.0) return -1;
      double n = sqrt(1.0 - r2);
      J->nm1[jx * J->ny + jy] = -r2 / (1.0 + n);
      J->ninv[jx * J->ny + jy] = 1.0 / n;
    }
  return 0;
}

static void pixel_free(job_t* J) {
  free(J->l); free(J->m); free(J->nm1); free(J->ninv);
}

static int run_threads(job_t* base, int64_t total, int nthreads, void* (*fn)(void*)) {
  if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
  if (nthreads < 1) nthreads = 1;
  if (total < nthreads) nthreads = total > 0 ? (int)total : 1;
  job_t* jobs = (job_t*)malloc(sizeof(job_t) * nthreads);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  /* interleaved chunks for balance: thread i gets elements i, i+T, ... via small blocks */
  int64_t chunk = (total + nthreads - 1) / nthreads;
  for (int i = 0; i < nthreads; ++i) {
    jobs[i] = *base;
    jobs[i].begin = (int64_t)i * chunk;
    jobs[i].end = jobs[i].begin + chunk < total ? jobs[i].begin + chunk : total;
    if (jobs[i].begin > total) jobs[i].begin = total;
    pthread_create(&th[i], NULL, fn, &jobs[i]);
  }
  for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
  free(jobs); free(th);
  return nthreads;
}

/*
 * oracle_degrid: vis_out[2t], vis_out[2t+1] = (R0 I)_k for k = vsel[t] (t < nvsel), or for
 * every k when vsel is NULL (then nvsel must equal nrows*nchan).  dirty is (nx, ny) C order.
 * Returns the number of threads used, or -1 for a pixel outside the unit disc.
 */
int oracle_degrid(const double* uvw, const double* freq, int64_t nrows, int64_t nchan,
                  const double* dirty, int64_t nx, int64_t ny, double psx, double psy,
                  const double* wgt, const uint8_t* mask, int do_wstacking,
                  const int64_t* vsel, int64_t nvsel, double* vis_out, int nthreads) {
  job_t J;
  memset(&J, 0, sizeof(J));
  J.uvw = uvw; J.freq = freq; J.nrows = nrows; J.nchan = nchan;
  J.nx = nx; J.ny = ny; J.psx = psx; J.psy = psy; J.do_w = do_wstacking;
  J.wgt = wgt; J.mask = mask; J.dirty = dirty; J.vis_out = vis_out;
  J.vsel = vsel; J.nvsel = nvsel;
  if (pixel_setup(&J) != 0) { pixel_free(&J); return -1; }
  int used = run_threads(&J, nvsel, nthreads, degrid_worker);
  pixel_free(&J);
  return used;
}

/*
 * oracle_grid: dirty_out[t] = (R0^dagger d)_p for flat pixel p = psel[t] (t < npsel), or
 * for every pixel when psel is NULL (then npsel must equal nx*ny).  vis is complex
 * interleaved (re, im), (nrows, nchan) C order.  Returns threads used, or -1 as above.
 */
int oracle_grid(const double* uvw, const double* freq, int64_t nrows, int64_t nchan,
                const double* vis, int64_t nx, int64_t ny, double psx, double psy,
                const double* wgt, const uint8_t* mask, int do_wstacking,
                const int64_t* psel, int64_t npsel, double* dirty_out, int nthreads) {
  job_t J;
  memset(&J, 0, sizeof(J));
  J.uvw = uvw; J.freq = freq; J.nrows = nrows; J.nchan = nchan;
  J.nx = nx; J.ny = ny; J.psx = psx; J.psy = psy; J.do_w = do_wstacking;
  J.wgt = wgt; J.mask = mask; J.vis_in = vis; J.dirty_out = dirty_out;
  J.psel = psel; J.npsel = npsel;
  if (pixel_setup(&J) != 0) { pixel_free(&J); return -1; }
  int used = run_threads(&J, npsel, nthreads, grid_worker);
  pixel_free(&J);
  return used;
}
