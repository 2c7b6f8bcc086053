// Visibility index on the device: uvw extent, bin-sort of visibilities into
// (uv tile, first w-plane) buckets, and the tile-sorted per-visibility records.
//
// This is the GPU counterpart of the paper's processing-order index (Sec. 4.3: 16x16 uv
// patches, first plane t_w, lexicographic order) built with a counting sort instead of the
// paper's mutex-guarded sorted structure (Sec. 4.4).
#include <cfloat>

#include "wgrid_internal.h"

namespace wg {

// ---------------------------------------------------------------------------------------
// uvw extent: max |u~|, max |v~|, min |w~|, max |w~| over rows.  Non-negative doubles order
// like their IEEE bit patterns, so 64-bit integer atomics give exact max / min.
// ---------------------------------------------------------------------------------------
__global__ void k_extent(const double* __restrict__ uvw, int64_t nrows,
                         unsigned long long* __restrict__ ext) {
  double mu = 0.0, mv = 0.0, wmn = DBL_MAX, wmx = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows;
       r += (int64_t)gridDim.x * blockDim.x) {
    double u = fabs(uvw[3 * r]), v = fabs(uvw[3 * r + 1]), w = fabs(uvw[3 * r + 2]);
    mu = fmax(mu, u); mv = fmax(mv, v); wmn = fmin(wmn, w); wmx = fmax(wmx, w);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mu = fmax(mu, __shfl_xor_sync(0xffffffffu, mu, o));
    mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, o));
    wmn = fmin(wmn, __shfl_xor_sync(0xffffffffu, wmn, o));
    wmx = fmax(wmx, __shfl_xor_sync(0xffffffffu, wmx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&ext[0], (unsigned long long)__double_as_longlong(mu));
    atomicMax(&ext[1], (unsigned long long)__double_as_longlong(mv));
    atomicMin(&ext[2], (unsigned long long)__double_as_longlong(wmn));
    atomicMax(&ext[3], (unsigned long long)__double_as_longlong(wmx));
  }
}

cudaError_t launch_extent(const double* uvw, int64_t nrows, unsigned long long* ext4,
                          cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((nrows + 255) / 256, 152 * 8);
  if (blocks < 1) blocks = 1;
  k_extent<<<blocks, 256, 0, s>>>(uvw, nrows, ext4);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Position of a visibility on the (u, v, w) grid (FP64).  Sec. 2: effective coordinates
// u = u~ f / c; Hermitian fold (u, v, w, d) -> (-u, -v, -w, d*) so that w >= 0; grid
// coordinate x = u dl N_u (cells); the alpha cells it touches start at ceil(x - alpha/2).
// w-plane coordinate z = (w - w_0) / dw; planes c0 .. c0 + alpha - 1 (Eq. approxw).
// chan4[4 ch + 0..3] = (f/c dl N_u, f/c dm N_v, f/c / dw, f/c).
// ---------------------------------------------------------------------------------------
struct VisPos {
  int64_t iu, iv;   // first cell, wrapped into [0, N)
  int c0;           // first plane
  double fu, fv, fw;  // first-cell offset minus coordinate, in [-alpha/2, -alpha/2 + 1)
  double wlam;      // folded w in wavelengths
  bool fold;
  bool bad;         // plane index had to be clamped (should not happen)
};

__device__ __forceinline__ void vis_position(const Geom& g, const double* __restrict__ uvw,
                                             const double* __restrict__ chan4, int64_t k,
                                             VisPos& p) {
  int64_t row = k / g.nchan;
  int ch = (int)(k - row * g.nchan);
  double ut = uvw[3 * row], vt = uvw[3 * row + 1], wt = uvw[3 * row + 2];
  p.fold = g.do_w && wt < 0.0;
  if (p.fold) { ut = -ut; vt = -vt; wt = -wt; }
  const double* sc = chan4 + 4 * ch;
  const double half = 0.5 * g.alpha;
  double x = __dmul_rn(ut, sc[0]);
  double y = __dmul_rn(vt, sc[1]);
  double cu = ceil(__dsub_rn(x, half));
  double cv = ceil(__dsub_rn(y, half));
  p.fu = __dsub_rn(cu, x);
  p.fv = __dsub_rn(cv, y);
  int64_t iu = (int64_t)cu % g.nu, iv = (int64_t)cv % g.nv;
  p.iu = iu < 0 ? iu + g.nu : iu;
  p.iv = iv < 0 ? iv + g.nv : iv;
  p.bad = false;
  p.wlam = g.do_w ? __dmul_rn(wt, sc[3]) : 0.0;
  if (g.do_w) {
    double z = __dsub_rn(__dmul_rn(wt, sc[2]), g.w0_dw);
    double cw = ceil(__dsub_rn(z, half));
    p.fw = __dsub_rn(cw, z);
    int c0 = (int)cw;
    if (c0 < 0) { c0 = 0; p.bad = true; }
    if (c0 > g.nw - g.alpha) { c0 = g.nw - g.alpha; p.bad = true; }
    p.c0 = c0;
  } else {
    p.c0 = 0;
    p.fw = -half;
  }
}

__device__ __forceinline__ uint32_t bucket_key(const Geom& g, const VisPos& p) {
  int tu = (int)(p.iu / g.tile), tv = (int)(p.iv / g.tile);
  return (uint32_t)(((int64_t)tu * g.ntv + tv) * g.nw + p.c0);
}

constexpr uint32_t kNoKey = 0xffffffffu;

// Histogram of bucket keys with warp-aggregated atomics: lanes that share a key (typically
// neighbouring channels of one row) elect one lane that adds their count; every lane gets its
// rank inside the bucket.
__global__ void k_bin_count(const Geom g, const double* __restrict__ uvw,
                            const double* __restrict__ chan4, const uint8_t* __restrict__ mask,
                            uint32_t* __restrict__ hist, uint32_t* __restrict__ key,
                            uint32_t* __restrict__ rank, int* __restrict__ err) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool valid = k < g.nvis && (mask == nullptr || mask[k] != 0);
  uint32_t kk = kNoKey;
  if (valid) {
    VisPos p;
    vis_position(g, uvw, chan4, k, p);
    if (p.bad) atomicOr(err, 1);
    kk = bucket_key(g, p);
  }
  unsigned active = __ballot_sync(0xffffffffu, valid);
  if (valid) {
    unsigned peers = __match_any_sync(active, kk);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    unsigned below = peers & ((1u << lane) - 1u);
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&hist[kk], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    rank[k] = base + (uint32_t)__popc(below);
  }
  if (k < g.nvis) key[k] = kk;
}

cudaError_t launch_bin_count(const Geom& g, const double* uvw, const double* chan4,
                             const uint8_t* mask, uint32_t* hist, uint32_t* key,
                             uint32_t* rank, int* err, cudaStream_t s) {
  int64_t blocks = (g.nvis + 255) / 256;
  if (blocks == 0) return cudaSuccess;
  k_bin_count<<<(unsigned)blocks, 256, 0, s>>>(g, uvw, chan4, mask, hist, key, rank, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Exclusive scan of uint32 counts (multi-level: 4096 elements per block).
// ---------------------------------------------------------------------------------------
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads) k_scan_block(uint32_t* __restrict__ data,
                                                             int64_t n,
                                                             uint32_t* __restrict__ bsum) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t tsum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? data[base + i] : 0u;
    tsum += v[i];
  }
  // inclusive warp scan of thread sums
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;  // inclusive
  }
  __syncthreads();
  uint32_t run = x - tsum + (wid > 0 ? warp_tot[wid - 1] : 0u);  // exclusive start of thread
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) data[base + i] = run;
    run += v[i];
  }
  if (bsum != nullptr && threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = run;
}

__global__ void k_scan_add(uint32_t* __restrict__ data, int64_t n,
                           const uint32_t* __restrict__ boff) {
  uint32_t add = boff[blockIdx.x];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
    if (base + i < n) data[base + i] += add;
}

size_t scan_scratch_elems(int64_t n) {
  size_t tot = 0;
  while (n > kScanTile) {
    n = (n + kScanTile - 1) / kScanTile;
    tot += (size_t)n;
  }
  return tot + 1;
}

cudaError_t launch_scan(uint32_t* data, int64_t n, uint32_t* scratch, cudaStream_t s) {
  if (n <= kScanTile) {
    k_scan_block<<<1, kScanThreads, 0, s>>>(data, n, nullptr);
    return cudaGetLastError();
  }
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  k_scan_block<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan(scratch, nb, scratch + nb, s);
  if (e != cudaSuccess) return e;
  k_scan_add<<<(unsigned)nb, 256, 0, s>>>(data, n, scratch);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// The record of visibility k at index position pos: meta (first cell inside its tile, first
// plane), Horner coordinates of the first kernel piece, and e^{2 pi i w_k nshift}.
// ---------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void write_record(const Geom& g, const VisPos& p, uint32_t pos,
                                             uint32_t* __restrict__ meta, Z4<R>* __restrict__ z,
                                             typename C2<R>::T* __restrict__ ph) {
  int du = (int)(p.iu % g.tile), dv = (int)(p.iv % g.tile);
  meta[pos] = (uint32_t)du | ((uint32_t)dv << 8) | ((uint32_t)p.c0 << 16);
  // Horner coordinate of the first piece: z = 2 (f + alpha/2) - 1 (Sec. 4.2)
  Z4<R> zz;
  zz.u = (R)(2.0 * p.fu + (g.alpha - 1));
  zz.v = (R)(2.0 * p.fv + (g.alpha - 1));
  zz.w = (R)(2.0 * p.fw + (g.alpha - 1));
  zz.pad = (R)0;
  z[pos] = zz;
  if (ph != nullptr) {
    // exp(2 pi i w_k nshift): the part of the w-term carried by the shifted reference
    double cyc = p.wlam * g.nshift;
    cyc -= rint(cyc);
    double sn, cs;
    sincospi(2.0 * cyc, &sn, &cs);
    typename C2<R>::T v;
    v.x = (R)cs; v.y = (R)sn;
    ph[pos] = v;
  }
}

// ---------------------------------------------------------------------------------------
// Scatter: each visibility writes its index entry (k | fold bit) at off[key] + rank, and, for
// a full index, its record (meta, z, ph may be null for a compact index).
// ---------------------------------------------------------------------------------------
template <typename R>
__global__ void k_bin_scatter(const Geom g, const double* __restrict__ uvw,
                              const double* __restrict__ chan4,
                              const uint32_t* __restrict__ key, const uint32_t* __restrict__ rank,
                              const uint32_t* __restrict__ off, uint32_t* __restrict__ idx,
                              uint32_t* __restrict__ meta, Z4<R>* __restrict__ z,
                              typename C2<R>::T* __restrict__ ph) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= g.nvis) return;
  uint32_t kk = key[k];
  if (kk == kNoKey) return;
  uint32_t pos = off[kk] + rank[k];
  VisPos p;
  vis_position(g, uvw, chan4, k, p);
  idx[pos] = (uint32_t)k | (p.fold ? kFoldBit : 0u);
  if (meta != nullptr) write_record<R>(g, p, pos, meta, z, ph);
}

template <typename R>
cudaError_t launch_bin_scatter(const Geom& g, const double* uvw, const double* chan4,
                               const uint32_t* key, const uint32_t* rank, const uint32_t* off,
                               uint32_t* idx, uint32_t* meta, Z4<R>* z,
                               typename C2<R>::T* ph, cudaStream_t s) {
  int64_t blocks = (g.nvis + 255) / 256;
  if (blocks == 0) return cudaSuccess;
  k_bin_scatter<R><<<(unsigned)blocks, 256, 0, s>>>(g, uvw, chan4, key, rank, off, idx, meta,
                                                     z, ph);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Expansion of a compact index: the records of index positions 0 .. nvis_idx - 1 recomputed
// from the plan's copy of uvw and the channel scales (the same FP64 arithmetic as the scatter,
// so the records are identical to a full index's).
// ---------------------------------------------------------------------------------------
template <typename R>
__global__ void k_expand(const Geom g, const double* __restrict__ uvw,
                         const double* __restrict__ chan4, const uint32_t* __restrict__ idx,
                         int64_t nvis_idx, uint32_t* __restrict__ meta, Z4<R>* __restrict__ z,
                         typename C2<R>::T* __restrict__ ph) {
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= nvis_idx) return;
  const int64_t k = idx[pos] & ~kFoldBit;
  VisPos p;
  vis_position(g, uvw, chan4, k, p);
  write_record<R>(g, p, (uint32_t)pos, meta, z, ph);
}

template <typename R>
cudaError_t launch_expand(const Geom& g, const double* uvw, const double* chan4,
                          const uint32_t* idx, int64_t nvis_idx, uint32_t* meta, Z4<R>* z,
                          typename C2<R>::T* ph, cudaStream_t s) {
  if (nvis_idx == 0) return cudaSuccess;
  k_expand<R><<<(unsigned)((nvis_idx + 255) / 256), 256, 0, s>>>(g, uvw, chan4, idx, nvis_idx,
                                                                  meta, z, ph);
  return cudaGetLastError();
}

template cudaError_t launch_expand<float>(const Geom&, const double*, const double*,
                                          const uint32_t*, int64_t, uint32_t*, Z4<float>*,
                                          float2*, cudaStream_t);
template cudaError_t launch_expand<double>(const Geom&, const double*, const double*,
                                           const uint32_t*, int64_t, uint32_t*, Z4<double>*,
                                           double2*, cudaStream_t);
template cudaError_t launch_bin_scatter<float>(const Geom&, const double*, const double*,
                                               const uint32_t*, const uint32_t*,
                                               const uint32_t*, uint32_t*, uint32_t*,
                                               Z4<float>*, float2*, cudaStream_t);
template cudaError_t launch_bin_scatter<double>(const Geom&, const double*, const double*,
                                                const uint32_t*, const uint32_t*,
                                                const uint32_t*, uint32_t*, uint32_t*,
                                                Z4<double>*, double2*, cudaStream_t);

}  // namespace wg
