// Degridding (Eq. R3) and gridding (Eq. Rad2) kernels of the w-gridder.
//
// Work decomposition (GPU counterpart of Secs. 4.3-4.4):
//  * the uv grid is cut into T x T tiles; visibilities are binned by (tile of their first
//    cell, first w-plane c0) — the device index;
//  * a group of G lanes (G = 4, 8 or 16 >= alpha) handles one visibility: lane j evaluates
//    the j-th kernel piece in u, v and w by Horner (Sec. 4.2) and owns column j of the
//    alpha x alpha footprint;
//  * degrid: one CTA per tile stages tile + (alpha - 1) halo of each plane of a sub-batch in
//    shared memory and accumulates every visibility of the tile over its planes; lanes reduce
//    by shuffles and one lane updates the visibility (deterministic: each visibility belongs
//    to one tile, whose CTA walks the sub-batches in order);
//  * grid: one CTA per (tile, sub-batch of planes) owns the T x T cells of those planes and
//    accumulates contributions of visibilities from its own tile and the three tiles whose
//    footprints reach into it, then writes every cell exactly once (no global atomics, no
//    separate zeroing pass; empty tiles write zeros).  Two accumulation schemes: shared-memory
//    atomics (cheap in FP32) or warps that each own whole planes (no atomics, deterministic;
//    used for FP64, where shared-memory double atomics occupy the FP64 pipe).
#include "wgrid_internal.h"

namespace wg {

constexpr int kThreads = 256;

template <typename R>
__device__ __forceinline__ R horner(const R* __restrict__ sc, int deg, int j, R z) {
  R r = sc[deg * kMaxG + j];
  for (int d = deg - 1; d >= 0; --d) r = fma(r, z, sc[d * kMaxG + j]);
  return r;
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
  const int lane = threadIdx.x & 31;
  return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
}

// ---------------------------------------------------------------------------------------
// degrid
// ---------------------------------------------------------------------------------------
template <typename R, int G>
__global__ void __launch_bounds__(kThreads)
k_degrid(const Geom g, const __grid_constant__ Coef<R> coef, const IndexView<R> ix,
         const typename C2<R>::T* __restrict__ planes, int b0, int nb, int bs,
         const R* __restrict__ wgt, typename C2<R>::T* __restrict__ vis) {
  using CT = typename C2<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  R* sc = reinterpret_cast<R*>(smem);
  CT* st = reinterpret_cast<CT*>(smem + (kMaxDeg + 1) * kMaxG * sizeof(R));
  const int T = g.tile, alpha = g.alpha, aw = g.alpha_w;
  const int TH = T + alpha - 1;
  const int t = blockIdx.x;
  const int tu = t / g.ntv, tv = t - tu * g.ntv;
  const uint32_t* offt = ix.off + (int64_t)t * g.nw;
  for (int i = threadIdx.x; i < (g.deg + 1) * kMaxG; i += blockDim.x) sc[i] = coef.c[i];
  const int j = threadIdx.x & (G - 1);
  const int grp = threadIdx.x / G, ngrp = blockDim.x / G;
  const unsigned gmask = group_mask<G>();
  const int64_t pstride = (int64_t)g.nu * g.nv;

  for (int s0 = b0; s0 < b0 + nb; s0 += bs) {
    const int sb = min(bs, b0 + nb - s0);
    const uint32_t lo = offt[max(0, s0 - aw + 1)], hi = offt[min(g.nw, s0 + sb)];
    if (lo == hi) continue;
    __syncthreads();
    for (int pl = 0; pl < sb; ++pl) {
      const int p = s0 + pl;
      if (offt[max(0, p - aw + 1)] == offt[min(p + 1, g.nw)]) continue;  // plane unused here
      const CT* src = planes + (int64_t)(p - b0) * pstride;
      CT* dst = st + pl * TH * TH;
      for (int e = threadIdx.x; e < TH * TH; e += blockDim.x) {
        int r = e / TH, c = e - r * TH;
        int gu = tu * T + r; if (gu >= g.nu) gu -= g.nu;
        int gv = tv * T + c; if (gv >= g.nv) gv -= g.nv;
        dst[e] = src[(int64_t)gu * g.nv + gv];
      }
    }
    __syncthreads();
    for (uint32_t v0 = lo; v0 < hi; v0 += ngrp) {
      const uint32_t vi = v0 + grp;
      if (vi >= hi) continue;  // whole group
      const uint32_t mt = ix.meta[vi];
      const Z4<R> zz = ix.z[vi];
      const int du = mt & 255, dv = (mt >> 8) & 255, c0 = (int)(mt >> 16);
      const bool lj = j < alpha;
      R pu = lj ? horner(sc, g.deg, j, zz.u) : (R)0;
      R pv = lj ? horner(sc, g.deg, j, zz.v) : (R)0;
      R pw = g.do_w ? (lj ? horner(sc, g.deg, j, zz.w) : (R)0) : (j == 0 ? (R)1 : (R)0);
      R wu[G], ww[G];
#pragma unroll
      for (int i = 0; i < G; ++i) {
        wu[i] = __shfl_sync(gmask, pu, i, G);
        ww[i] = __shfl_sync(gmask, pw, i, G);
      }
      R ar = (R)0, ai = (R)0;
      if (lj) {
#pragma unroll
        for (int q = 0; q < G; ++q) {
          const int p = c0 + q;
          if (q < aw && p >= s0 && p < s0 + sb) {
            const CT* row = st + (p - s0) * TH * TH + du * TH + dv + j;
            R sr = (R)0, si = (R)0;
#pragma unroll
            for (int i = 0; i < G; ++i) {
              if (i < alpha) {
                CT gv = row[i * TH];
                sr = fma(wu[i], gv.x, sr);
                si = fma(wu[i], gv.y, si);
              }
            }
            ar = fma(ww[q], sr, ar);
            ai = fma(ww[q], si, ai);
          }
        }
        ar *= pv;
        ai *= pv;
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(gmask, ar, o, G);
        ai += __shfl_xor_sync(gmask, ai, o, G);
      }
      if (j == 0) {
        const uint32_t id = ix.idx[vi];
        const int64_t k = id & ~kFoldBit;
        if (ix.ph != nullptr) {  // exp(2 pi i w nshift) times the gridded sum
          CT ph = ix.ph[vi];
          R r = ar * ph.x - ai * ph.y;
          ai = ar * ph.y + ai * ph.x;
          ar = r;
        }
        if (id & kFoldBit) ai = -ai;  // Hermitian fold undone: d = conj(d')
        if (wgt != nullptr) { R w = wgt[k]; ar *= w; ai *= w; }
        CT o = vis[k];
        o.x += ar; o.y += ai;
        vis[k] = o;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// grid, plane-owner variant (default for FP64)
//
// CTA = (uv tile, sub-batch of bs planes).  Warp w owns planes w, w + 8, ... of the
// sub-batch: it alone updates their T x T accumulators, so the updates are plain shared-memory
// read-modify-writes (no atomics, deterministic order).  Visibilities are handled in chunks:
// first every thread group computes the chunk's kernel weights (alpha values in u, v and w,
// Horner, Sec. 4.2) and weighted data into shared memory; then each warp walks the chunk and,
// for every visibility touching one of its planes, its 32 lanes cover distinct cells of the
// alpha x alpha footprint (lane -> column j, row group rg; rows rg, rg + 32/G, ...).
// ---------------------------------------------------------------------------------------
constexpr int kChunk = 64;   // visibilities staged per chunk

template <typename R>
struct GridStage {
  R wu[kChunk][kMaxG];
  R wv[kChunk][kMaxG];
  R ww[kChunk][kMaxG];
  typename C2<R>::T d[kChunk];
  int ru[kChunk], rv[kChunk], c0[kChunk];
};

template <typename R, int G>
__global__ void __launch_bounds__(kThreads)
k_grid_owner(const Geom g, const __grid_constant__ Coef<R> coef, const IndexView<R> ix,
       const typename C2<R>::T* __restrict__ vis, const R* __restrict__ wgt,
       typename C2<R>::T* __restrict__ planes, int b0, int nb, int bs, int pitch) {
  using CT = typename C2<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  R* sc = reinterpret_cast<R*>(smem);
  GridStage<R>* stg = reinterpret_cast<GridStage<R>*>(smem + (kMaxDeg + 1) * kMaxG * sizeof(R));
  CT* acc = reinterpret_cast<CT*>(reinterpret_cast<unsigned char*>(stg) + sizeof(GridStage<R>));
  const int T = g.tile, alpha = g.alpha, aw = g.alpha_w;
  const int t = blockIdx.x;
  const int tu = t / g.ntv, tv = t - tu * g.ntv;
  const int s0 = b0 + blockIdx.y * bs;
  const int sb = min(bs, b0 + nb - s0);
  const int plane_elems = T * pitch;
  for (int i = threadIdx.x; i < (g.deg + 1) * kMaxG; i += blockDim.x) sc[i] = coef.c[i];
  for (int e = threadIdx.x; e < sb * plane_elems; e += blockDim.x) {
    CT z; z.x = (R)0; z.y = (R)0;
    acc[e] = z;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // phase-1 mapping: groups of G lanes, one visibility each
  const int j1 = threadIdx.x & (G - 1), grp = threadIdx.x / G, ngrp = blockDim.x / G;
  // phase-2 mapping: lane -> column jc, first row rg; rows advance by 32 / G
  const int jc = lane & (G - 1), rg = lane / G;
  constexpr int RSTEP = 32 / G;

  for (int src = 0; src < 4; ++src) {
    const int ou = (src & 1) ? -1 : 0, ov = (src & 2) ? -1 : 0;
    int stu = tu + ou; if (stu < 0) stu += g.ntu;
    int stv = tv + ov; if (stv < 0) stv += g.ntv;
    const uint32_t* offs = ix.off + ((int64_t)stu * g.ntv + stv) * g.nw;
    const uint32_t lo = offs[max(0, s0 - aw + 1)], hi = offs[min(g.nw, s0 + sb)];
    for (uint32_t cs = lo; cs < hi; cs += kChunk) {
      const int nch = (int)min((uint32_t)kChunk, hi - cs);
      __syncthreads();  // previous chunk consumed (and accumulators zeroed)
      // ---- phase 1: weights and data of the chunk ----
      for (int v = grp; v < nch; v += ngrp) {
        const uint32_t vi = cs + v;
        const uint32_t mt = ix.meta[vi];
        const int ru = (int)(mt & 255) + ou * T, rv = (int)((mt >> 8) & 255) + ov * T;
        const bool hit = (ru + alpha > 0) && (rv + alpha > 0);
        if (j1 == 0) {
          stg->ru[v] = ru; stg->rv[v] = rv;
          stg->c0[v] = hit ? (int)(mt >> 16) : -(1 << 20);
        }
        if (!hit) continue;
        const Z4<R> zz = ix.z[vi];
        const bool lj = j1 < alpha;
        stg->wu[v][j1] = lj ? horner(sc, g.deg, j1, zz.u) : (R)0;
        stg->wv[v][j1] = lj ? horner(sc, g.deg, j1, zz.v) : (R)0;
        stg->ww[v][j1] = g.do_w ? (lj ? horner(sc, g.deg, j1, zz.w) : (R)0) : (j1 == 0 ? (R)1 : (R)0);
        if (j1 == 0) {
          const uint32_t id = ix.idx[vi];
          const int64_t k = id & ~kFoldBit;
          CT d = vis[k];
          R dr = d.x, di = d.y;
          if (wgt != nullptr) { R w = wgt[k]; dr *= w; di *= w; }
          if (id & kFoldBit) di = -di;      // grid conj(d) at the folded coordinates
          if (ix.ph != nullptr) {           // times conj(exp(2 pi i w nshift))
            CT ph = ix.ph[vi];
            R r = dr * ph.x + di * ph.y;
            di = di * ph.x - dr * ph.y;
            dr = r;
          }
          CT o; o.x = dr; o.y = di;
          stg->d[v] = o;
        }
      }
      __syncthreads();
      // ---- phase 2: each warp adds the chunk into its own planes ----
      for (int v = 0; v < nch; ++v) {
        const int c0 = stg->c0[v];
        if (c0 < -1000) continue;
        const int ru = stg->ru[v], rv = stg->rv[v];
        const int col = rv + jc;
        const bool colok = jc < alpha && col >= 0 && col < T;
        const CT d = stg->d[v];
        const R wvj = stg->wv[v][jc];
        for (int pl = warp; pl < sb; pl += nwarps) {
          const int q = s0 + pl - c0;
          if (q < 0 || q >= aw) continue;
          if (!colok) continue;
          const R wq = stg->ww[v][q] * wvj;
          const R dr = d.x * wq, di = d.y * wq;
          CT* base = acc + pl * plane_elems + col;
#pragma unroll
          for (int m = 0; m < (G + RSTEP - 1) / RSTEP; ++m) {
            const int i = rg + m * RSTEP;
            const int row = ru + i;
            if (i < alpha && row >= 0 && row < T) {
              const R wui = stg->wu[v][i];
              CT a = base[row * pitch];
              a.x = fma(dr, wui, a.x);
              a.y = fma(di, wui, a.y);
              base[row * pitch] = a;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  const int64_t pstride = (int64_t)g.nu * g.nv;
  for (int e = threadIdx.x; e < sb * T * T; e += blockDim.x) {
    const int pl = e / (T * T), rem = e - pl * T * T;
    const int r = rem / T, c = rem - r * T;
    planes[(int64_t)(s0 - b0 + pl) * pstride + (int64_t)(tu * T + r) * g.nv + tv * T + c] =
        acc[pl * plane_elems + r * pitch + c];
  }
}

// ---------------------------------------------------------------------------------------
// grid, shared-atomic variant (default for FP32)
//
// CTA = (uv tile, sub-batch of planes), owning the T x T cells of those planes.  A group of G
// lanes handles one visibility (lane j = footprint column j) and adds its alpha x alpha x
// alpha contributions with shared-memory float atomics; groups run concurrently, so cells
// shared by overlapping footprints are combined by the atomics (summation order not fixed).
// ---------------------------------------------------------------------------------------
template <typename R, int G>
__global__ void __launch_bounds__(kThreads)
k_grid_atomic(const Geom g, const __grid_constant__ Coef<R> coef, const IndexView<R> ix,
       const typename C2<R>::T* __restrict__ vis, const R* __restrict__ wgt,
       typename C2<R>::T* __restrict__ planes, int b0, int nb, int bs) {
  using CT = typename C2<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  R* sc = reinterpret_cast<R*>(smem);
  CT* acc = reinterpret_cast<CT*>(smem + (kMaxDeg + 1) * kMaxG * sizeof(R));
  const int T = g.tile, alpha = g.alpha, aw = g.alpha_w;
  const int t = blockIdx.x;
  const int tu = t / g.ntv, tv = t - tu * g.ntv;
  const int s0 = b0 + blockIdx.y * bs;
  const int sb = min(bs, b0 + nb - s0);
  for (int i = threadIdx.x; i < (g.deg + 1) * kMaxG; i += blockDim.x) sc[i] = coef.c[i];
  for (int e = threadIdx.x; e < sb * T * T; e += blockDim.x) {
    CT z; z.x = (R)0; z.y = (R)0;
    acc[e] = z;
  }
  __syncthreads();
  const int j = threadIdx.x & (G - 1);
  const int grp = threadIdx.x / G, ngrp = blockDim.x / G;
  const unsigned gmask = group_mask<G>();
  const bool lj = j < alpha;

  // sources: this tile and the tiles one to the left / above / both, whose visibilities'
  // alpha x alpha footprints can reach into this tile (alpha - 1 <= T)
  for (int src = 0; src < 4; ++src) {
    const int ou = (src & 1) ? -1 : 0, ov = (src & 2) ? -1 : 0;
    int stu = tu + ou; if (stu < 0) stu += g.ntu;
    int stv = tv + ov; if (stv < 0) stv += g.ntv;
    const uint32_t* offs = ix.off + ((int64_t)stu * g.ntv + stv) * g.nw;
    const uint32_t lo = offs[max(0, s0 - aw + 1)], hi = offs[min(g.nw, s0 + sb)];
    for (uint32_t v0 = lo; v0 < hi; v0 += ngrp) {
      const uint32_t vi = v0 + grp;
      if (vi >= hi) continue;
      const uint32_t mt = ix.meta[vi];
      const int ru = (int)(mt & 255) + ou * T, rv = (int)((mt >> 8) & 255) + ov * T;
      if (ru + alpha <= 0 || rv + alpha <= 0) continue;  // footprint misses this tile
      const int c0 = (int)(mt >> 16);
      const Z4<R> zz = ix.z[vi];
      const uint32_t id = ix.idx[vi];
      const int64_t k = id & ~kFoldBit;
      R pu = lj ? horner(sc, g.deg, j, zz.u) : (R)0;
      R pv = lj ? horner(sc, g.deg, j, zz.v) : (R)0;
      R pw = g.do_w ? (lj ? horner(sc, g.deg, j, zz.w) : (R)0) : (j == 0 ? (R)1 : (R)0);
      R wu[G], ww[G];
#pragma unroll
      for (int i = 0; i < G; ++i) {
        wu[i] = __shfl_sync(gmask, pu, i, G);
        ww[i] = __shfl_sync(gmask, pw, i, G);
      }
      const int col = rv + j;
      if (!lj || col < 0 || col >= T) continue;
      CT d = vis[k];
      R dr = d.x, di = d.y;
      if (wgt != nullptr) { R w = wgt[k]; dr *= w; di *= w; }
      if (id & kFoldBit) di = -di;      // grid conj(d) at the folded coordinates
      if (ix.ph != nullptr) {           // times conj(exp(2 pi i w nshift))
        CT ph = ix.ph[vi];
        R r = dr * ph.x + di * ph.y;
        di = di * ph.x - dr * ph.y;
        dr = r;
      }
      dr *= pv;
      di *= pv;
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const int p = c0 + q;
        if (q < aw && p >= s0 && p < s0 + sb) {
          const R qr = dr * ww[q], qi = di * ww[q];
          CT* base = acc + (p - s0) * T * T + col;
#pragma unroll
          for (int i = 0; i < G; ++i) {
            const int row = ru + i;
            if (i < alpha && row >= 0 && row < T) {
              atomicAdd(&base[row * T].x, qr * wu[i]);
              atomicAdd(&base[row * T].y, qi * wu[i]);
            }
          }
        }
      }
    }
  }
  __syncthreads();
  const int64_t pstride = (int64_t)g.nu * g.nv;
  for (int e = threadIdx.x; e < sb * T * T; e += blockDim.x) {
    const int pl = e / (T * T), rem = e - pl * T * T;
    const int r = rem / T, c = rem - r * T;
    planes[(int64_t)(s0 - b0 + pl) * pstride + (int64_t)(tu * T + r) * g.nv + tv * T + c] = acc[e];
  }
}

// ---------------------------------------------------------------------------------------
// launchers: sub-batch sizes from a shared-memory budget per CTA
// ---------------------------------------------------------------------------------------
constexpr size_t kDegridSmemBudget = 100 * 1024;
constexpr size_t kGridSmemBudget = 110 * 1024;
constexpr size_t kGridAtomicSmemBudget = 72 * 1024;

template <typename R>
static size_t coef_bytes() { return (kMaxDeg + 1) * kMaxG * sizeof(R); }

template <typename R, int G>
static cudaError_t degrid_g(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                            const typename C2<R>::T* planes, int b0, int nb, const R* wgt,
                            typename C2<R>::T* vis, cudaStream_t s) {
  const int TH = g.tile + g.alpha - 1;
  const size_t per = (size_t)TH * TH * sizeof(typename C2<R>::T);
  int bs = (int)std::max<size_t>(1, (kDegridSmemBudget - coef_bytes<R>()) / per);
  bs = std::min(bs, nb);
  size_t smem = coef_bytes<R>() + (size_t)bs * per;
  cudaError_t e = cudaFuncSetAttribute(k_degrid<R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int64_t ntiles = (int64_t)g.ntu * g.ntv;
  k_degrid<R, G><<<(unsigned)ntiles, kThreads, smem, s>>>(g, coef, ix, planes, b0, nb, bs, wgt, vis);
  return cudaGetLastError();
}

template <typename R, int G>
static cudaError_t grid_owner_g(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                                const typename C2<R>::T* vis, const R* wgt,
                                typename C2<R>::T* planes, int b0, int nb, cudaStream_t s) {
  // accumulator rows padded so that the row groups of a warp fall on different banks (FP32)
  const int pitch = g.tile + (sizeof(R) == 4 ? 8 : 0);
  const size_t per = (size_t)g.tile * pitch * sizeof(typename C2<R>::T);
  const size_t fixed = coef_bytes<R>() + sizeof(GridStage<R>);
  const int nwarps = kThreads / 32;
  int bs = (int)std::max<size_t>(1, (kGridSmemBudget - fixed) / per);
  if (bs > nwarps) bs -= bs % nwarps;  // equal planes per warp
  bs = std::min(bs, nb);
  size_t smem = fixed + (size_t)bs * per;
  cudaError_t e = cudaFuncSetAttribute(k_grid_owner<R, G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t ntiles = (int64_t)g.ntu * g.ntv;
  dim3 grid((unsigned)ntiles, (unsigned)((nb + bs - 1) / bs));
  k_grid_owner<R, G><<<grid, kThreads, smem, s>>>(g, coef, ix, vis, wgt, planes, b0, nb, bs, pitch);
  return cudaGetLastError();
}

template <typename R, int G>
static cudaError_t grid_atomic_g(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                                 const typename C2<R>::T* vis, const R* wgt,
                                 typename C2<R>::T* planes, int b0, int nb, cudaStream_t s) {
  const size_t per = (size_t)g.tile * g.tile * sizeof(typename C2<R>::T);
  int bs = (int)std::max<size_t>(1, (kGridAtomicSmemBudget - coef_bytes<R>()) / per);
  bs = std::min(bs, nb);
  size_t smem = coef_bytes<R>() + (size_t)bs * per;
  cudaError_t e = cudaFuncSetAttribute(k_grid_atomic<R, G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t ntiles = (int64_t)g.ntu * g.ntv;
  dim3 grid((unsigned)ntiles, (unsigned)((nb + bs - 1) / bs));
  k_grid_atomic<R, G><<<grid, kThreads, smem, s>>>(g, coef, ix, vis, wgt, planes, b0, nb, bs);
  return cudaGetLastError();
}

template <typename R, int G>
static cudaError_t grid_g(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                          const typename C2<R>::T* vis, const R* wgt,
                          typename C2<R>::T* planes, int b0, int nb, cudaStream_t s) {
  const bool owner = g.grid_variant == 2 || (g.grid_variant == 0 && sizeof(R) == 8);
  if (owner) return grid_owner_g<R, G>(g, coef, ix, vis, wgt, planes, b0, nb, s);
  return grid_atomic_g<R, G>(g, coef, ix, vis, wgt, planes, b0, nb, s);
}

template <typename R>
cudaError_t launch_degrid(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                          const typename C2<R>::T* planes, int b0, int nb, const R* wgt,
                          typename C2<R>::T* vis, cudaStream_t s) {
  if (g.alpha <= 4) return degrid_g<R, 4>(g, coef, ix, planes, b0, nb, wgt, vis, s);
  if (g.alpha <= 8) return degrid_g<R, 8>(g, coef, ix, planes, b0, nb, wgt, vis, s);
  return degrid_g<R, 16>(g, coef, ix, planes, b0, nb, wgt, vis, s);
}

template <typename R>
cudaError_t launch_grid(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                        const typename C2<R>::T* vis, const R* wgt, typename C2<R>::T* planes,
                        int b0, int nb, cudaStream_t s) {
  if (g.alpha <= 4) return grid_g<R, 4>(g, coef, ix, vis, wgt, planes, b0, nb, s);
  if (g.alpha <= 8) return grid_g<R, 8>(g, coef, ix, vis, wgt, planes, b0, nb, s);
  return grid_g<R, 16>(g, coef, ix, vis, wgt, planes, b0, nb, s);
}

template cudaError_t launch_degrid<float>(const Geom&, const Coef<float>&, const IndexView<float>&,
                                          const float2*, int, int, const float*, float2*,
                                          cudaStream_t);
template cudaError_t launch_degrid<double>(const Geom&, const Coef<double>&,
                                           const IndexView<double>&, const double2*, int, int,
                                           const double*, double2*, cudaStream_t);
template cudaError_t launch_grid<float>(const Geom&, const Coef<float>&, const IndexView<float>&,
                                        const float2*, const float*, float2*, int, int,
                                        cudaStream_t);
template cudaError_t launch_grid<double>(const Geom&, const Coef<double>&,
                                         const IndexView<double>&, const double2*,
                                         const double*, double2*, int, int, cudaStream_t);

}  // namespace wg
