// Degridding (Eq. R3) and gridding (Eq. Rad2) kernels of the w-gridder.
//
// Work decomposition (GPU counterpart of Secs. 4.3-4.4):
//  * the uv grid is cut into T x T tiles; visibilities are binned by (tile of their first
//    cell, first w-plane c0) — the device index;
//  * a group of G lanes (G = 4, 8 or 16 >= alpha) handles one visibility: lane j evaluates
//    the j-th kernel piece in u, v and w by Horner (Sec. 4.2) and owns column j of the
//    alpha x alpha footprint;
//  * degrid: one CTA per (tile, sub-batch of planes) stages tile + (alpha - 1) halo of those
//    planes in shared memory; each visibility of the tile sums its footprint over the staged
//    planes, lanes reduce by shuffles, and the partial sum goes to a fixed slot; a finalize
//    pass adds the slots in order (deterministic, no atomics);
//  * grid: one CTA per (tile, sub-batch of planes) owns the T x T cells of those planes and
//    accumulates contributions of visibilities from its own tile and the three tiles whose
//    footprints reach into it, then writes every cell exactly once (no global atomics, no
//    separate zeroing pass; empty tiles write zeros).  Two accumulation schemes: shared-memory
//    atomics (cheap in FP32) or warps that each own whole planes (no atomics, deterministic;
//    used for FP64, where shared-memory double atomics occupy the FP64 pipe);
//  * FP64 plans with the double-float FFT keep the planes as double-float pairs and run the
//    degridding and plane-owner gridding in pair arithmetic on the FP32 pipes (df64.cuh).
#include "df64.cuh"
#include "wgrid_internal.h"

namespace wg {

constexpr int kThreads = 256;


// asynchronous 8- or 16-byte global -> shared copy (cp.async) of one plane cell; completed by
// stage_wait() before the block's barrier
template <typename CT>
__device__ __forceinline__ void stage_copy(CT* d, const CT* g) {
  static_assert(sizeof(CT) == 8 || sizeof(CT) == 16, "plane cell size");
  const unsigned sa = (unsigned)__cvta_generic_to_shared(d);
  if (sizeof(CT) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(g) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void stage_wait() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <typename R>
__device__ __forceinline__ R horner(const R* __restrict__ sc, int deg, int j, R z) {
  R r = sc[deg * kMaxG + j];
  for (int d = deg - 1; d >= 0; --d) r = fma(r, z, sc[d * kMaxG + j]);
  return r;
}

// piece j of direction d (0 u, 1 v, 2 w) of indexed visibility vi: from the per-call table when
// present, else by Horner from the shared-memory coefficients
template <typename R>
__device__ __forceinline__ R kernel_value(const IndexView<R>& ix, const R* __restrict__ sc,
                                          int deg, uint32_t vi, int d, int j, R z) {
  if (ix.wts != nullptr) return ix.wts[(int64_t)vi * (3 * kMaxG) + d * kMaxG + j];
  return horner(sc, deg, j, z);
}

// The coefficients of one kernel piece held in a lane's registers (FP32 kernels, where a lane
// evaluates the same piece for every visibility it handles): zero-padded up to degree G + 3
// (alpha <= G), so Horner runs a fixed number of steps with no shared-memory loads.
template <typename R, int G>
struct LanePiece {
  static constexpr int kDeg = G + 3;
  R c[kDeg + 1];
  __device__ __forceinline__ void load(const R* __restrict__ sc, int deg, int j) {
#pragma unroll
    for (int d = 0; d <= kDeg; ++d) c[d] = d <= deg ? sc[d * kMaxG + j] : (R)0;
  }
  __device__ __forceinline__ R eval(R z) const {
    R r = c[kDeg];
#pragma unroll
    for (int d = kDeg - 1; d >= 0; --d) r = fma(r, z, c[d]);
    return r;
  }
};
// register pieces for FP32 only (an FP64 piece would take 40 registers; FP64 plans read the
// per-call or plan-resident value table, or Horner from shared memory)
template <typename R, int G>
using LanePieceOf = LanePiece<R, sizeof(R) == 4 ? G : 0>;

template <typename R, int G>
__device__ __forceinline__ R kernel_value(const IndexView<R>& ix, const LanePieceOf<R, G>& pc,
                                          const R* __restrict__ sc, int deg, uint32_t vi, int d,
                                          int j, R z) {
  if (ix.wts != nullptr) return ix.wts[(int64_t)vi * (3 * kMaxG) + d * kMaxG + j];
  if (sizeof(R) == 4) return pc.eval(z);
  return horner(sc, deg, j, z);
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
  const int lane = threadIdx.x & 31;
  return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
}

// ---------------------------------------------------------------------------------------
// degrid
//
// CTA = (uv tile, sub-batch of bs planes).  The CTA stages tile + (alpha - 1) halo of each plane
// of its sub-batch that some visibility of the tile needs, then every visibility of the tile
// whose planes meet the sub-batch computes its partial sum over those planes and stores it, as
// is, in slot (sub-batch id - first sub-batch id of the visibility) of a partial-sum array
// indexed by the visibility's position in the index.  Sub-batches are aligned to multiples of
// bs over the whole plane range, so a visibility meets at most `nslot` of them; a finalize pass
// adds its slots in slot order (deterministic, no atomics) and applies the w-reference phase,
// the Hermitian fold and the weight.
// ---------------------------------------------------------------------------------------
template <typename R, int G>
__global__ void __launch_bounds__(kThreads)
k_degrid(const Geom g, const __grid_constant__ Coef<R> coef, const IndexView<R> ix,
         const typename C2<R>::T* __restrict__ planes, int b0, int nb, int bs,
         typename C2<R>::T* __restrict__ partial, int64_t nvis_idx) {
  using CT = typename C2<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  R* sc = reinterpret_cast<R*>(smem);
  CT* st = reinterpret_cast<CT*>(smem + (kMaxDeg + 1) * kMaxG * sizeof(R));
  const int T = g.tile, alpha = g.alpha, aw = g.alpha_w;
  const int TH = T + alpha - 1;
  const int t = blockIdx.x;
  const int tu = t / g.ntv, tv = t - tu * g.ntv;
  const int s0 = b0 + blockIdx.y * bs;
  const int sb = min(bs, b0 + nb - s0);
  const int sbid = s0 / bs;                       // global sub-batch id (s0 is a multiple of bs)
  const uint32_t* offt = ix.off + (int64_t)t * g.nw;
  const uint32_t lo = offt[max(0, s0 - aw + 1)], hi = offt[min(g.nw, s0 + sb)];
  if (lo == hi) return;                           // no visibility of this tile meets these planes
  for (int i = threadIdx.x; i < (g.deg + 1) * kMaxG; i += blockDim.x) sc[i] = coef.c[i];
  const int64_t pstride = (int64_t)g.nu * g.nv;
  for (int pl = 0; pl < sb; ++pl) {
    const int p = s0 + pl;
    if (offt[max(0, p - aw + 1)] == offt[min(p + 1, g.nw)]) continue;  // plane unused here
    const CT* src = planes + (int64_t)(p - b0) * pstride;
    CT* dst = st + pl * TH * TH;
    for (int e = threadIdx.x; e < TH * TH; e += blockDim.x) {
      int r = e / TH, c = e - r * TH;
      int gu = tu * T + r; if (gu >= g.nu) gu -= g.nu;
      int gv = tv * T + c; if (gv >= g.nv) gv -= g.nv;
      stage_copy(dst + e, src + (int64_t)gu * g.nv + gv);
    }
  }
  stage_wait();
  __syncthreads();
  // G lanes per visibility (lane j = piece / footprint column j).  Visibilities of a tile are
  // sorted by first plane, so the groups of a warp have nearly the same plane range: the plane
  // loop runs over the union of the warp's ranges (warp-uniform bounds, per-group predicate)
  // instead of all G candidate planes.
  const int j = threadIdx.x & (G - 1);
  LanePieceOf<R, G> pc;
  if (sizeof(R) == 4) pc.load(sc, g.deg, j);
  const int grp = threadIdx.x / G, ngrp = blockDim.x / G;
  const unsigned gmask = group_mask<G>();
  for (uint32_t v0 = lo + (threadIdx.x >> 5) * (32 / G); v0 < hi; v0 += ngrp) {
    const uint32_t vi = v0 + (grp % (32 / G));
    const bool act = vi < hi;
    uint32_t mt = 0;
    Z4<R> zz;
    zz.u = zz.v = zz.w = zz.pad = (R)0;
    if (act) { mt = ix.meta[vi]; zz = ix.z[vi]; }
    const int du = mt & 255, dv = (mt >> 8) & 255, c0 = (int)(mt >> 16);
    const bool lj = act && j < alpha;
    R pu = lj ? kernel_value<R, G>(ix, pc, sc, g.deg, vi, 0, j, zz.u) : (R)0;
    R pv = lj ? kernel_value<R, G>(ix, pc, sc, g.deg, vi, 1, j, zz.v) : (R)0;
    R pw = g.do_w ? (lj ? kernel_value<R, G>(ix, pc, sc, g.deg, vi, 2, j, zz.w) : (R)0)
                  : (j == 0 ? (R)1 : (R)0);
    R wu[G];
#pragma unroll
    for (int i = 0; i < G; ++i) wu[i] = __shfl_sync(0xffffffffu, pu, i, G);
    const int qlo = act ? max(0, s0 - c0) : G, qhi = act ? min(aw, s0 + sb - c0) : 0;
    const int wlo = __reduce_min_sync(0xffffffffu, (unsigned)qlo);
    const int whi = __reduce_max_sync(0xffffffffu, (unsigned)qhi);
    R ar = (R)0, ai = (R)0;
    for (int q = wlo; q < whi; ++q) {
      const R wq = __shfl_sync(0xffffffffu, pw, q, G);
      if (lj && q >= qlo && q < qhi) {
        const CT* row = st + (c0 + q - s0) * TH * TH + du * TH + dv + j;
        R sr = (R)0, si = (R)0;
#pragma unroll
        for (int i = 0; i < G; ++i) {
          if (i < alpha) {
            CT gv = row[i * TH];
            sr = fma(wu[i], gv.x, sr);
            si = fma(wu[i], gv.y, si);
          }
        }
        ar = fma(wq, sr, ar);
        ai = fma(wq, si, ai);
      }
    }
    ar *= pv;
    ai *= pv;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o, G);
      ai += __shfl_xor_sync(0xffffffffu, ai, o, G);
    }
    if (act && j == 0) {
      const int slot = sbid - c0 / bs;
      CT o; o.x = ar; o.y = ai;
      partial[(int64_t)slot * nvis_idx + vi] = o;
    }
  }
}

// ---------------------------------------------------------------------------------------
// degrid of double-float planes (FP64 plans with the double-float FFT)
//
// The same decomposition as k_degrid, on planes whose cells are double-float pairs (float4:
// re hi, re lo, im hi, im lo): the tile + halo is staged as is, kernel values come as pairs
// (the kernel-value table stores them split), and the footprint sum runs in pair arithmetic on
// the FP32 pipes (dd_fma: 15 FP32 instructions for an FP64 FMA, which GB300 issues at 1/64 of
// the FP32 rate).  Each lane sums its column over rows and planes, the lanes' sums are reduced
// by shuffles in pair arithmetic, and the partial sum is stored in FP64 as in k_degrid.
// ---------------------------------------------------------------------------------------
// piece j of direction d of indexed visibility vi as a double-float pair
__device__ __forceinline__ dd kernel_value_dd(const IndexView<double>& ix, const double* __restrict__ sc,
                                              int deg, uint32_t vi, int d, int j, double z) {
  if (ix.wts != nullptr) {
    const float2 p = reinterpret_cast<const float2*>(ix.wts)[(int64_t)vi * (3 * kMaxG) + d * kMaxG + j];
    return dd_make(p.x, p.y);
  }
  return split_double(horner(sc, deg, j, z));
}

__device__ __forceinline__ dd shfl_dd(dd x, int src, int width) {
  return dd_make(__shfl_sync(0xffffffffu, x.h, src, width), __shfl_sync(0xffffffffu, x.l, src, width));
}

template <int G>
__global__ void __launch_bounds__(kThreads)
k_degrid_dd(const Geom g, const __grid_constant__ Coef<double> coef, const IndexView<double> ix,
            const double2* __restrict__ planes, int b0, int nb, int bs,
            double2* __restrict__ partial, int64_t nvis_idx) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* sc = reinterpret_cast<double*>(smem);
  double2* st = reinterpret_cast<double2*>(smem + (kMaxDeg + 1) * kMaxG * sizeof(double));
  const int T = g.tile, alpha = g.alpha, aw = g.alpha_w;
  const int TH = T + alpha - 1;
  const int t = blockIdx.x;
  const int tu = t / g.ntv, tv = t - tu * g.ntv;
  const int s0 = b0 + blockIdx.y * bs;
  const int sb = min(bs, b0 + nb - s0);
  const int sbid = s0 / bs;                       // global sub-batch id (s0 is a multiple of bs)
  const uint32_t* offt = ix.off + (int64_t)t * g.nw;
  const uint32_t lo = offt[max(0, s0 - aw + 1)], hi = offt[min(g.nw, s0 + sb)];
  if (lo == hi) return;                           // no visibility of this tile meets these planes
  for (int i = threadIdx.x; i < (g.deg + 1) * kMaxG; i += blockDim.x) sc[i] = coef.c[i];
  const int64_t pstride = (int64_t)g.nu * g.nv;
  for (int pl = 0; pl < sb; ++pl) {
    const int p = s0 + pl;
    if (offt[max(0, p - aw + 1)] == offt[min(p + 1, g.nw)]) continue;  // plane unused here
    const double2* src = planes + (int64_t)(p - b0) * pstride;
    double2* dst = st + pl * TH * TH;
    for (int e = threadIdx.x; e < TH * TH; e += blockDim.x) {
      int r = e / TH, c = e - r * TH;
      int gu = tu * T + r; if (gu >= g.nu) gu -= g.nu;
      int gv = tv * T + c; if (gv >= g.nv) gv -= g.nv;
      stage_copy(dst + e, src + (int64_t)gu * g.nv + gv);   // 16 bytes, copied as they are
    }
  }
  stage_wait();
  __syncthreads();
  const int j = threadIdx.x & (G - 1);
  const int grp = threadIdx.x / G, ngrp = blockDim.x / G;
  const dd zero = dd_make(0.f, 0.f);
  // with a kernel-value table, the group's next visibility's index entry and table values are
  // loaded while the current one is summed (the loads' latency is otherwise exposed)
  const float2* tw = reinterpret_cast<const float2*>(ix.wts);
  const uint32_t gofs = grp % (32 / G);
  uint32_t mt_n = 0;
  float2 pu_n = make_float2(0.f, 0.f), pv_n = pu_n, pw_n = pu_n;
  auto prefetch = [&](uint32_t vi) {
    if (vi < hi) {
      mt_n = ix.meta[vi];
      if (tw != nullptr && j < alpha) {
        const int64_t b = (int64_t)vi * (3 * kMaxG) + j;
        pu_n = tw[b]; pv_n = tw[b + kMaxG]; pw_n = tw[b + 2 * kMaxG];
      }
    }
  };
  uint32_t v0 = lo + (threadIdx.x >> 5) * (32 / G);
  prefetch(v0 + gofs);
  for (; v0 < hi; v0 += ngrp) {
    const uint32_t vi = v0 + gofs;
    const bool act = vi < hi;
    const uint32_t mt = act ? mt_n : 0u;
    const float2 tu = pu_n, tv = pv_n, tww = pw_n;
    prefetch(v0 + ngrp + gofs);
    Z4<double> zz;
    zz.u = zz.v = zz.w = zz.pad = 0.0;
    if (act && tw == nullptr) zz = ix.z[vi];
    const int du = mt & 255, dv = (mt >> 8) & 255, c0 = (int)(mt >> 16);
    const bool lj = act && j < alpha;
    dd pu = zero, pv = zero, pw = zero;
    if (lj) {
      if (tw != nullptr) {
        pu = dd_make(tu.x, tu.y); pv = dd_make(tv.x, tv.y); pw = dd_make(tww.x, tww.y);
      } else {
        pu = kernel_value_dd(ix, sc, g.deg, vi, 0, j, zz.u);
        pv = kernel_value_dd(ix, sc, g.deg, vi, 1, j, zz.v);
        pw = kernel_value_dd(ix, sc, g.deg, vi, 2, j, zz.w);
      }
    }
    if (!g.do_w) pw = j == 0 ? dd_make(1.f, 0.f) : zero;
    dd wu[G];
#pragma unroll
    for (int i = 0; i < G; ++i) wu[i] = shfl_dd(pu, i, G);
    const int qlo = act ? max(0, s0 - c0) : G, qhi = act ? min(aw, s0 + sb - c0) : 0;
    const int wlo = __reduce_min_sync(0xffffffffu, (unsigned)qlo);
    const int whi = __reduce_max_sync(0xffffffffu, (unsigned)qhi);
    dd ar = zero, ai = zero;
    for (int q = wlo; q < whi; ++q) {
      const dd wq = shfl_dd(pw, q, G);
      if (lj && q >= qlo && q < qhi) {
        const float4* row = reinterpret_cast<const float4*>(st + (c0 + q - s0) * TH * TH + du * TH + dv + j);
        dd sr = zero, si = zero;
#pragma unroll
        for (int i = 0; i < G; ++i) {
          if (i < alpha) {
            const float4 gv = row[i * TH];
            sr = dd_fma(wu[i], dd_make(gv.x, gv.y), sr);
            si = dd_fma(wu[i], dd_make(gv.z, gv.w), si);
          }
        }
        ar = dd_fma(wq, sr, ar);
        ai = dd_fma(wq, si, ai);
      }
    }
    ar = dd_mul(ar, pv);
    ai = dd_mul(ai, pv);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      ar = dd_add(ar, dd_make(__shfl_xor_sync(0xffffffffu, ar.h, o, G), __shfl_xor_sync(0xffffffffu, ar.l, o, G)));
      ai = dd_add(ai, dd_make(__shfl_xor_sync(0xffffffffu, ai.h, o, G), __shfl_xor_sync(0xffffffffu, ai.l, o, G)));
    }
    if (act && j == 0) {
      const int slot = sbid - c0 / bs;
      partial[(int64_t)slot * nvis_idx + vi] = make_double2(join_double(ar), join_double(ai));
    }
  }
}

// vis[k] = wgt_k * fold(e^{2 pi i w_k nshift} * sum of the visibility's partial-sum slots)
template <typename R>
__global__ void k_degrid_finalize(const Geom g, const IndexView<R> ix,
                                  const typename C2<R>::T* __restrict__ partial, int64_t nvis_idx,
                                  int bs, const R* __restrict__ wgt,
                                  typename C2<R>::T* __restrict__ vis) {
  using CT = typename C2<R>::T;
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= nvis_idx) return;
  const uint32_t id = ix.idx[pos];
  const int c0 = (int)(ix.meta[pos] >> 16);
  const int nsl = (c0 + g.alpha_w - 1) / bs - c0 / bs + 1;
  R ar = (R)0, ai = (R)0;
  for (int sl = 0; sl < nsl; ++sl) {
    CT v = partial[(int64_t)sl * nvis_idx + pos];
    ar += v.x; ai += v.y;
  }
  if (ix.ph != nullptr) {  // exp(2 pi i w nshift) times the gridded sum
    CT ph = ix.ph[pos];
    R r = ar * ph.x - ai * ph.y;
    ai = ar * ph.y + ai * ph.x;
    ar = r;
  }
  if (id & kFoldBit) ai = -ai;  // Hermitian fold undone: d = conj(d')
  const int64_t k = id & ~kFoldBit;
  if (wgt != nullptr) { R w = wgt[k]; ar *= w; ai *= w; }
  CT o; o.x = ar; o.y = ai;
  vis[k] = o;
}

// ---------------------------------------------------------------------------------------
// grid, plane-owner variant (default for FP64)
//
// CTA = (uv tile, sub-batch of bs planes).  Warp w owns planes w, w + 8, ... of the
// sub-batch: it alone updates their T x T accumulators, so the updates are plain shared-memory
// read-modify-writes (no atomics, deterministic order).  Visibilities are handled in chunks:
// first a group of G lanes per visibility stages its kernel values in u and v (Sec. 4.2) and
// its data times the w kernel value of each of its planes; then each warp walks the chunk and,
// for every visibility touching one of its planes, spreads the 32 lanes over the cells of the
// footprint that fall inside the tile (the clipped footprint, row-major) and adds their
// staged 2-D weights wu * wv times the visibility's plane-weighted data into each of its planes
// the visibility touches.  The 2-D weights are formed once per visibility in phase 1 (by the
// visibility's lane group, exchanging its u and v values by shuffles), not once per warp.
// ---------------------------------------------------------------------------------------
// visibilities staged per chunk: the staged 2-D weights of a chunk take kChunk x G^2 values
template <int G>
struct OwnerChunk {
  static constexpr int value = G > 8 ? 12 : 48;
};
// plane-owner gridding CTA: 8 warps (4 warps with 4 planes each measured 10 % slower: fewer
// warps to hide the shared-memory latency of the updates)
constexpr int kOwnerThreads = 256;
constexpr int kOwnerWarps = kOwnerThreads / 32;   // warp w owns planes w, w + kOwnerWarps, ...

template <typename R, int G>
struct GridStage {
  static constexpr int kChunk = OwnerChunk<G>::value;
  R wt[kChunk][G * G];                  // wu_i * wv_j of the clipped footprint cells, row-major
  typename C2<R>::T dq[kChunk][G];      // data x w kernel value of plane q of the visibility
  int ru[kChunk], rv[kChunk], c0[kChunk];
};

// The part of a visibility's footprint inside the tile: rows i0.., columns j0..j0 + w - 1 of
// the footprint, `cells` cells in all, footprint origin at tile cell (ru, rv).
struct OwnerFootprint {
  int i0, j0, w, cells, ru, rv;
};

// Add visibility v of the chunk into the warp's planes p1, p1 + kOwnerWarps, .. < phi: lane
// takes cells lane + 32 m (m < MC) of the clipped footprint in row-major order, loads their
// staged 2-D weights and updates each plane (plane pl uses the staged data x w value of the
// visibility's plane pl + qoff).  Lanes past the last cell update a private cell of the row
// padding (columns T, T + 1) with weight 0, so every update is unconditional.
template <typename R, int G, int MC>
__device__ __forceinline__ void owner_add(const GridStage<R, G>* __restrict__ stg, int v,
                                          const OwnerFootprint& fp, int lane, int T, int pitch,
                                          int p1, int phi, int qoff,
                                          typename C2<R>::T* __restrict__ acc, int plane_elems) {
  using CT = typename C2<R>::T;
  const float rw = 1.0f / (float)fp.w;
  const int dummy = (lane >> 1) * pitch + T + (lane & 1);
  R wt[MC];
  int off[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    const int c = lane + 32 * m;
    // c = ii * w + jj; exact in float: c < 256 and w <= 16 keep (c + 0.5) / w at least 1 / 32
    // away from an integer
    const int ii = (int)(((float)c + 0.5f) * rw), jj = c - ii * fp.w;
    const bool ok = c < fp.cells;
    const int i = fp.i0 + (ok ? ii : 0), j = fp.j0 + (ok ? jj : 0);
    wt[m] = ok ? stg->wt[v][c] : (R)0;
    off[m] = ok ? (fp.ru + i) * pitch + fp.rv + j : dummy;
  }
  // loads, arithmetic and stores in separate sweeps (see owner_add_dd)
  for (int pl = p1; pl < phi; pl += kOwnerWarps) {
    const CT dq = stg->dq[v][pl + qoff];
    CT* base = acc + pl * plane_elems;
    CT a[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m) a[m] = base[off[m]];
#pragma unroll
    for (int m = 0; m < MC; ++m) {
      a[m].x = fma(dq.x, wt[m], a[m].x);
      a[m].y = fma(dq.y, wt[m], a[m].y);
    }
#pragma unroll
    for (int m = 0; m < MC; ++m) base[off[m]] = a[m];
  }
}

template <typename R, int G>
__global__ void __launch_bounds__(kOwnerThreads)
k_grid_owner(const Geom g, const __grid_constant__ Coef<R> coef, const IndexView<R> ix,
       const typename C2<R>::T* __restrict__ vis, const R* __restrict__ wgt,
       typename C2<R>::T* __restrict__ planes, int b0, int nb, int bs, int pitch) {
  using CT = typename C2<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  R* sc = reinterpret_cast<R*>(smem);
  using Stage = GridStage<R, G>;
  constexpr int kChunk = Stage::kChunk;
  Stage* stg = reinterpret_cast<Stage*>(smem + (kMaxDeg + 1) * kMaxG * sizeof(R));
  CT* acc = reinterpret_cast<CT*>(reinterpret_cast<unsigned char*>(stg) + sizeof(Stage));
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
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // phase-1 mapping: groups of G lanes, one visibility each
  const int j1 = threadIdx.x & (G - 1), grp = threadIdx.x / G, ngrp = blockDim.x / G;
  const unsigned gmask = group_mask<G>();
  __syncthreads();   // coefficients staged
  LanePieceOf<R, G> pc;
  if (sizeof(R) == 4) pc.load(sc, g.deg, j1);

  for (int src = 0; src < 4; ++src) {
    const int ou = (src & 1) ? -1 : 0, ov = (src & 2) ? -1 : 0;
    int stu = tu + ou; if (stu < 0) stu += g.ntu;
    int stv = tv + ov; if (stv < 0) stv += g.ntv;
    const uint32_t* offs = ix.off + ((int64_t)stu * g.ntv + stv) * g.nw;
    const uint32_t lo = offs[max(0, s0 - aw + 1)], hi = offs[min(g.nw, s0 + sb)];
    for (uint32_t cs = lo; cs < hi; cs += kChunk) {
      const int nch = (int)min((uint32_t)kChunk, hi - cs);
      __syncthreads();  // previous chunk consumed (and accumulators zeroed)
      // ---- phase 1: kernel values and plane-weighted data of the chunk ----
      for (int v = grp; v < nch; v += ngrp) {
        const uint32_t vi = cs + v;
        const uint32_t mt = ix.meta[vi];
        const int ru = (int)(mt & 255) + ou * T, rv = (int)((mt >> 8) & 255) + ov * T;
        const bool hit = (ru + alpha > 0) && (rv + alpha > 0);
        if (j1 == 0) {
          stg->ru[v] = ru; stg->rv[v] = rv;
          stg->c0[v] = hit ? (int)(mt >> 16) : -(1 << 20);
        }
        if (!hit) continue;   // uniform within the group
        const Z4<R> zz = ix.z[vi];
        const bool lj = j1 < alpha;
        const R pu = lj ? kernel_value<R, G>(ix, pc, sc, g.deg, vi, 0, j1, zz.u) : (R)0;
        const R pv = lj ? kernel_value<R, G>(ix, pc, sc, g.deg, vi, 1, j1, zz.v) : (R)0;
        // 2-D weights of the footprint cells inside the tile (rows i0.., columns j0..j0+w-1),
        // row-major: lane j1 forms cells j1, j1 + G, ... from the group's u and v values
        {
          const int i0 = max(0, -ru), i1 = min(alpha, T - ru);
          const int j0 = max(0, -rv), w = min(alpha, T - rv) - j0;
          const int cells = (i1 - i0) * w;
          const float rw = 1.0f / (float)w;
          const int nt = (cells + G - 1) / G;   // same trip count for the whole group
          for (int tq = 0; tq < nt; ++tq) {
            const int c = j1 + G * tq;
            // exact in float: c < 256 and w <= 16 keep (c + 0.5) / w at least 1 / 32 away
            // from an integer
            const int ii = (int)(((float)c + 0.5f) * rw), jj = c - ii * w;
            const bool ok = c < cells;
            const R a = __shfl_sync(gmask, pu, ok ? i0 + ii : 0, G);
            const R b = __shfl_sync(gmask, pv, ok ? j0 + jj : 0, G);
            if (ok) stg->wt[v][c] = a * b;
          }
        }
        const R wwj = g.do_w ? (lj ? kernel_value<R, G>(ix, pc, sc, g.deg, vi, 2, j1, zz.w) : (R)0)
                             : (j1 == 0 ? (R)1 : (R)0);
        R dr = (R)0, di = (R)0;
        if (j1 == 0) {
          const uint32_t id = ix.idx[vi];
          const int64_t k = id & ~kFoldBit;
          CT d = vis[k];
          dr = d.x; di = d.y;
          if (wgt != nullptr) { R w = wgt[k]; dr *= w; di *= w; }
          if (id & kFoldBit) di = -di;      // grid conj(d) at the folded coordinates
          if (ix.ph != nullptr) {           // times conj(exp(2 pi i w nshift))
            CT ph = ix.ph[vi];
            R r = dr * ph.x + di * ph.y;
            di = di * ph.x - dr * ph.y;
            dr = r;
          }
        }
        dr = __shfl_sync(gmask, dr, 0, G);
        di = __shfl_sync(gmask, di, 0, G);
        CT o; o.x = dr * wwj; o.y = di * wwj;
        stg->dq[v][j1] = o;
      }
      __syncthreads();
      // ---- phase 2: each warp adds the chunk into its own planes ----
      for (int v = 0; v < nch; ++v) {
        const int c0 = stg->c0[v];
        if (c0 < -1000) continue;
        // this warp's planes among the visibility's planes c0 .. c0 + aw - 1
        const int plo = max(0, c0 - s0), phi = min(sb, c0 - s0 + aw);
        const int p1 = plo + ((warp - plo) & (kOwnerWarps - 1));
        if (p1 >= phi) continue;
        const int ru = stg->ru[v], rv = stg->rv[v];
        // footprint rows i0..i1-1 and columns j0..j1-1 inside the tile
        const int i0 = max(0, -ru), i1 = min(alpha, T - ru);
        const int j0 = max(0, -rv), j1c = min(alpha, T - rv);
        const int w = j1c - j0, cells = (i1 - i0) * w;
        // dispatch on the warp-uniform number of cells per lane, so that each case runs
        // exactly its updates (no predicated-off FP64 instructions)
        const OwnerFootprint fp{i0, j0, w, cells, ru, rv};
        switch ((cells + 31) >> 5) {
          case 1: owner_add<R, G, 1>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 2: owner_add<R, G, 2>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 3: owner_add<R, G, (G > 8 ? 3 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 4: owner_add<R, G, (G > 8 ? 4 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 5: owner_add<R, G, (G > 8 ? 5 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 6: owner_add<R, G, (G > 8 ? 6 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 7: owner_add<R, G, (G > 8 ? 7 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          default: owner_add<R, G, (G > 8 ? 8 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
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
// per-call visibility data for the pair-arithmetic gridding: position pos of the index gets
// wgt_k * d_k, conjugated where the visibility was folded (Hermitian symmetry), times
// conj(e^{2 pi i w nshift}) (the w reference shift), as double-float pairs -- the FP64 work that
// the gridding kernel would otherwise repeat on every (tile, sub-batch) visit
// ---------------------------------------------------------------------------------------
__global__ void k_grid_vis_dd(const IndexView<double> ix, const double2* __restrict__ vis,
                              const double* __restrict__ wgt, int64_t nvis_idx,
                              float4* __restrict__ out) {
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= nvis_idx) return;
  const uint32_t id = ix.idx[pos];
  const int64_t k = id & ~kFoldBit;
  const double2 d = vis[k];
  double xr = d.x, xi = d.y;
  if (wgt != nullptr) { const double w = wgt[k]; xr *= w; xi *= w; }
  if (id & kFoldBit) xi = -xi;      // grid conj(d) at the folded coordinates
  if (ix.ph != nullptr) {           // times conj(exp(2 pi i w nshift))
    const double2 ph = ix.ph[pos];
    const double r = xr * ph.x + xi * ph.y;
    xi = xi * ph.x - xr * ph.y;
    xr = r;
  }
  const dd a = split_double(xr), b = split_double(xi);
  out[pos] = make_float4(a.h, a.l, b.h, b.l);
}

cudaError_t launch_grid_vis_dd(const IndexView<double>& ix, const double2* vis, const double* wgt,
                               int64_t nvis_idx, float4* out, cudaStream_t s) {
  if (nvis_idx == 0) return cudaSuccess;
  k_grid_vis_dd<<<(unsigned)((nvis_idx + 255) / 256), 256, 0, s>>>(ix, vis, wgt, nvis_idx, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// grid of double-float planes (FP64 plans with the double-float FFT): the plane-owner scheme
// of k_grid_owner with the staged 2-D weights, the plane-weighted data and the accumulators as
// double-float pairs, updated in pair arithmetic on the FP32 pipes (dd_fma), and the planes
// written as pairs (float4 per cell) for the double-float FFT.
// ---------------------------------------------------------------------------------------
template <int G>
struct GridStageDD {
  // kernel values in u and v as pairs (the 2-D weight of a cell, one pair product, is formed
  // where it is used: 7 FP32 instructions, cheaper than staging G^2 weights), and the data
  // times the w kernel value of plane q (re hi, re lo, im hi, im lo)
  static constexpr int kChunk = 48;
  float2 wu[kChunk][G];
  float2 wv[kChunk][G];
  float4 dq[kChunk][G];
  int ru[kChunk], rv[kChunk], c0[kChunk];
};

template <int G, int MC>
__device__ __forceinline__ void owner_add_dd(const GridStageDD<G>* __restrict__ stg, int v,
                                             const OwnerFootprint& fp, int lane, int T, int pitch,
                                             int p1, int phi, int qoff, float4* __restrict__ acc,
                                             int plane_elems) {
  const float rw = 1.0f / (float)fp.w;
  const int dummy = (lane >> 1) * pitch + T + (lane & 1);
  dd wt[MC];
  int off[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    const int c = lane + 32 * m;
    // c = ii * w + jj; exact in float (see owner_add)
    const int ii = (int)(((float)c + 0.5f) * rw), jj = c - ii * fp.w;
    const bool ok = c < fp.cells;
    const int i = fp.i0 + (ok ? ii : 0), j = fp.j0 + (ok ? jj : 0);
    const float2 a = stg->wu[v][i], b = stg->wv[v][j];
    wt[m] = ok ? dd_mul(dd_make(a.x, a.y), dd_make(b.x, b.y)) : dd_make(0.f, 0.f);
    off[m] = ok ? (fp.ru + i) * pitch + fp.rv + j : dummy;
  }
  // all loads of a plane first, then the arithmetic, then all stores: the cells of one lane are
  // distinct (its idle slots share a padding cell, updated with weight 0), but the compiler
  // cannot see that, and interleaved load / store would serialise the MC update chains
  for (int pl = p1; pl < phi; pl += kOwnerWarps) {
    const float4 q = stg->dq[v][pl + qoff];
    float4* base = acc + pl * plane_elems;
    float4 a[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m) a[m] = base[off[m]];
#pragma unroll
    for (int m = 0; m < MC; ++m) {
      const dd re = dd_fma(dd_make(q.x, q.y), wt[m], dd_make(a[m].x, a[m].y));
      const dd im = dd_fma(dd_make(q.z, q.w), wt[m], dd_make(a[m].z, a[m].w));
      a[m] = make_float4(re.h, re.l, im.h, im.l);
    }
#pragma unroll
    for (int m = 0; m < MC; ++m) base[off[m]] = a[m];
  }
}

// vis: the per-position data of k_grid_vis_dd (float4 pairs, 16 bytes like a double2), which
// already carry the weights, the fold and the w-reference phase
template <int G>
__global__ void __launch_bounds__(kOwnerThreads)
k_grid_owner_dd(const Geom g, const __grid_constant__ Coef<double> coef, const IndexView<double> ix,
                const double2* __restrict__ vis, double2* __restrict__ planes, int b0, int nb,
                int bs, int pitch) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* sc = reinterpret_cast<double*>(smem);
  using Stage = GridStageDD<G>;
  constexpr int kChunk = Stage::kChunk;
  Stage* stg = reinterpret_cast<Stage*>(smem + (kMaxDeg + 1) * kMaxG * sizeof(double));
  float4* acc = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(stg) + sizeof(Stage));
  const int T = g.tile, alpha = g.alpha, aw = g.alpha_w;
  const int t = blockIdx.x;
  const int tu = t / g.ntv, tv = t - tu * g.ntv;
  const int s0 = b0 + blockIdx.y * bs;
  const int sb = min(bs, b0 + nb - s0);
  const int plane_elems = T * pitch;
  for (int i = threadIdx.x; i < (g.deg + 1) * kMaxG; i += blockDim.x) sc[i] = coef.c[i];
  for (int e = threadIdx.x; e < sb * plane_elems; e += blockDim.x) acc[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j1 = threadIdx.x & (G - 1), grp = threadIdx.x / G, ngrp = blockDim.x / G;
  const unsigned gmask = group_mask<G>();
  const dd zero = dd_make(0.f, 0.f);
  __syncthreads();   // coefficients staged

  for (int src = 0; src < 4; ++src) {
    const int ou = (src & 1) ? -1 : 0, ov = (src & 2) ? -1 : 0;
    int stu = tu + ou; if (stu < 0) stu += g.ntu;
    int stv = tv + ov; if (stv < 0) stv += g.ntv;
    const uint32_t* offs = ix.off + ((int64_t)stu * g.ntv + stv) * g.nw;
    const uint32_t lo = offs[max(0, s0 - aw + 1)], hi = offs[min(g.nw, s0 + sb)];
    for (uint32_t cs = lo; cs < hi; cs += kChunk) {
      const int nch = (int)min((uint32_t)kChunk, hi - cs);
      __syncthreads();  // previous chunk consumed (and accumulators zeroed)
      // ---- phase 1: kernel values and plane-weighted data of the chunk, as pairs ----
      for (int v = grp; v < nch; v += ngrp) {
        const uint32_t vi = cs + v;
        const uint32_t mt = ix.meta[vi];
        // with a kernel-value table, the visibility's table entries and data are loaded
        // together with its index entry (before the tile test), so their latencies overlap
        const float2* tw = reinterpret_cast<const float2*>(ix.wts);
        float2 tu = make_float2(0.f, 0.f), tv = tu, tww = tu;
        if (tw != nullptr) {
          const int64_t b = (int64_t)vi * (3 * kMaxG) + j1;
          tu = tw[b]; tv = tw[b + kMaxG]; tww = tw[b + 2 * kMaxG];
        }
        // the visibility's weighted, folded and phase-rotated data, prepared once per call by
        // k_grid_vis_dd as pairs in index order (`vis` holds them, 16 bytes per position)
        const float4 q = reinterpret_cast<const float4*>(vis)[vi];
        const int ru = (int)(mt & 255) + ou * T, rv = (int)((mt >> 8) & 255) + ov * T;
        const bool hit = (ru + alpha > 0) && (rv + alpha > 0);
        if (j1 == 0) {
          stg->ru[v] = ru; stg->rv[v] = rv;
          stg->c0[v] = hit ? (int)(mt >> 16) : -(1 << 20);
        }
        if (!hit) continue;   // uniform within the group
        const bool lj = j1 < alpha;
        dd pu = zero, pv = zero, pw = zero;
        if (lj) {
          if (tw != nullptr) {   // the table holds zeros beyond alpha as well
            pu = dd_make(tu.x, tu.y); pv = dd_make(tv.x, tv.y); pw = dd_make(tww.x, tww.y);
          } else {
            const Z4<double> zz = ix.z[vi];
            pu = kernel_value_dd(ix, sc, g.deg, vi, 0, j1, zz.u);
            pv = kernel_value_dd(ix, sc, g.deg, vi, 1, j1, zz.v);
            pw = kernel_value_dd(ix, sc, g.deg, vi, 2, j1, zz.w);
          }
        }
        stg->wu[v][j1] = make_float2(pu.h, pu.l);
        stg->wv[v][j1] = make_float2(pv.h, pv.l);
        const dd wwj = g.do_w ? pw : (j1 == 0 ? dd_make(1.f, 0.f) : zero);
        const dd dr = dd_make(q.x, q.y), di = dd_make(q.z, q.w);
        const dd qr = dd_mul(dr, wwj), qi = dd_mul(di, wwj);
        stg->dq[v][j1] = make_float4(qr.h, qr.l, qi.h, qi.l);
      }
      __syncthreads();
      // ---- phase 2: each warp adds the chunk into its own planes ----
      for (int v = 0; v < nch; ++v) {
        const int c0 = stg->c0[v];
        if (c0 < -1000) continue;
        const int plo = max(0, c0 - s0), phi = min(sb, c0 - s0 + aw);
        const int p1 = plo + ((warp - plo) & (kOwnerWarps - 1));
        if (p1 >= phi) continue;
        const int ru = stg->ru[v], rv = stg->rv[v];
        const int i0 = max(0, -ru), i1 = min(alpha, T - ru);
        const int j0 = max(0, -rv), j1c = min(alpha, T - rv);
        const int w = j1c - j0, cells = (i1 - i0) * w;
        const OwnerFootprint fp{i0, j0, w, cells, ru, rv};
        switch ((cells + 31) >> 5) {
          case 1: owner_add_dd<G, 1>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 2: owner_add_dd<G, 2>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 3: owner_add_dd<G, (G > 8 ? 3 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 4: owner_add_dd<G, (G > 8 ? 4 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 5: owner_add_dd<G, (G > 8 ? 5 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 6: owner_add_dd<G, (G > 8 ? 6 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          case 7: owner_add_dd<G, (G > 8 ? 7 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
          default: owner_add_dd<G, (G > 8 ? 8 : 1)>(stg, v, fp, lane, T, pitch, p1, phi, s0 - c0, acc, plane_elems); break;
        }
      }
    }
  }
  __syncthreads();
  const int64_t pstride = (int64_t)g.nu * g.nv;
  float4* out = reinterpret_cast<float4*>(planes);
  for (int e = threadIdx.x; e < sb * T * T; e += blockDim.x) {
    const int pl = e / (T * T), rem = e - pl * T * T;
    const int r = rem / T, c = rem - r * T;
    out[(int64_t)(s0 - b0 + pl) * pstride + (int64_t)(tu * T + r) * g.nv + tv * T + c] =
        acc[pl * plane_elems + r * pitch + c];
  }
}

// ---------------------------------------------------------------------------------------
// grid, shared-atomic variant (default for FP32)
//
// CTA = (uv tile, sub-batch of planes), owning the T x T cells of those planes as separate real
// and imaginary accumulators in shared memory.  A warp handles one visibility at a time: lane
// (j, rg) = (lane mod G, lane / G) takes footprint column j and rows rg, rg + 32 / G, ...;
// with the accumulator row pitch = G (mod 32), the 32 lanes of every atomic add hit 32
// different banks.  Kernel values (Sec. 4.2): each lane evaluates piece j in u (rg = 0) or v
// (rg > 0) and in w, and the warp exchanges them by shuffles.  Warps run concurrently, so cells
// shared by overlapping footprints are combined by the atomics (summation order not fixed).
// ---------------------------------------------------------------------------------------
// Shared memory per gridding CTA, 54 KB: four gridding CTAs per SM (with the kernel held to 64 registers).  The kernel is
// latency-bound (the atomics' read-modify-write); measured on the 1e8-visibility FP32 workload:
// two CTAs per SM (110 KB) 244 ms, three (72 KB) 197-263 ms, four 175 ms
constexpr size_t kGridAtomicSmemBudget = 54 * 1024;
constexpr int kGridAtomicMinBlocks = 4;

// shared-memory atomic add without a returned value (PTX red; 2 % faster than atomicAdd on the
// 1e8-visibility FP32 gridding)
__device__ __forceinline__ void red_add(float* p, float v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("red.shared.add.f32 [%0], %1;" :: "r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(double* p, double v) { atomicAdd(p, v); }

template <int G>
struct AtomicLayout {
  static constexpr int kRowGroups = 32 / G;                      // rows handled at once
  static constexpr int kRowsPerLane = G * G / 32 > 0 ? G * G / 32 : 1;   // ceil(G / kRowGroups)
};

template <typename R, int G>
__global__ void __launch_bounds__(kThreads, kGridAtomicMinBlocks)
k_grid_atomic(const Geom g, const __grid_constant__ Coef<R> coef, const IndexView<R> ix,
              const typename C2<R>::T* __restrict__ vis, const R* __restrict__ wgt,
              typename C2<R>::T* __restrict__ planes, int b0, int nb, int bs, int pitch) {
  using CT = typename C2<R>::T;
  constexpr int RG = AtomicLayout<G>::kRowGroups;
  constexpr int KR = AtomicLayout<G>::kRowsPerLane;
  extern __shared__ __align__(16) unsigned char smem[];
  R* sc = reinterpret_cast<R*>(smem);
  R* acc = reinterpret_cast<R*>(smem + (kMaxDeg + 1) * kMaxG * sizeof(R));
  const int T = g.tile, alpha = g.alpha, aw = g.alpha_w;
  const int t = blockIdx.x;
  const int tu = t / g.ntv, tv = t - tu * g.ntv;
  const int s0 = b0 + blockIdx.y * bs;
  const int sb = min(bs, b0 + nb - s0);
  const int plane_elems = T * pitch;
  R* acc_im = acc + sb * plane_elems;   // real parts of the sb planes, then imaginary parts
  for (int i = threadIdx.x; i < (g.deg + 1) * kMaxG; i += blockDim.x) sc[i] = coef.c[i];
  for (int e = threadIdx.x; e < 2 * sb * plane_elems; e += blockDim.x) acc[e] = (R)0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int j = lane & (G - 1), rg = lane / G;
  LanePieceOf<R, G> pc;
  if (sizeof(R) == 4) pc.load(sc, g.deg, j);
  const bool lj = j < alpha;

  // sources: this tile and the tiles one to the left / above / both, whose visibilities'
  // alpha x alpha footprints can reach into this tile (alpha - 1 <= T)
  for (int src = 0; src < 4; ++src) {
    const int ou = (src & 1) ? -1 : 0, ov = (src & 2) ? -1 : 0;
    int stu = tu + ou; if (stu < 0) stu += g.ntu;
    int stv = tv + ov; if (stv < 0) stv += g.ntv;
    const uint32_t* offs = ix.off + ((int64_t)stu * g.ntv + stv) * g.nw;
    const uint32_t lo = offs[max(0, s0 - aw + 1)], hi = offs[min(g.nw, s0 + sb)];
    // blocks of 32 visibilities per warp, interleaved over the warps (visibility vb + l nwarps
    // of block vb goes to lane l): each lane loads the coordinates and data of its visibility
    // (one round trip for 32), then the warp takes the block's visibilities whose footprint
    // meets the tile one at a time, broadcast by shuffles
    for (uint32_t vb = lo + warp; vb < hi; vb += 32 * nwarps) {
      const uint32_t vl = vb + lane * nwarps;
      uint32_t mtl = 0;
      Z4<R> zl;
      zl.u = zl.v = zl.w = zl.pad = (R)0;
      R drl = (R)0, dil = (R)0;
      bool hitl = false;
      if (vl < hi) {
        mtl = ix.meta[vl];
        const int ru = (int)(mtl & 255) + ou * T, rv = (int)((mtl >> 8) & 255) + ov * T;
        hitl = ru + alpha > 0 && rv + alpha > 0;   // footprint meets this tile
        if (hitl) {
          zl = ix.z[vl];
          const uint32_t id = ix.idx[vl];
          const int64_t k = id & ~kFoldBit;
          const CT d = vis[k];
          drl = d.x; dil = d.y;
          if (wgt != nullptr) { const R w = wgt[k]; drl *= w; dil *= w; }
          if (id & kFoldBit) dil = -dil;    // grid conj(d) at the folded coordinates
          if (ix.ph != nullptr) {           // times conj(exp(2 pi i w nshift))
            const CT ph = ix.ph[vl];
            const R r = drl * ph.x + dil * ph.y;
            dil = dil * ph.x - drl * ph.y;
            drl = r;
          }
        }
      }
      unsigned hits = __ballot_sync(0xffffffffu, hitl);
      while (hits != 0u) {
        const int v = __ffs(hits) - 1;
        hits &= hits - 1u;
        const uint32_t vi = vb + v * nwarps;
        const uint32_t mt = __shfl_sync(0xffffffffu, mtl, v);
        const int ru = (int)(mt & 255) + ou * T, rv = (int)((mt >> 8) & 255) + ov * T;
        const int c0 = (int)(mt >> 16);
        const R zu = __shfl_sync(0xffffffffu, zl.u, v), zv = __shfl_sync(0xffffffffu, zl.v, v);
        const R zw = __shfl_sync(0xffffffffu, zl.w, v);
        const R dr = __shfl_sync(0xffffffffu, drl, v), di = __shfl_sync(0xffffffffu, dil, v);
        // piece j in u (row group 0) or v (the others), and in w
        const R puv = lj ? kernel_value<R, G>(ix, pc, sc, g.deg, vi, rg == 0 ? 0 : 1, j,
                                              rg == 0 ? zu : zv) : (R)0;
        const R pw = g.do_w ? (lj ? kernel_value<R, G>(ix, pc, sc, g.deg, vi, 2, j, zw) : (R)0)
                            : (j == 0 ? (R)1 : (R)0);
        // this lane's column weight and the 2-D weights of its rows, clipped to the tile
        const R pv = __shfl_sync(0xffffffffu, puv, G + j);   // lane G + j holds v piece j
        const int col = rv + j;
        const bool colok = lj && col >= 0 && col < T;
        R cw[KR];
        int off[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) {
          const int i = rg + k * RG;
          const R pu = __shfl_sync(0xffffffffu, puv, i < G ? i : 0);   // lane i holds u piece i
          const int row = ru + i;
          const bool ok = colok && i < alpha && row >= 0 && row < T;
          cw[k] = ok ? pu * pv : (R)0;
          off[k] = ok ? row * pitch + col : -1;
        }
        const int qlo = max(0, s0 - c0), qhi = min(aw, s0 + sb - c0);
        for (int q = qlo; q < qhi; ++q) {
          const R wq = __shfl_sync(0xffffffffu, pw, q);
          const R qr = dr * wq, qi = di * wq;
          R* bre = acc + (c0 + q - s0) * plane_elems;
          R* bim = acc_im + (c0 + q - s0) * plane_elems;
#pragma unroll
          for (int k = 0; k < KR; ++k) {
            if (off[k] >= 0) {
              red_add(bre + off[k], qr * cw[k]);
              red_add(bim + off[k], qi * cw[k]);
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
    CT o;
    o.x = acc[pl * plane_elems + r * pitch + c];
    o.y = acc_im[pl * plane_elems + r * pitch + c];
    planes[(int64_t)(s0 - b0 + pl) * pstride + (int64_t)(tu * T + r) * g.nv + tv * T + c] = o;
  }
}

// ---------------------------------------------------------------------------------------
// grid, row-band owner variant (FP32, alpha <= 8, 32-cell tiles; deterministic)
//
// CTA = (32 x 32 uv tile, sub-batch of up to kBandPlanes planes), accumulators in shared memory
// as (re, im) float pairs with a row pitch of kBandPitch pairs.  Warp w owns tile rows 4w ..
// 4w + 3 of every plane of the sub-batch, so its updates are plain read-modify-writes (no
// atomics, each cell updated in index order: deterministic) and the 32 lanes of an update --
// (row r, footprint column j) = (lane / 8, lane mod 8) -- touch 32 distinct cells in two
// shared-memory wavefronts (pitch = 8 mod 16 pairs).  Visibilities of the tile and of the three
// tiles whose footprints reach into it are taken in chunks of kBandChunk:
//  1a. each visibility's footprint is tested against the tile (a bit of a 64-bit hit mask);
//  1b. the hits are staged in index order (slot = hits before it): kernel values in u and v,
//      and the data times the w kernel value of each of its planes (a group of 8 lanes per
//      visibility, lane j evaluating piece j by Horner from registers, Sec. 4.2); each staged
//      visibility sets its bit in the 64-bit masks of the row bands its footprint meets;
//  2.  each warp walks the set bits of its band's mask and adds those visibilities into its
//      rows, with the loop over the visibility's planes in the sub-batch unrolled per count.
// ---------------------------------------------------------------------------------------
constexpr int kBandTile = 32, kBandRows = 4, kBandPitch = 40, kBandChunk = 64, kBandPlanes = 8;
constexpr int kBandWarps = kBandTile / kBandRows;
static_assert(kBandRows * 8 == 32 && kBandWarps * 32 == 256, "band layout");
static_assert(kBandPitch % 16 == 8 && kBandPitch >= kBandTile + 8, "band pitch");

struct BandStage {
  float wu[kBandChunk][8], wv[kBandChunk][8];
  float2 dq[kBandChunk][8];   // data x w kernel value of plane q of the visibility
  int ru[kBandChunk], rv[kBandChunk], c0[kBandChunk];
  unsigned long long hits;                 // chunk positions whose footprint meets the tile
  unsigned long long band[kBandWarps];     // staged slots whose footprint meets band w
};

// add staged visibility v into planes pl0 .. pl0 + NQ - 1 of this lane's cell
template <int NQ>
__device__ __forceinline__ void band_add(float2* __restrict__ base, const float2* __restrict__ dq,
                                         float w2) {
  constexpr int kPlane = kBandTile * kBandPitch;
  float2 a[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) a[q] = base[q * kPlane];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const float2 d = dq[q];
    a[q].x = fmaf(d.x, w2, a[q].x);
    a[q].y = fmaf(d.y, w2, a[q].y);
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) base[q * kPlane] = a[q];
}

__global__ void __launch_bounds__(256, 2)
k_grid_band(const Geom g, const __grid_constant__ Coef<float> coef, const IndexView<float> ix,
            const float2* __restrict__ vis, const float* __restrict__ wgt,
            float2* __restrict__ planes, int b0, int nb, int bs) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* sc = reinterpret_cast<float*>(smem);
  BandStage* stg = reinterpret_cast<BandStage*>(smem + (kMaxDeg + 1) * kMaxG * sizeof(float));
  float2* acc = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(stg) + sizeof(BandStage));
  constexpr int T = kBandTile, kPlane = kBandTile * kBandPitch;
  const int alpha = g.alpha, aw = g.alpha_w;
  const int t = blockIdx.x;
  const int tu = t / g.ntv, tv = t - tu * g.ntv;
  const int s0 = b0 + blockIdx.y * bs;
  const int sb = min(bs, b0 + nb - s0);
  for (int i = threadIdx.x; i < (g.deg + 1) * kMaxG; i += blockDim.x) sc[i] = coef.c[i];
  for (int e = threadIdx.x; e < sb * kPlane; e += blockDim.x) acc[e] = make_float2(0.f, 0.f);
  if (threadIdx.x <= kBandWarps) {
    if (threadIdx.x == kBandWarps) stg->hits = 0ull;
    else stg->band[threadIdx.x] = 0ull;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // phase 1: groups of 8 lanes, one visibility each, lane j1 = kernel piece j1
  const int j1 = threadIdx.x & 7, grp = threadIdx.x >> 3;
  constexpr int kGroups = 256 / 8;
  const unsigned gmask = 0xffu << (lane & 24);
  LanePiece<float, 8> pc;
  pc.load(sc, g.deg, j1);
  // phase 2: this warp's rows band0 .. band0 + 3; lane (r, j)
  const int band0 = warp * kBandRows;
  const int row = band0 + (lane >> 3), j = lane & 7;
  for (int src = 0; src < 4; ++src) {
    // sources: this tile and the tiles one to the left / above / both, whose visibilities'
    // footprints can reach into this tile (alpha - 1 <= T)
    const int ou = (src & 1) ? -1 : 0, ov = (src & 2) ? -1 : 0;
    int stu = tu + ou; if (stu < 0) stu += g.ntu;
    int stv = tv + ov; if (stv < 0) stv += g.ntv;
    const uint32_t* offs = ix.off + ((int64_t)stu * g.ntv + stv) * g.nw;
    const uint32_t lo = offs[max(0, s0 - aw + 1)], hi = offs[min(g.nw, s0 + sb)];
    for (uint32_t cs = lo; cs < hi; cs += kBandChunk) {
      const int nch = (int)min((uint32_t)kBandChunk, hi - cs);
      // 1a: hit test (each group keeps its visibilities' index entries for 1b)
      uint32_t mt[kBandChunk / kGroups];
#pragma unroll
      for (int pass = 0; pass < kBandChunk / kGroups; ++pass) {
        const int v = grp + pass * kGroups;
        mt[pass] = 0u;
        if (v < nch) {
          mt[pass] = ix.meta[cs + v];
          const int ru = (int)(mt[pass] & 255) + ou * T, rv = (int)((mt[pass] >> 8) & 255) + ov * T;
          if (j1 == 0 && ru + alpha > 0 && rv + alpha > 0) atomicOr(&stg->hits, 1ull << v);
        }
      }
      __syncthreads();
      const unsigned long long hits = stg->hits;
      // 1b: stage the hits in index order
#pragma unroll
      for (int pass = 0; pass < kBandChunk / kGroups; ++pass) {
        const int v = grp + pass * kGroups;
        if (v >= nch || !((hits >> v) & 1ull)) continue;   // uniform within the group
        const int slot = __popcll(hits & ((1ull << v) - 1ull));
        const uint32_t vi = cs + v;
        const int ru = (int)(mt[pass] & 255) + ou * T, rv = (int)((mt[pass] >> 8) & 255) + ov * T;
        const Z4<float> zz = ix.z[vi];
        const bool lj = j1 < alpha;
        stg->wu[slot][j1] = lj ? pc.eval(zz.u) : 0.f;
        stg->wv[slot][j1] = lj ? pc.eval(zz.v) : 0.f;
        const float ww = g.do_w ? (lj ? pc.eval(zz.w) : 0.f) : (j1 == 0 ? 1.f : 0.f);
        float dr = 0.f, di = 0.f;
        if (j1 == 0) {
          const uint32_t id = ix.idx[vi];
          const int64_t k = id & ~kFoldBit;
          const float2 d = vis[k];
          dr = d.x; di = d.y;
          if (wgt != nullptr) { const float w = wgt[k]; dr *= w; di *= w; }
          if (id & kFoldBit) di = -di;      // grid conj(d) at the folded coordinates
          if (ix.ph != nullptr) {           // times conj(exp(2 pi i w nshift))
            const float2 ph = ix.ph[vi];
            const float rr = dr * ph.x + di * ph.y;
            di = di * ph.x - dr * ph.y;
            dr = rr;
          }
          stg->ru[slot] = ru; stg->rv[slot] = rv; stg->c0[slot] = (int)(mt[pass] >> 16);
        }
        // the row bands the footprint meets (lanes 1 .. : one band each)
        const int blo = max(ru, 0) / kBandRows, bhi = min(ru + alpha - 1, T - 1) / kBandRows;
        if (j1 >= 1 && blo + j1 - 1 <= bhi) atomicOr(&stg->band[blo + j1 - 1], 1ull << slot);
        dr = __shfl_sync(gmask, dr, 0, 8);
        di = __shfl_sync(gmask, di, 0, 8);
        stg->dq[slot][j1] = make_float2(dr * ww, di * ww);
      }
      __syncthreads();
      if (threadIdx.x == 0) stg->hits = 0ull;   // read again only after the next barrier
      // 2: this warp's visibilities
      unsigned long long m = stg->band[warp];
      __syncwarp();
      if (lane == 0) stg->band[warp] = 0ull;
      while (m != 0ull) {
        const int v = __ffsll((long long)m) - 1;
        m &= m - 1ull;
        const int c0 = stg->c0[v], ru = stg->ru[v], rv = stg->rv[v];
        const int qlo = max(0, s0 - c0), qhi = min(aw, s0 + sb - c0);
        const int i = row - ru, col = rv + j;
        const bool ok = i >= 0 && i < alpha && j < alpha && col >= 0 && col < T;
        const float w2 = ok ? stg->wu[v][ok ? i : 0] * stg->wv[v][j] : 0.f;
        // idle lanes update a private padding cell of their row with weight 0
        float2* base = acc + (c0 + qlo - s0) * kPlane + row * kBandPitch + (ok ? col : T + j);
        const float2* dqv = stg->dq[v] + qlo;
        switch (qhi - qlo) {
          case 1: band_add<1>(base, dqv, w2); break;
          case 2: band_add<2>(base, dqv, w2); break;
          case 3: band_add<3>(base, dqv, w2); break;
          case 4: band_add<4>(base, dqv, w2); break;
          case 5: band_add<5>(base, dqv, w2); break;
          case 6: band_add<6>(base, dqv, w2); break;
          case 7: band_add<7>(base, dqv, w2); break;
          case 8: band_add<8>(base, dqv, w2); break;
          default: break;
        }
      }
      __syncthreads();   // the staged chunk has been consumed
    }
  }
  const int64_t pstride = (int64_t)g.nu * g.nv;
  for (int e = threadIdx.x; e < sb * T * T; e += blockDim.x) {
    const int pl = e / (T * T), rem = e - pl * T * T;
    const int r = rem / T, c = rem - r * T;
    planes[(int64_t)(s0 - b0 + pl) * pstride + (int64_t)(tu * T + r) * g.nv + tv * T + c] =
        acc[pl * kPlane + r * kBandPitch + c];
  }
}

// ---------------------------------------------------------------------------------------
// per-call kernel values: one thread per (visibility, direction, piece), Horner (Sec. 4.2)
// ---------------------------------------------------------------------------------------
template <typename R>
__global__ void k_weights(const Geom g, const __grid_constant__ Coef<R> coef, const IndexView<R> ix,
                          int64_t nvis_idx, R* __restrict__ wts) {
  __shared__ R sc[(kMaxDeg + 1) * kMaxG];
  for (int i = threadIdx.x; i < (g.deg + 1) * kMaxG; i += blockDim.x) sc[i] = coef.c[i];
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nvis_idx * 3 * kMaxG) return;
  const int64_t pos = e / (3 * kMaxG);
  const int r = (int)(e - pos * 3 * kMaxG), d = r / kMaxG, j = r - d * kMaxG;
  const Z4<R> zz = ix.z[pos];
  R v = (R)0;
  if (j < g.alpha) v = horner(sc, g.deg, j, d == 0 ? zz.u : (d == 1 ? zz.v : zz.w));
  if (sizeof(R) == 8 && g.df64_planes) {
    // the pair-arithmetic kernels read the value as a double-float pair (same 8 bytes)
    const dd p = split_double((double)v);
    reinterpret_cast<float2*>(wts)[e] = make_float2(p.h, p.l);
  } else {
    wts[e] = v;
  }
}

template <typename R>
cudaError_t launch_weights(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                           int64_t nvis_idx, R* wts, cudaStream_t s) {
  if (nvis_idx == 0) return cudaSuccess;
  const int64_t n = nvis_idx * 3 * kMaxG;
  k_weights<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, coef, ix, nvis_idx, wts);
  return cudaGetLastError();
}
template cudaError_t launch_weights<float>(const Geom&, const Coef<float>&, const IndexView<float>&,
                                           int64_t, float*, cudaStream_t);
template cudaError_t launch_weights<double>(const Geom&, const Coef<double>&,
                                            const IndexView<double>&, int64_t, double*,
                                            cudaStream_t);

// ---------------------------------------------------------------------------------------
// launchers: sub-batch sizes from a shared-memory budget per CTA
// ---------------------------------------------------------------------------------------
// degridding CTA shared memory: FP32 54 KB, four CTAs per SM (measured on the 1e8-visibility
// workload: 72 KB 71.9 ms, 54 KB 61.3 ms, 44 KB 66.8 ms -- fewer planes per CTA against more
// warps to hide the staging loads); FP64 72 KB (FP64-pipe bound: more planes per CTA, fewer
// visits per visibility)
template <typename R>
constexpr size_t degrid_smem_budget() { return sizeof(R) == 4 ? 54 * 1024 : 72 * 1024; }
constexpr size_t kGridSmemBudget = 110 * 1024;

template <typename R>
static size_t coef_bytes() { return (kMaxDeg + 1) * kMaxG * sizeof(R); }

template <typename R>
static size_t degrid_plane_bytes(const Geom& g) {
  const int TH = g.tile + g.alpha - 1;
  return (size_t)TH * TH * sizeof(typename C2<R>::T);
}

template <typename R>
int degrid_subbatch(const Geom& g) {
  return (int)std::max<size_t>(1, (degrid_smem_budget<R>() - coef_bytes<R>()) / degrid_plane_bytes<R>(g));
}

template <typename R, int G>
static cudaError_t degrid_g(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                            const typename C2<R>::T* planes, int b0, int nb, int bs,
                            typename C2<R>::T* partial, int64_t nvis_idx, cudaStream_t s) {
  size_t smem = coef_bytes<R>() + (size_t)std::min(bs, nb) * degrid_plane_bytes<R>(g);
  int64_t ntiles = (int64_t)g.ntu * g.ntv;
  dim3 grid((unsigned)ntiles, (unsigned)((nb + bs - 1) / bs));
  if constexpr (sizeof(R) == 8) {
    if (g.df64_planes) {
      cudaError_t e = cudaFuncSetAttribute(k_degrid_dd<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
      k_degrid_dd<G><<<grid, kThreads, smem, s>>>(g, coef, ix, planes, b0, nb, bs, partial, nvis_idx);
      return cudaGetLastError();
    }
  }
  cudaError_t e = cudaFuncSetAttribute(k_degrid<R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_degrid<R, G><<<grid, kThreads, smem, s>>>(g, coef, ix, planes, b0, nb, bs, partial, nvis_idx);
  return cudaGetLastError();
}

template <typename R, int G>
static cudaError_t grid_owner_g(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                                const typename C2<R>::T* vis, const R* wgt,
                                typename C2<R>::T* planes, int b0, int nb, cudaStream_t s) {
  // accumulator rows padded by two cells: rows of a clipped footprint start on different
  // banks, and the 2 x T padding cells of a plane give each lane of its owner warp a private
  // cell for idle updates
  const int pitch = g.tile + 2;
  const size_t per = (size_t)g.tile * pitch * sizeof(typename C2<R>::T);
  const size_t stage = (sizeof(R) == 8 && g.df64_planes) ? sizeof(GridStageDD<G>) : sizeof(GridStage<R, G>);
  const size_t fixed = coef_bytes<R>() + stage;
  const int nwarps = kOwnerWarps;
  int bs = (int)std::max<size_t>(1, (kGridSmemBudget - fixed) / per);
  if (bs > nwarps) bs -= bs % nwarps;  // equal planes per warp
  bs = std::min(bs, nb);
  size_t smem = fixed + (size_t)bs * per;
  int64_t ntiles = (int64_t)g.ntu * g.ntv;
  dim3 grid((unsigned)ntiles, (unsigned)((nb + bs - 1) / bs));
  if constexpr (sizeof(R) == 8) {
    if (g.df64_planes) {
      cudaError_t e = cudaFuncSetAttribute(k_grid_owner_dd<G>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_grid_owner_dd<G><<<grid, kOwnerThreads, smem, s>>>(g, coef, ix, vis, planes, b0, nb, bs, pitch);
      return cudaGetLastError();
    }
  }
  cudaError_t e = cudaFuncSetAttribute(k_grid_owner<R, G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_grid_owner<R, G><<<grid, kOwnerThreads, smem, s>>>(g, coef, ix, vis, wgt, planes, b0, nb, bs, pitch);
  return cudaGetLastError();
}

template <typename R, int G>
static cudaError_t grid_atomic_g(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                                 const typename C2<R>::T* vis, const R* wgt,
                                 typename C2<R>::T* planes, int b0, int nb, cudaStream_t s) {
  // row pitch = G (mod 32) words: the 32 lanes of an atomic add (G columns x 32 / G rows)
  // fall in 32 different banks
  int pitch = g.tile;
  while (pitch % 32 != G % 32) ++pitch;
  const size_t per = (size_t)g.tile * pitch * sizeof(typename C2<R>::T);
  int bs = (int)std::max<size_t>(1, (kGridAtomicSmemBudget - coef_bytes<R>()) / per);
  bs = std::min(bs, nb);
  size_t smem = coef_bytes<R>() + (size_t)bs * per;
  cudaError_t e = cudaFuncSetAttribute(k_grid_atomic<R, G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t ntiles = (int64_t)g.ntu * g.ntv;
  dim3 grid((unsigned)ntiles, (unsigned)((nb + bs - 1) / bs));
  k_grid_atomic<R, G><<<grid, kThreads, smem, s>>>(g, coef, ix, vis, wgt, planes, b0, nb, bs, pitch);
  return cudaGetLastError();
}

static cudaError_t grid_band(const Geom& g, const Coef<float>& coef, const IndexView<float>& ix,
                             const float2* vis, const float* wgt, float2* planes, int b0, int nb,
                             cudaStream_t s) {
  const int bs = std::min(kBandPlanes, nb);
  const size_t smem = coef_bytes<float>() + sizeof(BandStage) +
                      (size_t)bs * kBandTile * kBandPitch * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_grid_band, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int64_t ntiles = (int64_t)g.ntu * g.ntv;
  dim3 grid((unsigned)ntiles, (unsigned)((nb + bs - 1) / bs));
  k_grid_band<<<grid, 256, smem, s>>>(g, coef, ix, vis, wgt, planes, b0, nb, bs);
  return cudaGetLastError();
}

// the gridding variant a plan uses (Geom::grid_variant 0 = automatic).  Automatic FP32 takes the
// shared-memory atomics: on the 1e8-visibility workload the row-band owners measured 289 ms
// against 171 ms (ncu on 1.6e6 visibilities: 37 % fewer instructions, but barrier- and
// latency-bound at 16 warps per SM, issue active 26 % against 74 %)
template <typename R>
static int grid_variant_of(const Geom& g) {
  // double-float planes are written by the plane-owner kernel only
  if (g.df64_planes) return 2;
  const bool band_ok = sizeof(R) == 4 && g.alpha <= 8 && g.tile == kBandTile;
  if (g.grid_variant == 3) return band_ok ? 3 : 1;
  if (g.grid_variant != 0) return g.grid_variant;
  return sizeof(R) == 8 ? 2 : 1;
}

template <typename R, int G>
static cudaError_t grid_g(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                          const typename C2<R>::T* vis, const R* wgt,
                          typename C2<R>::T* planes, int b0, int nb, cudaStream_t s) {
  const int variant = grid_variant_of<R>(g);
  if (variant == 2) return grid_owner_g<R, G>(g, coef, ix, vis, wgt, planes, b0, nb, s);
  if constexpr (sizeof(R) == 4 && G <= 8) {
    if (variant == 3)
      return grid_band(g, coef, ix, (const float2*)vis, (const float*)wgt, (float2*)planes, b0,
                       nb, s);
  }
  return grid_atomic_g<R, G>(g, coef, ix, vis, wgt, planes, b0, nb, s);
}

template <typename R>
cudaError_t launch_degrid(const Geom& g, const Coef<R>& coef, const IndexView<R>& ix,
                          const typename C2<R>::T* planes, int b0, int nb, int bs,
                          typename C2<R>::T* partial, int64_t nvis_idx, cudaStream_t s) {
  if (g.alpha <= 4) return degrid_g<R, 4>(g, coef, ix, planes, b0, nb, bs, partial, nvis_idx, s);
  if (g.alpha <= 8) return degrid_g<R, 8>(g, coef, ix, planes, b0, nb, bs, partial, nvis_idx, s);
  return degrid_g<R, 16>(g, coef, ix, planes, b0, nb, bs, partial, nvis_idx, s);
}

template <typename R>
cudaError_t launch_degrid_finalize(const Geom& g, const IndexView<R>& ix,
                                   const typename C2<R>::T* partial, int64_t nvis_idx, int bs,
                                   const R* wgt, typename C2<R>::T* vis, cudaStream_t s) {
  if (nvis_idx == 0) return cudaSuccess;
  k_degrid_finalize<R><<<(unsigned)((nvis_idx + 255) / 256), 256, 0, s>>>(g, ix, partial, nvis_idx,
                                                                          bs, wgt, vis);
  return cudaGetLastError();
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
                                          const float2*, int, int, int, float2*, int64_t,
                                          cudaStream_t);
template cudaError_t launch_degrid<double>(const Geom&, const Coef<double>&,
                                           const IndexView<double>&, const double2*, int, int, int,
                                           double2*, int64_t, cudaStream_t);
template cudaError_t launch_degrid_finalize<float>(const Geom&, const IndexView<float>&,
                                                   const float2*, int64_t, int, const float*,
                                                   float2*, cudaStream_t);
template cudaError_t launch_degrid_finalize<double>(const Geom&, const IndexView<double>&,
                                                    const double2*, int64_t, int, const double*,
                                                    double2*, cudaStream_t);
template int degrid_subbatch<float>(const Geom&);
template int degrid_subbatch<double>(const Geom&);
template cudaError_t launch_grid<float>(const Geom&, const Coef<float>&, const IndexView<float>&,
                                        const float2*, const float*, float2*, int, int,
                                        cudaStream_t);
template cudaError_t launch_grid<double>(const Geom&, const Coef<double>&,
                                         const IndexView<double>&, const double2*,
                                         const double*, double2*, int, int, cudaStream_t);

}  // namespace wg
