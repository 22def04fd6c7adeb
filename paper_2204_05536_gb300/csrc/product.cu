// The HODLR2D product (Alg. 2) over one factor layout, in four arithmetic
// policies: binary64 (F64A), float-float (DF32A), binary32 (F32A) and
// binary32 sums over bfloat16 factors (BF16A).
//
// Far field.  The plan gives every level up to three forms; each product
// picks one per level from the mode and the number of right-hand sides
// (two_pass_end, box_as_pairs):
//   two-pass: a projection pass t = V^T x over row chunks, a fixed-order sum
//     of the chunk partials (k_tsum2; k_tsum64 for few chunks in binary64),
//     and an expansion pass y_X += U t per row box into the level's slab
//     (k_exp2).  The projection kernel depends on the arithmetic: k_proj2
//     (one warp per column), k_proj64 (binary64: column groups, one halving
//     exchange), k_projm (binary32, many right-hand sides), and for bfloat16
//     with several right-hand sides the tcgen05 tensor-core kernels
//     k_projg_t5 (tasks sharing a box stacked into one GEMM) and k_exp_t5;
//   pairs: one block, warp or sub-warp per stored pair (X,Y) computes
//     t1 = V^T x_Y, t2 = U^T x_X and writes the partial results U t1 (rows
//     of X) and V t2 (rows of Y).  The pairs of a level are split into size
//     classes, one launch each: k_pairs / k_pairg (one right-hand side) and
//     k_pairm (several) keep each thread's rows of U and V in registers
//     between the two uses, so each factor value is read once (in
//     float-float the small forms stage the next column group through
//     shared memory with cp.async); in binary64, k_pair (one warp per
//     column, the pair read twice) and k_pair64 (boxes of <= 128 points: one
//     warp per pair, lane-owned dot products from shared memory);
//   box (binary64, boxes of <= kBoxRows points): one warp per row box, the
//     box's pairs staged in shared memory; own sums to the slab, partials for
//     the column side.
// Near field: every leaf against itself and its edge sharers in work items of
// at most 32 targets, entries evaluated from the points (k_near_warp;
// k_near64 in binary64).  The combine pass adds the near field, the slabs
// and the partials of each point in a fixed order.  No atomics anywhere: a
// product is bitwise reproducible.
#include <algorithm>
#include <type_traits>
#include <array>
#include <vector>

#include "arith.cuh"
#include "internal.h"
#include "tc5.cuh"

namespace h2d {

#ifndef H2D_FUSE_ROWS
#define H2D_FUSE_ROWS 2048
#endif
#ifndef H2D_BOX_STAGE
#define H2D_BOX_STAGE 960
#endif
constexpr int kFuseRows = H2D_FUSE_ROWS;  // largest box handled by the single-read kernels
constexpr int kSmallPair = 256;   // boxes up to this size: 64-thread pair blocks
constexpr int kChunk2 = 256;      // rows of one expansion task of the two-pass levels
constexpr int kExpMaxEnt = 64;    // largest list of a box (15 pairs, two sides, margin)
constexpr int kExpQ = 64;         // t columns staged at a time (several right-hand sides)
constexpr int kChunkP = 512;      // rows of one projection task (16 per lane)
// Two-pass levels whose boxes hold at most kDualRows points (with ranks of
// at most kDualKmax and at least two pairs per SM) also get a pair plan; products with one
// right-hand side (not binary64) run them as pairs (each factor value read
// once) instead of in two passes.
constexpr int kDualRows = 512 * 9;
constexpr int kDualKmax = 64;
// With several right-hand sides, boxes of more than kMultiRows points run in
// two passes (each factor value read twice for all of them); smaller ones run
// with the multi-RHS register pair kernel.
constexpr int kMultiRows = 256;
// With few right-hand sides (binary32 sums: 2-8, bfloat16 factors: 2-4),
// pairs of boxes up to kMultiRowsFew points run as pairs too (one 256-thread
// block each), and bfloat16 stays off the tensor cores.  Measured at N = 2^20
// against two passes above 256 points: binary32 2/4/8 RHS 7.62/8.85/11.83 ->
// 7.56/8.56/11.03 ms, bfloat16 2/4 RHS 11.35/11.57 -> 9.65/10.62 ms;
// float-float and bfloat16 with 8 RHS were slower this way.
constexpr int kFewRhs = 8;
constexpr int kMultiRowsFew = 1024;
__host__ __device__ constexpr bool few_rhs(int nrhs, int mode) {
  return nrhs > 1 && ((mode == HODLR2D_MODE_F32 && nrhs <= kFewRhs) ||
                      (mode == HODLR2D_MODE_BF16 && nrhs <= 4));
}

struct LevelV2 {
  const int32_t* px;
  const int32_t* py;
  const int32_t* rank;
  const int64_t* foff;
  const int64_t* prow;
  const int64_t* ppoff;
  const int64_t* toff;
  const int32_t* ent_off;
  const int32_t* ent;
  const void* fac;
  const PairMeta* meta;
  const int64_t* entpp;  // per entry: partial offset << 1 | side
};

enum { LMODE_TWO = 0, LMODE_PAIR = 1, LMODE_BOX = 2 };

struct ArgsV2 {
  LevelV2 lev[HODLR2D_MAX_LEVELS];
  int lmode[HODLR2D_MAX_LEVELS];
  const int32_t* leaf_off;
  int kappa;
  int lfuse;
  int64_t n;
  int nrhs;
  int64_t pstride;  // partial values per right-hand side
};

__device__ __forceinline__ int32_t bstart(const int32_t* leaf_off, int kappa, int l, uint32_t b) {
  return leaf_off[(int64_t)b << (2 * (kappa - l))];
}
__device__ __forceinline__ int32_t bsize(const int32_t* leaf_off, int kappa, int l, uint32_t b) {
  const int sh = 2 * (kappa - l);
  return leaf_off[(int64_t)(b + 1) << sh] - leaf_off[(int64_t)b << sh];
}

__device__ __forceinline__ double shfl_val(double v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ float shfl_val(float v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ float2 shfl_val(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ double shfl_idx(double v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ float shfl_idx(float v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ float2 shfl_idx(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// ---------------------------------------------------------------------------
// gather x into tree order
// ---------------------------------------------------------------------------
// The kernels of the two-pass product are written as device bodies with an
// explicit work index (a point, a warp's item or a block's task) under thin
// kernel wrappers, so that the persistent batch kernel (k_batch) runs the
// same code.
template <class A>
__device__ __forceinline__ void gather2_body(const double* __restrict__ x,
                                             const int64_t* __restrict__ perm, int64_t n,
                                             int nrhs, typename A::val* __restrict__ xt,
                                             int64_t i) {
  if (i >= n) return;
  const int64_t g = perm[i];
  for (int c = 0; c < nrhs; ++c) xt[i + c * n] = A::from_double(x[g + c * n]);
}
template <class A>
__global__ void k_gather2(const double* __restrict__ x, const int64_t* __restrict__ perm,
                          int64_t n, int nrhs, typename A::val* __restrict__ xt) {
  gather2_body<A>(x, perm, n, nrhs, xt, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// near field, every mode: one warp per work item (a leaf, at most 32 of its
// targets; point, entry and sum types come from the policy).  With
// G = 32 / (targets per round) lanes per target (G = 4 for <= 8 points, 2 for
// <= 16, else 1), lane group h takes the sources s = h (mod G) of the
// concatenated source list (the leaf itself, then its edge sharers in
// ascending Morton order); the G partial sums meet in a fixed shuffle tree.
// ---------------------------------------------------------------------------
constexpr int kNearWarps = 4;

// kMinBlocks: resident blocks per SM the near kernel asks the compiler for
struct NearDF32 {  // float-float points, entries and sums
  static constexpr int kMinBlocks = 10;
  typedef float2 pt;
  typedef KernelFF K;
  typedef DF32A A;
  static __device__ __forceinline__ float2 entry(const K& k, pt xi, pt yi, int64_t gi, pt xj,
                                                 pt yj, int64_t gj) {
    return entry_ff(k, xi, yi, gi, xj, yj, gj);
  }
};
struct NearF32 {  // binary32 points, entries and sums (mixed form)
  static constexpr int kMinBlocks = 10;
  typedef float pt;
  typedef KernelF32 K;
  typedef F32A A;
  static __device__ __forceinline__ float entry(const K& k, pt xi, pt yi, int64_t gi, pt xj,
                                                pt yj, int64_t gj) {
    return entry_f32(k, xi, yi, gi, xj, yj, gj);
  }
};
struct NearF64 {  // binary64 points, entries and sums (bound by the binary64 pipe, not occupancy)
  static constexpr int kMinBlocks = 4;
  typedef double pt;
  typedef KernelParams K;
  typedef F64A A;
  static __device__ __forceinline__ double entry(const K& k, pt xi, pt yi, int64_t gi, pt xj,
                                                 pt yj, int64_t gj) {
    return h2d::entry(k, xi, yi, gi, xj, yj, gj);
  }
};

// NRH right-hand sides per pass (each entry evaluated once per pass).  At
// least NP::kMinBlocks blocks per SM: 10 (40 warps) for the float-float and
// binary32 entry chains, which need the occupancy more than registers
// (measured 0.85 -> 0.68 ms at N = 2^20).
template <class NP, int NRH>
__device__ __forceinline__ void near_warp_body(
    const typename NP::pt* __restrict__ xf, const typename NP::pt* __restrict__ yf,
    const int32_t* __restrict__ leaf_off, int kappa, const int2* __restrict__ work, int64_t nwork,
    const typename NP::K& kp, const typename NP::A::val* __restrict__ xt, int64_t n, int nrhs,
    typename NP::A::val* __restrict__ yout, int64_t wi) {
  using A = typename NP::A;
  using Val = typename A::val;
  using Pt = typename NP::pt;
  const int lane = threadIdx.x & 31;
  if (wi >= nwork) return;
  // work item: (leaf, first target); a leaf of more than 32 points is split
  // into items of 32 targets, each against all of the leaf's sources
  const int2 wk = work[wi];
  const uint32_t b = (uint32_t)wk.x;
  const int32_t s0 = leaf_off[b] + wk.y;
  const int32_t m = min(leaf_off[b + 1] - s0, 32);
  if (m <= 0) return;
  int cx, cy;
  morton_decode(b, cx, cy);
  const int side = 1 << kappa;
  int32_t sb[5], se[5];
  int ns = 0;
  sb[0] = leaf_off[b];
  se[0] = leaf_off[b + 1];
  ns = 1;
  uint32_t nb[4];
  int nn = 0;
  const int dx[4] = {-1, 1, 0, 0}, dy[4] = {0, 0, -1, 1};
  for (int e = 0; e < 4; ++e) {
    const int qx = cx + dx[e], qy = cy + dy[e];
    if (qx < 0 || qy < 0 || qx >= side || qy >= side) continue;
    nb[nn++] = morton_encode((uint32_t)qx, (uint32_t)qy);
  }
  for (int i = 1; i < nn; ++i) {
    const uint32_t v = nb[i];
    int j = i - 1;
    while (j >= 0 && nb[j] > v) { nb[j + 1] = nb[j]; --j; }
    nb[j + 1] = v;
  }
  for (int i = 0; i < nn; ++i) {
    sb[ns] = leaf_off[nb[i]];
    se[ns] = leaf_off[nb[i] + 1];
    ++ns;
  }
  const int G = m <= 8 ? 4 : (m <= 16 ? 2 : 1);
  const int tpr = 32 / G;
  const int h = lane / tpr, tl = lane - h * tpr;
  for (int t0 = 0; t0 < m; t0 += tpr) {
    const int t = t0 + tl;
    const bool act = t < m;
    const int64_t it = s0 + (act ? t : 0);
    const Pt xi = xf[it], yi = yf[it];
    for (int c0 = 0; c0 < nrhs; c0 += NRH) {
      const int nc = min(NRH, nrhs - c0);
      typename A::acc acc[NRH];
#pragma unroll
      for (int r = 0; r < NRH; ++r) acc[r] = A::zero();
      int sidx = 0;  // running index over the concatenated sources
      for (int q = 0; q < ns; ++q) {
        const int32_t len = se[q] - sb[q];
        // first source of this box whose running index is = h (mod G)
        int j = (h - sidx) % G;
        if (j < 0) j += G;
        // the diagonal is found by tree position, a bijection of the
        // original index
        for (int cnt = 1; j < len; j += G, ++cnt) {
          const int64_t js = sb[q] + j;
          const Val kij = NP::entry(kp, xi, yi, it, xf[js], yf[js], js);
#pragma unroll
          for (int r = 0; r < NRH; ++r)
            if (r < nc) A::fma(acc[r], kij, xt[(int64_t)(c0 + r) * n + js]);
          if (cnt % kRenorm == 0)
#pragma unroll
            for (int r = 0; r < NRH; ++r) A::renorm(acc[r]);
        }
        sidx += len;
      }
      Val res[NRH];
#pragma unroll
      for (int r = 0; r < NRH; ++r) {
        Val v = A::fin(acc[r]);
        for (int o = tpr; o < 32; o <<= 1) v = A::add(v, shfl_val(v, o));
        res[r] = v;
      }
      if (act && h == 0)
        for (int r = 0; r < nc; ++r) yout[(int64_t)(c0 + r) * n + it] = res[r];
    }
  }
}
template <class NP, int NRH>
__global__ void __launch_bounds__(32 * kNearWarps, NP::kMinBlocks)
    k_near_warp(const typename NP::pt* __restrict__ xf, const typename NP::pt* __restrict__ yf,
                const int32_t* __restrict__ leaf_off, int kappa, const int2* __restrict__ work,
                int64_t nwork, typename NP::K kp, const typename NP::A::val* __restrict__ xt,
                int64_t n, int nrhs, typename NP::A::val* __restrict__ yout) {
  near_warp_body<NP, NRH>(xf, yf, leaf_off, kappa, work, nwork, kp, xt, n, nrhs, yout,
                          (int64_t)blockIdx.x * kNearWarps + (threadIdx.x >> 5));
}

// ---------------------------------------------------------------------------
// near field in binary64: one warp per work item (a leaf, at most 32 of its
// targets).  A binary64 warp instruction costs the same whatever its active
// lanes, so the targets are spread over all lanes: with m targets the item
// runs m G units (target i, slice g), G in [1, 8] chosen for the fewest idle
// lanes over at most two passes, and unit (i, g) sums the sources whose
// index in the concatenated source list (the leaf, then its edge sharers in
// ascending Morton order) is g mod G.  Sources are staged in shared memory
// kNearChunk at a time (coordinates and x), so the lanes of one slice read
// the same source (a broadcast).  The G partials of a target are added in
// slice order.  The multiquadric and inverse multiquadric form r^2 + a^2 as
// dx dx + (dy dy + a^2) with two fused multiply-adds.
// ---------------------------------------------------------------------------
constexpr int kNear64Warps = 4;
constexpr int kNearChunk = 128;

__device__ __forceinline__ double near64_entry(const KernelParams& k, double dx, double dy) {
  if (k.kind == HODLR2D_MQ) return sqrt(fma(dx, dx, fma(dy, dy, k.a2)));
  if (k.kind == HODLR2D_IMQ) return 1.0 / sqrt(fma(dx, dx, fma(dy, dy, k.a2)));
  return phi_r2(k, dx * dx + dy * dy);
}

template <int NRH>
__global__ void __launch_bounds__(32 * kNear64Warps)
    k_near64(const double* __restrict__ xf, const double* __restrict__ yf,
             const int32_t* __restrict__ leaf_off, int kappa, const int2* __restrict__ work,
             int64_t nwork, KernelParams kp, const double* __restrict__ xt, int64_t n, int nrhs,
             double* __restrict__ yout) {
  __shared__ double s_x[kNear64Warps][kNearChunk], s_y[kNear64Warps][kNearChunk];
  __shared__ double s_v[kNear64Warps][NRH][kNearChunk];
  __shared__ double s_p[kNear64Warps][NRH][64];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t wi = (int64_t)blockIdx.x * kNear64Warps + w;
  if (wi >= nwork) return;
  const int2 wk = work[wi];
  const uint32_t b = (uint32_t)wk.x;
  const int32_t s0 = leaf_off[b] + wk.y;
  const int m = min(leaf_off[b + 1] - s0, 32);
  if (m <= 0) return;
  int cx, cy;
  morton_decode(b, cx, cy);
  const int side = 1 << kappa;
  int32_t sb[5], se[5];
  sb[0] = leaf_off[b];
  se[0] = leaf_off[b + 1];
  int ns = 1;
  uint32_t nb[4];
  int nn = 0;
  const int dxs[4] = {-1, 1, 0, 0}, dys[4] = {0, 0, -1, 1};
  for (int e = 0; e < 4; ++e) {
    const int qx = cx + dxs[e], qy = cy + dys[e];
    if (qx < 0 || qy < 0 || qx >= side || qy >= side) continue;
    nb[nn++] = morton_encode((uint32_t)qx, (uint32_t)qy);
  }
  for (int i = 1; i < nn; ++i) {
    const uint32_t v = nb[i];
    int j = i - 1;
    while (j >= 0 && nb[j] > v) { nb[j + 1] = nb[j]; --j; }
    nb[j + 1] = v;
  }
  for (int i = 0; i < nn; ++i) {
    sb[ns] = leaf_off[nb[i]];
    se[ns] = leaf_off[nb[i] + 1];
    ++ns;
  }
  int total = 0;
  for (int q = 0; q < ns; ++q) total += se[q] - sb[q];
  // slices: the fewest idle lanes over at most 64 units (two passes)
  int G = 1, bu = m, bp = (m + 31) / 32;
  for (int g = 2; g <= 8 && m * g <= 64; ++g) {
    const int u = m * g, pss = (u + 31) / 32;
    if ((int64_t)u * bp > (int64_t)bu * pss) {
      G = g;
      bu = u;
      bp = pss;
    }
  }
  const int units = m * G;
  int ui[2], ug[2];
  double xi[2], yi[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int u = lane + 32 * p;
    ui[p] = u < units ? u % m : 0;
    ug[p] = u < units ? u / m : 0;
    xi[p] = xf[s0 + ui[p]];
    yi[p] = yf[s0 + ui[p]];
  }
  double* sx = s_x[w];
  double* sy = s_y[w];
  for (int c0 = 0; c0 < nrhs; c0 += NRH) {
    const int nc = min(NRH, nrhs - c0);
    double acc[2][NRH];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int r = 0; r < NRH; ++r) acc[p][r] = 0.0;
    for (int base = 0; base < total; base += kNearChunk) {
      const int cnt = min(kNearChunk, total - base);
      for (int sl = lane; sl < cnt; sl += 32) {  // source base + sl -> tree position
        int gsrc = base + sl, q = 0;
        while (gsrc >= se[q] - sb[q]) {
          gsrc -= se[q] - sb[q];
          ++q;
        }
        const int64_t pos = sb[q] + gsrc;
        sx[sl] = xf[pos];
        sy[sl] = yf[pos];
#pragma unroll
        for (int r = 0; r < NRH; ++r)
          if (r < nc) s_v[w][r][sl] = xt[(int64_t)(c0 + r) * n + pos];
      }
      __syncwarp();
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        if (lane + 32 * p >= units) continue;
        const int g = ug[p];
        const int diag = wk.y + ui[p] - base;  // the target's own index in this chunk
        int sl = (g - base % G + G) % G;
        for (; sl < cnt; sl += G) {
          const double e =
              sl == diag ? kp.diag : near64_entry(kp, xi[p] - sx[sl], yi[p] - sy[sl]);
#pragma unroll
          for (int r = 0; r < NRH; ++r)
            if (r < nc) acc[p][r] = fma(e, s_v[w][r][sl], acc[p][r]);
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int p = 0; p < 2; ++p)
      if (lane + 32 * p < units)
#pragma unroll
        for (int r = 0; r < NRH; ++r) s_p[w][r][lane + 32 * p] = acc[p][r];
    __syncwarp();
    if (lane < m)
      for (int r = 0; r < nc; ++r) {
        double y = s_p[w][r][lane];
        for (int g = 1; g < G; ++g) y += s_p[w][r][lane + m * g];
        yout[(int64_t)(c0 + r) * n + s0 + lane] = y;
      }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// pair mode (mid levels): one block per stored pair (X,Y).  Phase 1: one warp
// per column computes t1 = V^T x_Y and t2 = U^T x_X (rows over lanes, shuffle
// sum).  Phase 2: one thread per row writes U t1 (rows of X) and V t2 (rows of
// Y) as partial results.  Phase 2 re-reads U and V: from L2 when the pairs in
// flight fit it (small boxes), else from HBM.
// ---------------------------------------------------------------------------
constexpr int kPairKmax = 256;

template <class A, int T>
__global__ void __launch_bounds__(T)
    k_pair(ArgsV2 P, const int2* __restrict__ work, const typename A::val* __restrict__ xt,
           typename A::val* __restrict__ ppart) {
  using V = typename A::val;
  using Acc = typename A::acc;
  __shared__ V ts[2 * kPairKmax];
  constexpr int NW = T / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int2 wk = work[blockIdx.x];
  const int l = wk.x;
  const int64_t p = wk.y;
  const LevelV2& L = P.lev[l];
  const PairMeta PM = L.meta[p];
  const int32_t xs = PM.xs, m = PM.m, ys = PM.ys, n = PM.n;
  const int64_t lm = ldpad(m), ln = ldpad(n);
  const int k = PM.k;
  using F = typename A::fac;
  const F* Ug = reinterpret_cast<const F*>(L.fac) + PM.foff;
  const F* Vg = Ug + lm * k;
  for (int c = 0; c < P.nrhs; ++c) {
    const V* xc = xt + (int64_t)c * P.n;
    for (int job = warp; job < 2 * k; job += NW) {
      const bool isV = job < k;
      const int q = isV ? job : job - k;
      const int rows = isV ? n : m;
      const F* col = (isV ? Vg + q * ln : Ug + q * lm);
      const V* xv = xc + (isV ? ys : xs);
      Acc a = A::zero();
      int r = lane;
      for (; r + 224 < rows; r += 256) {  // eight loads of each kind in flight
        F v[8];
        V xx[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          v[u] = col[r + 32 * u];
          xx[u] = xv[r + 32 * u];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) A::fma(a, A::ld(v[u]), xx[u]);
      }
      for (; r + 96 < rows; r += 128) {
        const F v0 = col[r], v1 = col[r + 32], v2 = col[r + 64], v3 = col[r + 96];
        const V x0 = xv[r], x1 = xv[r + 32], x2 = xv[r + 64], x3 = xv[r + 96];
        A::fma(a, A::ld(v0), x0);
        A::fma(a, A::ld(v1), x1);
        A::fma(a, A::ld(v2), x2);
        A::fma(a, A::ld(v3), x3);
      }
      for (; r < rows; r += 32) A::fma(a, A::ld(col[r]), xv[r]);
      const V sum = A::warp_sum(a);
      if (lane == 0) ts[job] = sum;
    }
    __syncthreads();
    V* outx = ppart + (int64_t)c * P.pstride + PM.ppx;
    V* outy = ppart + (int64_t)c * P.pstride + PM.ppy;
    for (int r = tid; r < m + n; r += T) {
      const bool own = r < m;
      const int i = own ? r : r - m;
      const F* M = own ? Ug + i : Vg + i;
      const int64_t ld = own ? lm : ln;
      const V* tv = own ? ts : ts + k;  // U pairs with t1, V with t2
      Acc a = A::zero();
      int q = 0;
      for (; q + 8 <= k; q += 8) {
        F mv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) mv[u] = M[(q + u) * ld];
#pragma unroll
        for (int u = 0; u < 8; ++u) A::fma(a, A::ld(mv[u]), tv[q + u]);
        if ((q + 8) % kRenorm == 0) A::renorm(a);
      }
      for (; q < k; ++q) A::fma(a, A::ld(M[q * ld]), tv[q]);
      (own ? outx : outy)[i] = A::fin(a);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// register pair mode: one block of T threads per stored pair (X,Y), one
// right-hand side.  Thread t owns rows t, t + T, ... (at most RM) of X and of
// Y and keeps x, and the partial results y, of those rows in registers.  The
// columns are visited in groups of G: the group's values of U and V are
// loaded once into registers, the block sums
//   t1_q = sum over Y rows of V(r,q) x(r),   t2_q = sum over X rows of U(r,q) x(r)
// are formed (below), and the same registers are then used for y_X += U t1
// and y_Y += V t2.  Every factor value is read from HBM exactly once.
//
// The 2G sums of a warp are reduced by halving exchanges: at each of the
// first log2(2G) steps a lane keeps half of its values and adds the other
// half received from its partner, so that after them lane L holds one
// column's partial (column L >> (5 - log2 2G)); the remaining steps are plain
// butterflies.  Warps then combine through shared memory in warp order.
// ---------------------------------------------------------------------------
template <class F>
__device__ __forceinline__ F fac_zero();
template <>
__device__ __forceinline__ double fac_zero<double>() { return 0.0; }
template <>
__device__ __forceinline__ float fac_zero<float>() { return 0.f; }
template <>
__device__ __forceinline__ float2 fac_zero<float2>() { return make_float2(0.f, 0.f); }
template <>
__device__ __forceinline__ __nv_bfloat16 fac_zero<__nv_bfloat16>() {
  return __float2bfloat16_rn(0.f);
}

__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

// asynchronous global -> shared copies (cp.async): 16 bytes bypassing L1, or
// 4 / 8 bytes through L1; each thread waits for its own groups
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
template <int B>
__device__ __forceinline__ void cp_async_small(void* dst, const void* src) {
  static_assert(B == 4 || B == 8, "cp.async.ca copies 4 or 8 bytes here");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "n"(B)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// v[NV] per lane -> the total over the W-lane group (W a power of two, W >=
// NV) of column ((lane % W) >> (log2 W - log2 NV)), returned
template <class A, int NV, int W = 32>
__device__ __forceinline__ typename A::val warp_reduce_scatter(typename A::val (&v)[NV],
                                                               int lane) {
  using V = typename A::val;
  constexpr int LG = ilog2c(NV);
  static_assert(NV <= W, "one value per lane at least");
#pragma unroll
  for (int st = 0; st < LG; ++st) {
    const int o = (W / 2) >> st;
    const int M = NV >> st;  // values still held
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < M / 2; ++j) {
      const V mine = up ? v[j + M / 2] : v[j];
      const V other = up ? v[j] : v[j + M / 2];
      v[j] = A::add(mine, shfl_val(other, o));
    }
  }
  V r = v[0];
#pragma unroll
  for (int o = (W / 2) >> LG; o > 0; o >>= 1) r = A::add(r, shfl_val(r, o));
  return r;
}

// A step's factor column values held as loaded (CVT false: converted at each
// use) or converted to the arithmetic type at load (CVT true).
template <class A, bool CVT>
struct ColType {
  using type = typename std::conditional<CVT, typename A::val, typename A::fac>::type;
  static __device__ __forceinline__ type load(typename A::fac f) {
    if constexpr (CVT) return A::ld(f);
    else return f;
  }
  static __device__ __forceinline__ typename A::val use(type x) {
    if constexpr (CVT) return x;
    else return A::ld(x);
  }
};

// k_pairg stages its factor loads through shared memory for float-float
// factors in blocks of at most 128 threads (measured: these gain, the larger
// blocks and the binary32 forms lose occupancy for nothing); bytes of dynamic
// shared memory:
template <class A, int T>
__host__ __device__ constexpr bool pairg_async() {
  return sizeof(typename A::fac) == 8 && sizeof(typename A::acc) == 8 && T <= 128;
}
constexpr int kPairgStages = 2;  // column groups in flight: kPairgStages - 1 (3 measured slower)
template <class A, int T, int RM, int G>
__host__ __device__ constexpr int pairg_smem() {
  return pairg_async<A, T>() ? kPairgStages * 2 * RM * G * T * (int)sizeof(typename A::fac) : 0;
}

template <class A, int T, int RM, int G>
__global__ void __launch_bounds__(T)
    k_pairg(ArgsV2 P, const int2* __restrict__ work, const typename A::val* __restrict__ xt,
            typename A::val* __restrict__ ppart) {
  using V = typename A::val;
  using F = typename A::fac;
  using Acc = typename A::acc;
  constexpr int NW = T / 32;
  constexpr int NV = 2 * G;              // sums per group (power of two)
  constexpr int SH = 5 - ilog2c(NV);     // lane >> SH = column held after the scatter
  __shared__ V red[2][NW > 1 ? NW : 1][NV];
  __shared__ V tot[2][NV];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int2 wk = work[blockIdx.x];
  const LevelV2& L = P.lev[wk.x];
  const PairMeta PM = L.meta[wk.y];
  const int m = PM.m, n = PM.n, k = PM.k;
  const int64_t lm = ldpad(m), ln = ldpad(n);
  const F* Ug = reinterpret_cast<const F*>(L.fac) + PM.foff;
  const F* Vg = Ug + lm * k;
  const int mn = max(m, n);
  V xX[RM], xY[RM];
  Acc yX[RM], yY[RM];
#pragma unroll
  for (int a = 0; a < RM; ++a) {
    const int i = tid + a * T;
    xX[a] = i < m ? xt[PM.xs + i] : A::vzero();
    xY[a] = i < n ? xt[PM.ys + i] : A::vzero();
    yX[a] = A::zero();
    yY[a] = A::zero();
  }
  // staged forms: the next column groups are copied to this thread's
  // shared-memory slots (kPairgStages stages) while the current one is
  // computed; every step commits one copy group (empty past the last column)
  constexpr bool kAsync = pairg_async<A, T>();
  extern __shared__ __align__(16) unsigned char pairg_smem[];
  F* const stage = reinterpret_cast<F*>(pairg_smem);  // [stage][u, v][RM][G][T]
  auto slot = [&](int b, int uv, int a, int g) {
    return stage + ((((b * 2 + uv) * RM + a) * G + g) * T + tid);
  };
  auto issue = [&](int q0, int b) {  // columns q0 .. q0 + G - 1 (those < k)
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const bool qok = q0 + g < k;
      const F* uc = Ug + (int64_t)(q0 + g) * lm;
      const F* vc = Vg + (int64_t)(q0 + g) * ln;
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        const int i = tid + a * T;
        if constexpr (kAsync) {
          if (qok && i < m) cp_async_small<sizeof(F)>(slot(b, 0, a, g), uc + i);
          if (qok && i < n) cp_async_small<sizeof(F)>(slot(b, 1, a, g), vc + i);
        }
      }
    }
    cp_async_commit();
  };
  if constexpr (kAsync) {
#pragma unroll
    for (int sidx = 0; sidx < kPairgStages - 1; ++sidx) issue(sidx * G, sidx);
  }
  int par = 0, stb = 0;
  // blocks of 256 and 512 threads convert the step's columns to the
  // arithmetic type once, at load (bfloat16, N = 2^20: their levels 0.95 ->
  // 0.81 ms); the smaller ones, like k_pairs, keep the factor type and
  // convert where used (with both converting at load, the levels of boxes of
  // <= 256 points went 0.25 -> 0.37 ms)
  using CT = ColType<A, (T >= 256)>;
  for (int q0 = 0; q0 < k; q0 += G) {
    typename CT::type u[RM][G], v[RM][G];
    if constexpr (kAsync) {
      // group q0 + (S - 1) G into the slot freed by the previous step
      issue(q0 + (kPairgStages - 1) * G, (stb + kPairgStages - 1) % kPairgStages);
      cp_async_wait<kPairgStages - 1>();  // this step's group has landed
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const bool qok = q0 + g < k;
#pragma unroll
        for (int a = 0; a < RM; ++a) {
          const int i = tid + a * T;
          u[a][g] = CT::load((qok && i < m) ? *slot(stb, 0, a, g) : fac_zero<F>());
          v[a][g] = CT::load((qok && i < n) ? *slot(stb, 1, a, g) : fac_zero<F>());
        }
      }
      stb = (stb + 1) % kPairgStages;
    } else {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const bool qok = q0 + g < k;
        const F* uc = Ug + (int64_t)(q0 + g) * lm;
        const F* vc = Vg + (int64_t)(q0 + g) * ln;
#pragma unroll
        for (int a = 0; a < RM; ++a) {
          const int i = tid + a * T;
          u[a][g] = CT::load((qok && i < m) ? uc[i] : fac_zero<F>());
          v[a][g] = CT::load((qok && i < n) ? vc[i] : fac_zero<F>());
        }
      }
    }
    // s[g] = partial t1_{q0+g} (V), s[G+g] = partial t2_{q0+g} (U)
    V s[NV];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      Acc a1 = A::zero(), a2 = A::zero();
#pragma unroll
      for (int a = 0; a < RM; ++a)  // row groups past the box are skipped (block-uniform)
        if (a * T < mn) {
          A::fma(a1, CT::use(v[a][g]), xY[a]);
          A::fma(a2, CT::use(u[a][g]), xX[a]);
        }
      s[g] = A::fin(a1);
      s[G + g] = A::fin(a2);
    }
    const V mine = warp_reduce_scatter<A, NV>(s, lane);
    V t[NV];
    if (NW == 1) {
#pragma unroll
      for (int c = 0; c < NV; ++c) t[c] = shfl_idx(mine, c << SH);
    } else {
      if ((lane & ((1 << SH) - 1)) == 0) red[par][warp][lane >> SH] = mine;
      __syncthreads();
      if (tid < NV) {
        V acc = red[par][0][tid];
#pragma unroll
        for (int w = 1; w < NW; ++w) acc = A::add(acc, red[par][w][tid]);
        tot[par][tid] = acc;
      }
      __syncthreads();
#pragma unroll
      for (int c = 0; c < NV; ++c) t[c] = tot[par][c];
      par ^= 1;
    }
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int a = 0; a < RM; ++a)
        if (a * T < mn) {
          A::fma(yX[a], CT::use(u[a][g]), t[g]);      // U with t1
          A::fma(yY[a], CT::use(v[a][g]), t[G + g]);  // V with t2
        }
    if ((q0 / G + 1) % (kRenorm / G) == 0)
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        A::renorm(yX[a]);
        A::renorm(yY[a]);
      }
  }
  V* outx = ppart + PM.ppx;
  V* outy = ppart + PM.ppy;
#pragma unroll
  for (int a = 0; a < RM; ++a) {
    const int i = tid + a * T;
    if (i < m) outx[i] = A::fin(yX[a]);
    if (i < n) outy[i] = A::fin(yY[a]);
  }
}

// Several right-hand sides: k_pairg with one column per step and NR
// right-hand sides per pass.  Thread t keeps x and y of its rows (at most RM
// of X and of Y) for the pass's NR right-hand sides in registers; each column
// of U and V is loaded once per pass and used for all of them.  The 2 NR
// sums of a column reduce like k_pairg's.
// (the T threads tid = 0 .. T - 1 of group gid, whole warps, take pair wk
// together.  With T = 32 they are one warp and never synchronise; with NG = 1
// they are the whole block and synchronise it; with NG > 1 groups of one
// block they synchronise on the named barrier B0 + gid, T threads.  A block
// whose groups may drift into the next unit before the others finish must
// give each group size its own barrier ids, so that one id is always used by
// the same warps with the same count.)
template <int T, int NG, int B0>
__device__ __forceinline__ void group_sync(int gid) {
  if constexpr (NG == 1) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(B0 + gid), "r"(T) : "memory");
}
template <class A, int T, int RM, int NR, int NG = 1, int B0 = 1>
__device__ __forceinline__ void pairm_body(const ArgsV2& P, const int2 wk,
                                           const typename A::val* __restrict__ xt,
                                           typename A::val* __restrict__ ppart, const int tid,
                                           const int gid = 0) {
  using V = typename A::val;
  using F = typename A::fac;
  using Acc = typename A::acc;
  constexpr int NW = T / 32;
  constexpr int NV = 2 * NR;
  constexpr int SH = 5 - ilog2c(NV);
  __shared__ V red_all[NG][2][NW > 1 ? NW : 1][NV];
  __shared__ V tot_all[NG][2][NV];
  auto& red = red_all[gid];
  auto& tot = tot_all[gid];
  const int lane = tid & 31, warp = tid >> 5;
  const LevelV2& L = P.lev[wk.x];
  const PairMeta PM = L.meta[wk.y];
  const int m = PM.m, n = PM.n, k = PM.k;
  const int64_t lm = ldpad(m), ln = ldpad(n);
  const F* Ug = reinterpret_cast<const F*>(L.fac) + PM.foff;
  const F* Vg = Ug + lm * k;
  const int mn = max(m, n);
  int par = 0;
  for (int c0 = 0; c0 < P.nrhs; c0 += NR) {
    V xX[RM][NR], xY[RM][NR];
    Acc yX[RM][NR], yY[RM][NR];
#pragma unroll
    for (int a = 0; a < RM; ++a) {
      const int i = tid + a * T;
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        const bool ok = c0 + c < P.nrhs;
        const V* xc = xt + (int64_t)(c0 + c) * P.n;
        xX[a][c] = (ok && i < m) ? xc[PM.xs + i] : A::vzero();
        xY[a][c] = (ok && i < n) ? xc[PM.ys + i] : A::vzero();
        yX[a][c] = A::zero();
        yY[a][c] = A::zero();
      }
    }
    // column q + 1 of U and V is loaded while column q is reduced
    F u[RM], v[RM];
#pragma unroll
    for (int a = 0; a < RM; ++a) {
      const int i = tid + a * T;
      u[a] = i < m && k > 0 ? Ug[i] : fac_zero<F>();
      v[a] = i < n && k > 0 ? Vg[i] : fac_zero<F>();
    }
    for (int q = 0; q < k; ++q) {
      F un[RM], vn[RM];
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        const int i = tid + a * T;
        un[a] = i < m && q + 1 < k ? Ug[(int64_t)(q + 1) * lm + i] : fac_zero<F>();
        vn[a] = i < n && q + 1 < k ? Vg[(int64_t)(q + 1) * ln + i] : fac_zero<F>();
      }
      V uf[RM], vf[RM];  // the column in the arithmetic type, converted once
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        uf[a] = A::ld(u[a]);
        vf[a] = A::ld(v[a]);
      }
      V s[NV];  // s[c] = partial t1 of RHS c (V), s[NR + c] = partial t2 (U)
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        Acc a1 = A::zero(), a2 = A::zero();
#pragma unroll
        for (int a = 0; a < RM; ++a)
          if (a * T < mn) {
            A::fma(a1, vf[a], xY[a][c]);
            A::fma(a2, uf[a], xX[a][c]);
          }
        s[c] = A::fin(a1);
        s[NR + c] = A::fin(a2);
      }
      const V mine = warp_reduce_scatter<A, NV>(s, lane);
      V t[NV];
      if constexpr (NW == 1) {
#pragma unroll
        for (int c = 0; c < NV; ++c) t[c] = shfl_idx(mine, c << SH);
      } else {
        if ((lane & ((1 << SH) - 1)) == 0) red[par][warp][lane >> SH] = mine;
        group_sync<T, NG, B0>(gid);
        if (tid < NV) {
          V acc = red[par][0][tid];
#pragma unroll
          for (int w = 1; w < NW; ++w) acc = A::add(acc, red[par][w][tid]);
          tot[par][tid] = acc;
        }
        group_sync<T, NG, B0>(gid);
#pragma unroll
        for (int c = 0; c < NV; ++c) t[c] = tot[par][c];
        par ^= 1;
      }
#pragma unroll
      for (int c = 0; c < NR; ++c)
#pragma unroll
        for (int a = 0; a < RM; ++a)
          if (a * T < mn) {
            A::fma(yX[a][c], uf[a], t[c]);       // U with t1
            A::fma(yY[a][c], vf[a], t[NR + c]);  // V with t2
          }
      if ((q + 1) % kRenorm == 0)
#pragma unroll
        for (int c = 0; c < NR; ++c)
#pragma unroll
          for (int a = 0; a < RM; ++a) {
            A::renorm(yX[a][c]);
            A::renorm(yY[a][c]);
          }
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        u[a] = un[a];
        v[a] = vn[a];
      }
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      if (c0 + c >= P.nrhs) break;
      V* outx = ppart + (int64_t)(c0 + c) * P.pstride + PM.ppx;
      V* outy = ppart + (int64_t)(c0 + c) * P.pstride + PM.ppy;
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        const int i = tid + a * T;
        if (i < m) outx[i] = A::fin(yX[a][c]);
        if (i < n) outy[i] = A::fin(yY[a][c]);
      }
    }
  }
}
template <class A, int T, int RM, int NR>
__global__ void __launch_bounds__(T)
    k_pairm(ArgsV2 P, const int2* __restrict__ work, const typename A::val* __restrict__ xt,
            typename A::val* __restrict__ ppart) {
  pairm_body<A, T, RM, NR>(P, work[blockIdx.x], xt, ppart, threadIdx.x);
}

// Sub-warp form of k_pairm for small boxes: S lanes per pair
// (S = 8 or 16), 32 / S pairs per warp, the items item0, item0 + 1, ... of
// the work list; lane s of a segment takes rows s, s + S, ... (RM of them)
// of X and of Y.  The column loop runs to the largest rank of the warp's
// pairs (columns beyond a pair's own rank add zeros); the 2 NR sums of a
// column reduce within the segment (reduce-scatter over S lanes) and come
// back from the lanes that hold them.
template <class A, int S, int RM, int NR>
__device__ __forceinline__ void pairms_body(const ArgsV2& P, const int2* __restrict__ work,
                                            int64_t nwork,
                                            const typename A::val* __restrict__ xt,
                                            typename A::val* __restrict__ ppart, int64_t item0) {
  using V = typename A::val;
  using F = typename A::fac;
  using Acc = typename A::acc;
  constexpr int NV = 2 * NR;
  static_assert(NV <= S && S <= 32, "one sum per lane of a segment at least");
  constexpr int SH = ilog2c(S) - ilog2c(NV);
  const int lane = threadIdx.x & 31, g = lane / S, sl = lane % S, sbase = g * S;
  const int64_t it = item0 + g;
  int m = 0, n = 0, k = 0;
  int64_t lm = 0, ln = 0, ppx = 0, ppy = 0;
  int32_t xs = 0, ys = 0;
  const F* Ug = nullptr;
  const F* Vg = nullptr;
  if (it < nwork) {
    const int2 wk = work[it];
    const LevelV2& L = P.lev[wk.x];
    const PairMeta PM = L.meta[wk.y];
    m = PM.m;
    n = PM.n;
    k = PM.k;
    lm = ldpad(m);
    ln = ldpad(n);
    xs = PM.xs;
    ys = PM.ys;
    ppx = PM.ppx;
    ppy = PM.ppy;
    Ug = reinterpret_cast<const F*>(L.fac) + PM.foff;
    Vg = Ug + lm * k;
  }
  int kmax = k;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
  for (int c0 = 0; c0 < P.nrhs; c0 += NR) {
    V xX[RM][NR], xY[RM][NR];
    Acc yX[RM][NR], yY[RM][NR];
#pragma unroll
    for (int a = 0; a < RM; ++a) {
      const int i = sl + a * S;
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        const bool ok = c0 + c < P.nrhs;
        const V* xc = xt + (int64_t)(c0 + c) * P.n;
        xX[a][c] = (ok && i < m) ? xc[xs + i] : A::vzero();
        xY[a][c] = (ok && i < n) ? xc[ys + i] : A::vzero();
        yX[a][c] = A::zero();
        yY[a][c] = A::zero();
      }
    }
    F u[RM], v[RM];  // column q + 1 is loaded while column q is reduced
#pragma unroll
    for (int a = 0; a < RM; ++a) {
      const int i = sl + a * S;
      u[a] = i < m && k > 0 ? Ug[i] : fac_zero<F>();
      v[a] = i < n && k > 0 ? Vg[i] : fac_zero<F>();
    }
    for (int q = 0; q < kmax; ++q) {
      F un[RM], vn[RM];
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        const int i = sl + a * S;
        un[a] = i < m && q + 1 < k ? Ug[(int64_t)(q + 1) * lm + i] : fac_zero<F>();
        vn[a] = i < n && q + 1 < k ? Vg[(int64_t)(q + 1) * ln + i] : fac_zero<F>();
      }
      V uf[RM], vf[RM];  // the column in the arithmetic type, converted once
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        uf[a] = A::ld(u[a]);
        vf[a] = A::ld(v[a]);
      }
      V sv[NV];  // sv[c]: partial t1 of RHS c (V), sv[NR + c]: partial t2 (U)
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        Acc a1 = A::zero(), a2 = A::zero();
#pragma unroll
        for (int a = 0; a < RM; ++a) {
          A::fma(a1, vf[a], xY[a][c]);
          A::fma(a2, uf[a], xX[a][c]);
        }
        sv[c] = A::fin(a1);
        sv[NR + c] = A::fin(a2);
      }
      const V mine = warp_reduce_scatter<A, NV, S>(sv, lane);
      V t[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) t[c] = shfl_idx(mine, sbase + (c << SH));
#pragma unroll
      for (int c = 0; c < NR; ++c)
#pragma unroll
        for (int a = 0; a < RM; ++a) {
          A::fma(yX[a][c], uf[a], t[c]);       // U with t1
          A::fma(yY[a][c], vf[a], t[NR + c]);  // V with t2
        }
      if ((q + 1) % kRenorm == 0)
#pragma unroll
        for (int c = 0; c < NR; ++c)
#pragma unroll
          for (int a = 0; a < RM; ++a) {
            A::renorm(yX[a][c]);
            A::renorm(yY[a][c]);
          }
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        u[a] = un[a];
        v[a] = vn[a];
      }
    }
    if (it >= nwork) continue;
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      if (c0 + c >= P.nrhs) break;
      V* outx = ppart + (int64_t)(c0 + c) * P.pstride + ppx;
      V* outy = ppart + (int64_t)(c0 + c) * P.pstride + ppy;
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        const int i = sl + a * S;
        if (i < m) outx[i] = A::fin(yX[a][c]);
        if (i < n) outy[i] = A::fin(yY[a][c]);
      }
    }
  }
}
constexpr int kPairmsWarps = 4;
template <class A, int S, int RM, int NR>
__global__ void __launch_bounds__(32 * kPairmsWarps)
    k_pairms(ArgsV2 P, const int2* __restrict__ work, int64_t nwork,
             const typename A::val* __restrict__ xt, typename A::val* __restrict__ ppart) {
  pairms_body<A, S, RM, NR>(P, work, nwork, xt, ppart,
                            ((int64_t)blockIdx.x * kPairmsWarps + (threadIdx.x >> 5)) * (32 / S));
}

// Sub-warp form of k_pairg for the finest levels (boxes of <= kBoxRows
// points): S lanes per pair, 32 / S pairs per warp, rows t, t + S, ... (at
// most RM) of X and Y per lane.  The column loop runs to the largest rank of
// the warp's pairs; the sums reduce within each S-lane group.
// k_pairs stages its factor loads like k_pairg for float-float factors (the
// binary32 forms measured slower with the slots):
template <class A, int S>
__host__ __device__ constexpr bool pairs_async() {
  return sizeof(typename A::fac) == 8 && sizeof(typename A::acc) == 8;
}
template <class A, int S, int RM, int G>
__host__ __device__ constexpr int pairs_smem() {
  return pairs_async<A, S>() ? 2 * 2 * RM * G * 128 * (int)sizeof(typename A::fac) : 0;
}

template <class A, int S, int RM, int G>
__global__ void __launch_bounds__(128)
    k_pairs(ArgsV2 P, const int2* __restrict__ work, int64_t nwork,
            const typename A::val* __restrict__ xt, typename A::val* __restrict__ ppart) {
  using V = typename A::val;
  using F = typename A::fac;
  using Acc = typename A::acc;
  constexpr int NV = 2 * G;
  constexpr int SH = ilog2c(S) - ilog2c(NV);  // (lane % S) >> SH = column after the scatter
  const int lane = threadIdx.x & 31;
  const int sl = lane & (S - 1), gb = lane & ~(S - 1);
  const int64_t w = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 / S) +
                    lane / S;
  int m = 0, n = 0, k = 0;
  PairMeta PM{};
  const F* Ug = nullptr;
  if (w < nwork) {
    const int2 wk = work[w];
    const LevelV2& L = P.lev[wk.x];
    PM = L.meta[wk.y];
    m = PM.m;
    n = PM.n;
    k = PM.k;
    Ug = reinterpret_cast<const F*>(L.fac) + PM.foff;
  }
  const int kw = __reduce_max_sync(0xffffffffu, k);  // columns the warp visits
  const int mnw = __reduce_max_sync(0xffffffffu, max(m, n));  // rows the warp visits
  const int64_t lm = ldpad(m), ln = ldpad(n);
  const F* Vg = Ug + lm * k;
  V xX[RM], xY[RM];
  Acc yX[RM], yY[RM];
#pragma unroll
  for (int a = 0; a < RM; ++a) {
    const int i = sl + a * S;
    xX[a] = i < m ? xt[PM.xs + i] : A::vzero();
    xY[a] = i < n ? xt[PM.ys + i] : A::vzero();
    yX[a] = A::zero();
    yY[a] = A::zero();
  }
  // staged forms: the next column group goes to this thread's shared-memory
  // slots (two stages, one commit group per step) while the current one is
  // computed
  constexpr bool kAsync = pairs_async<A, S>();
  extern __shared__ __align__(16) unsigned char pairs_smem_buf[];
  F* const stage = reinterpret_cast<F*>(pairs_smem_buf);  // [2][u, v][RM][G][128]
  auto slot = [&](int b, int uv, int a, int g) {
    return stage + ((((b * 2 + uv) * RM + a) * G + g) * 128 + threadIdx.x);
  };
  auto issue = [&](int q0, int b) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const bool qok = q0 + g < k;
      const F* uc = Ug + (int64_t)(q0 + g) * lm;
      const F* vc = Vg + (int64_t)(q0 + g) * ln;
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        const int i = sl + a * S;
        if constexpr (kAsync) {
          if (qok && i < m) cp_async_small<sizeof(F)>(slot(b, 0, a, g), uc + i);
          if (qok && i < n) cp_async_small<sizeof(F)>(slot(b, 1, a, g), vc + i);
        }
      }
    }
    cp_async_commit();
  };
  if constexpr (kAsync) issue(0, 0);
  int stb = 0;
  for (int q0 = 0; q0 < kw; q0 += G) {
    F u[RM][G], v[RM][G];  // the step's columns in the factor type (converted where used)
    if constexpr (kAsync) {
      issue(q0 + G, stb ^ 1);
      cp_async_wait<1>();
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const bool qok = q0 + g < k;
#pragma unroll
        for (int a = 0; a < RM; ++a) {
          const int i = sl + a * S;
          u[a][g] = (qok && i < m) ? *slot(stb, 0, a, g) : fac_zero<F>();
          v[a][g] = (qok && i < n) ? *slot(stb, 1, a, g) : fac_zero<F>();
        }
      }
      stb ^= 1;
    } else {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const bool qok = q0 + g < k;
        const F* uc = Ug + (int64_t)(q0 + g) * lm;
        const F* vc = Vg + (int64_t)(q0 + g) * ln;
#pragma unroll
        for (int a = 0; a < RM; ++a) {
          const int i = sl + a * S;
          u[a][g] = (qok && i < m) ? uc[i] : fac_zero<F>();
          v[a][g] = (qok && i < n) ? vc[i] : fac_zero<F>();
        }
      }
    }
    V s[NV];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      Acc a1 = A::zero(), a2 = A::zero();
#pragma unroll
      for (int a = 0; a < RM; ++a)  // row groups past the warp's boxes are skipped
        if (a * S < mnw) {
          A::fma(a1, A::ld(v[a][g]), xY[a]);
          A::fma(a2, A::ld(u[a][g]), xX[a]);
        }
      s[g] = A::fin(a1);
      s[G + g] = A::fin(a2);
    }
    const V mine = warp_reduce_scatter<A, NV, S>(s, lane);
    V t[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) t[c] = shfl_idx(mine, gb + (c << SH));
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int a = 0; a < RM; ++a)
        if (a * S < mnw) {
          A::fma(yX[a], A::ld(u[a][g]), t[g]);      // U with t1
          A::fma(yY[a], A::ld(v[a][g]), t[G + g]);  // V with t2
        }
    if ((q0 / G + 1) % (kRenorm / G) == 0)
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        A::renorm(yX[a]);
        A::renorm(yY[a]);
      }
  }
  if (w >= nwork) return;
  V* outx = ppart + PM.ppx;
  V* outy = ppart + PM.ppy;
#pragma unroll
  for (int a = 0; a < RM; ++a) {
    const int i = sl + a * S;
    if (i < m) outx[i] = A::fin(yX[a]);
    if (i < n) outy[i] = A::fin(yY[a]);
  }
}

// ---------------------------------------------------------------------------
// box mode (finest levels, boxes of <= kBoxRows points): one warp per row box
// X, its stored pairs one after another.  A pair that fits kBoxStage values is
// copied to one of the warp's two shared-memory slices with asynchronous
// copies (cp.async, 16 bytes per lane and copy) while the previous pair is
// computed from the other slice, then
//   lane q < 2k: one column's dot product (V columns -> t1, U columns -> t2),
//                rows visited from q onwards (mod rows) so that the lanes hit
//                distinct banks;
//   lanes over rows: y_X += U t1 kept in registers, V t2 written as the
//                partial of Y.
// A larger pair is read from global memory with one warp per column instead.
// The slices are dynamic shared memory (kBoxSmem bytes per block).
// ---------------------------------------------------------------------------
constexpr int kBoxRows = 64;
constexpr int kBoxStage = H2D_BOX_STAGE;
constexpr int kBoxK = 64;
constexpr int kBoxWarps = 4;

constexpr int kBoxMaxPairs = 16;  // row pairs of one box (at most 15)

// bytes per warp: two factor slices (8-byte values at most), two x_Y slices,
// x_X, the 2k projections and the box's pair records
constexpr int kBoxWarpSmem = 2 * kBoxStage * 8 + 2 * kBoxRows * 8 + kBoxRows * 8 +
                             2 * kBoxK * 8 + kBoxMaxPairs * (int)sizeof(PairMeta);
constexpr int kBoxSmem = kBoxWarps * kBoxWarpSmem;
static_assert(kBoxStage % 2 == 0 && kBoxWarpSmem % 16 == 0, "16-byte aligned slices");

template <class A>
__global__ void __launch_bounds__(32 * kBoxWarps)
    k_box(ArgsV2 P, const BoxWork* __restrict__ work, int64_t nwork,
          const typename A::val* __restrict__ xt, typename A::val* __restrict__ yl,
          typename A::val* __restrict__ ppart) {
  using V = typename A::val;
  using F = typename A::fac;
  using Acc = typename A::acc;
  static_assert(sizeof(F) <= 8 && sizeof(V) <= 8, "slice sizes assume 8-byte values at most");
  extern __shared__ __align__(16) unsigned char box_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t wid = (int64_t)blockIdx.x * kBoxWarps + warp;
  if (wid >= nwork) return;
  unsigned char* ws = box_smem + (size_t)warp * kBoxWarpSmem;
  F* st2 = reinterpret_cast<F*>(ws);                        // [2][kBoxStage]
  V* xy2 = reinterpret_cast<V*>(ws + 2 * kBoxStage * 8);  // [2][kBoxRows]
  V* xx = xy2 + 2 * kBoxRows;
  V* ts = xx + kBoxRows;
  PairMeta* pm = reinterpret_cast<PairMeta*>(ts + 2 * kBoxK);
  const BoxWork wk = work[wid];
  const int l = wk.level;
  if (P.lmode[l] != LMODE_BOX) return;  // this level runs as pairs in this product
  const LevelV2& L = P.lev[l];
  const int32_t xs = wk.xs, m = wk.m;
  const int64_t lm = ldpad(m);
  const int npb = wk.np;
  if (lane < npb) pm[lane] = L.meta[wk.p0 + lane];
  __syncwarp();
  const F* fac = reinterpret_cast<const F*>(L.fac);
  auto fits = [&](const PairMeta& PM) {
    return (ldpad(PM.m) + ldpad(PM.n)) * (int64_t)PM.k <= kBoxStage && PM.k <= kBoxK;
  };
  for (int c = 0; c < P.nrhs; ++c) {
    const V* xc = xt + (int64_t)c * P.n;
    // copies of pair ip (factors if they fit, and x_Y) into slice b
    auto issue = [&](int ip, int b) {
      const PairMeta& PM = pm[ip];
      F* st = st2 + b * kBoxStage;
      V* xy = xy2 + b * kBoxRows;
      if (fits(PM)) {
        const F* Ug = fac + PM.foff;
        const int64_t tot = (ldpad(m) + ldpad(PM.n)) * (int64_t)PM.k;
        // pairs start at even values and hold an even count: copies of two
        // values (16, 8 or 4 bytes) stay aligned
        if constexpr (sizeof(F) == 8) {
          for (int64_t e = lane; 2 * e < tot; e += 32) cp_async16(st + 2 * e, Ug + 2 * e);
        } else {
          for (int64_t e = lane; 2 * e < tot; e += 32)
            cp_async_small<2 * sizeof(F)>(st + 2 * e, Ug + 2 * e);
        }
      }
      for (int j = lane; j < PM.n; j += 32) cp_async_small<sizeof(V)>(xy + j, xc + PM.ys + j);
      cp_async_commit();
    };
    for (int i = lane; i < m; i += 32) xx[i] = xc[xs + i];
    if (npb > 0) issue(0, 0);
    Acc y0 = A::zero(), y1 = A::zero();  // rows lane and lane + 32
    for (int ip = 0; ip < npb; ++ip) {
      const int b = ip & 1;
      if (ip + 1 < npb) {
        issue(ip + 1, b ^ 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();  // every lane's copies of slice b (and x_X) are visible
      const PairMeta& PM = pm[ip];
      const int k = PM.k;
      const int32_t n = PM.n;
      const int64_t ln = ldpad(n);
      const F* Ug = fac + PM.foff;
      const F* Vg = Ug + lm * k;
      const V* xy = xy2 + b * kBoxRows;
      V* outy = ppart + (int64_t)c * P.pstride + PM.ppy;
      if (fits(PM)) {
        const F* Us = st2 + b * kBoxStage;
        const F* Vs = Us + lm * k;
        for (int job = lane; job < 2 * k; job += 32) {
          const bool isV = job < k;
          const int q = isV ? job : job - k;
          const int rows = isV ? n : m;
          const F* col = isV ? Vs + q * ln : Us + q * lm;
          const V* xv = isV ? xy : xx;
          Acc a = A::zero();
          int r = q;  // q < k <= rows
          for (int u = 0; u < rows; ++u) {
            A::fma(a, A::ld(col[r]), xv[r]);
            if (++r == rows) r = 0;
          }
          ts[job] = A::fin(a);
        }
        __syncwarp();
        for (int r = lane; r < m + n; r += 32) {
          const bool own = r < m;
          const int i = own ? r : r - m;
          const F* M = own ? Us + i : Vs + i;
          const int64_t ld = own ? lm : ln;
          const V* tv = own ? ts : ts + k;
          Acc a = own ? (i < 32 ? y0 : y1) : A::zero();
          for (int q = 0; q < k; ++q) A::fma(a, A::ld(M[q * ld]), tv[q]);
          if (own) {
            if (i < 32) y0 = a;
            else y1 = a;
          } else {
            outy[i] = A::fin(a);
          }
        }
      } else {
        // the pair does not fit the slice: warp-per-column from global memory
        for (int job = 0; job < 2 * k; ++job) {
          const bool isV = job < k;
          const int q = isV ? job : job - k;
          const int rows = isV ? n : m;
          const F* col = isV ? Vg + q * ln : Ug + q * lm;
          const V* xv = isV ? xy : xx;
          Acc a = A::zero();
          for (int r = lane; r < rows; r += 32) A::fma(a, A::ld(col[r]), xv[r]);
          const V sum = A::warp_sum(a);
          if (lane == 0) ts[job] = sum;
        }
        __syncwarp();
        for (int r = lane; r < m + n; r += 32) {
          const bool own = r < m;
          const int i = own ? r : r - m;
          const F* M = own ? Ug + i : Vg + i;
          const int64_t ld = own ? lm : ln;
          const V* tv = own ? ts : ts + k;
          Acc a = own ? (i < 32 ? y0 : y1) : A::zero();
          for (int q = 0; q < k; ++q) A::fma(a, A::ld(M[q * ld]), tv[q]);
          if (own) {
            if (i < 32) y0 = a;
            else y1 = a;
          } else {
            outy[i] = A::fin(a);
          }
        }
      }
      __syncwarp();  // slice b and ts are free for the next copies
    }
    V* own = yl + ((int64_t)l * P.nrhs + c) * P.n + xs;
    if (lane < m) own[lane] = A::fin(y0);
    if (lane + 32 < m) own[lane + 32] = A::fin(y1);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// binary64 far field.  GB300 runs binary64 at 2 FMA per clock per SM, and a
// binary64 warp instruction costs the same whatever its active lanes, so the
// binary64 kernels are shaped to keep every lane of every binary64
// instruction useful and to spend as few additions as possible on sums
// across lanes:
//   - two-pass projection (k_proj64): one warp per (task, group of <= 32
//     columns); lanes over rows (coalesced loads), each lane accumulating all
//     columns of the group over its 16 rows, then one halving exchange sums
//     the group (NV - 1 additions for NV columns, against 5 per column for
//     a butterfly per column);
//   - small boxes (k_pair64): one warp per stored pair, the pair's factors
//     and vectors staged in shared memory; the projection is split into
//     units of one column and one row segment, one unit per lane, summed by
//     its lane alone (then the few segment partials of a column by one
//     lane); the expansion runs one lane per row.
// ---------------------------------------------------------------------------
// Row segments per column for `jobs` dot products of `rows` rows on one warp:
// the S in [1, 8] with the fewest binary64 instructions (passes over the
// units times the segment length, plus the S - 1 additions per column), at
// most 256 units.
__device__ __forceinline__ int f64_segments(int jobs, int rows, int& seglen) {
  int best = 1, bl = rows, bc = 1 << 30;
  for (int S = 1; S <= 8 && jobs * S <= 256; ++S) {
    const int L = (rows + S - 1) / S;
    if (S > 1 && (S - 1) * L >= rows) break;  // the last segment would be empty
    const int cost = ((jobs * S + 31) >> 5) * L + (S - 1) * ((jobs + 31) >> 5);
    if (cost < bc) {
      bc = cost;
      best = S;
      bl = L;
    }
  }
  seglen = bl;
  return best;
}

// One column group of a two-pass projection task: NV >= c columns q0 ..
// q0 + c - 1 of `mat` (leading dimension ld) against x over the task's rows
// [r0, r0 + nr), 16 rows per lane in two halves of 8 (the half's x kept in
// registers); within a half the columns are visited one after another, so
// the warp's loads stream one contiguous column slice at a time; column
// q0 + j's total goes to out[j].
template <int NV>
__device__ __forceinline__ void proj64_group(const double* __restrict__ mat, int64_t ld, int c,
                                             const double* __restrict__ xv, int r0, int nr,
                                             int lane, double* __restrict__ out) {
  constexpr int H = kChunkP / 64;  // rows per lane and half
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    const int rb = 32 * H * hf;  // first row of the half, relative to r0
    if (rb >= nr) break;         // uniform
    double xr[H];
#pragma unroll
    for (int u = 0; u < H; ++u) {
      const int r = rb + lane + 32 * u;
      xr[u] = r < nr ? xv[r0 + r] : 0.0;
    }
    const bool full = rb + 32 * H <= nr;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      if (j < c) {
        const double* col = mat + j * ld + r0 + rb + lane;
        if (full) {
#pragma unroll
          for (int u = 0; u < H; ++u) acc[j] = fma(__ldg(col + 32 * u), xr[u], acc[j]);
        } else {
#pragma unroll
          for (int u = 0; u < H; ++u) {
            const int r = rb + lane + 32 * u;
            if (rb + 32 * u < nr) acc[j] = fma(r < nr ? __ldg(col + 32 * u) : 0.0, xr[u], acc[j]);
          }
        }
      }
    }
  }
  const double s = warp_reduce_scatter<F64A, NV>(acc, lane);
  constexpr int per = 32 / NV;  // lanes holding each column's total
  const int col = lane / per;
  if (lane % per == 0 && col < c) out[col] = s;
}

// Two-pass projection in binary64: one warp per (task, group of <= 8
// columns) of the work list pg (task index, first column); the task's k
// partial sums per right-hand side go where k_proj2 puts them.  Eight
// columns per warp, 9 additions per 8 columns; registers are kept to 64 so
// that 32 warps per SM keep enough loads in flight.
constexpr int kProj64Cols = 8;
__global__ void __launch_bounds__(256, 4)
    k_proj64(ArgsV2 P, const ProjTask* __restrict__ tasks, const int2* __restrict__ pg,
             int64_t ngroups, const double* __restrict__ xt, double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= ngroups) return;
  const int2 g = pg[w];
  const ProjTask T = tasks[g.x];
  const int q0 = g.y, k = T.k;
  const int c = min(kProj64Cols, k - q0);
  const double* mat = reinterpret_cast<const double*>(P.lev[T.level].fac) + T.mat +
                      (int64_t)q0 * T.ld;
  for (int rc = 0; rc < P.nrhs; ++rc) {
    const double* xv = xt + (int64_t)rc * P.n + T.base;
    double* out = part + T.out * P.nrhs + (int64_t)rc * k + q0;
    if (c <= 4)
      proj64_group<4>(mat, T.ld, c, xv, T.r0, T.nr, lane, out);
    else
      proj64_group<kProj64Cols>(mat, T.ld, c, xv, T.r0, T.nr, lane, out);
  }
}

// Chunk sums of the two-pass levels in binary64 for pair sides of at most
// kTsumThread chunks: one thread per (pair side, column), the chunk partials
// added in chunk order (no cross-lane sums); sides of more chunks are left
// to k_tsum2 (lanes over chunks, then a shuffle tree).
constexpr int kTsumThread = 32;
__global__ void __launch_bounds__(256)
    k_tsum64(ArgsV2 P, const ProjTask* __restrict__ tasks, const int64_t* __restrict__ red,
             const int64_t* __restrict__ sideq, int64_t nwork, const double* __restrict__ part,
             double* __restrict__ t) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w >= nwork) return;
  const int64_t s = sideq[2 * w];
  const int q = (int)sideq[2 * w + 1];
  const int64_t first = red[2 * s], count = red[2 * s + 1];
  if (count > kTsumThread) return;
  const ProjTask T0 = tasks[first];
  const LevelV2& L = P.lev[T0.level];
  const int k = L.rank[T0.pair];
  double* out = t + L.toff[T0.pair] * P.nrhs + (int64_t)T0.side * k * P.nrhs;
  for (int c = 0; c < P.nrhs; ++c) {
    double acc = part[tasks[first].out * P.nrhs + c * k + q];
    for (int64_t j = 1; j < count; ++j) acc += part[tasks[first + j].out * P.nrhs + c * k + q];
    out[c * k + q] = acc;
  }
}

// Pair levels of small boxes in binary64: one warp per stored pair (X,Y).
// x_X and x_Y are copied to the warp's shared-memory slice; then, block by
// block of cb columns (as many as fit kP64Slice values), the columns of U
// and V are copied there too, and their projections t1 = V^T x_Y and
// t2 = U^T x_X run as lane-owned (column, segment) units, each lane starting
// its segment at its own offset (mod the segment length) so that the lanes
// spread over the banks.  Then U t1 (rows of X) and V t2 (rows of Y), one
// lane per row with the factors read from global memory (coalesced), are
// written as the pair's partial results.
constexpr int kPair64Warps = 8;
constexpr int kP64Slice = 512;  // factor values staged per warp and column block
constexpr int kP64Rows = 128;   // largest box of a level run by this kernel
constexpr int kP64Kmax = 64;    // largest rank of a level run by this kernel
constexpr int kP64Warp = kP64Slice + 2 * kP64Rows + 256 + 2 * kP64Kmax;  // doubles per warp
constexpr int kPair64Smem = kPair64Warps * kP64Warp * 8;
__device__ __forceinline__ double f64_dot_rot(const double* __restrict__ col,
                                              const double* __restrict__ x, int len, int rot) {
  double a0 = 0.0, a1 = 0.0;
  int t = rot % len;
  int i = 0;
  for (; i + 1 < len; i += 2) {
    a0 = fma(col[t], x[t], a0);
    if (++t == len) t = 0;
    a1 = fma(col[t], x[t], a1);
    if (++t == len) t = 0;
  }
  if (i < len) a0 = fma(col[t], x[t], a0);
  return a0 + a1;
}

__global__ void __launch_bounds__(32 * kPair64Warps)
    k_pair64(ArgsV2 P, const int2* __restrict__ work, int64_t nw, const double* __restrict__ xt,
             double* __restrict__ ppart) {
  extern __shared__ __align__(16) double p64_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t wi = (int64_t)blockIdx.x * kPair64Warps + warp;
  if (wi >= nw) return;
  double* fs = p64_smem + (size_t)warp * kP64Warp;  // column block of U, then of V
  double* xx = fs + kP64Slice;                      // x_X
  double* xy = xx + kP64Rows;                       // x_Y
  double* sp = xy + kP64Rows;                       // segment partials
  double* tw = sp + 256;                            // t1 (k), t2 (k)
  const int2 wk = work[wi];
  const LevelV2& Lv = P.lev[wk.x];
  const PairMeta PM = Lv.meta[wk.y];
  const int32_t xs = PM.xs, m = PM.m, ys = PM.ys, n = PM.n;
  const int lm = (int)ldpad(m), ln = (int)ldpad(n);
  const int k = PM.k;
  const double* Ug = reinterpret_cast<const double*>(Lv.fac) + PM.foff;
  const double* Vg = Ug + (int64_t)lm * k;
  const int cb = max(1, min(k, kP64Slice / (lm + ln)));  // columns per block
  int L;
  const int S = f64_segments(2 * cb, max(m, n), L);
  for (int c = 0; c < P.nrhs; ++c) {
    const double* xc = xt + (int64_t)c * P.n;
    for (int i = lane; i < m; i += 32) cp_async_small<8>(xx + i, xc + xs + i);
    for (int i = lane; i < n; i += 32) cp_async_small<8>(xy + i, xc + ys + i);
    for (int q0 = 0; q0 < k; q0 += cb) {
      const int nc = min(cb, k - q0);
      // columns q0 .. q0 + nc - 1 of U, then of V (16-byte copies: columns
      // start on 16-byte boundaries and hold an even count)
      const double* us = Ug + (int64_t)q0 * lm;
      const double* vs = Vg + (int64_t)q0 * ln;
      for (int e = lane; 2 * e < nc * lm; e += 32) cp_async16(fs + 2 * e, us + 2 * e);
      for (int e = lane; 2 * e < nc * ln; e += 32) cp_async16(fs + nc * lm + 2 * e, vs + 2 * e);
      cp_async_commit();
      cp_async_wait<0>();
      __syncwarp();
      for (int u = lane; u < 2 * nc * S; u += 32) {
        const int job = u / S, sg = u - job * S;
        const bool isV = job < nc;  // V columns against x_Y give t1
        const int q = isV ? job : job - nc;
        const int rows = isV ? n : m;
        const double* col = isV ? fs + nc * lm + q * ln : fs + q * lm;
        const int r0 = sg * L, len = min(rows - r0, L);
        sp[u] = len > 0 ? f64_dot_rot(col + r0, (isV ? xy : xx) + r0, len, u) : 0.0;
      }
      __syncwarp();
      for (int j = lane; j < 2 * nc; j += 32) {
        double a = sp[j * S];
        for (int sg = 1; sg < S; ++sg) a += sp[j * S + sg];
        tw[j < nc ? q0 + j : k + q0 + j - nc] = a;
      }
      __syncwarp();
    }
    double* outx = ppart + (int64_t)c * P.pstride + PM.ppx;
    double* outy = ppart + (int64_t)c * P.pstride + PM.ppy;
    for (int r = lane; r < m + n; r += 32) {
      const bool own = r < m;
      const int i = own ? r : r - m;
      const double* M = own ? Ug + i : Vg + i;
      const int64_t ld = own ? lm : ln;
      const double* tv = own ? tw : tw + k;  // U pairs with t1, V with t2
      double a = 0.0;
      int q = 0;
      for (; q + 4 <= k; q += 4) {
        const double m0 = __ldg(M + q * ld), m1 = __ldg(M + (q + 1) * ld),
                     m2 = __ldg(M + (q + 2) * ld), m3 = __ldg(M + (q + 3) * ld);
        a = fma(m0, tv[q], a);
        a = fma(m1, tv[q + 1], a);
        a = fma(m2, tv[q + 2], a);
        a = fma(m3, tv[q + 3], a);
      }
      for (; q < k; ++q) a = fma(__ldg(M + q * ld), tv[q], a);
      (own ? outx : outy)[i] = a;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// two-pass far field (levels < lfuse)
// ---------------------------------------------------------------------------
// One warp per (task, column): lanes read rows r0 + lane + 32 u (coalesced),
// keep them in registers across the right-hand sides, and reduce by shuffles.
// wtask[w] is the task of warp w; its column is w - out[task].
template <class A>
__device__ __forceinline__ void proj2_body(const ArgsV2& P, const ProjTask* __restrict__ tasks,
                                           const int32_t* __restrict__ wtask, int64_t nwarps,
                                           const typename A::val* __restrict__ xt,
                                           typename A::val* __restrict__ part, int64_t w) {
  using V = typename A::val;
  using Acc = typename A::acc;
  constexpr int R = kChunkP / 32;
  const int lane = threadIdx.x & 31;
  if (w >= nwarps) return;
  const int64_t lo = wtask[w];
  const ProjTask T = tasks[lo];
  const int q = (int)(w - T.out);
  const LevelV2& L = P.lev[T.level];
  const int32_t base = T.base;
  const int k = T.k;
  using F = typename A::fac;
  const F* col = reinterpret_cast<const F*>(L.fac) + T.mat + (int64_t)q * T.ld;
  V v[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int r = T.r0 + lane + 32 * u;
    v[u] = r < T.r0 + T.nr ? A::ld(col[r]) : A::vzero();
  }
  for (int c = 0; c < P.nrhs; ++c) {
    const V* xv = xt + c * P.n + base;
    Acc a = A::zero();
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int r = T.r0 + lane + 32 * u;
      if (r < T.r0 + T.nr) A::fma(a, v[u], xv[r]);
    }
    const V sum = A::warp_sum(a);
    if (lane == 0) part[T.out * P.nrhs + (int64_t)c * k + q] = sum;
  }
}
template <class A>
__global__ void __launch_bounds__(256)
    k_proj2(ArgsV2 P, const ProjTask* __restrict__ tasks, const int32_t* __restrict__ wtask,
            int64_t nwarps, const typename A::val* __restrict__ xt,
            typename A::val* __restrict__ part) {
  proj2_body<A>(P, tasks, wtask, nwarps, xt, part,
                (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
}

// Several right-hand sides (two-pass levels): one block of 256 threads per
// projection task computes its k x R partial sums (R <= 32 right-hand sides
// per pass, 64 columns per pass) from shared-memory tiles of 64 rows (32 for
// 8-byte values): the
// task's rows of the matrix (transposed, row r of the tile = the task's row)
// and of x.  Thread (qg, cg) owns columns 4 qg .. 4 qg + 3 and right-hand
// sides 2 cg, 2 cg + 1, summed over the rows in row order.
constexpr int kPmRows = 64;  // rows per tile
constexpr int kPmCols = 64;  // columns per pass
constexpr int kPmRhs = 32;   // right-hand sides per pass

template <class A>
__global__ void __launch_bounds__(256)
    k_projm(ArgsV2 P, const ProjTask* __restrict__ tasks, const typename A::val* __restrict__ xt,
            typename A::val* __restrict__ part) {
  using V = typename A::val;
  using F = typename A::fac;
  using Acc = typename A::acc;
  constexpr int RT = sizeof(V) == 4 ? kPmRows : kPmRows / 2;  // tile rows (48 KB static limit)
  static_assert(sizeof(V) == 4 || RT == kPmRows / 2, "tile fits static shared memory");
  __shared__ V Ms[RT][kPmCols + 1];
  __shared__ V Xs[RT][kPmRhs + 1];
  const int tid = threadIdx.x;
  const int qg = tid & 15, cg = tid >> 4;
  const ProjTask T = tasks[blockIdx.x];
  const LevelV2& L = P.lev[T.level];
  const F* M = reinterpret_cast<const F*>(L.fac) + T.mat;
  const int k = T.k;
  for (int q0 = 0; q0 < k; q0 += kPmCols) {
    const int kc = min(kPmCols, k - q0);
    for (int c0 = 0; c0 < P.nrhs; c0 += kPmRhs) {
      const int rc = min(kPmRhs, P.nrhs - c0);
      Acc acc[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = A::zero();
      for (int r0 = 0; r0 < T.nr; r0 += RT) {
        const int rows = min(RT, T.nr - r0);
        __syncthreads();  // the previous tile is consumed
        for (int e = tid; e < RT * kPmCols; e += 256) {
          const int rr = e & (RT - 1), q = e / RT;
          Ms[rr][q] = (rr < rows && q < kc) ? A::ld(M[(int64_t)(q0 + q) * T.ld + T.r0 + r0 + rr])
                                            : A::vzero();
        }
        for (int e = tid; e < RT * kPmRhs; e += 256) {
          const int rr = e & (RT - 1), c = e / RT;
          Xs[rr][c] = (rr < rows && c < rc)
                          ? xt[(int64_t)(c0 + c) * P.n + T.base + T.r0 + r0 + rr]
                          : A::vzero();
        }
        __syncthreads();
        for (int rr = 0; rr < rows; ++rr) {
          const V x0 = Xs[rr][2 * cg], x1 = Xs[rr][2 * cg + 1];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const V mv = Ms[rr][4 * qg + i];
            A::fma(acc[i][0], mv, x0);
            A::fma(acc[i][1], mv, x1);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int q = 4 * qg + i, c = 2 * cg + j;
          if (q < kc && c < rc)
            part[T.out * P.nrhs + (int64_t)(c0 + c) * k + q0 + q] = A::fin(acc[i][j]);
        }
    }
  }
}

// ---------------------------------------------------------------------------
// bfloat16 pairs: packing and the split of a binary32 value into two
// bfloat16 terms (hi + lo, about 2^-17 relative)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bf2_pack(__nv_bfloat16 lo_idx, __nv_bfloat16 hi_idx) {
  return (uint32_t)__bfloat16_as_ushort(lo_idx) | ((uint32_t)__bfloat16_as_ushort(hi_idx) << 16);
}
__device__ __forceinline__ void bf_split(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(v - __bfloat162float(h));
}
// ---------------------------------------------------------------------------
// bfloat16 factors, several right-hand sides, two-pass levels, on the
// fifth-generation tensor cores (tcgen05): the accumulators live in tensor
// memory (TMEM), the operands are staged in shared memory in the K-major
// core-matrix layout (tc5.cuh), one thread issues the MMAs, and an mbarrier
// per staging buffer reports their completion.  Two buffers: the next stage
// is copied in while the tensor core works on the current one.  x and t
// enter as two bfloat16 terms (hi + lo, about 2^-17 relative), side by side
// in the N dimension (32 right-hand sides per pass: N = 64), so the result
// keeps the bfloat16 mode's accuracy (set by the factors).  Every wait is
// bounded: a wait that gives up sets *status, stops issuing work, waits
// (bounded) for the MMAs in flight, frees the TMEM and returns.
// ---------------------------------------------------------------------------
constexpr int kT5K = 64;                      // K-elements per stage (4 MMAs of K = 16)
// Core matrices adjacent in K sit 144 bytes apart (128 + 16): the eight
// 16-byte pieces of one row's 64 K-elements then fall on distinct banks, so
// a warp storing one row (two K-elements per lane) writes conflict-free.
constexpr int kT5Lbo = 144;
constexpr int kT5Sbo = kT5K / 8 * kT5Lbo;     // bytes between 8-row groups
constexpr int kT5ABytes = 128 / 8 * kT5Sbo;   // A stage: M = 128 rows
constexpr int kT5BBytes = 64 / 8 * kT5Sbo;    // B stage: N = 64 rows (32 hi, 32 lo)
constexpr int kT5Smem = 2 * (kT5ABytes + kT5BBytes);
constexpr uint32_t kT5Polls = 1u << 24;       // polls of an mbarrier before giving up
constexpr uint32_t kT5Idesc = tc5::idesc_bf16(128, 64);

__device__ __forceinline__ int t5_off(int row, int k) {
  return (row >> 3) * kT5Sbo + (k >> 3) * kT5Lbo + (row & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint32_t bf2u(float a, float b) {
  return bf2_pack(__float2bfloat16_rn(a), __float2bfloat16_rn(b));
}
// eight binary32 values -> their hi and lo bfloat16 terms, 16 bytes each
__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo) {
  __nv_bfloat16 h[8], l[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) bf_split(v[e], h[e], l[e]);
  hi = make_uint4(bf2_pack(h[0], h[1]), bf2_pack(h[2], h[3]), bf2_pack(h[4], h[5]),
                  bf2_pack(h[6], h[7]));
  lo = make_uint4(bf2_pack(l[0], l[1]), bf2_pack(l[2], l[3]), bf2_pack(l[4], l[5]),
                  bf2_pack(l[6], l[7]));
}

// Shared pipeline state of the two kernels below.  Every thread of the block
// waits on the mbarrier itself; the outcome is agreed on by a block-wide
// vote, so that every thread takes the same branch afterwards.
struct T5Pipe {
  uint64_t* bar;   // [2] mbarriers, one per staging buffer
  int gs = 0;      // stages issued so far
  bool ok = true;  // no wait gave up (the same in every thread)
  __device__ __forceinline__ void wait_stage(int g, int* status) {
    const bool got = tc5::mbar_wait(&bar[g & 1], (g >> 1) & 1, kT5Polls);
    ok = __syncthreads_and(got) != 0;
    if (!ok && threadIdx.x == 0) atomicOr(status, 1);
  }
  // before refilling the buffer of stage gs: the MMAs of stage gs - 2 are done
  __device__ __forceinline__ void acquire(int* status) {
    if (gs >= 2 && ok) wait_stage(gs - 2, status);
  }
  // all MMAs issued so far are done
  __device__ __forceinline__ void drain(int* status) {
    if (gs >= 1 && ok) wait_stage(gs - 1, status);
  }
  // before the TMEM is freed: after a wait gave up, one more bounded wait
  // for the MMAs still in flight
  __device__ __forceinline__ void finish() {
    if (gs >= 1 && !ok) (void)tc5::mbar_wait(&bar[(gs - 1) & 1], ((gs - 1) >> 1) & 1, kT5Polls);
  }
};

// Projection: blocks of 128 threads walk the projection tasks (grid-stride),
// keeping their TMEM and mbarriers.  Per task, pass of 32 right-hand sides
// and tile of 128 columns q, D[q, n] = sum over the task's rows r of
// M(r, q) B(n, r), B = (x_hi | x_lo); stages of 64 rows, each column of the
// stage loaded by one warp (two rows per lane, coalesced) and stored
// conflict-free (kT5Lbo).  Then thread (warp w, lane i) holds column
// q = 32 w + i of D in TMEM and writes t_q = D[q, c] + D[q, 32 + c] where
// k_proj2 puts it.
__global__ void __launch_bounds__(128)
    k_proj_t5(ArgsV2 P, const ProjTask* __restrict__ tasks, int64_t ntasks,
              const float* __restrict__ xt, float* __restrict__ part, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char t5_smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc5::mbar_init(&bar[0], 1);
    tc5::mbar_init(&bar[1], 1);
  }
  if (warp == 0) tc5::tmem_alloc(&tslot, 64);
  tc5::fence_before();
  __syncthreads();
  tc5::fence_after();
  const uint32_t tm = tslot;
  T5Pipe pp;
  pp.bar = bar;
  for (int64_t ti = blockIdx.x; ti < ntasks && pp.ok; ti += gridDim.x) {
    const ProjTask T = tasks[ti];
    const __nv_bfloat16* M =
        reinterpret_cast<const __nv_bfloat16*>(P.lev[T.level].fac) + T.mat + T.r0;
    const int k = T.k, nr = T.nr;
    const int nst = (nr + kT5K - 1) / kT5K;
    const float* xb = xt + T.base + T.r0;
    for (int c0 = 0; c0 < P.nrhs && pp.ok; c0 += 32) {
      for (int q0 = 0; q0 < k && pp.ok; q0 += 128) {
        for (int st = 0; st < nst && pp.ok; ++st) {
          pp.acquire(status);
          if (!pp.ok) break;
          unsigned char* sA = t5_smem + (pp.gs & 1) * kT5ABytes;
          unsigned char* sB = t5_smem + 2 * kT5ABytes + (pp.gs & 1) * kT5BBytes;
          const int r = st * kT5K + 2 * lane;  // this lane's two rows of the stage
          const bool r0ok = r < nr, r1ok = r + 1 < nr;
          // A: columns q0 + warp + 4 i (those < k; rows of A past k are left
          // as they are: they only feed rows of D that are not read)
          for (int ql = warp; ql < 128 && q0 + ql < k; ql += 4) {
            const __nv_bfloat16* col = M + (int64_t)(q0 + ql) * T.ld + r;
            uint32_t w = 0u;
            if (r1ok)
              w = *reinterpret_cast<const uint32_t*>(col);  // even offset
            else if (r0ok)
              w = bf2_pack(col[0], __float2bfloat16_rn(0.f));
            *reinterpret_cast<uint32_t*>(sA + t5_off(ql, 2 * lane)) = w;
          }
          // B: right-hand sides c0 + warp + 4 i, hi and lo terms
          for (int c = warp; c < 32; c += 4) {
            const bool okc = c0 + c < P.nrhs;
            const float* xc = xb + (int64_t)(c0 + c) * P.n;
            const float v0 = (okc && r0ok) ? xc[r] : 0.f;
            const float v1 = (okc && r1ok) ? xc[r + 1] : 0.f;
            __nv_bfloat16 h0, l0, h1, l1;
            bf_split(v0, h0, l0);
            bf_split(v1, h1, l1);
            *reinterpret_cast<uint32_t*>(sB + t5_off(c, 2 * lane)) = bf2_pack(h0, h1);
            *reinterpret_cast<uint32_t*>(sB + t5_off(32 + c, 2 * lane)) = bf2_pack(l0, l1);
          }
          tc5::fence_smem_to_async();
          __syncthreads();
          if (tid == 0) {
            tc5::fence_after();
            const int nk = min(kT5K, nr - st * kT5K);
            for (int kk = 0; 16 * kk < nk; ++kk)
              tc5::mma_bf16(tm, tc5::sdesc(tc5::smem_addr(sA) + kk * 2 * kT5Lbo, kT5Lbo, kT5Sbo),
                            tc5::sdesc(tc5::smem_addr(sB) + kk * 2 * kT5Lbo, kT5Lbo, kT5Sbo),
                            kT5Idesc, st > 0 || kk > 0);
            tc5::mma_commit(&bar[pp.gs & 1]);
          }
          ++pp.gs;
        }
        pp.drain(status);
        tc5::fence_after();
        if (pp.ok) {
          float hv[32], lv[32];
          const uint32_t ta = tm + ((uint32_t)(32 * warp) << 16);
          tc5::tmem_ld32(ta, hv);
          tc5::tmem_ld32(ta + 32, lv);
          const int q = q0 + 32 * warp + lane;
          if (q < k)
#pragma unroll
            for (int c = 0; c < 32; ++c)
              if (c0 + c < P.nrhs)
                part[T.out * P.nrhs + (int64_t)(c0 + c) * k + q] = hv[c] + lv[c];
        }
        tc5::fence_before();
        __syncthreads();  // TMEM read before the next tile's MMAs overwrite it
        tc5::fence_after();
      }
    }
  }
  pp.drain(status);
  pp.finish();
  tc5::fence_before();
  __syncthreads();
  if (warp == 0) tc5::tmem_dealloc(tm, 64);
}

// Projection grouped by box: every projection task of one level that reads
// the same rows of x (the same box, the same row chunk) multiplies the same
// B = (x_hi | x_lo) tile, so the group's matrices are stacked along M: D row
// j of the group is column q of task t, D[j, n] = sum over the rows r of
// M_t(r, q) B(n, r).  x is loaded once per group and stage instead of once
// per task.  Blocks of 256 threads walk the groups (grid-stride); a group
// holds at most kGrpRows D rows (kGrpRows / 128 tiles of 128 rows, 64 TMEM
// columns each).  Per stage of 64 rows: B is loaded into one of two buffers
// with the stage's first tile, and each tile's A (128 rows of 64 K-elements,
// four-byte asynchronous copies, two rows per lane) into one of two
// buffers; the next tile's copies are issued before the current tile's MMAs.
constexpr int kGrpRows = 256;                  // D rows per group, at most
constexpr int kGrpTmem = kGrpRows / 128 * 64;  // TMEM columns
constexpr int kGrpSmem = 2 * kT5ABytes + 2 * kT5BBytes;
struct GrpRow {
  int64_t col;  // first value of the column (its row 0 in the chunk) in the level's factors
  int64_t out;  // the task's partial-sum offset
  int32_t k, q;
};

__global__ void __launch_bounds__(256)
    k_projg_t5(ArgsV2 P, const ProjTask* __restrict__ tasks, const int32_t* __restrict__ gtask,
               const int4* __restrict__ grp, int64_t ngrp, const float* __restrict__ xt,
               float* __restrict__ part, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char t5_smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tslot;
  __shared__ GrpRow srow[kGrpRows];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc5::mbar_init(&bar[0], 1);
    tc5::mbar_init(&bar[1], 1);
  }
  if (warp == 0) tc5::tmem_alloc(&tslot, kGrpTmem);
  tc5::fence_before();
  __syncthreads();
  tc5::fence_after();
  const uint32_t tm = tslot;
  T5Pipe pp;
  pp.bar = bar;
  for (int64_t gi = blockIdx.x; gi < ngrp && pp.ok; gi += gridDim.x) {
    const int4 G = grp[gi];  // first sorted task, tasks, D rows, unused
    const ProjTask T0 = tasks[gtask[G.x]];
    const __nv_bfloat16* fac = reinterpret_cast<const __nv_bfloat16*>(P.lev[T0.level].fac);
    const int nr = T0.nr, rows = G.z;
    const int nt = (rows + 127) / 128, nst = (nr + kT5K - 1) / kT5K;
    if (warp == 0) {  // the group's D rows: lanes read 32 tasks at a time
      int j0 = 0;
      for (int i0 = 0; i0 < G.y; i0 += 32) {
        const int i = i0 + lane;
        ProjTask T{};
        if (i < G.y) T = tasks[gtask[G.x + i]];
        const int kk = i < G.y ? T.k : 0;
        int incl = kk;  // inclusive prefix of the ranks over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const int j = j0 + incl - kk;
        for (int q = 0; q < kk; ++q)
          srow[j + q] = GrpRow{T.mat + (int64_t)q * T.ld + T.r0, T.out, T.k, q};
        j0 += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncthreads();
    const float* xb = xt + T0.base + T0.r0;
    for (int c0 = 0; c0 < P.nrhs && pp.ok; c0 += 32) {
      const int nf = nst * nt;
      // fill i: stage i / nt, tile i % nt (B with the stage's first tile)
      auto issue = [&](int i) {
        pp.acquire(status);
        if (!pp.ok) return;
        const int st = i / nt, m = i - st * nt;
        unsigned char* sA = t5_smem + (pp.gs & 1) * kT5ABytes;
        const int r = st * kT5K + 2 * lane;
        const bool r0ok = r < nr, r1ok = r + 1 < nr;
        for (int jl = warp; jl < 128; jl += 8) {
          const int j = 128 * m + jl;
          if (j >= rows) break;
          unsigned char* dst = sA + t5_off(jl, 2 * lane);
          const __nv_bfloat16* src = fac + srow[j].col + r;
          if (r1ok)
            cp_async_small<4>(dst, src);  // even element offset
          else
            *reinterpret_cast<uint32_t*>(dst) =
                r0ok ? bf2_pack(src[0], __float2bfloat16_rn(0.f)) : 0u;
        }
        if (m == 0) {
          unsigned char* sB = t5_smem + 2 * kT5ABytes + (st & 1) * kT5BBytes;
          for (int c = warp; c < 32; c += 8) {
            const bool okc = c0 + c < P.nrhs;
            const float* xc = xb + (int64_t)(c0 + c) * P.n;
            const float v0 = (okc && r0ok) ? xc[r] : 0.f;
            const float v1 = (okc && r1ok) ? xc[r + 1] : 0.f;
            __nv_bfloat16 h0, l0, h1, l1;
            bf_split(v0, h0, l0);
            bf_split(v1, h1, l1);
            *reinterpret_cast<uint32_t*>(sB + t5_off(c, 2 * lane)) = bf2_pack(h0, h1);
            *reinterpret_cast<uint32_t*>(sB + t5_off(32 + c, 2 * lane)) = bf2_pack(l0, l1);
          }
        }
        cp_async_commit();
        ++pp.gs;
      };
      issue(0);
      for (int i = 0; i < nf && pp.ok; ++i) {
        if (i + 1 < nf) {
          issue(i + 1);
          if (!pp.ok) break;
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        tc5::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
          tc5::fence_after();
          const int st = i / nt, m = i - st * nt;
          const int fb = (pp.gs - (i + 1 < nf ? 2 : 1)) & 1;  // buffer of fill i
          unsigned char* sA = t5_smem + fb * kT5ABytes;
          unsigned char* sB = t5_smem + 2 * kT5ABytes + (st & 1) * kT5BBytes;
          const int nk = min(kT5K, nr - st * kT5K);
          for (int kk = 0; 16 * kk < nk; ++kk)
            tc5::mma_bf16(tm + 64 * m,
                          tc5::sdesc(tc5::smem_addr(sA) + kk * 2 * kT5Lbo, kT5Lbo, kT5Sbo),
                          tc5::sdesc(tc5::smem_addr(sB) + kk * 2 * kT5Lbo, kT5Lbo, kT5Sbo),
                          kT5Idesc, st > 0 || kk > 0);
          tc5::mma_commit(&bar[fb]);
        }
      }
      cp_async_wait<0>();
      pp.drain(status);
      tc5::fence_after();
      if (pp.ok) {
        for (int m = warp >> 2; m < nt; m += 2) {
          float hv[32], lv[32];
          const uint32_t ta = tm + ((uint32_t)(32 * (warp & 3)) << 16) + 64 * m;
          tc5::tmem_ld32(ta, hv);
          tc5::tmem_ld32(ta + 32, lv);
          const int j = 128 * m + 32 * (warp & 3) + lane;
          if (j < rows) {
            const GrpRow R = srow[j];
#pragma unroll
            for (int c = 0; c < 32; ++c)
              if (c0 + c < P.nrhs) part[R.out * P.nrhs + (int64_t)(c0 + c) * R.k + R.q] = hv[c] + lv[c];
          }
        }
      }
      tc5::fence_before();
      __syncthreads();  // TMEM and the row table read before the next pass or group
      tc5::fence_after();
    }
  }
  cp_async_wait<0>();
  pp.drain(status);
  pp.finish();
  tc5::fence_before();
  __syncthreads();
  if (warp == 0) tc5::tmem_dealloc(tm, kGrpTmem);
}

// Expansion: blocks of 128 threads walk the expansion tasks (<= 256 rows of
// one box each, grid-stride), 128-row tiles.  The columns of all the box's
// list entries are packed along K (entry after entry, in partner order):
// K-position j is column q of entry e, A(r, j) = U_e(r, q), B(n, j) = t_e
// (hi | lo) of column q, so that one MMA of K = 16 may span entries and a
// 16-point box with fifteen entries of rank 10 takes three stages, not
// fifteen.  Per pass of 32 right-hand sides, D[r, n] = sum over j; thread
// (warp w, lane i) holds row r = 32 w + i of D and writes
// y_r = D[r, c] + D[r, 32 + c] to the level's slab, where k_exp2 puts it.
__device__ __forceinline__ int t5_entry(const int* kpre, int ne, int j) {
  int e = 0;
  while (e + 1 < ne && kpre[e + 1] <= j) ++e;
  return e;
}

__global__ void __launch_bounds__(128)
    k_exp_t5(ArgsV2 P, const ExpTask* __restrict__ tasks, int64_t ntasks,
             const float* __restrict__ t, float* __restrict__ yl, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char t5_smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tslot;
  __shared__ int64_t s_off[kExpMaxEnt];
  __shared__ int64_t s_toff[kExpMaxEnt];
  __shared__ int s_k[kExpMaxEnt];
  __shared__ int s_kpre[kExpMaxEnt + 1];  // K-positions before entry e
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc5::mbar_init(&bar[0], 1);
    tc5::mbar_init(&bar[1], 1);
  }
  if (warp == 0) tc5::tmem_alloc(&tslot, 64);
  tc5::fence_before();
  __syncthreads();
  tc5::fence_after();
  const uint32_t tm = tslot;
  T5Pipe pp;
  pp.bar = bar;
  for (int64_t ti = blockIdx.x; ti < ntasks && pp.ok; ti += gridDim.x) {
    const ExpTask T = tasks[ti];
    const int l = T.level;
    const LevelV2& L = P.lev[l];
    const uint32_t X = (uint32_t)T.box;
    const int32_t e0 = L.ent_off[X], ne = L.ent_off[X + 1] - e0;
    for (int e = tid; e < ne; e += blockDim.x) {
      const int32_t code = L.ent[e0 + e];
      const int64_t p = code >> 1;
      const int side = code & 1;
      const int k = L.rank[p];
      int64_t off = L.foff[p];
      if (side == 1) off += ldpad(bsize(P.leaf_off, P.kappa, l, (uint32_t)L.px[p])) * k;
      s_off[e] = off;
      s_k[e] = k;
      s_toff[e] = L.toff[p] * P.nrhs + (int64_t)side * k * P.nrhs;
    }
    __syncthreads();
    if (tid == 0) {
      int a = 0;
      for (int e = 0; e < ne; ++e) {
        s_kpre[e] = a;
        a += s_k[e];
      }
      s_kpre[ne] = a;
    }
    __syncthreads();
    const int ktot = s_kpre[ne];
    const int nst = (ktot + kT5K - 1) / kT5K;
    const int32_t base = bstart(P.leaf_off, P.kappa, l, X);
    const int64_t ld = ldpad(bsize(P.leaf_off, P.kappa, l, X));
    const __nv_bfloat16* fac = reinterpret_cast<const __nv_bfloat16*>(L.fac);
    for (int c0 = 0; c0 < P.nrhs && pp.ok; c0 += 32) {
      for (int rt = 0; rt < T.nr && pp.ok; rt += 128) {
        const int rows = min(128, T.nr - rt);
        for (int st = 0; st < nst && pp.ok; ++st) {
          pp.acquire(status);
          if (!pp.ok) break;
          unsigned char* sA = t5_smem + (pp.gs & 1) * kT5ABytes;
          unsigned char* sB = t5_smem + 2 * kT5ABytes + (pp.gs & 1) * kT5BBytes;
          const int j0 = st * kT5K;
          // A: rows (2 rp, 2 rp + 1) of the tile, K-positions j0 + 8 q8 .. + 7
          // (rows past the tile are left as they are: they only feed rows of
          // D that are not written)
          for (int it = tid; it < 64 * (kT5K / 8); it += 128) {
            const int rp = it & 63, q8 = it >> 6;
            const int r = 2 * rp;
            if (r >= rows) continue;
            uint32_t w[8];
            int e = t5_entry(s_kpre, ne, min(j0 + 8 * q8, ktot - 1));
#pragma unroll
            for (int e2 = 0; e2 < 8; ++e2) {
              const int j = j0 + 8 * q8 + e2;
              w[e2] = 0u;
              if (j < ktot) {
                while (s_kpre[e + 1] <= j) ++e;
                const __nv_bfloat16* c =
                    fac + s_off[e] + (int64_t)(j - s_kpre[e]) * ld + T.r0 + rt + r;
                if (r + 1 < rows)
                  w[e2] = *reinterpret_cast<const uint32_t*>(c);  // even offset
                else
                  w[e2] = bf2_pack(c[0], __float2bfloat16_rn(0.f));
              }
            }
            uint4 ra, rb;  // row r: the low halves, row r + 1: the high halves
            ra.x = __byte_perm(w[0], w[1], 0x5410);
            ra.y = __byte_perm(w[2], w[3], 0x5410);
            ra.z = __byte_perm(w[4], w[5], 0x5410);
            ra.w = __byte_perm(w[6], w[7], 0x5410);
            rb.x = __byte_perm(w[0], w[1], 0x7632);
            rb.y = __byte_perm(w[2], w[3], 0x7632);
            rb.z = __byte_perm(w[4], w[5], 0x7632);
            rb.w = __byte_perm(w[6], w[7], 0x7632);
            *reinterpret_cast<uint4*>(sA + t5_off(r, 8 * q8)) = ra;
            *reinterpret_cast<uint4*>(sA + t5_off(r + 1, 8 * q8)) = rb;
          }
          // B: t of right-hand side c0 + c at K-positions j0 + 8 q8 .. + 7
          for (int it = tid; it < 32 * (kT5K / 8); it += 128) {
            const int c = it & 31, q8 = it >> 5;
            const bool okc = c0 + c < P.nrhs;
            float v[8];
            int e = t5_entry(s_kpre, ne, min(j0 + 8 * q8, ktot - 1));
#pragma unroll
            for (int e2 = 0; e2 < 8; ++e2) {
              const int j = j0 + 8 * q8 + e2;
              v[e2] = 0.f;
              if (okc && j < ktot) {
                while (s_kpre[e + 1] <= j) ++e;
                v[e2] = t[s_toff[e] + (int64_t)(c0 + c) * s_k[e] + (j - s_kpre[e])];
              }
            }
            uint4 hi, lo;
            split8(v, hi, lo);
            *reinterpret_cast<uint4*>(sB + t5_off(c, 8 * q8)) = hi;
            *reinterpret_cast<uint4*>(sB + t5_off(32 + c, 8 * q8)) = lo;
          }
          tc5::fence_smem_to_async();
          __syncthreads();
          if (tid == 0) {
            tc5::fence_after();
            const int nk = min(kT5K, ktot - j0);
            for (int kk = 0; 16 * kk < nk; ++kk)
              tc5::mma_bf16(tm, tc5::sdesc(tc5::smem_addr(sA) + kk * 2 * kT5Lbo, kT5Lbo, kT5Sbo),
                            tc5::sdesc(tc5::smem_addr(sB) + kk * 2 * kT5Lbo, kT5Lbo, kT5Sbo),
                            kT5Idesc, st > 0 || kk > 0);
            tc5::mma_commit(&bar[pp.gs & 1]);
          }
          ++pp.gs;
        }
        pp.drain(status);
        tc5::fence_after();
        if (pp.ok) {
          float hv[32], lv[32];
          if (nst > 0) {
            const uint32_t ta = tm + ((uint32_t)(32 * warp) << 16);
            tc5::tmem_ld32(ta, hv);
            tc5::tmem_ld32(ta + 32, lv);
          } else {  // no entries: the level adds nothing to these rows
#pragma unroll
            for (int c = 0; c < 32; ++c) hv[c] = lv[c] = 0.f;
          }
          const int r = 32 * warp + lane;
          if (r < rows)
#pragma unroll
            for (int c = 0; c < 32; ++c)
              if (c0 + c < P.nrhs)
                yl[((int64_t)l * P.nrhs + c0 + c) * P.n + base + T.r0 + rt + r] = hv[c] + lv[c];
        }
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();
      }
    }
  }
  pp.drain(status);
  pp.finish();
  tc5::fence_before();
  __syncthreads();
  if (warp == 0) tc5::tmem_dealloc(tm, 64);
}

// t[pair, side, q] = sum of the chunk partials in chunk order: one warp per
// (pair, side, column); lane j sums chunks j, j + 32, ..., then a fixed
// shuffle tree adds the 32 lane sums (one right-hand side), or lane c sums
// all chunks of right-hand side c (several).  red[2 s] = {first task, count}.
template <class A>
__device__ __forceinline__ void tsum2_body(const ArgsV2& P, const ProjTask* __restrict__ tasks,
                                           const int64_t* __restrict__ red,
                                           const int64_t* __restrict__ sideq, int64_t nwork,
                                           const typename A::val* __restrict__ part,
                                           typename A::val* __restrict__ t, int64_t min_count,
                                           int64_t w) {
  using V = typename A::val;
  const int lane = threadIdx.x & 31;
  if (w >= nwork) return;
  const int64_t s = sideq[2 * w];
  const int q = (int)sideq[2 * w + 1];
  const int64_t first = red[2 * s], count = red[2 * s + 1];
  if (count < min_count) return;  // left to a thread-per-column form
  const ProjTask T0 = tasks[first];
  const LevelV2& L = P.lev[T0.level];
  const int k = L.rank[T0.pair];
  V* out = t + L.toff[T0.pair] * P.nrhs + (int64_t)T0.side * k * P.nrhs;
  if (P.nrhs > 1) {  // lane per right-hand side, chunks in order
    for (int c = lane; c < P.nrhs; c += 32) {
      V acc = A::vzero();
      for (int64_t j = 0; j < count; ++j)
        acc = A::add(acc, part[tasks[first + j].out * P.nrhs + c * k + q]);
      out[c * k + q] = acc;
    }
    return;
  }
  for (int c = 0; c < P.nrhs; ++c) {
    V acc = A::vzero();
    for (int64_t j = lane; j < count; j += 32)
      acc = A::add(acc, part[tasks[first + j].out * P.nrhs + c * k + q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = A::add(acc, shfl_val(acc, o));
    if (lane == 0) out[c * k + q] = acc;
  }
}
template <class A>
__global__ void __launch_bounds__(256)
    k_tsum2(ArgsV2 P, const ProjTask* __restrict__ tasks, const int64_t* __restrict__ red,
            const int64_t* __restrict__ sideq, int64_t nwork,
            const typename A::val* __restrict__ part, typename A::val* __restrict__ t,
            int64_t min_count = 0) {
  tsum2_body<A>(P, tasks, red, sideq, nwork, part, t, min_count,
                (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
}

// One block per expansion task (256 rows of one box): the box's list
// (matrix offset, rank, t offset per entry) is staged in shared memory once,
// then one thread per row sums U t1 / V t2 over the list in ascending partner
// order, eight independent loads at a time.

// The several-RHS expansion of one row (exp2_body), EC right-hand sides per
// pass over the box's list: each factor value is loaded once per pass.
template <class A, int EC>
__device__ __forceinline__ void exp2_multi(const ArgsV2& P, int ne, const int* s_k,
                                           const int64_t* s_off, const int64_t* s_toff,
                                           const typename A::fac* __restrict__ fac,
                                           const typename A::val* __restrict__ t,
                                           typename A::val* __restrict__ yl, int l, int64_t ld,
                                           int32_t base, int r) {
  using V = typename A::val;
  using Acc = typename A::acc;
  using F = typename A::fac;
  for (int c0 = 0; c0 < P.nrhs; c0 += EC) {
    Acc a[EC];
#pragma unroll
    for (int c = 0; c < EC; ++c) a[c] = A::zero();
    for (int e = 0; e < ne; ++e) {
      const int k = s_k[e];
      const F* M = fac + s_off[e] + r;
      const V* tv = t + s_toff[e];
#pragma unroll 4
      for (int q = 0; q < k; ++q) {
        const V mv = A::ld(M[q * ld]);
#pragma unroll
        for (int c = 0; c < EC; ++c)
          if (c0 + c < P.nrhs) A::fma(a[c], mv, tv[(int64_t)(c0 + c) * k + q]);
        if ((q + 1) % kRenorm == 0)
#pragma unroll
          for (int c = 0; c < EC; ++c) A::renorm(a[c]);
      }
#pragma unroll
      for (int c = 0; c < EC; ++c) A::renorm(a[c]);
    }
#pragma unroll
    for (int c = 0; c < EC; ++c)
      if (c0 + c < P.nrhs) yl[((int64_t)l * P.nrhs + c0 + c) * P.n + base + r] = A::fin(a[c]);
  }
}

// (blocks of 256 threads; every thread of the block calls it with the same
// task: it synchronises the block once)
template <class A>
__device__ __forceinline__ void exp2_body(const ArgsV2& P, const ExpTask* __restrict__ tasks,
                                          const typename A::val* __restrict__ t,
                                          typename A::val* __restrict__ yl, int64_t bid) {
  using V = typename A::val;
  using Acc = typename A::acc;
  using F = typename A::fac;
  __shared__ int64_t s_off[kExpMaxEnt];
  __shared__ int64_t s_toff[kExpMaxEnt];
  __shared__ int s_k[kExpMaxEnt];
  const ExpTask T = tasks[bid];
  const int l = T.level;
  const LevelV2& L = P.lev[l];
  const uint32_t X = (uint32_t)T.box;
  const int32_t e0 = L.ent_off[X], ne = L.ent_off[X + 1] - e0;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const int32_t code = L.ent[e0 + e];
    const int64_t p = code >> 1;
    const int side = code & 1;
    const int k = L.rank[p];
    int64_t off = L.foff[p];
    if (side == 1) off += ldpad(bsize(P.leaf_off, P.kappa, l, (uint32_t)L.px[p])) * k;
    s_off[e] = off;
    s_k[e] = k;
    s_toff[e] = L.toff[p] * P.nrhs + (int64_t)side * k * P.nrhs;
  }
  __syncthreads();
  const int r = T.r0 + (int)threadIdx.x;
  const bool act = r < T.r0 + T.nr;
  const int32_t base = bstart(P.leaf_off, P.kappa, l, X);
  const int64_t ld = ldpad(bsize(P.leaf_off, P.kappa, l, X));
  const F* fac = reinterpret_cast<const F*>(L.fac);
  if ((sizeof(F) == 2 || (std::is_same<A, F32A>::value && P.nrhs > 8)) && P.nrhs > 1) {
    // bfloat16 factors with several right-hand sides, binary32 with many:
    // the pass's t values of an entry are staged in shared memory, kExpQ
    // columns at a time, right-hand sides adjacent: one shared vector read
    // serves all EC sums of a factor value (the whole block takes part).
    // Measured at N = 2^20, 4 RHS: bfloat16 3.07 -> 1.42 ms; binary32 1.63 ->
    // 2.37 and float-float 3.81 -> 4.51 ms, so those keep the direct loads;
    // binary32 at 32 RHS gains (9.06 -> 8.41 ms) and stages above 8.
    constexpr int EC = sizeof(typename A::acc) == 4 ? 8 : 4;
    __shared__ __align__(16) V s_t[kExpQ][EC];
    for (int c0 = 0; c0 < P.nrhs; c0 += EC) {
      const int nc = min(EC, P.nrhs - c0);
      Acc a[EC];
#pragma unroll
      for (int c = 0; c < EC; ++c) a[c] = A::zero();
      for (int e = 0; e < ne; ++e) {
        const int k = s_k[e];
        const F* M = fac + s_off[e] + (act ? r : T.r0);
        const V* tv = t + s_toff[e];
        for (int q0 = 0; q0 < k; q0 += kExpQ) {
          const int qn = min(kExpQ, k - q0);
          __syncthreads();  // the previous columns are used up
          for (int i = threadIdx.x; i < EC * qn; i += blockDim.x) {
            const int c = i / qn, q = i - c * qn;
            s_t[q][c] = c < nc ? tv[(int64_t)(c0 + c) * k + q0 + q] : A::vzero();
          }
          __syncthreads();
          if (!act) continue;
#pragma unroll 4
          for (int q = 0; q < qn; ++q) {
            const V mv = A::ld(M[(int64_t)(q0 + q) * ld]);
#pragma unroll
            for (int c = 0; c < EC; ++c)
              if (c < nc) A::fma(a[c], mv, s_t[q][c]);
            if ((q0 + q + 1) % kRenorm == 0)
#pragma unroll
              for (int c = 0; c < EC; ++c) A::renorm(a[c]);
          }
        }
#pragma unroll
        for (int c = 0; c < EC; ++c) A::renorm(a[c]);
      }
      if (act)
#pragma unroll
        for (int c = 0; c < EC; ++c)
          if (c < nc) yl[((int64_t)l * P.nrhs + c0 + c) * P.n + base + r] = A::fin(a[c]);
    }
    return;
  }
  if (!act) return;
  if (P.nrhs > 1) {  // EC right-hand sides per pass: each factor value loaded once per pass
    // (float-float: 8 per pass above 8 right-hand sides, half the passes
    // over the factors; 32 RHS at N = 2^20: 126 -> 115 ms for the product,
    // where binary32 with 16 per pass lost: expansions 9.06 -> 9.58 ms)
    constexpr int EC = sizeof(typename A::acc) == 4 ? 8 : 4;
    if (std::is_same<A, DF32A>::value && P.nrhs > 8)
      exp2_multi<A, 2 * EC>(P, ne, s_k, s_off, s_toff, fac, t, yl, l, ld, base, r);
    else
      exp2_multi<A, EC>(P, ne, s_k, s_off, s_toff, fac, t, yl, l, ld, base, r);
    return;
  }
  for (int c = 0; c < P.nrhs; ++c) {
    Acc a = A::zero();
    for (int e = 0; e < ne; ++e) {
      const int k = s_k[e];
      const F* M = fac + s_off[e] + r;
      const V* tv = t + s_toff[e] + (int64_t)c * k;
      int q = 0;
      for (; q + 8 <= k; q += 8) {  // eight independent loads in flight
        F mv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) mv[u] = M[(q + u) * ld];
#pragma unroll
        for (int u = 0; u < 8; ++u) A::fma(a, A::ld(mv[u]), tv[q + u]);
        if ((q + 8) % kRenorm == 0) A::renorm(a);
      }
      for (; q < k; ++q) A::fma(a, A::ld(M[q * ld]), tv[q]);
      A::renorm(a);  // one renormalisation per list entry at least
    }
    yl[((int64_t)l * P.nrhs + c) * P.n + base + r] = A::fin(a);
  }
}
template <class A>
__global__ void __launch_bounds__(256)
    k_exp2(ArgsV2 P, const ExpTask* __restrict__ tasks, const typename A::val* __restrict__ t,
           typename A::val* __restrict__ yl) {
  exp2_body<A>(P, tasks, t, yl, blockIdx.x);
}

// ---------------------------------------------------------------------------
// combine: y[perm[i]] = near + sum over levels of (own / two-pass result)
// + the partials of the pairs in which the point's box is the column side
// ---------------------------------------------------------------------------
template <class A>
__device__ __forceinline__ void combine2_body(const ArgsV2& P,
                                              const typename A::val* __restrict__ yl,
                                              const typename A::val* __restrict__ ppart,
                                              const int32_t* __restrict__ leaf_of,
                                              const int64_t* __restrict__ perm,
                                              double* __restrict__ y, int64_t i) {
  using V = typename A::val;
  if (i >= P.n) return;
  const uint32_t leaf = (uint32_t)leaf_of[i];
  const int64_t g = perm[i];
  for (int c = 0; c < P.nrhs; ++c) {
    V acc = yl[(int64_t)c * P.n + i];
    const V* pc = ppart + (int64_t)c * P.pstride;
    for (int l = 1; l <= P.kappa; ++l) {
      const int mode = P.lmode[l];
      if (mode != LMODE_PAIR) acc = A::add(acc, yl[((int64_t)l * P.nrhs + c) * P.n + i]);
      if (mode == LMODE_TWO) continue;
      const LevelV2& L = P.lev[l];
      const uint32_t B = leaf >> (2 * (P.kappa - l));
      const int64_t loc = i - bstart(P.leaf_off, P.kappa, l, B);
      const int32_t e1 = L.ent_off[B + 1];
#pragma unroll 4
      for (int32_t e = L.ent_off[B]; e < e1; ++e) {
        const int64_t w = L.entpp[e];
        if (mode == LMODE_BOX && (w & 1) == 0) continue;  // own sums are in the slab
        acc = A::add(acc, pc[(w >> 1) + loc]);
      }
    }
    y[g + (int64_t)c * P.n] = A::to_double(acc);
  }
}
template <class A>
__global__ void k_combine2(ArgsV2 P, const typename A::val* __restrict__ yl,
                           const typename A::val* __restrict__ ppart,
                           const int32_t* __restrict__ leaf_of, const int64_t* __restrict__ perm,
                           double* __restrict__ y) {
  combine2_body<A>(P, yl, ppart, leaf_of, perm, y, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// entry e of a box list (pair * 2 + side) -> that side's partial offset << 1 | side
__global__ void k_entpp(const int32_t* __restrict__ ent, int64_t nent,
                        const int64_t* __restrict__ ppoff, int64_t* __restrict__ entpp) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nent) return;
  const int32_t code = ent[e];
  entpp[e] = (ppoff[code] << 1) | (code & 1);
}

__global__ void k_leaf_of(const int32_t* __restrict__ leaf_off, int64_t nleaf,
                          int32_t* __restrict__ leaf_of) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nleaf) return;
  for (int32_t i = leaf_off[b]; i < leaf_off[b + 1]; ++i) leaf_of[i] = (int32_t)b;
}

__global__ void k_to_ff(const double* __restrict__ a, float2* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = DF32A::from_double(a[i]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// A box level runs the box kernel in binary64 only; the other modes run it as
// pairs (the sub-warp register kernel for one right-hand side, staged in
// float-float, measured faster than the box kernel; the multi-RHS register
// kernel for several).
static bool box_as_pairs(const hodlr2d* h, int l, int nrhs, int mode) {
  (void)h;
  (void)l;
  (void)nrhs;
  return mode != HODLR2D_MODE_F64;
}

// First level that is not run in two passes by a product:
//   binary64                    lfuse (pairs from there on)
//   several right-hand sides    l2max (boxes of <= kMultiRows points as pairs;
//                               few_rhs: l2few, boxes of <= kMultiRowsFew)
//   one right-hand side         ldual (the 512 x 9 register forms hold the
//                               boxes of [ldual, lfuse): two columns per
//                               step in binary32, one in float-float)
static int two_pass_end(const hodlr2d* h, int nrhs, int mode) {
  const V2Plan& V = h->v2;
  if (mode == HODLR2D_MODE_F64) return V.lfuse;
  if (nrhs > 1) return few_rhs(nrhs, mode) ? V.l2few : V.l2max;
  return V.ldual;
}

static ArgsV2 args_v2(const hodlr2d* h, int nrhs, int mode) {
  ArgsV2 P;
  for (int l = 0; l < HODLR2D_MAX_LEVELS; ++l) {
    const Level& L = h->lev[l];
    const void* fac = mode == HODLR2D_MODE_F64 ? (const void*)L.d_fac : L.d_fac_mode[mode];
    P.lev[l] = LevelV2{L.d_px, L.d_py, L.d_rank, L.d_foff, L.d_prow, L.d_ppoff,
                       L.d_toff, L.d_ent_off, L.d_ent, fac, L.d_meta, L.d_entpp};
  }
  const int l2end = two_pass_end(h, nrhs, mode);
  for (int l = 0; l < HODLR2D_MAX_LEVELS; ++l) {
    const int base = h->v2.lmode[l];
    if (l < l2end)
      P.lmode[l] = LMODE_TWO;
    else if (base == LMODE_BOX)
      P.lmode[l] = box_as_pairs(h, l, nrhs, mode) ? LMODE_PAIR : LMODE_BOX;
    else
      P.lmode[l] = LMODE_PAIR;  // pair levels, and two-pass levels with a pair plan
  }
  P.leaf_off = h->d_leaf_off;
  P.kappa = h->kappa;
  P.lfuse = h->v2.lfuse;
  P.n = h->n;
  P.nrhs = nrhs;
  P.pstride = h->v2.pstride;
  return P;
}

// Two-pass plan of levels [1, lmax): the projection tasks (pair, side, row
// chunk), their grouping by box for the tensor cores and by column group for
// binary64, the chunk-sum work and the expansion tasks (one per 256 rows of
// a box).  Built for [1, l2max) with the plan, and for every level the first
// time a product runs all levels in two passes (bfloat16, several
// right-hand sides).
static int build_two_pass(hodlr2d* h, int lmax) {
  V2Plan& V = h->v2;
  const int kappa = h->kappa;
  for (void* q : {(void*)V.d_proj, (void*)V.d_exp, (void*)V.d_red, (void*)V.d_wtask,
                  (void*)V.d_sideq, (void*)V.d_pgrp, (void*)V.d_gtask, (void*)V.d_grp})
    cudaFree(q);
  V.d_proj = nullptr;
  V.d_exp = nullptr;
  V.d_red = nullptr;
  V.d_wtask = nullptr;
  V.d_sideq = nullptr;
  V.d_pgrp = nullptr;
  V.d_gtask = nullptr;
  V.d_grp = nullptr;
  V.grp_ok = true;
  std::vector<ProjTask> proj;
  std::vector<ExpTask> exps;
  std::vector<int64_t> red;
  int64_t out = 0;
  int64_t pre_sides[HODLR2D_MAX_LEVELS + 1] = {};
  for (int l = 1; l < lmax; ++l) {
    // the task lists are level-ordered: record the counts below level l
    V.pre_proj[l] = (int64_t)proj.size();
    V.pre_exp[l] = (int64_t)exps.size();
    V.pre_part[l] = out;
    pre_sides[l] = (int64_t)red.size() / 2;
    Level& L = h->lev[l];
    const int64_t np = L.npairs;
    const int sh = 2 * (kappa - l);
    auto cnt = [&](int32_t b) {
      return (int32_t)(h->h_leaf_off[(int64_t)(b + 1) << sh] - h->h_leaf_off[(int64_t)b << sh]);
    };
    std::vector<int32_t> px(np), py(np);
    if (np) {
      H2D_CK(cudaMemcpy(px.data(), L.d_px, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
      H2D_CK(cudaMemcpy(py.data(), L.d_py, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    }
    for (int64_t p = 0; p < np; ++p) {
      const int k = L.h_rank[p];
      for (int side = 0; side < 2; ++side) {
        const int32_t rows = side == 0 ? cnt(py[p]) : cnt(px[p]);
        const int64_t first = (int64_t)proj.size();
        if (k > 0)
          for (int32_t r0 = 0; r0 < rows; r0 += kChunkP) {
            ProjTask T;
            T.level = l;
            T.side = side;
            T.pair = p;
            T.r0 = r0;
            T.nr = std::min(kChunkP, rows - r0);
            T.out = out;
            T.mat = L.h_foff[p] + (side == 0 ? ldpad(cnt(px[p])) * k : 0);
            T.ld = (int32_t)ldpad(rows);
            T.base = (int32_t)h->h_leaf_off[(int64_t)(side == 0 ? py[p] : px[p]) << sh];
            T.k = k;
            T.pad = 0;
            out += k;
            proj.push_back(T);
          }
        red.push_back(first);
        red.push_back((int64_t)proj.size() - first);
      }
    }
    for (int64_t b = 0; b < ((int64_t)1 << (2 * l)); ++b) {
      const int32_t rows = cnt((int32_t)b);
      for (int32_t r0 = 0; r0 < rows; r0 += kChunk2)
        exps.push_back(ExpTask{l, (int32_t)b, r0, std::min(kChunk2, rows - r0)});
    }
  }
  V.nproj = (int64_t)proj.size();
  V.nexp = (int64_t)exps.size();
  for (int l = lmax; l <= HODLR2D_MAX_LEVELS; ++l) {
    V.pre_proj[l] = V.nproj;
    V.pre_exp[l] = V.nexp;
    V.pre_part[l] = out;
    pre_sides[l] = (int64_t)red.size() / 2;
  }
  {  // bfloat16 tensor-core projection: tasks grouped by (level, box, row chunk)
    std::vector<int32_t> order(proj.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      const ProjTask &A = proj[a], &B = proj[b];
      if (A.level != B.level) return A.level < B.level;
      if (A.base != B.base) return A.base < B.base;
      return A.r0 < B.r0;
    });
    std::vector<int4> grp;
    size_t i = 0;
    while (i < order.size()) {
      const ProjTask& T = proj[order[i]];
      int4 g = make_int4((int)i, 0, 0, T.level);
      while (i < order.size()) {
        const ProjTask& U = proj[order[i]];
        if (U.level != T.level || U.base != T.base || U.r0 != T.r0) break;
        if (g.y > 0 && g.z + U.k > kGrpRows) break;
        if (U.k > kGrpRows) V.grp_ok = false;  // a rank beyond one group: per-task kernel
        g.y += 1;
        g.z += U.k;
        ++i;
      }
      grp.push_back(g);
    }
    for (int l = 1; l <= HODLR2D_MAX_LEVELS; ++l) {
      int64_t c = 0;
      while (c < (int64_t)grp.size() && grp[c].w < l) ++c;
      V.pre_grp[l] = c;
    }
    H2D_CK(cudaMalloc(&V.d_gtask, sizeof(int32_t) * std::max<size_t>(order.size(), 1)));
    H2D_CK(cudaMalloc(&V.d_grp, sizeof(int4) * std::max<size_t>(grp.size(), 1)));
    if (!order.empty())
      H2D_CK(cudaMemcpy(V.d_gtask, order.data(), sizeof(int32_t) * order.size(),
                        cudaMemcpyHostToDevice));
    if (!grp.empty())
      H2D_CK(cudaMemcpy(V.d_grp, grp.data(), sizeof(int4) * grp.size(), cudaMemcpyHostToDevice));
  }
  {  // binary64 projection work: (task, first column) per group of kProj64Cols columns
    std::vector<int2> pg;
    for (int64_t t = 0; t < (int64_t)proj.size(); ++t) {
      for (int q0 = 0; q0 < proj[t].k; q0 += kProj64Cols) pg.push_back(make_int2((int)t, q0));
    }
    // groups of the tasks below level l (the task list is level-ordered)
    {
      int64_t gi = 0;
      int l = 1;
      for (int64_t t = 0; t <= (int64_t)proj.size(); ++t) {
        while (l <= HODLR2D_MAX_LEVELS && V.pre_proj[l] <= t) V.pre_pgrp[l++] = gi;
        if (t < (int64_t)proj.size()) gi += (proj[t].k + kProj64Cols - 1) / kProj64Cols;
      }
      while (l <= HODLR2D_MAX_LEVELS) V.pre_pgrp[l++] = gi;
    }
    H2D_CK(cudaMalloc(&V.d_pgrp, sizeof(int2) * std::max<size_t>(pg.size(), 1)));
    if (!pg.empty())
      H2D_CK(cudaMemcpy(V.d_pgrp, pg.data(), sizeof(int2) * pg.size(), cudaMemcpyHostToDevice));
  }
  {
    std::vector<int32_t> wt(std::max<int64_t>(out, 1));
    for (int64_t t = 0; t < V.nproj; ++t) {
      const int k = h->lev[proj[t].level].h_rank[proj[t].pair];
      for (int q = 0; q < k; ++q) wt[proj[t].out + q] = (int32_t)t;
    }
    std::vector<int64_t> sq;
    std::vector<int64_t> sq_at_side((int64_t)red.size() / 2 + 1, 0);  // sq entries before side sd
    for (int64_t sd = 0; sd < (int64_t)red.size() / 2; ++sd) {
      sq_at_side[sd] = (int64_t)sq.size() / 2;
      if (red[2 * sd + 1] == 0) continue;
      const ProjTask& T0 = proj[red[2 * sd]];
      const int k = h->lev[T0.level].h_rank[T0.pair];
      for (int q = 0; q < k; ++q) {
        sq.push_back(sd);
        sq.push_back(q);
      }
    }
    V.ntsum = (int64_t)sq.size() / 2;
    sq_at_side[(int64_t)red.size() / 2] = V.ntsum;
    for (int l = 1; l <= HODLR2D_MAX_LEVELS; ++l) V.pre_tsum[l] = sq_at_side[pre_sides[l]];
    H2D_CK(cudaMalloc(&V.d_wtask, sizeof(int32_t) * wt.size()));
    H2D_CK(cudaMemcpy(V.d_wtask, wt.data(), sizeof(int32_t) * wt.size(), cudaMemcpyHostToDevice));
    H2D_CK(cudaMalloc(&V.d_sideq, sizeof(int64_t) * std::max<size_t>(sq.size(), 2)));
    if (!sq.empty())
      H2D_CK(cudaMemcpy(V.d_sideq, sq.data(), sizeof(int64_t) * sq.size(), cudaMemcpyHostToDevice));
  }
  V.proj_partials = out;
  V.nsides = (int64_t)red.size() / 2;
  H2D_CK(cudaMalloc(&V.d_proj, sizeof(ProjTask) * std::max<int64_t>(V.nproj, 1)));
  H2D_CK(cudaMalloc(&V.d_exp, sizeof(ExpTask) * std::max<int64_t>(V.nexp, 1)));
  H2D_CK(cudaMalloc(&V.d_red, sizeof(int64_t) * std::max<int64_t>((int64_t)red.size(), 2)));
  if (V.nproj)
    H2D_CK(cudaMemcpy(V.d_proj, proj.data(), sizeof(ProjTask) * V.nproj, cudaMemcpyHostToDevice));
  if (V.nexp)
    H2D_CK(cudaMemcpy(V.d_exp, exps.data(), sizeof(ExpTask) * V.nexp, cudaMemcpyHostToDevice));
  if (!red.empty())
    H2D_CK(cudaMemcpy(V.d_red, red.data(), sizeof(int64_t) * red.size(), cudaMemcpyHostToDevice));
  V.two_levels = lmax;
  ++h->gen;
  return HODLR2D_OK;
}

// Plan of the v2 product (once per handle, after the factors exist).
int plan_v2(hodlr2d* h) {
  V2Plan& V = h->v2;
  if (V.ready) return HODLR2D_OK;
  const int kappa = h->kappa;
  // the box kernel's two slices per warp exceed the default 48 KB
  H2D_CK(cudaFuncSetAttribute(k_box<F64A>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBoxSmem));
  H2D_CK(cudaFuncSetAttribute(k_box<DF32A>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBoxSmem));
  H2D_CK(cudaFuncSetAttribute(k_box<F32A>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBoxSmem));
  H2D_CK(cudaFuncSetAttribute(k_box<BF16A>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBoxSmem));
  H2D_CK(cudaFuncSetAttribute(k_pair64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kPair64Smem));
  H2D_CK(cudaFuncSetAttribute(k_proj_t5, cudaFuncAttributeMaxDynamicSharedMemorySize, kT5Smem));
  H2D_CK(cudaFuncSetAttribute(k_projg_t5, cudaFuncAttributeMaxDynamicSharedMemorySize, kGrpSmem));
  H2D_CK(cudaFuncSetAttribute(k_exp_t5, cudaFuncAttributeMaxDynamicSharedMemorySize, kT5Smem));
  H2D_CK(cudaMalloc(&V.d_status, sizeof(int)));
  H2D_CK(cudaMemset(V.d_status, 0, sizeof(int)));
  auto maxcount = [&](int l) {
    const int sh = 2 * (kappa - l);
    int64_t mx = 0;
    for (int64_t b = 0; b < ((int64_t)1 << (2 * l)); ++b)
      mx = std::max<int64_t>(mx, h->h_leaf_off[(b + 1) << sh] - h->h_leaf_off[b << sh]);
    return mx;
  };
  V.lfuse = kappa + 1;
  for (int l = 1; l <= kappa; ++l)
    if (maxcount(l) <= kFuseRows) { V.lfuse = l; break; }
  for (int l = V.lfuse; l <= kappa; ++l)  // the pair kernel holds at most kPairKmax terms
    if (h->lev[l].max_rank > kPairKmax) V.lfuse = l + 1;
  // two-pass levels that may also run as pairs, [ldual, lfuse): boxes of at
  // most kDualRows points, ranks of at most kDualKmax (a pair block steps
  // through its columns one reduction at a time), and enough pairs (two per
  // SM) that one block per pair fills the GPU
  {
    int dev = 0;
    H2D_CK(cudaGetDevice(&dev));
    H2D_CK(cudaDeviceGetAttribute(&V.nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  V.ldual = V.lfuse;
  while (V.ldual > 1 && maxcount(V.ldual - 1) <= kDualRows &&
         h->lev[V.ldual - 1].max_rank <= kDualKmax &&
         h->lev[V.ldual - 1].npairs >= 2 * (int64_t)V.nsm)
    --V.ldual;
  // pair levels with boxes of more than kMultiRows points also get a two-pass
  // plan, which several right-hand sides use: [lfuse, l2max)
  V.l2max = V.lfuse;
  while (V.l2max <= kappa && maxcount(V.l2max) > kMultiRows) ++V.l2max;
  V.l2few = V.lfuse;
  while (V.l2few <= kappa && maxcount(V.l2few) > kMultiRowsFew) ++V.l2few;
  H2D_TRY(build_two_pass(h, V.l2max));
  // single-read levels: pair mode (one block per pair, partials for both
  // sides) or box mode (one warp per row box, partials for the column side)
  std::vector<BoxWork> bw;
  int64_t pbase = 0;
  for (int l = 1; l <= kappa; ++l) V.lmode[l] = l < V.lfuse ? LMODE_TWO : LMODE_PAIR;
  V.lpair_small = kappa + 1;
  for (int l = V.ldual; l <= kappa; ++l) {
    Level& L = h->lev[l];
    const int64_t np = L.npairs;
    const int sh = 2 * (kappa - l);
    const int64_t mc = maxcount(l);
    if (l >= V.lfuse) V.lmode[l] = mc <= kBoxRows ? LMODE_BOX : LMODE_PAIR;
    std::vector<int32_t> px(np), py(np);
    if (np) {
      H2D_CK(cudaMemcpy(px.data(), L.d_px, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
      H2D_CK(cudaMemcpy(py.data(), L.d_py, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    }
    auto cnt = [&](int32_t b) {
      return h->h_leaf_off[(int64_t)(b + 1) << sh] - h->h_leaf_off[(int64_t)b << sh];
    };
    std::vector<int64_t> pp(2 * np + 2);
    for (int64_t p = 0; p < np; ++p) {
      pp[2 * p] = pbase;  // pair layout also for box levels (they may run as pairs)
      pbase += cnt(px[p]);
      pp[2 * p + 1] = pbase;
      pbase += cnt(py[p]);
    }
    pp[2 * np] = pp[2 * np + 1] = pbase;
    H2D_CK(cudaMalloc(&L.d_ppoff, sizeof(int64_t) * (2 * np + 2)));
    H2D_CK(cudaMemcpy(L.d_ppoff, pp.data(), sizeof(int64_t) * (2 * np + 2), cudaMemcpyHostToDevice));
    H2D_CK(cudaMalloc(&L.d_entpp, sizeof(int64_t) * std::max<int64_t>(L.nent, 1)));
    if (L.nent > 0) {
      k_entpp<<<(unsigned)((L.nent + 255) / 256), 256>>>(L.d_ent, L.nent, L.d_ppoff, L.d_entpp);
      H2D_CK(cudaGetLastError());
    }
    if (V.lmode[l] == LMODE_TWO) {
      // dual level: pair plan only
    } else if (V.lmode[l] == LMODE_PAIR) {
      if (mc <= kSmallPair) V.lpair_small = std::min(V.lpair_small, l);
    } else {
      std::vector<int64_t> prow(((int64_t)1 << (2 * l)) + 1);
      H2D_CK(cudaMemcpy(prow.data(), L.d_prow, sizeof(int64_t) * prow.size(),
                        cudaMemcpyDeviceToHost));
      for (int64_t b = 0; b < ((int64_t)1 << (2 * l)); ++b)
        if (cnt((int32_t)b) > 0) {
          BoxWork w;
          w.level = l;
          w.np = (int32_t)(prow[b + 1] - prow[b]);
          w.p0 = prow[b];
          w.xs = (int32_t)h->h_leaf_off[b << sh];
          w.m = (int32_t)cnt((int32_t)b);
          bw.push_back(w);
        }
    }
  }
  V.pstride = std::max<int64_t>(pbase, 1);
  for (int l = 1; l <= kappa; ++l) {  // one record per stored pair
    Level& L = h->lev[l];
    const int64_t np = L.npairs;
    if (!np) continue;
    const int sh = 2 * (kappa - l);
    std::vector<int32_t> px(np), py(np);
    H2D_CK(cudaMemcpy(px.data(), L.d_px, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    H2D_CK(cudaMemcpy(py.data(), L.d_py, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    std::vector<int64_t> pp(2 * np + 2, 0);
    if (L.d_ppoff)
      H2D_CK(cudaMemcpy(pp.data(), L.d_ppoff, sizeof(int64_t) * (2 * np + 2), cudaMemcpyDeviceToHost));
    std::vector<PairMeta> meta(np);
    for (int64_t p = 0; p < np; ++p) {
      PairMeta& M = meta[p];
      M.foff = L.h_foff[p];
      M.ppx = pp[2 * p];
      M.ppy = pp[2 * p + 1];
      M.k = L.h_rank[p];
      M.xs = h->h_leaf_off[(int64_t)px[p] << sh];
      M.m = h->h_leaf_off[(int64_t)(px[p] + 1) << sh] - M.xs;
      M.ys = h->h_leaf_off[(int64_t)py[p] << sh];
      M.n = h->h_leaf_off[(int64_t)(py[p] + 1) << sh] - M.ys;
      M.pad = 0;
    }
    H2D_CK(cudaMalloc(&L.d_meta, sizeof(PairMeta) * np));
    H2D_CK(cudaMemcpy(L.d_meta, meta.data(), sizeof(PairMeta) * np, cudaMemcpyHostToDevice));
  }
  // pair work lists, one per single-read or dual level
  for (int l = V.ldual; l <= kappa; ++l) {
    Level& L = h->lev[l];
    PairLevel& G = V.plev[l];
    const int64_t np = L.npairs;
    const int sh = 2 * (kappa - l);
    std::vector<int32_t> px(np), py(np);
    if (np) {
      H2D_CK(cudaMemcpy(px.data(), L.d_px, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
      H2D_CK(cudaMemcpy(py.data(), L.d_py, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    }
    auto cnt = [&](int32_t b) {
      return h->h_leaf_off[(int64_t)(b + 1) << sh] - h->h_leaf_off[(int64_t)b << sh];
    };
    std::vector<int2> cls_work[kPairClasses];
    for (int64_t p = 0; p < np; ++p) {
      if (L.h_rank[p] <= 0) continue;
      const int rows = (int)std::max(cnt(px[p]), cnt(py[p]));
      int c = 0;
      while (rows > kPairClassRows[c]) ++c;
      cls_work[c].push_back(make_int2(l, (int)p));
      G.cls_rows[c] = std::max(G.cls_rows[c], rows);
      G.max_rows = std::max(G.max_rows, rows);
    }
    std::vector<int2> wl;
    for (int c = 0; c < kPairClasses; ++c) {
      G.off[c] = (int64_t)wl.size();
      wl.insert(wl.end(), cls_work[c].begin(), cls_work[c].end());
    }
    G.off[kPairClasses] = (int64_t)wl.size();
    G.nwork = (int64_t)wl.size();
    G.h_work = wl;
    H2D_CK(cudaMalloc(&G.d_work, sizeof(int2) * std::max<int64_t>(G.nwork, 1)));
    if (G.nwork)
      H2D_CK(cudaMemcpy(G.d_work, wl.data(), sizeof(int2) * G.nwork, cudaMemcpyHostToDevice));
  }
  V.nbw = (int64_t)bw.size();
  H2D_CK(cudaMalloc(&V.d_bw, sizeof(BoxWork) * std::max<int64_t>(V.nbw, 1)));
  if (V.nbw) H2D_CK(cudaMemcpy(V.d_bw, bw.data(), sizeof(BoxWork) * V.nbw, cudaMemcpyHostToDevice));
  // pair-mode values of partial results need zero for pairs of rank 0
  V.zero_partials = false;
  for (int l = V.ldual; l <= kappa; ++l)
    for (int64_t p = 0; p < h->lev[l].npairs; ++p)
      if (h->lev[l].h_rank[p] == 0) V.zero_partials = true;
  // near-field work items: (leaf, first target), at most 32 targets each
  {
    std::vector<int2> nw;
    const int64_t nl = (int64_t)1 << (2 * kappa);
    const int side = 1 << kappa;
    V.near_entries = 0;
    for (int64_t b = 0; b < nl; ++b) {
      const int64_t m = h->h_leaf_off[b + 1] - h->h_leaf_off[b];
      for (int32_t t = 0; t < m; t += 32) nw.push_back(make_int2((int)b, t));
      int cx, cy;
      morton_decode((uint32_t)b, cx, cy);
      int64_t cols = m;
      const int ex[4] = {-1, 1, 0, 0}, ey[4] = {0, 0, -1, 1};
      for (int e = 0; e < 4; ++e) {
        const int qx = cx + ex[e], qy = cy + ey[e];
        if (qx < 0 || qy < 0 || qx >= side || qy >= side) continue;
        const uint32_t q = morton_encode((uint32_t)qx, (uint32_t)qy);
        cols += h->h_leaf_off[q + 1] - h->h_leaf_off[q];
      }
      V.near_entries += m * cols;
    }
    V.nnearw = (int64_t)nw.size();
    H2D_CK(cudaMalloc(&V.d_nearw, sizeof(int2) * std::max<int64_t>(V.nnearw, 1)));
    if (V.nnearw)
      H2D_CK(cudaMemcpy(V.d_nearw, nw.data(), sizeof(int2) * V.nnearw, cudaMemcpyHostToDevice));
  }
  // leaf of every tree position
  const int64_t nleaf = (int64_t)1 << (2 * kappa);
  H2D_CK(cudaMalloc(&V.d_leaf_of, sizeof(int32_t) * h->n));
  k_leaf_of<<<(unsigned)((nleaf + 255) / 256), 256>>>(h->d_leaf_off, nleaf, V.d_leaf_of);
  H2D_CK(cudaGetLastError());
  H2D_CK(cudaDeviceSynchronize());
  H2D_CK(cudaStreamCreateWithFlags(&V.s_near, cudaStreamNonBlocking));
  H2D_CK(cudaStreamCreateWithFlags(&V.s_far, cudaStreamNonBlocking));
  H2D_CK(cudaEventCreateWithFlags(&V.ev_in, cudaEventDisableTiming));
  H2D_CK(cudaEventCreateWithFlags(&V.ev_near, cudaEventDisableTiming));
  H2D_CK(cudaEventCreateWithFlags(&V.ev_far, cudaEventDisableTiming));
  V.ready = true;
  return HODLR2D_OK;
}

int scratch_v2(hodlr2d* h, int nrhs) {
  V2Plan& V = h->v2;
  if (V.scratch_nrhs >= nrhs) return HODLR2D_OK;
  cudaFree(V.d_xt);
  cudaFree(V.d_yl);
  cudaFree(V.d_ppart);
  cudaFree(V.d_part);
  cudaFree(V.d_t);
  V.d_xt = V.d_yl = V.d_ppart = V.d_part = V.d_t = nullptr;
  V.scratch_nrhs = 0;
  const int64_t n = h->n;
  // every element is 8 bytes (double, or a float pair)
  H2D_CK(cudaMalloc(&V.d_xt, 8 * n * nrhs + 16));  // + bulk-copy slack
  H2D_CK(cudaMalloc(&V.d_yl, 8 * n * nrhs * (h->kappa + 1)));
  H2D_CK(cudaMalloc(&V.d_ppart, 8 * V.pstride * nrhs));
  H2D_CK(cudaMalloc(&V.d_part, 8 * std::max<int64_t>(V.proj_partials, 1) * nrhs));
  H2D_CK(cudaMalloc(&V.d_t, 8 * std::max<int64_t>(h->t_total, 1) * nrhs));
  V.scratch_nrhs = nrhs;
  ++h->gen;
  return HODLR2D_OK;
}

template <class A>
static int launch_pair_plain(const int2* work, int64_t nw, int rows, const ArgsV2& P,
                             const typename A::val* xt, typename A::val* ppart, cudaStream_t st) {
  if (rows <= kSmallPair)
    k_pair<A, 64><<<(unsigned)nw, 64, 0, st>>>(P, work, xt, ppart);
  else
    k_pair<A, 256><<<(unsigned)nw, 256, 0, st>>>(P, work, xt, ppart);
  H2D_CK(cudaGetLastError());
  return HODLR2D_OK;
}

// one launch of k_pairg<A, T, RM, G> with its staging slots
template <class A, int T, int RM, int G>
static void launch_pairg(unsigned nb, const ArgsV2& P, const int2* work,
                         const typename A::val* xt, typename A::val* ppart, cudaStream_t st) {
  constexpr int smem = pairg_smem<A, T, RM, G>();
  static_assert(smem <= 48 * 1024, "staging slots within the default dynamic shared memory");
  k_pairg<A, T, RM, G><<<nb, T, smem, st>>>(P, work, xt, ppart);
}

template <class A>
static int launch_pair_reg(const int2* work, int64_t nw, int rows, const ArgsV2& P,
                           const typename A::val* xt, typename A::val* ppart, cudaStream_t st) {
  // column group of the small-box forms: 4, or 2 for float-float (registers)
  constexpr bool b32 = sizeof(typename A::acc) == 4;
  constexpr int GS = b32 ? 4 : 2;
  const unsigned nb = (unsigned)nw;
  if (rows <= 48)  // 16 pairs per 128-thread block
    k_pairs<A, 8, 6, GS><<<(unsigned)((nw + 15) / 16), 128, pairs_smem<A, 8, 6, GS>(), st>>>(
        P, work, nw, xt, ppart);
  else if (rows <= 64)  // 8 pairs per block
    k_pairs<A, 16, 4, GS><<<(unsigned)((nw + 7) / 8), 128, pairs_smem<A, 16, 4, GS>(), st>>>(
        P, work, nw, xt, ppart);
  else if (rows <= 128)
    launch_pairg<A, 32, 4, GS>(nb, P, work, xt, ppart, st);
  else if (rows <= 256)
    launch_pairg<A, 64, 4, GS>(nb, P, work, xt, ppart, st);
  else if (rows <= 384)
    launch_pairg<A, 128, 3, GS>(nb, P, work, xt, ppart, st);
  else if (rows <= 1280)
    launch_pairg<A, 256, 5, 2>(nb, P, work, xt, ppart, st);
  else if (rows <= 2560)
    launch_pairg<A, 512, 5, 2>(nb, P, work, xt, ppart, st);
  else if (rows <= kDualRows && b32) {
    if constexpr (b32) launch_pairg<A, 512, 9, 2>(nb, P, work, xt, ppart, st);
  } else if (rows <= kDualRows && !b32) {
    if constexpr (!b32) launch_pairg<A, 512, 9, 1>(nb, P, work, xt, ppart, st);
  } else
    return launch_pair_plain<A>(work, nw, rows, P, xt, ppart, st);
  H2D_CK(cudaGetLastError());
  return HODLR2D_OK;
}

template <class A>
static int launch_pair_multi(const int2* work, int64_t nw, int rows, const ArgsV2& P,
                             const typename A::val* xt, typename A::val* ppart,
                             cudaStream_t st) {
  constexpr bool b32 = sizeof(typename A::acc) == 4;
  constexpr int NR = b32 ? 8 : 4;  // right-hand sides per pass
  const unsigned nb = (unsigned)nw;
  if (rows <= 16) {  // four pairs per warp
    k_pairms<A, 8, 2, 4><<<(unsigned)((nw + 4 * kPairmsWarps - 1) / (4 * kPairmsWarps)),
                           32 * kPairmsWarps, 0, st>>>(P, work, nw, xt, ppart);
  } else if (rows <= 32) {  // two pairs per warp
    k_pairms<A, 16, 2, 4><<<(unsigned)((nw + 2 * kPairmsWarps - 1) / (2 * kPairmsWarps)),
                            32 * kPairmsWarps, 0, st>>>(P, work, nw, xt, ppart);
  } else if (rows <= 64)
    k_pairm<A, 32, 2, NR><<<nb, 32, 0, st>>>(P, work, xt, ppart);
  else if (rows <= 128)
    k_pairm<A, 64, 2, NR><<<nb, 64, 0, st>>>(P, work, xt, ppart);
  else if (rows <= kMultiRows)
    k_pairm<A, 128, 2, NR><<<nb, 128, 0, st>>>(P, work, xt, ppart);
  else if (rows <= 512 && P.nrhs <= kFewRhs)
    k_pairm<A, 256, 2, NR><<<nb, 256, 0, st>>>(P, work, xt, ppart);
  else if (rows <= kMultiRowsFew && P.nrhs <= kFewRhs)  // four rows a thread: half the RHS a pass
    k_pairm<A, 256, 4, NR / 2><<<nb, 256, 0, st>>>(P, work, xt, ppart);
  else
    return launch_pair_plain<A>(work, nw, rows, P, xt, ppart, st);
  H2D_CK(cudaGetLastError());
  return HODLR2D_OK;
}

// Which kernel form the launchers above pick for a size class of boxes of at
// most `rows` points (their branch conditions, in order): consecutive
// classes of the same form share one launch.
template <class A>
static int pair_form(int rows, int nrhs) {
  if constexpr (std::is_same<A, F64A>::value) return rows <= kSmallPair ? 100 : 101;
  constexpr bool b32 = sizeof(typename A::acc) == 4;
  if (nrhs == 1) {
    const int lim[8] = {48, 64, 128, 256, 384, 1280, 2560, kDualRows};
    for (int i = 0; i < 8; ++i)
      if (rows <= lim[i]) return i;
    return rows <= kSmallPair ? 100 : 101;
  }
  if (rows <= 16) return 10;
  if (rows <= 32) return 11;
  if (rows <= 64) return 12;
  if (rows <= 128) return 13;
  if (rows <= kMultiRows) return 14;
  if (rows <= 512 && nrhs <= kFewRhs) return 15;
  if (rows <= kMultiRowsFew && nrhs <= kFewRhs) return 16;
  return rows <= kSmallPair ? 100 : 101;
}

// Runs of consecutive size classes with one form (empty classes join any
// run): calls f(first work item, items, largest box) once per run and
// returns the number of runs.
template <class A, class Fn>
static int pair_runs(const PairLevel& G, int nrhs, Fn&& f) {
  int runs = 0;
  for (int c = 0; c < kPairClasses;) {
    if (G.off[c + 1] == G.off[c]) {
      ++c;
      continue;
    }
    const int form = pair_form<A>(G.cls_rows[c], nrhs);
    int rows = G.cls_rows[c], c2 = c + 1;
    while (c2 < kPairClasses && (G.off[c2 + 1] == G.off[c2] ||
                                 pair_form<A>(G.cls_rows[c2], nrhs) == form)) {
      if (G.off[c2 + 1] > G.off[c2]) rows = std::max(rows, G.cls_rows[c2]);
      ++c2;
    }
    const int rc = f(G.off[c], G.off[c2] - G.off[c], rows);
    if (rc) return rc < 0 ? rc : -1;
    ++runs;
    c = c2;
  }
  return runs;
}

// Runs the pairs of level l, one launch per run of size classes of one form:
// k_pairg / k_pairs (each factor value read once) for one right-hand side,
// block shape by the run's largest box; k_pairm / k_pairms for several
// right-hand sides; k_pair for binary64 sums (its shuffle-free second phase
// suits the slow binary64 pipe).
template <class A>
static int launch_pairs(hodlr2d* h, int l, const ArgsV2& P, const typename A::val* xt,
                        typename A::val* ppart, cudaStream_t st) {
  const PairLevel& G = h->v2.plev[l];
  if constexpr (std::is_same<A, F64A>::value) {
    // binary64, small boxes: one warp per pair, every size class at once
    if (G.max_rows <= kP64Rows && h->lev[l].max_rank <= kP64Kmax) {
      if (G.nwork)
        k_pair64<<<(unsigned)((G.nwork + kPair64Warps - 1) / kPair64Warps), 32 * kPair64Warps,
                   kPair64Smem, st>>>(P, G.d_work, G.nwork, xt, ppart);
      H2D_CK(cudaGetLastError());
      return HODLR2D_OK;
    }
  }
  const int runs = pair_runs<A>(G, P.nrhs, [&](int64_t first, int64_t nw, int rows) {
    const int2* work = G.d_work + first;
    if constexpr (std::is_same<A, F64A>::value)  // binary64: warp per column, two reads
      return launch_pair_plain<A>(work, nw, rows, P, xt, ppart, st);
    else if (P.nrhs == 1)
      return launch_pair_reg<A>(work, nw, rows, P, xt, ppart, st);
    else
      return launch_pair_multi<A>(work, nw, rows, P, xt, ppart, st);
  });
  return runs < 0 ? runs : HODLR2D_OK;
}

// The near field with one right-hand side per pass, or NM per pass for
// several.
template <class NP, int NM>
static void launch_near(const V2Plan& V, const hodlr2d* h, cudaStream_t sn,
                        const typename NP::pt* xf, const typename NP::pt* yf,
                        const typename NP::K& kp, const typename NP::A::val* xt, int nrhs,
                        typename NP::A::val* yl) {
  const unsigned g = (unsigned)((V.nnearw + kNearWarps - 1) / kNearWarps);
  if (nrhs == 1)
    k_near_warp<NP, 1><<<g, 32 * kNearWarps, 0, sn>>>(xf, yf, h->d_leaf_off, h->kappa,
                                                      V.d_nearw, V.nnearw, kp, xt, h->n, nrhs, yl);
  else
    k_near_warp<NP, NM><<<g, 32 * kNearWarps, 0, sn>>>(xf, yf, h->d_leaf_off, h->kappa,
                                                       V.d_nearw, V.nnearw, kp, xt, h->n, nrhs, yl);
}

// Operations of one kernel entry's formula, each elementary function (sqrt,
// log, division) counted as one: the algorithmic cost c_K of a near-field
// entry, before the multiply-add with x.
static int64_t near_formula_ops(int kind) {
  switch (kind) {
    case HODLR2D_IMQ: return 8;   // dx, dy, dx^2, dy^2, +, + a^2, sqrt, 1/
    case HODLR2D_PHI1: return 8;  // dx, dy, dx^2, dy^2, +, sqrt, log, / (either branch)
    default: return 7;            // MQ: ..., + a^2, sqrt; INV_R, PHI2: sqrt, /; LOG: log, * 0.5
  }
}

template <class A>
static int run_v2(hodlr2d* h, const double* x, double* y, int nrhs, int mode) {
  using Val = typename A::val;
  V2Plan& V = h->v2;
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  const unsigned g = (unsigned)((n + 255) / 256);
  const ArgsV2 P = args_v2(h, nrhs, mode);
  Val* xt = reinterpret_cast<Val*>(V.d_xt);
  Val* yl = reinterpret_cast<Val*>(V.d_yl);
  Val* ppart = reinterpret_cast<Val*>(V.d_ppart);
  const int64_t fs = (int64_t)sizeof(typename A::fac);  // bytes per factor value
  const int64_t vs = (int64_t)sizeof(Val);                // bytes per vector value
  const int64_t vb = vs * n * nrhs;                       // one vector block
  {
    PhaseScope ps(h, 0, 1, vb + 8 * n + 8 * n * nrhs);
    k_gather2<A><<<g, 256, 0, s>>>(x, h->d_perm, n, nrhs, xt);
  }
  // the near field (arithmetic-bound) and the single-read levels run on side
  // streams, concurrently with the two-pass levels on the caller's stream
  // (while profiling, everything stays on the caller's stream so that the
  // per-phase event times are those of each kernel alone)
  const cudaStream_t sn = h->prof_on ? s : V.s_near;
  const cudaStream_t sf = h->prof_on ? s : V.s_far;
  H2D_CK(cudaEventRecord(V.ev_in, s));
  H2D_CK(cudaStreamWaitEvent(sn, V.ev_in, 0));
  H2D_CK(cudaStreamWaitEvent(sf, V.ev_in, 0));
  {
    PhaseScope ps(h, 1, 1, 24 * n + 2 * vb, sn);
    ps.flops(V.near_entries * (near_formula_ops(h->kp.kind) + 2 * (int64_t)nrhs));
    if (mode == HODLR2D_MODE_F64) {
      const unsigned gn = (unsigned)((V.nnearw + kNear64Warps - 1) / kNear64Warps);
      if (nrhs == 1)
        k_near64<1><<<gn, 32 * kNear64Warps, 0, sn>>>(
            h->d_x, h->d_y, h->d_leaf_off, h->kappa, V.d_nearw, V.nnearw, h->kp,
            reinterpret_cast<const double*>(xt), h->n, nrhs, reinterpret_cast<double*>(yl));
      else
        k_near64<4><<<gn, 32 * kNear64Warps, 0, sn>>>(
            h->d_x, h->d_y, h->d_leaf_off, h->kappa, V.d_nearw, V.nnearw, h->kp,
            reinterpret_cast<const double*>(xt), h->n, nrhs, reinterpret_cast<double*>(yl));
    }
    else if (mode == HODLR2D_MODE_DF32)
      launch_near<NearDF32, 4>(V, h, sn, reinterpret_cast<const float2*>(V.d_xf),
                               reinterpret_cast<const float2*>(V.d_yf), V.kff,
                               reinterpret_cast<const float2*>(xt), nrhs,
                               reinterpret_cast<float2*>(yl));
    else
      launch_near<NearF32, 4>(V, h, sn, reinterpret_cast<const float*>(V.d_x32),
                              reinterpret_cast<const float*>(V.d_y32), V.kf32,
                              reinterpret_cast<const float*>(xt), nrhs,
                              reinterpret_cast<float*>(yl));
  }
  // two-pass levels [1, l2end): level-ordered prefixes of the task lists
  const int l2end = two_pass_end(h, nrhs, mode);
  const int64_t nproj = V.pre_proj[l2end];
  const int64_t npart = V.pre_part[l2end];
  const int64_t ntsum = V.pre_tsum[l2end];
  const int64_t nexp = V.pre_exp[l2end];
  int64_t two_pass_vals = 0;
  for (int l = 1; l < l2end; ++l) two_pass_vals += h->lev[l].nstored;
  if (nproj) {
    {
      PhaseScope ps(h, 2, 1, fs * two_pass_vals + vs * npart * nrhs);
      ps.flops(2 * two_pass_vals * nrhs);
      const int64_t thr = npart * 32;  // one warp per (task, column)
      if (std::is_same<A, BF16A>::value && nrhs > 1 && !few_rhs(nrhs, mode))  // tensor cores
        if (V.grp_ok)  // tasks grouped by box: x loaded once per group
          k_projg_t5<<<(unsigned)std::min<int64_t>(V.pre_grp[l2end], 3 * V.nsm), 256, kGrpSmem,
                       s>>>(P, V.d_proj, V.d_gtask, V.d_grp, V.pre_grp[l2end],
                            reinterpret_cast<const float*>(xt),
                            reinterpret_cast<float*>(V.d_part), V.d_status);
        else
          k_proj_t5<<<(unsigned)std::min<int64_t>(nproj, 4 * V.nsm), 128, kT5Smem, s>>>(
              P, V.d_proj, nproj, reinterpret_cast<const float*>(xt),
              reinterpret_cast<float*>(V.d_part), V.d_status);
      else if (nrhs >= 24 && sizeof(Val) == 4)  // binary32 sums: tiled over many right-hand sides
        k_projm<A><<<(unsigned)nproj, 256, 0, s>>>(P, V.d_proj, xt,
                                                   reinterpret_cast<Val*>(V.d_part));
      else if (std::is_same<A, F64A>::value) {  // binary64: column groups, halving exchange
        const int64_t ng = V.pre_pgrp[l2end];
        k_proj64<<<(unsigned)((ng * 32 + 255) / 256), 256, 0, s>>>(
            P, V.d_proj, V.d_pgrp, ng, reinterpret_cast<const double*>(xt),
            reinterpret_cast<double*>(V.d_part));
      }
      else
        k_proj2<A><<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(
            P, V.d_proj, V.d_wtask, npart, xt, reinterpret_cast<Val*>(V.d_part));
    }
    {
      PhaseScope ps(h, 3, std::is_same<A, F64A>::value ? 2 : 1, vs * (npart + h->t_total) * nrhs);
      const int64_t thr = ntsum * 32;
      if (std::is_same<A, F64A>::value) {  // binary64: one thread per (side, column)
        k_tsum64<<<(unsigned)((ntsum + 255) / 256), 256, 0, s>>>(
            P, V.d_proj, V.d_red, V.d_sideq, ntsum, reinterpret_cast<const double*>(V.d_part),
            reinterpret_cast<double*>(V.d_t));
        k_tsum2<A><<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(
            P, V.d_proj, V.d_red, V.d_sideq, ntsum, reinterpret_cast<const Val*>(V.d_part),
            reinterpret_cast<Val*>(V.d_t), kTsumThread + 1);
      } else
      k_tsum2<A><<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(
          P, V.d_proj, V.d_red, V.d_sideq, ntsum, reinterpret_cast<const Val*>(V.d_part),
          reinterpret_cast<Val*>(V.d_t));
    }
  }
  if (nexp) {
    PhaseScope ps(h, 4, 1, fs * two_pass_vals + vb * (l2end - 1));
    ps.flops(2 * two_pass_vals * nrhs);
    if (std::is_same<A, BF16A>::value && nrhs > 1 && !few_rhs(nrhs, mode))  // tensor cores
      k_exp_t5<<<(unsigned)std::min<int64_t>(nexp, 4 * V.nsm), 128, kT5Smem, s>>>(
          P, V.d_exp, nexp, reinterpret_cast<const float*>(V.d_t), reinterpret_cast<float*>(yl),
          V.d_status);
    else
      k_exp2<A><<<(unsigned)nexp, 256, 0, s>>>(P, V.d_exp, reinterpret_cast<const Val*>(V.d_t),
                                               yl);
  }
  H2D_CK(cudaEventRecord(V.ev_near, sn));
  bool any_pair = false;
  for (int l = l2end; l <= h->kappa; ++l) any_pair = any_pair || P.lmode[l] == LMODE_PAIR;
  if (V.zero_partials && any_pair)
    H2D_CK(cudaMemsetAsync(V.d_ppart, 0, 8 * V.pstride * nrhs, sf));
  for (int l = l2end; l <= h->kappa; ++l) {
    if (P.lmode[l] != LMODE_PAIR || V.plev[l].nwork == 0) continue;
    const int phase = V.lmode[l] == LMODE_BOX ? 7 : l < V.lpair_small ? 6 : 8;
    // one launch per run of size classes of one form (binary64 small boxes: one per level)
    int nlaunch = pair_runs<A>(V.plev[l], nrhs, [](int64_t, int64_t, int) { return 0; });
    if (std::is_same<A, F64A>::value && V.plev[l].max_rows <= kP64Rows &&
        h->lev[l].max_rank <= kP64Kmax)
      nlaunch = 1;
    PhaseScope ps(h, phase, nlaunch, fs * h->lev[l].nstored, sf);
    ps.flops(4 * h->lev[l].nstored * nrhs);
    H2D_TRY(launch_pairs<A>(h, l, P, xt, ppart, sf));
  }
  int64_t box_vals = 0;  // levels left to the box kernel in this product
  for (int l = V.lfuse; l <= h->kappa; ++l)
    if (P.lmode[l] == LMODE_BOX) box_vals += h->lev[l].nstored;
  if (V.nbw && box_vals) {
    PhaseScope ps(h, 7, 1, fs * box_vals, sf);
    ps.flops(4 * box_vals * nrhs);
    k_box<A><<<(unsigned)((V.nbw + kBoxWarps - 1) / kBoxWarps), 32 * kBoxWarps, kBoxSmem, sf>>>(
        P, V.d_bw, V.nbw, xt, yl, ppart);
  }
  H2D_CK(cudaEventRecord(V.ev_far, sf));
  H2D_CK(cudaStreamWaitEvent(s, V.ev_near, 0));
  H2D_CK(cudaStreamWaitEvent(s, V.ev_far, 0));
  {
    PhaseScope ps(h, 5, 1, vb * (h->kappa + 1) + vs * V.pstride * nrhs + 16 * n + 8 * n * nrhs);
    k_combine2<A><<<g, 256, 0, s>>>(P, yl, ppart, V.d_leaf_of, h->d_perm, y);
  }
  H2D_CK(cudaGetLastError());
  return HODLR2D_OK;
}

// ---------------------------------------------------------------------------
// Persistent batch product: the products of many independent handles (point
// sets of uneven size) in one cooperative kernel launch.  Per set, the levels
// whose boxes hold at most pair_rows points run as pairs (each stored pair
// read once: t1 = V^T x_Y and t2 = U^T x_X, then U t1 and V t2 into the
// pair's partial results); the coarser levels run in two passes
// (projections over row chunks, chunk sums, expansions).  The work falls
// into five phases, each a flat list of units over all sets (a unit is the
// work of one 256-thread block, named by a descriptor: set, kind, index):
//   0 gather x into tree order;
//   1 pairs (by their larger box: up to 2048 points one pair per unit, up
//     to 256 two per unit of 128 threads each, up to 128 four per unit of 64
//     threads each, up to warp_rows one per warp), the two-pass projections
//     and the near field -- independent work, longest units first.  The
//     groups of one unit do not wait for each other at its end: the groups
//     of 128 threads synchronise on named barriers 1-2, those of 64 on 3-6,
//     each id always used by the same warps;
//   2 chunk sums; 3 expansions; 4 combine.
// The near field and the one-warp pairs depend only on the gathered x, so
// they may instead run beside the expansions and the chunk sums (place).
// Blocks walk a phase's units grid-stride, then meet at a grid barrier.  All
// blocks are resident (cooperative launch), and every barrier wait is
// bounded: a block that polls `polls` times in vain records it in the status
// word and leaves, so the launch always ends.  The last block out resets the
// barrier counters for the next launch, so one launch is the whole product.
// ---------------------------------------------------------------------------
// largest box of a one-pair-per-unit item: 2048 points (8 rows a thread,
// one right-hand side per pass) for 4-byte sums, 1024 for binary64
constexpr int kBatchBlockRows = 2048;
constexpr int kBatchWarp = 5, kBatchW16 = 6, kBatchW8 = 7;  // the warp-level pair kinds
// pair items by the box size they take, largest first: one per unit with
// 8, 4 or 2 rows a thread, two per unit (128 threads each), four per unit
// (64 threads each), one per warp
constexpr int kBatchPairKinds = 8;
// (the last three kinds take pairs of at most warp_rows points: a warp, or
// 2 or 4 pairs per warp for boxes of at most 32 or 16 points)
constexpr int kBatchKindRows[kBatchPairKinds - 3] = {2048, 1024, 512, 256, 128};

struct BatchSet {
  ArgsV2 P;                   // LMODE_TWO below the first pair level, LMODE_PAIR from it on
  const double* x;            // caller's x and y (n x nrhs, column-major)
  double* y;
  const int64_t* perm;
  const int32_t* leaf_of;
  void* xt;                   // the handle's scratch
  void* yl;
  void* ppart;
  void* part;
  void* t;
  const void* xf;             // near-field points of the mode
  const void* yf;
  KernelParams kp;            // binary64 entries
  KernelF32 kf32;             // binary32 entries
  const int2* nearw;
  int64_t nnearw;
  const ProjTask* proj;
  const int32_t* wtask;
  int64_t npart;              // projection warps
  const int64_t* red;
  const int64_t* sideq;
  int64_t ntsum;              // chunk-sum warps
  const ExpTask* exps;
  int64_t nexp;
  // pair items (level, pair) by kind (kBatchKindRows): kind q at
  // pwork[p0[q] .. p0[q + 1])
  const int2* pwork;
  int64_t p0[kBatchPairKinds + 1];
  int64_t u_proj, u_near;     // phase-1 units of the projections and of the near field
};

// Device words of a persistent launch.
struct BatchSync {
  unsigned bar;     // barrier arrivals of the running launch
  unsigned exit;    // blocks that have left
  int status;       // nonzero: a barrier wait gave up
  int pad;
  unsigned long long ts[6];  // %globaltimer: start, after each barrier, end
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool batch_barrier(BatchSync* sy, unsigned target, uint32_t polls) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this block's writes before its arrival
    atomicAdd(&sy->bar, 1u);
    int ok = 0;
    for (uint32_t it = 0; it < polls; ++it) {
      if (*reinterpret_cast<volatile unsigned*>(&sy->bar) >= target) {
        ok = 1;
        break;
      }
      __nanosleep(64);
    }
    if (!ok) atomicOr(&sy->status, 1);
    __threadfence();  // the other blocks' writes before this block's reads
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Unit kinds of the persistent product, and the unit descriptors: set
// << 44 | kind << 40 | index of the unit among the set's units of its kind.
enum BatchKind {
  BK_GATHER = 0,  // 256 points
  BK_BLK8,        // one pair of at most 2048 points (4-byte sums only)
  BK_BLK4,        // one pair of at most 1024 points
  BK_BLK,         // one pair of at most 512 points
  BK_G128,        // two pairs of at most 256 points (128 threads each)
  BK_G64,         // four pairs of at most 128 points (64 threads each)
  BK_PROJ,        // eight projection warps
  BK_NEAR,        // eight near-field warps
  BK_WARP,        // eight pairs of at most warp_rows points (a warp each)
  BK_W16,         // sixteen pairs of at most 32 points (16 lanes each)
  BK_W8,          // thirty-two pairs of at most 16 points (8 lanes each)
  BK_TSUM,        // eight chunk-sum warps
  BK_EXP,         // one expansion task
  BK_COMBINE,     // 256 points
  BK_COUNT
};
__host__ __device__ constexpr uint64_t batch_desc(int set, int kind, int64_t i) {
  return (uint64_t)set << 44 | (uint64_t)kind << 40 | (uint64_t)i;
}

template <class A, class NP>
__device__ __forceinline__ void batch_unit(const BatchSet& S, int kind, int64_t lv) {
  using V = typename A::val;
  constexpr int NRM = sizeof(typename A::acc) == 4 ? 4 : 2;  // right-hand sides per pair pass
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  V* xt = reinterpret_cast<V*>(S.xt);
  V* yl = reinterpret_cast<V*>(S.yl);
  V* part = reinterpret_cast<V*>(S.part);
  V* tt = reinterpret_cast<V*>(S.t);
  V* ppart = reinterpret_cast<V*>(S.ppart);
  const bool one = S.P.nrhs == 1;
  constexpr bool b32 = sizeof(typename A::acc) == 4;
  switch (kind) {
    case BK_GATHER:
      gather2_body<A>(S.x, S.perm, S.P.n, S.P.nrhs, xt, lv * 256 + tid);
      return;
    case BK_BLK8:
      if constexpr (b32) pairm_body<A, 256, 8, 1>(S.P, S.pwork[S.p0[0] + lv], xt, ppart, tid);
      return;
    case BK_BLK4:
      if (one || !b32) pairm_body<A, 256, 4, 1>(S.P, S.pwork[S.p0[1] + lv], xt, ppart, tid);
      else pairm_body<A, 256, 4, 2>(S.P, S.pwork[S.p0[1] + lv], xt, ppart, tid);
      return;
    case BK_BLK:
      if (one) pairm_body<A, 256, 2, 1>(S.P, S.pwork[S.p0[2] + lv], xt, ppart, tid);
      else pairm_body<A, 256, 2, NRM>(S.P, S.pwork[S.p0[2] + lv], xt, ppart, tid);
      return;
    case BK_G128: {
      const int g = tid >> 7;
      const int64_t j = S.p0[3] + lv * 2 + g;
      if (j >= S.p0[4]) return;
      const int2 wk = S.pwork[j];
      if (one) pairm_body<A, 128, 2, 1, 2, 1>(S.P, wk, xt, ppart, tid & 127, g);
      else pairm_body<A, 128, 2, NRM, 2, 1>(S.P, wk, xt, ppart, tid & 127, g);
      return;
    }
    case BK_G64: {
      const int g = tid >> 6;
      const int64_t j = S.p0[4] + lv * 4 + g;
      if (j >= S.p0[5]) return;
      const int2 wk = S.pwork[j];
      if (one) pairm_body<A, 64, 2, 1, 4, 3>(S.P, wk, xt, ppart, tid & 63, g);
      else pairm_body<A, 64, 2, NRM, 4, 3>(S.P, wk, xt, ppart, tid & 63, g);
      return;
    }
    case BK_PROJ:
      proj2_body<A>(S.P, S.proj, S.wtask, S.npart, xt, part, lv * 8 + warp);
      return;
    case BK_NEAR: {
      const typename NP::K* kpp;
      if constexpr (std::is_same<typename NP::K, KernelParams>::value) kpp = &S.kp;
      else kpp = &S.kf32;
      const typename NP::pt* xf = reinterpret_cast<const typename NP::pt*>(S.xf);
      const typename NP::pt* yf = reinterpret_cast<const typename NP::pt*>(S.yf);
      if (one)
        near_warp_body<NP, 1>(xf, yf, S.P.leaf_off, S.P.kappa, S.nearw, S.nnearw, *kpp, xt,
                              S.P.n, S.P.nrhs, yl, lv * 8 + warp);
      else
        near_warp_body<NP, 4>(xf, yf, S.P.leaf_off, S.P.kappa, S.nearw, S.nnearw, *kpp, xt,
                              S.P.n, S.P.nrhs, yl, lv * 8 + warp);
      return;
    }
    case BK_WARP: {
      const int64_t j = S.p0[kBatchWarp] + lv * 8 + warp;
      if (j >= S.p0[kBatchWarp + 1]) return;
      const int2 wk = S.pwork[j];
      if (one) pairm_body<A, 32, 2, 1>(S.P, wk, xt, ppart, lane);
      else pairm_body<A, 32, 2, NRM>(S.P, wk, xt, ppart, lane);
      return;
    }
    case BK_W16: {
      const int2* w = S.pwork + S.p0[kBatchW16];
      const int64_t nw = S.p0[kBatchW16 + 1] - S.p0[kBatchW16], i0 = (lv * 8 + warp) * 2;
      if (i0 >= nw) return;  // uniform in the warp
      if (one) pairms_body<A, 16, 2, 1>(S.P, w, nw, xt, ppart, i0);
      else pairms_body<A, 16, 2, NRM>(S.P, w, nw, xt, ppart, i0);
      return;
    }
    case BK_W8: {
      const int2* w = S.pwork + S.p0[kBatchW8];
      const int64_t nw = S.p0[kBatchW8 + 1] - S.p0[kBatchW8], i0 = (lv * 8 + warp) * 4;
      if (i0 >= nw) return;
      if (one) pairms_body<A, 8, 2, 1>(S.P, w, nw, xt, ppart, i0);
      else pairms_body<A, 8, 2, NRM>(S.P, w, nw, xt, ppart, i0);
      return;
    }
    case BK_TSUM:
      tsum2_body<A>(S.P, S.proj, S.red, S.sideq, S.ntsum, part, tt, 0, lv * 8 + warp);
      return;
    case BK_EXP:
      exp2_body<A>(S.P, S.exps, tt, yl, lv);
      __syncthreads();  // its shared list is refilled by the next unit
      return;
    default:
      combine2_body<A>(S.P, yl, ppart, S.leaf_of, S.perm, S.y, lv * 256 + tid);
  }
}

// MINB: resident blocks per SM the compiler is asked for (registers a thread
// 65536 / (256 MINB)); the batch picks one of 2, 3, 4.  tab holds the unit
// descriptors of the five phases, phase p at [off[p], off[p + 1]); a block
// walks its units grid-stride, loading the next descriptor before it runs
// the current unit.
template <class A, class NP, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_batch(const BatchSet* __restrict__ sets, const uint64_t* __restrict__ tab,
            const int64_t* __restrict__ off, BatchSync* sy, uint32_t polls) {
  if (blockIdx.x == 0 && threadIdx.x == 0) sy->ts[0] = global_ns();
  for (int ph = 0; ph < 5; ++ph) {
    const int64_t end = off[ph + 1];
    int64_t vb = off[ph] + blockIdx.x;
    uint64_t d = vb < end ? tab[vb] : 0;
    for (; vb < end; vb += gridDim.x) {
      const uint64_t cur = d;
      if (vb + gridDim.x < end) d = tab[vb + gridDim.x];
      batch_unit<A, NP>(sets[cur >> 44], (int)((cur >> 40) & 15),
                        (int64_t)(cur & ((uint64_t(1) << 40) - 1)));
    }
    if (ph == 4) break;
    if (!batch_barrier(sy, (unsigned)(ph + 1) * gridDim.x, polls)) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) sy->ts[ph + 1] = global_ns();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMax(&sy->ts[5], global_ns());
    __threadfence();
    if (atomicAdd(&sy->exit, 1u) == gridDim.x - 1) {  // every block has left: reset
      sy->bar = 0;
      sy->exit = 0;
      __threadfence();
    }
  }
}

// The instantiation of the batch's mode and registers a thread.
static const void* batch_kernel(const BatchPersist& bp) {
  const bool f64 = bp.mode == HODLR2D_MODE_F64;
  switch (bp.minb) {
    case 2: return f64 ? (const void*)k_batch<F64A, NearF64, 2> : (const void*)k_batch<F32A, NearF32, 2>;
    case 4: return f64 ? (const void*)k_batch<F64A, NearF64, 4> : (const void*)k_batch<F32A, NearF32, 4>;
    default: return f64 ? (const void*)k_batch<F64A, NearF64, 3> : (const void*)k_batch<F32A, NearF32, 3>;
  }
}

// First level of set h that runs as pairs in the persistent form: every
// level from it on has a pair plan and boxes of at most pair_rows points.
static int batch_first_pair_level(const hodlr2d* h, int pair_rows) {
  const V2Plan& V = h->v2;
  int lp = h->kappa + 1;
  for (int l = h->kappa; l >= std::max(1, V.ldual); --l) {
    if (V.plev[l].max_rows > pair_rows) break;
    lp = l;
  }
  return lp;
}

int batch_persist_setup(hodlr2d* const* hs, int count, const double* const* x, double* const* y,
                        const int* nrhs, int mode, BatchPersist* bp) {
  if (mode != HODLR2D_MODE_F64 && mode != HODLR2D_MODE_F32) return HODLR2D_ERR_ARG;
  const int pair_rows =
      std::min(bp->pair_rows, mode == HODLR2D_MODE_F64 ? kBatchBlockRows / 2 : kBatchBlockRows);
  const int warp_rows = std::min(bp->warp_rows, 64);  // two rows a lane
  if (count > (1 << 19)) return HODLR2D_ERR_ARG;  // set index of a unit descriptor
  std::vector<BatchSet> sets(count);
  std::vector<std::array<int64_t, BK_COUNT>> units(count);
  std::vector<int> lpair(count);
  for (int i = 0; i < count; ++i) {
    hodlr2d* h = hs[i];
    V2Plan& V = h->v2;
    H2D_TRY(plan_v2(h));
    lpair[i] = batch_first_pair_level(h, pair_rows);
    if (V.two_levels < lpair[i]) {
      H2D_CK(cudaStreamSynchronize(h->stream));
      H2D_TRY(build_two_pass(h, lpair[i]));
      V.scratch_nrhs = 0;  // the partial sums grew
    }
    H2D_TRY(scratch_v2(h, nrhs[i]));
  }
  batch_persist_free(bp);
  // pair items of every set, grouped by the threads that take one pair:
  // 256 (boxes of at most 512 points), 128 (256), 64 (128), 32 (warp_rows)
  std::vector<int2> items;
  std::vector<int64_t> item0(count);
  cudaStream_t s0 = hs[0]->stream;
  for (int i = 0; i < count; ++i) {
    hodlr2d* h = hs[i];
    V2Plan& V = h->v2;
    const int lp = lpair[i];
    BatchSet& S = sets[i];
    S.P = args_v2(h, nrhs[i], mode);
    for (int l = 0; l < HODLR2D_MAX_LEVELS; ++l) S.P.lmode[l] = l < lp ? LMODE_TWO : LMODE_PAIR;
    S.x = x[i];
    S.y = y[i];
    S.perm = h->d_perm;
    S.leaf_of = V.d_leaf_of;
    S.xt = V.d_xt;
    S.yl = V.d_yl;
    S.ppart = V.d_ppart;
    S.part = V.d_part;
    S.t = V.d_t;
    if (mode == HODLR2D_MODE_F64) {
      S.xf = h->d_x;
      S.yf = h->d_y;
    } else {
      S.xf = V.d_x32;
      S.yf = V.d_y32;
    }
    S.kp = h->kp;
    S.kf32 = V.kf32;
    S.nearw = V.d_nearw;
    S.nnearw = V.nnearw;
    S.proj = V.d_proj;
    S.wtask = V.d_wtask;
    S.npart = V.pre_part[lp];
    S.red = V.d_red;
    S.sideq = V.d_sideq;
    S.ntsum = V.pre_tsum[lp];
    S.exps = V.d_exp;
    S.nexp = V.pre_exp[lp];
    item0[i] = (int64_t)items.size();
    S.p0[0] = 0;
    for (int kind = 0; kind < kBatchPairKinds; ++kind) {
      S.p0[kind + 1] = S.p0[kind];
      for (int l = lp; l <= h->kappa; ++l) {
        const PairLevel& G = V.plev[l];
        for (int c = 0; c < kPairClasses; ++c) {
          const int r = G.cls_rows[c];
          int k;  // the smallest kind whose boxes hold r points
          if (r <= warp_rows)
            k = r <= 16 ? kBatchW8 : r <= 32 ? kBatchW16 : kBatchWarp;
          else
            for (k = kBatchWarp - 1; k > 0 && r > kBatchKindRows[k]; --k) {
            }
          if (k != kind) continue;
          items.insert(items.end(), G.h_work.begin() + G.off[c], G.h_work.begin() + G.off[c + 1]);
          S.p0[kind + 1] += G.off[c + 1] - G.off[c];
        }
      }
    }
    // slots of rank-0 pairs are read by the combine and written by no item
    H2D_CK(cudaMemsetAsync(V.d_ppart, 0, 8 * V.pstride * nrhs[i], s0));
    S.u_proj = (S.npart + 7) / 8;
    S.u_near = (V.nnearw + 7) / 8;
    auto& u = units[i];
    u[BK_GATHER] = u[BK_COMBINE] = (h->n + 255) / 256;
    u[BK_BLK8] = S.p0[1] - S.p0[0];
    u[BK_BLK4] = S.p0[2] - S.p0[1];
    u[BK_BLK] = S.p0[3] - S.p0[2];
    u[BK_G128] = (S.p0[4] - S.p0[3] + 1) / 2;
    u[BK_G64] = (S.p0[5] - S.p0[4] + 3) / 4;
    u[BK_PROJ] = S.u_proj;
    u[BK_NEAR] = S.u_near;
    u[BK_WARP] = (S.p0[kBatchWarp + 1] - S.p0[kBatchWarp] + 7) / 8;
    u[BK_W16] = (S.p0[kBatchW16 + 1] - S.p0[kBatchW16] + 15) / 16;
    u[BK_W8] = (S.p0[kBatchW8 + 1] - S.p0[kBatchW8] + 31) / 32;
    u[BK_TSUM] = (S.ntsum + 7) / 8;
    u[BK_EXP] = S.nexp;
  }
  // unit descriptors, phase by phase; within a phase kind by kind (longest
  // units first), set by set.  place bit 0 moves the near field from phase 1
  // to phase 3 (beside the expansions), bit 1 the one-warp pairs to phase 2
  // (beside the chunk sums).
  std::vector<int> kinds[5];
  kinds[0] = {BK_GATHER};
  kinds[1] = {BK_BLK8, BK_BLK4, BK_BLK, BK_G128, BK_G64, BK_PROJ};
  if (!(bp->place & 1)) kinds[1].push_back(BK_NEAR);
  for (int kd : {BK_WARP, BK_W16, BK_W8}) {
    if (!(bp->place & 2)) kinds[1].push_back(kd);
    else kinds[2].push_back(kd);
  }
  kinds[2].push_back(BK_TSUM);
  kinds[3] = {BK_EXP};
  if (bp->place & 1) kinds[3].push_back(BK_NEAR);
  kinds[4] = {BK_COMBINE};
  std::vector<uint64_t> tab;
  int64_t off[6] = {0, 0, 0, 0, 0, 0};
  for (int ph = 0; ph < 5; ++ph) {
    for (int kind : kinds[ph])
      for (int i = 0; i < count; ++i)
        for (int64_t j = 0; j < units[i][kind]; ++j) tab.push_back(batch_desc(i, kind, j));
    off[ph + 1] = (int64_t)tab.size();
  }
  H2D_CK(cudaMalloc(&bp->d_work, sizeof(int2) * std::max<size_t>(items.size(), 1)));
  for (int i = 0; i < count; ++i) sets[i].pwork = reinterpret_cast<int2*>(bp->d_work) + item0[i];
  if (!items.empty())
    H2D_CK(cudaMemcpyAsync(bp->d_work, items.data(), sizeof(int2) * items.size(),
                           cudaMemcpyHostToDevice, s0));
  H2D_CK(cudaMalloc(&bp->d_sets, sizeof(BatchSet) * count));
  H2D_CK(cudaMalloc(&bp->d_pre, sizeof(off)));
  H2D_CK(cudaMalloc(&bp->d_tab, sizeof(uint64_t) * std::max<size_t>(tab.size(), 1)));
  H2D_CK(cudaMalloc(&bp->d_sync, sizeof(BatchSync)));
  H2D_CK(cudaMemcpyAsync(bp->d_sets, sets.data(), sizeof(BatchSet) * count,
                         cudaMemcpyHostToDevice, s0));
  H2D_CK(cudaMemcpyAsync(bp->d_pre, off, sizeof(off), cudaMemcpyHostToDevice, s0));
  if (!tab.empty())
    H2D_CK(cudaMemcpyAsync(bp->d_tab, tab.data(), sizeof(uint64_t) * tab.size(),
                           cudaMemcpyHostToDevice, s0));
  H2D_CK(cudaMemsetAsync(bp->d_sync, 0, sizeof(BatchSync), s0));
  H2D_CK(cudaStreamSynchronize(s0));
  bp->count = count;
  bp->mode = mode;
  int dev = 0, nsm = 1, per = 0;
  H2D_CK(cudaGetDevice(&dev));
  H2D_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  H2D_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel(*bp), 256, 0));
  bp->grid = std::max(1, per) * nsm;
  return HODLR2D_OK;
}

// One persistent launch on stream s: the whole product of every set.
int batch_persist_launch(const BatchPersist& bp, cudaStream_t s) {
  BatchSync* sy = reinterpret_cast<BatchSync*>(bp.d_sync);
  void* args[] = {(void*)&bp.d_sets, (void*)&bp.d_tab, (void*)&bp.d_pre, (void*)&sy,
                  (void*)&bp.polls};
  H2D_CK(cudaLaunchCooperativeKernel(batch_kernel(bp), dim3((unsigned)bp.grid), dim3(256), args,
                                     0, s));
  return HODLR2D_OK;
}

// Reads and clears the status word (synchronises stream s): TIMEOUT if a
// barrier wait gave up since the previous call.
int batch_persist_status(const BatchPersist& bp, cudaStream_t s) {
  if (!bp.d_sync) return HODLR2D_OK;
  H2D_CK(cudaStreamSynchronize(s));
  BatchSync* sy = reinterpret_cast<BatchSync*>(bp.d_sync);
  int st = 0;
  H2D_CK(cudaMemcpy(&st, &sy->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) H2D_CK(cudaMemset(&sy->status, 0, sizeof(int)));
  return st ? HODLR2D_ERR_TIMEOUT : HODLR2D_OK;
}

// Milliseconds of the five phases of the last launch (block 0's view of the
// barriers; the last phase ends with the last block).
int batch_persist_phase_ms(const BatchPersist& bp, cudaStream_t s, double* ms) {
  if (!bp.d_sync) return HODLR2D_ERR_STATE;
  H2D_CK(cudaStreamSynchronize(s));
  BatchSync h{};
  H2D_CK(cudaMemcpy(&h, bp.d_sync, sizeof(BatchSync), cudaMemcpyDeviceToHost));
  for (int p = 0; p < 5; ++p) ms[p] = (double)(int64_t)(h.ts[p + 1] - h.ts[p]) * 1e-6;
  return HODLR2D_OK;
}

void batch_persist_free(BatchPersist* bp) {
  cudaFree(bp->d_sets);
  cudaFree(bp->d_pre);
  cudaFree(bp->d_tab);
  cudaFree(bp->d_sync);
  cudaFree(bp->d_work);
  bp->d_sets = nullptr;
  bp->d_pre = nullptr;
  bp->d_tab = nullptr;
  bp->d_sync = nullptr;
  bp->d_work = nullptr;
}

// Reads and clears the device status word of the product kernels (a bounded
// wait that gave up); synchronises the handle's stream.
int product_status(hodlr2d* h) {
  V2Plan& V = h->v2;
  if (!V.ready || !V.d_status) return HODLR2D_OK;
  int st = 0;
  H2D_CK(cudaStreamSynchronize(h->stream));
  H2D_CK(cudaMemcpy(&st, V.d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) H2D_CK(cudaMemset(V.d_status, 0, sizeof(int)));
  return st ? HODLR2D_ERR_TIMEOUT : HODLR2D_OK;
}

// The product in a prepared mode (F64 or DF32) with device x and y.
int product_device(hodlr2d* h, const double* x, double* y, int nrhs, int mode) {
  H2D_TRY(plan_v2(h));
  if (two_pass_end(h, nrhs, mode) > h->v2.two_levels) {  // first product of all levels in two passes
    H2D_CK(cudaStreamSynchronize(h->stream));
    H2D_TRY(build_two_pass(h, two_pass_end(h, nrhs, mode)));
    h->v2.scratch_nrhs = 0;  // the partial sums grew
  }
  H2D_TRY(scratch_v2(h, nrhs));
  if (mode == HODLR2D_MODE_F64) return run_v2<F64A>(h, x, y, nrhs, mode);
  if (mode == HODLR2D_MODE_DF32) return run_v2<DF32A>(h, x, y, nrhs, mode);
  if (mode == HODLR2D_MODE_F32) return run_v2<F32A>(h, x, y, nrhs, mode);
  if (mode == HODLR2D_MODE_BF16) return run_v2<BF16A>(h, x, y, nrhs, mode);
  return HODLR2D_ERR_STATE;
}

// Float-float copies of the factors, the points and the kernel parameters.
int prepare_df32(hodlr2d* h) {
  V2Plan& V = h->v2;
  for (int l = 1; l <= h->kappa; ++l) {
    Level& L = h->lev[l];
    if (L.d_fac_mode[HODLR2D_MODE_DF32]) continue;
    const int64_t nv = std::max<int64_t>(L.nvalues, 1);
    H2D_CK(cudaMalloc(&L.d_fac_mode[HODLR2D_MODE_DF32], 8 * nv + 16));  // + bulk-copy slack
    if (L.nvalues)
      k_to_ff<<<(unsigned)((L.nvalues + 255) / 256), 256, 0, h->stream>>>(
          L.d_fac, reinterpret_cast<float2*>(L.d_fac_mode[HODLR2D_MODE_DF32]), L.nvalues);
  }
  if (!V.d_xf) {
    H2D_CK(cudaMalloc(&V.d_xf, 8 * h->n));
    H2D_CK(cudaMalloc(&V.d_yf, 8 * h->n));
    k_to_ff<<<(unsigned)((h->n + 255) / 256), 256, 0, h->stream>>>(h->d_x, reinterpret_cast<float2*>(V.d_xf), h->n);
    k_to_ff<<<(unsigned)((h->n + 255) / 256), 256, 0, h->stream>>>(h->d_y, reinterpret_cast<float2*>(V.d_yf), h->n);
  }
  H2D_CK(cudaGetLastError());
  H2D_CK(cudaStreamSynchronize(h->stream));
  // kernel parameters as float pairs (host split of the binary64 values)
  auto split = [](double d) {
    const float hi = (float)d;
    return make_float2(hi, (float)(d - (double)hi));
  };
  V.kff.kind = h->kp.kind;
  V.kff.a = split(h->kp.a);
  V.kff.a2 = split(h->kp.a2);
  V.kff.inv_a = split(h->kp.inv_a);
  V.kff.diag = split(h->kp.diag);
  V.kff.inv_log_a = split(h->kp.log_a != 0.0 ? 1.0 / h->kp.log_a : 0.0);
  V.kff.inv_phi1_den = split(h->kp.phi1_den != 0.0 ? 1.0 / h->kp.phi1_den : 0.0);
  return HODLR2D_OK;
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = __double2float_rn(a[i]);
}
__global__ void k_to_bf16(const double* __restrict__ a, __nv_bfloat16* __restrict__ out,
                          int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = __double2bfloat16(a[i]);
}

// binary32 or bfloat16 factor copies, binary32 points and kernel parameters
int prepare_low(hodlr2d* h, int mode) {
  V2Plan& V = h->v2;
  for (int l = 1; l <= h->kappa; ++l) {
    Level& L = h->lev[l];
    if (L.d_fac_mode[mode]) continue;
    const int64_t nv = std::max<int64_t>(L.nvalues, 1);
    const int64_t es = mode == HODLR2D_MODE_F32 ? 4 : 2;
    H2D_CK(cudaMalloc(&L.d_fac_mode[mode], es * nv + 16));  // + bulk-copy slack
    if (!L.nvalues) continue;
    const unsigned g = (unsigned)((L.nvalues + 255) / 256);
    if (mode == HODLR2D_MODE_F32)
      k_to_f32<<<g, 256, 0, h->stream>>>(L.d_fac, reinterpret_cast<float*>(L.d_fac_mode[mode]),
                                         L.nvalues);
    else
      k_to_bf16<<<g, 256, 0, h->stream>>>(
          L.d_fac, reinterpret_cast<__nv_bfloat16*>(L.d_fac_mode[mode]), L.nvalues);
  }
  if (!V.d_x32) {
    H2D_CK(cudaMalloc(&V.d_x32, 4 * h->n));
    H2D_CK(cudaMalloc(&V.d_y32, 4 * h->n));
    const unsigned g = (unsigned)((h->n + 255) / 256);
    k_to_f32<<<g, 256, 0, h->stream>>>(h->d_x, reinterpret_cast<float*>(V.d_x32), h->n);
    k_to_f32<<<g, 256, 0, h->stream>>>(h->d_y, reinterpret_cast<float*>(V.d_y32), h->n);
  }
  H2D_CK(cudaGetLastError());
  H2D_CK(cudaStreamSynchronize(h->stream));
  V.kf32.kind = h->kp.kind;
  V.kf32.a = (float)h->kp.a;
  V.kf32.a2 = (float)h->kp.a2;
  V.kf32.inv_a = (float)h->kp.inv_a;
  V.kf32.log_a = (float)h->kp.log_a;
  V.kf32.phi1_den = (float)h->kp.phi1_den;
  V.kf32.diag = (float)h->kp.diag;
  return HODLR2D_OK;
}

void free_v2(hodlr2d* h) {
  V2Plan& V = h->v2;
  cudaFree(V.d_proj);
  cudaFree(V.d_exp);
  cudaFree(V.d_red);
  cudaFree(V.d_wtask);
  cudaFree(V.d_sideq);
  cudaFree(V.d_pgrp);
  cudaFree(V.d_status);
  cudaFree(V.d_gtask);
  cudaFree(V.d_grp);
  cudaFree(V.d_bw);
  cudaFree(V.d_nearw);
  cudaFree(V.d_leaf_of);
  cudaFree(V.d_xt);
  cudaFree(V.d_yl);
  cudaFree(V.d_ppart);
  cudaFree(V.d_part);
  cudaFree(V.d_t);
  cudaFree(V.d_xf);
  cudaFree(V.d_yf);
  cudaFree(V.d_x32);
  cudaFree(V.d_y32);
  for (int l = 0; l < HODLR2D_MAX_LEVELS; ++l) cudaFree(V.plev[l].d_work);
  if (V.s_near) cudaStreamDestroy(V.s_near);
  if (V.s_far) cudaStreamDestroy(V.s_far);
  if (V.ev_in) cudaEventDestroy(V.ev_in);
  if (V.ev_near) cudaEventDestroy(V.ev_near);
  if (V.ev_far) cudaEventDestroy(V.ev_far);
  V = V2Plan();
}

}  // namespace h2d
