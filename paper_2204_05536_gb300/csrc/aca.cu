// Batched ACA (the compression step of Alg. 1): one thread block per
// admissible pair, all pairs of a level in a few launches.
//
// Partially pivoted ACA with pivots fixed by the points' original indices, so
// that the result does not depend on where a point sits in memory:
//   - first row: the point of X with the smallest original index;
//   - column pivot: argmax |residual row|, ties to the smaller original index;
//   - a zero residual row marks the row used and moves to the unused row with
//     the smallest original index;
//   - term k: v = residual row / pivot, u = residual column (unscaled);
//   - |S_k|_F^2 += 2 sum_q (u_q.u)(v_q.v) + |u|^2 |v|^2;
//   - stop when |u| |v| <= eps |S_k|_F, at rank min(|X|, |Y|), or when every
//     row was used; a block that reaches the rank cap first is unconverged;
//   - next row: argmax |u| over unused rows, ties to the smaller index.
// Residual rows and columns are written straight into the factor workspace
// (U: |X| x cap, V: |Y| x cap, column-major), then compacted to rank k.
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "scan.cuh"

namespace h2d {

struct Piv {
  double a;   // |value| (or 0 / -1 for "any unused" / "none")
  int64_t g;  // original index (tie-break)
  int32_t pos;
};

__device__ __forceinline__ bool piv_better(const Piv& x, const Piv& y) {
  return x.a > y.a || (x.a == y.a && x.g < y.g);
}

__device__ __forceinline__ Piv piv_none() { return Piv{-1.0, INT64_MAX, -1}; }

__device__ __forceinline__ Piv warp_piv(Piv v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Piv w;
    w.a = __shfl_xor_sync(0xffffffffu, v.a, o);
    w.g = __shfl_xor_sync(0xffffffffu, v.g, o);
    w.pos = __shfl_xor_sync(0xffffffffu, v.pos, o);
    if (piv_better(w, v)) v = w;
  }
  return v;
}

// every thread gets the block's best; uses red[nwarps]
template <int T>
__device__ __forceinline__ Piv block_piv(Piv v, Piv* red) {
  v = warp_piv(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  Piv b = red[0];
#pragma unroll
  for (int w = 1; w < T / 32; ++w)
    if (piv_better(red[w], b)) b = red[w];
  __syncthreads();
  return b;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct AcaArgs {
  const double* x;
  const double* y;
  const int64_t* perm;
  const int32_t* leaf_off;
  int kappa, l;
  KernelParams kp;
  double eps;
  int max_rank;
  const int32_t* px;
  const int32_t* py;
  int64_t p0;             // first pair of the batch
  const int64_t* wsoff;   // per batch pair: workspace offset (values)
  const int64_t* fgoff;   // per batch pair: row-flag offset (bytes)
  double* ws;
  uint8_t* flags;
  int32_t* rank;          // per level pair
  int32_t* conv;          // per level pair
  const int64_t* plist;   // batch pair ids (fallback pass) or null: p0 + block
  const int32_t* bcap;    // per batch pair rank cap (predicted) or null
};

template <int T>
__global__ void __launch_bounds__(T) k_aca(AcaArgs A) {
  extern __shared__ double sm[];
  __shared__ Piv red[T / 32];
  const int capmax = A.max_rank;
  double* s_u = sm;                  // row i of U, q < k
  double* s_v = sm + capmax;         // row jp of V, q < k
  double* s_du = s_v + capmax;       // U_q . u, q <= k
  double* s_dv = s_du + capmax + 1;  // V_q . v, q <= k
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const int64_t p = A.plist ? A.plist[blockIdx.x] : A.p0 + blockIdx.x;
  const uint32_t bx = (uint32_t)A.px[p], by = (uint32_t)A.py[p];
  const int sh = 2 * (A.kappa - A.l);
  const int32_t xs = A.leaf_off[(int64_t)bx << sh];
  const int32_t m = A.leaf_off[(int64_t)(bx + 1) << sh] - xs;
  const int32_t ys = A.leaf_off[(int64_t)by << sh];
  const int32_t n = A.leaf_off[(int64_t)(by + 1) << sh] - ys;
  const int kfull = min(m, n);
  const int cap = A.bcap ? min(A.bcap[blockIdx.x], min(kfull, capmax)) : min(kfull, capmax);
  double* U = A.ws + A.wsoff[blockIdx.x];
  double* V = U + (int64_t)m * cap;
  uint8_t* used = A.flags + A.fgoff[blockIdx.x];
  const double* X0 = A.x + xs;
  const double* Y0 = A.y + xs;
  const double* X1 = A.x + ys;
  const double* Y1 = A.y + ys;
  const int64_t* G0 = A.perm + xs;
  const int64_t* G1 = A.perm + ys;

  for (int t = tid; t < m; t += T) used[t] = 0;
  Piv best = piv_none();
  for (int t = tid; t < m; t += T) {
    const Piv c{0.0, G0[t], t};
    if (piv_better(c, best)) best = c;
  }
  best = block_piv<T>(best, red);  // also orders the flag writes above
  int32_t i = best.pos;
  int k = 0, nused = 0;
  double S2 = 0.0;
  bool conv = false;

  while (k < cap && nused < m) {
    for (int q = tid; q < k; q += T) s_u[q] = U[(int64_t)q * m + i];
    __syncthreads();
    const double xi = X0[i], yi = Y0[i];
    const int64_t gi = G0[i];
    Piv jb = piv_none();
    double* Vk = V + (int64_t)k * n;
    for (int j = tid; j < n; j += T) {
      double r = entry(A.kp, xi, yi, gi, X1[j], Y1[j], G1[j]);
      for (int q = 0; q < k; ++q) r -= s_u[q] * V[(int64_t)q * n + j];
      Vk[j] = r;
      const Piv c{fabs(r), G1[j], j};
      if (piv_better(c, jb)) jb = c;
    }
    jb = block_piv<T>(jb, red);
    if (tid == 0) used[i] = 1;
    ++nused;
    const int32_t jp = jb.pos;
    if (jp < 0) break;  // every residual entry is NaN: give up on this block
    const double piv = Vk[jp];
    __syncthreads();  // everyone has read the pivot before its owner rescales it
    if (piv == 0.0) {
      Piv nb = piv_none();
      for (int t = tid; t < m; t += T)
        if (!used[t]) {
          const Piv c{0.0, G0[t], t};
          if (piv_better(c, nb)) nb = c;
        }
      nb = block_piv<T>(nb, red);
      if (nb.pos < 0) break;
      i = nb.pos;
      continue;
    }
    for (int j = tid; j < n; j += T) Vk[j] = Vk[j] / piv;
    for (int q = tid; q < k; q += T) s_v[q] = V[(int64_t)q * n + jp];
    __syncthreads();
    const double xj = X1[jp], yj = Y1[jp];
    const int64_t gj = G1[jp];
    double* Uk = U + (int64_t)k * m;
    for (int t = tid; t < m; t += T) {
      double u = entry(A.kp, X0[t], Y0[t], G0[t], xj, yj, gj);
      for (int q = 0; q < k; ++q) u -= U[(int64_t)q * m + t] * s_v[q];
      Uk[t] = u;
    }
    __syncthreads();
    for (int q = warp; q <= k; q += T / 32) {
      double a = 0.0, b = 0.0;
      const double* Uq = U + (int64_t)q * m;
      const double* Vq = V + (int64_t)q * n;
      for (int t = lane; t < m; t += 32) a += Uq[t] * Uk[t];
      for (int j = lane; j < n; j += 32) b += Vq[j] * Vk[j];
      a = warp_sum(a);
      b = warp_sum(b);
      if (lane == 0) {
        s_du[q] = a;
        s_dv[q] = b;
      }
    }
    __syncthreads();
    double cross = 0.0;
    for (int q = 0; q < k; ++q) cross += s_du[q] * s_dv[q];
    const double uu = s_du[k], vv = s_dv[k];
    S2 += 2.0 * cross + uu * vv;
    ++k;
    if (sqrt(uu) * sqrt(vv) <= A.eps * sqrt(fmax(S2, 0.0))) {
      conv = true;
      break;
    }
    Piv nb = piv_none();
    for (int t = tid; t < m; t += T)
      if (!used[t]) {
        const Piv c{fabs(Uk[t]), G0[t], t};
        if (piv_better(c, nb)) nb = c;
      }
    nb = block_piv<T>(nb, red);
    if (nb.pos < 0) break;
    i = nb.pos;
  }
  if (tid == 0) {
    A.rank[p] = k;
    A.conv[p] = (conv || k == kfull || nused == m) ? 1 : 0;
  }
}

// copy U[:, :k] and V[:, :k] of each batch pair (columns padded to even
// length) to dst + dstoff[b]; dstoff < 0 skips the pair
__global__ void k_compact(const double* __restrict__ ws, const int64_t* __restrict__ wsoff,
                          const int32_t* __restrict__ leaf_off, int kappa, int l,
                          const int32_t* __restrict__ px, const int32_t* __restrict__ py,
                          const int64_t* __restrict__ plist, const int32_t* __restrict__ rank,
                          const int32_t* __restrict__ bcap, const int64_t* __restrict__ dstoff,
                          double* __restrict__ dst) {
  const int64_t doff = dstoff[blockIdx.x];
  if (doff < 0) return;
  const int64_t p = plist[blockIdx.x];
  const int sh = 2 * (kappa - l);
  const uint32_t bx = (uint32_t)px[p], by = (uint32_t)py[p];
  const int64_t m = leaf_off[(int64_t)(bx + 1) << sh] - leaf_off[(int64_t)bx << sh];
  const int64_t n = leaf_off[(int64_t)(by + 1) << sh] - leaf_off[(int64_t)by << sh];
  const int64_t cap = bcap[blockIdx.x];
  const int64_t k = rank[p];
  const double* U = ws + wsoff[blockIdx.x];
  const double* V = U + m * cap;
  const int64_t lm = ldpad(m), ln = ldpad(n);
  double* out = dst + doff;
  for (int64_t t = threadIdx.x; t < lm * k; t += blockDim.x) {
    const int64_t q = t / lm, i = t - q * lm;
    out[t] = i < m ? U[q * m + i] : 0.0;
  }
  for (int64_t t = threadIdx.x; t < ln * k; t += blockDim.x) {
    const int64_t q = t / ln, j = t - q * ln;
    out[lm * k + t] = j < n ? V[q * n + j] : 0.0;
  }
}

// gather each pair's packed block from its staging place into the level
// buffer, in pair order
__global__ void k_pack_pairs(const double* const* __restrict__ src,
                             const int64_t* __restrict__ cnt, const int64_t* __restrict__ foff,
                             double* __restrict__ fac) {
  const int64_t p = blockIdx.x;
  const double* s = src[p];
  double* d = fac + foff[p];
  for (int64_t t = threadIdx.x; t < cnt[p]; t += blockDim.x) d[t] = s[t];
}

// ---------------------------------------------------------------------------
// Wide ACA: the same steps for pairs too large for one thread block (boxes of
// hundreds of thousands of points at the coarse levels), each step spread
// over many blocks and driven from the host one term at a time:
//   k_wrow   residual row i over column chunks; argmax partial per chunk
//   k_wpiv   pivot (chunk partials in chunk order), row i marked used; a zero
//            pivot moves to the unused row of smallest original index
//   k_wcol   v scaled by the pivot, residual column u over row chunks; chunk
//            partials of V_q . v, U_q . u (q <= k) and argmax |u| (unused)
//   k_wfin   |S_k|_F^2 update (partials in chunk order), stopping test, next
//            row
// The residual entries are the k_aca ones (same expressions, same order over
// q); the dot products sum in a different order, so the stopping test can in
// principle decide differently on an exact tie.
// ---------------------------------------------------------------------------
constexpr int kWideChunk = 4096;  // elements per block
constexpr int64_t kWideRows = 24576;  // |X| + |Y| from which a pair runs wide
constexpr int kWideT = 256;

struct WideState {
  int64_t p;             // pair of the level
  int64_t wsoff, fgoff;  // workspace (U then V) and row-flag offsets
  int32_t xs, m, ys, n, cap, kfull;
  int32_t k, i, jp, nused;
  int32_t active, conv, skip;  // skip: this term's column step is not run
  int32_t ncm, ncn;            // row / column chunks
  int64_t cm0, cn0;            // first chunk of this pair in the row / column chunk lists
  double S2, piv;
};

struct WideArgs {
  AcaArgs A;
  WideState* st;
  int nw;
  const int2* rchunks;  // (pair, chunk) over the rows of X
  const int2* cchunks;  // (pair, chunk) over the rows of Y
  int64_t nr;           // row chunks (column chunks follow them in ppiv, pdot)
  Piv* ppiv;            // per chunk argmax partials: rows of X, then rows of Y
  double* pdot;         // per chunk: dots of q = 0..cap (cap + 1 values)
  double* svec;         // per pair: V(jp, q), q < cap
  int cap;              // largest cap of the batch
};

__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kWideT / 32; ++w) s += red[w];
  __syncthreads();
  return s;
}

// first row of every wide pair: the point of X with the smallest original index
__global__ void __launch_bounds__(kWideT) k_winit(WideArgs W) {
  __shared__ Piv red[kWideT / 32];
  WideState& S = W.st[blockIdx.x];
  const AcaArgs& A = W.A;
  uint8_t* used = A.flags + S.fgoff;
  const int64_t* G0 = A.perm + S.xs;
  Piv best = piv_none();
  for (int t = threadIdx.x; t < S.m; t += kWideT) {
    used[t] = 0;
    const Piv c{0.0, G0[t], t};
    if (piv_better(c, best)) best = c;
  }
  best = block_piv<kWideT>(best, red);
  if (threadIdx.x == 0) {
    S.i = best.pos;
    S.k = 0;
    S.nused = 0;
    S.S2 = 0.0;
    S.active = S.cap > 0 && S.m > 0 ? 1 : 0;
    S.conv = S.active ? 0 : (S.kfull == 0 ? 1 : 0);
    S.skip = 0;
  }
}

__global__ void __launch_bounds__(kWideT) k_wrow(WideArgs W, int64_t nchunks) {
  __shared__ Piv red[kWideT / 32];
  __shared__ double s_u[256];
  const int64_t b = blockIdx.x;
  if (b >= nchunks) return;
  const int2 pc = W.cchunks[b];
  WideState& S = W.st[pc.x];
  if (!S.active) return;
  const AcaArgs& A = W.A;
  const int k = S.k, i = S.i;
  double* U = A.ws + S.wsoff;
  double* V = U + (int64_t)S.m * S.cap;
  for (int q = threadIdx.x; q < k; q += kWideT) s_u[q] = U[(int64_t)q * S.m + i];
  __syncthreads();
  const double xi = A.x[S.xs + i], yi = A.y[S.xs + i];
  const int64_t gi = A.perm[S.xs + i];
  const double* X1 = A.x + S.ys;
  const double* Y1 = A.y + S.ys;
  const int64_t* G1 = A.perm + S.ys;
  double* Vk = V + (int64_t)k * S.n;
  Piv jb = piv_none();
  const int j0 = pc.y * kWideChunk, j1 = min(S.n, j0 + kWideChunk);
  for (int j = j0 + threadIdx.x; j < j1; j += kWideT) {
    double r = entry(A.kp, xi, yi, gi, X1[j], Y1[j], G1[j]);
    for (int q = 0; q < k; ++q) r -= s_u[q] * V[(int64_t)q * S.n + j];
    Vk[j] = r;
    const Piv c{fabs(r), G1[j], j};
    if (piv_better(c, jb)) jb = c;
  }
  jb = block_piv<kWideT>(jb, red);
  if (threadIdx.x == 0) W.ppiv[W.nr + b] = jb;
}

__global__ void __launch_bounds__(kWideT) k_wpiv(WideArgs W) {
  __shared__ Piv red[kWideT / 32];
  WideState& S = W.st[blockIdx.x];
  if (!S.active) return;
  const AcaArgs& A = W.A;
  // column pivot: the best of the column chunks, in chunk order
  Piv jb = piv_none();
  for (int c = threadIdx.x; c < S.ncn; c += kWideT) {
    const Piv v = W.ppiv[W.nr + S.cn0 + c];
    if (piv_better(v, jb)) jb = v;
  }
  jb = block_piv<kWideT>(jb, red);
  uint8_t* used = A.flags + S.fgoff;
  double* U = A.ws + S.wsoff;
  double* V = U + (int64_t)S.m * S.cap;
  const int k = S.k;
  __syncthreads();
  if (threadIdx.x == 0) {
    used[S.i] = 1;
    S.nused += 1;
    S.skip = 0;
  }
  if (jb.pos < 0) {  // every residual entry is NaN: give up on this block
    if (threadIdx.x == 0) {
      S.active = 0;
      S.conv = (S.k == S.kfull || S.nused == S.m) ? 1 : 0;
    }
    return;
  }
  const double piv = V[(int64_t)k * S.n + jb.pos];
  __syncthreads();  // used[i] is set before the search below
  if (piv == 0.0) {  // next unused row of smallest original index
    const int64_t* G0 = A.perm + S.xs;
    Piv nb = piv_none();
    for (int t = threadIdx.x; t < S.m; t += kWideT)
      if (!used[t]) {
        const Piv c{0.0, G0[t], t};
        if (piv_better(c, nb)) nb = c;
      }
    nb = block_piv<kWideT>(nb, red);
    if (threadIdx.x == 0) {
      S.skip = 1;
      if (nb.pos < 0 || S.nused >= S.m) {
        S.active = 0;
        S.conv = (S.k == S.kfull || S.nused == S.m) ? 1 : 0;
      } else {
        S.i = nb.pos;
      }
    }
    return;
  }
  // V(jp, q) of the scaled columns q < k, for the residual column
  double* sv = W.svec + (int64_t)blockIdx.x * W.cap;
  for (int q = threadIdx.x; q < k; q += kWideT) sv[q] = V[(int64_t)q * S.n + jb.pos];
  if (threadIdx.x == 0) {
    S.jp = jb.pos;
    S.piv = piv;
  }
}

// blocks [0, nr) over the rows of X, then [nr, nr + nc) over the rows of Y
__global__ void __launch_bounds__(kWideT) k_wcol(WideArgs W, int64_t nc) {
  __shared__ Piv red[kWideT / 32];
  __shared__ double dred[kWideT / 32];
  __shared__ double s_v[256];
  const int64_t b = blockIdx.x, nr = W.nr;
  if (b >= nr + nc) return;
  const bool rows_x = b < nr;
  const int2 pc = rows_x ? W.rchunks[b] : W.cchunks[b - nr];
  WideState& S = W.st[pc.x];
  if (!S.active || S.skip) return;
  const AcaArgs& A = W.A;
  const int k = S.k;
  double* U = A.ws + S.wsoff;
  double* V = U + (int64_t)S.m * S.cap;
  double* out = W.pdot + b * (int64_t)(W.cap + 1);
  if (rows_x) {
    const double* sv = W.svec + (int64_t)pc.x * W.cap;
    for (int q = threadIdx.x; q < k; q += kWideT) s_v[q] = sv[q];
    __syncthreads();
    const int64_t gjp = A.perm[S.ys + S.jp];
    const double xj = A.x[S.ys + S.jp], yj = A.y[S.ys + S.jp];
    const double* X0 = A.x + S.xs;
    const double* Y0 = A.y + S.xs;
    const int64_t* G0 = A.perm + S.xs;
    const uint8_t* used = A.flags + S.fgoff;
    double* Uk = U + (int64_t)k * S.m;
    const int t0 = pc.y * kWideChunk, t1 = min(S.m, t0 + kWideChunk);
    Piv nb = piv_none();
    for (int t = t0 + threadIdx.x; t < t1; t += kWideT) {
      double u = entry(A.kp, X0[t], Y0[t], G0[t], xj, yj, gjp);
      for (int q = 0; q < k; ++q) u -= U[(int64_t)q * S.m + t] * s_v[q];
      Uk[t] = u;
      if (!used[t]) {
        const Piv c{fabs(u), G0[t], t};
        if (piv_better(c, nb)) nb = c;
      }
    }
    nb = block_piv<kWideT>(nb, red);
    if (threadIdx.x == 0) W.ppiv[b] = nb;
    __syncthreads();
    for (int q = 0; q <= k; ++q) {  // U_q . u over this chunk
      double a = 0.0;
      for (int t = t0 + threadIdx.x; t < t1; t += kWideT) a += U[(int64_t)q * S.m + t] * Uk[t];
      a = block_sum(a, dred);
      if (threadIdx.x == 0) out[q] = a;
    }
  } else {
    double* Vk = V + (int64_t)k * S.n;
    const int j0 = pc.y * kWideChunk, j1 = min(S.n, j0 + kWideChunk);
    for (int j = j0 + threadIdx.x; j < j1; j += kWideT) Vk[j] = Vk[j] / S.piv;
    __syncthreads();
    for (int q = 0; q <= k; ++q) {  // V_q . v over this chunk
      double a = 0.0;
      for (int j = j0 + threadIdx.x; j < j1; j += kWideT) a += V[(int64_t)q * S.n + j] * Vk[j];
      a = block_sum(a, dred);
      if (threadIdx.x == 0) out[q] = a;
    }
  }
}

__global__ void __launch_bounds__(kWideT) k_wfin(WideArgs W) {
  __shared__ Piv red[kWideT / 32];
  __shared__ double s_du[257], s_dv[257];
  WideState& S = W.st[blockIdx.x];
  if (!S.active || S.skip) return;
  const int k = S.k;
  const int64_t stride = W.cap + 1, nr = W.nr;
  for (int q = threadIdx.x; q <= k; q += kWideT) {  // chunk partials in chunk order
    double a = 0.0, v = 0.0;
    for (int c = 0; c < S.ncm; ++c) a += W.pdot[(S.cm0 + c) * stride + q];
    for (int c = 0; c < S.ncn; ++c) v += W.pdot[(nr + S.cn0 + c) * stride + q];
    s_du[q] = a;
    s_dv[q] = v;
  }
  Piv nb = piv_none();
  for (int c = threadIdx.x; c < S.ncm; c += kWideT) {
    const Piv v = W.ppiv[S.cm0 + c];
    if (piv_better(v, nb)) nb = v;
  }
  nb = block_piv<kWideT>(nb, red);  // also publishes s_du / s_dv
  if (threadIdx.x != 0) return;
  double cross = 0.0;
  for (int q = 0; q < k; ++q) cross += s_du[q] * s_dv[q];
  const double uu = s_du[k], vv = s_dv[k];
  S.S2 += 2.0 * cross + uu * vv;
  S.k = k + 1;
  if (sqrt(uu) * sqrt(vv) <= W.A.eps * sqrt(fmax(S.S2, 0.0))) {
    S.active = 0;
    S.conv = 1;
    return;
  }
  if (S.k >= S.cap || S.nused >= S.m || nb.pos < 0) {
    S.active = 0;
    S.conv = (S.k == S.kfull || S.nused == S.m) ? 1 : 0;
    return;
  }
  S.i = nb.pos;
}

__global__ void k_wdone(const WideState* __restrict__ st, int nw, int32_t* __restrict__ rank,
                        int32_t* __restrict__ conv, int32_t* __restrict__ nactive) {
  int a = 0;
  for (int w = threadIdx.x; w < nw; w += blockDim.x) {
    const WideState& S = st[w];
    rank[S.p] = S.k;
    conv[S.p] = S.active ? 0 : S.conv;
    a += S.active;
  }
  a = __reduce_add_sync(0xffffffffu, a);
  if (threadIdx.x == 0) *nactive = a;
}

// Runs the wide pairs of a batch to completion (states filled with p, wsoff,
// fgoff, xs, m, ys, n, cap <= 256, kfull); fills rank[p] and conv[p] like
// k_aca.
static int aca_wide(const AcaArgs& A, std::vector<WideState> st, cudaStream_t s) {
  const int nw = (int)st.size();
  if (nw == 0) return HODLR2D_OK;
  std::vector<int2> rch, cch;
  int cap = 1;
  int64_t max_rounds = 0;
  for (int w = 0; w < nw; ++w) {
    WideState& S = st[w];
    S.ncm = (int32_t)((S.m + kWideChunk - 1) / kWideChunk);
    S.ncn = (int32_t)((S.n + kWideChunk - 1) / kWideChunk);
    S.cm0 = (int64_t)rch.size();
    S.cn0 = (int64_t)cch.size();
    for (int c = 0; c < S.ncm; ++c) rch.push_back(make_int2(w, c));
    for (int c = 0; c < S.ncn; ++c) cch.push_back(make_int2(w, c));
    cap = std::max(cap, S.cap);
    // a term per round, or a used row without a term (zero pivot)
    max_rounds = std::max<int64_t>(max_rounds, (int64_t)S.cap + S.m);
  }
  if (cap > 256) return HODLR2D_ERR_ARG;  // the shared vectors hold 256 terms
  const int64_t nr = (int64_t)rch.size(), nc = (int64_t)cch.size();
  WideArgs W;
  W.A = A;
  W.nw = nw;
  W.cap = cap;
  W.nr = nr;
  WideState* d_st = nullptr;
  int2 *d_r = nullptr, *d_c = nullptr;
  Piv* d_piv = nullptr;
  double *d_dot = nullptr, *d_sv = nullptr;
  int32_t* d_na = nullptr;
  int rc = HODLR2D_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == HODLR2D_OK) {
      (void)cudaGetLastError();
      rc = e == cudaErrorMemoryAllocation ? HODLR2D_ERR_OOM : HODLR2D_ERR_CUDA;
    }
  };
  ck(cudaMalloc(&d_st, sizeof(WideState) * nw));
  ck(cudaMalloc(&d_r, sizeof(int2) * nr));
  ck(cudaMalloc(&d_c, sizeof(int2) * nc));
  ck(cudaMalloc(&d_piv, sizeof(Piv) * (nr + nc)));
  ck(cudaMalloc(&d_dot, sizeof(double) * (nr + nc) * (cap + 1)));
  ck(cudaMalloc(&d_sv, sizeof(double) * nw * cap));
  ck(cudaMalloc(&d_na, sizeof(int32_t)));
  int32_t* h_na = nullptr;
  ck(cudaMallocHost(&h_na, sizeof(int32_t)));
  if (rc == HODLR2D_OK) {
    ck(cudaMemcpyAsync(d_st, st.data(), sizeof(WideState) * nw, cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(d_r, rch.data(), sizeof(int2) * nr, cudaMemcpyHostToDevice, s));
    ck(cudaMemcpyAsync(d_c, cch.data(), sizeof(int2) * nc, cudaMemcpyHostToDevice, s));
  }
  W.st = d_st;
  W.rchunks = d_r;
  W.cchunks = d_c;
  W.ppiv = d_piv;
  W.pdot = d_dot;
  W.svec = d_sv;
  if (rc == HODLR2D_OK) {
    k_winit<<<nw, kWideT, 0, s>>>(W);
    ck(cudaGetLastError());
  }
  for (int64_t round = 0; rc == HODLR2D_OK && round < max_rounds; ++round) {
    k_wrow<<<(unsigned)nc, kWideT, 0, s>>>(W, nc);
    k_wpiv<<<nw, kWideT, 0, s>>>(W);
    k_wcol<<<(unsigned)(nr + nc), kWideT, 0, s>>>(W, nc);
    k_wfin<<<nw, kWideT, 0, s>>>(W);
    ck(cudaGetLastError());
    if (round % 4 == 3 || round + 1 == max_rounds) {  // poll every fourth round
      k_wdone<<<1, 32, 0, s>>>(d_st, nw, A.rank, A.conv, d_na);
      ck(cudaGetLastError());
      ck(cudaMemcpyAsync(h_na, d_na, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      ck(cudaStreamSynchronize(s));
      if (rc == HODLR2D_OK && *h_na == 0) break;
    }
  }
  if (rc == HODLR2D_OK) {  // ranks of pairs that finished before the last poll
    k_wdone<<<1, 32, 0, s>>>(d_st, nw, A.rank, A.conv, d_na);
    ck(cudaGetLastError());
    ck(cudaStreamSynchronize(s));
  }
  cudaFree(d_st);
  cudaFree(d_r);
  cudaFree(d_c);
  cudaFree(d_piv);
  cudaFree(d_dot);
  cudaFree(d_sv);
  cudaFree(d_na);
  cudaFreeHost(h_na);
  return rc;
}

int mlp_predict_device(hodlr2d_rank_model* M, const float* d_feats, int64_t n, float* d_out,
                       cudaStream_t s);

// The 8 geometry features of a stored pair (X, Y) at level l: level, offset
// of Y from X in box units, box sizes (log2), kernel parameter relative to
// the box width, -log10(eps), kernel kind.  Inputs of the rank predictor.
void pair_features(const hodlr2d* h, int l, int32_t bx, int32_t by, int64_t m, int64_t n,
                   float* f) {
  int ax, ay, cx, cy;
  morton_decode((uint32_t)bx, ax, ay);
  morton_decode((uint32_t)by, cx, cy);
  const double wl = h->root[2] / (double)(1 << l);
  f[0] = (float)l / 16.f;
  f[1] = (float)(cx - ax) / 3.f;
  f[2] = (float)(cy - ay) / 3.f;
  f[3] = (float)(log2((double)std::max<int64_t>(m, 1)) / 16.0);
  f[4] = (float)(log2((double)std::max<int64_t>(n, 1)) / 16.0);
  f[5] = (float)(std::min(h->kp.a / wl, 4.0) / 4.0);
  f[6] = (float)(-log10(h->eps) / 16.0);
  f[7] = (float)h->kp.kind / 8.f;
}

// Compress every pair of every level; fills Level::{d_rank, d_foff, d_fac,
// nvalues, nstored, max_rank, h_rank, h_foff}, the unconverged count, and the
// predictor statistics.
//
// With a rank model in the options, each pair's ACA runs with the cap the
// model predicts (1.25 (2^y - 1) + 4, within min(|X|, |Y|, max_rank)): the
// workspace is sized from the predictions.  A pair that reaches its
// predicted cap without meeting eps is compressed again with the full cap
// (plain adaptive ACA); the first terms are the same, so the factors equal
// those of a build without the model.
int aca_build(hodlr2d* h) {
  cudaStream_t s = h->stream;
  const int capmax = h->opts.max_rank;
  const size_t smem = sizeof(double) * (4 * (size_t)capmax + 2);
  // workspace values per batch: an eighth of the free device memory, between
  // 2 and 16 GiB, so that the few huge coarse pairs share batches
  int64_t ws_budget = (int64_t)1 << 28;
  {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
      ws_budget = std::min<int64_t>(std::max<int64_t>((int64_t)(free_b / 8 / sizeof(double)),
                                                      (int64_t)1 << 28),
                                    (int64_t)1 << 31);
    else
      (void)cudaGetLastError();
  }
  hodlr2d_rank_model* model = reinterpret_cast<hodlr2d_rank_model*>(h->opts.rank_model);
  int64_t unconverged = 0, fallbacks = 0, ws_peak = 0;
  for (int l = h->kappa; l >= 1; --l) {  // Alg. 1: levels kappa down to 1
    Level& L = h->lev[l];
    const int64_t np = L.npairs;
    H2D_CK(cudaMalloc(&L.d_rank, sizeof(int32_t) * (np + 1)));
    H2D_CK(cudaMalloc(&L.d_foff, sizeof(int64_t) * (np + 1)));
    L.h_rank.assign(np, 0);
    L.h_foff.assign(np + 1, 0);
    if (np == 0) {
      H2D_CK(cudaMemsetAsync(L.d_foff, 0, sizeof(int64_t), s));
      H2D_CK(cudaMalloc(&L.d_fac, sizeof(double)));
      continue;
    }
    std::vector<int32_t> px(np), py(np);
    H2D_CK(cudaMemcpyAsync(px.data(), L.d_px, sizeof(int32_t) * np, cudaMemcpyDeviceToHost, s));
    H2D_CK(cudaMemcpyAsync(py.data(), L.d_py, sizeof(int32_t) * np, cudaMemcpyDeviceToHost, s));
    H2D_CK(cudaStreamSynchronize(s));
    const int sh = 2 * (h->kappa - l);
    auto cnt = [&](int32_t b) {
      return (int64_t)h->h_leaf_off[(int64_t)(b + 1) << sh] - h->h_leaf_off[(int64_t)b << sh];
    };
    std::vector<int64_t> mm(np), nn(np);
    std::vector<int32_t> full(np), capv(np);
    int64_t tot_rows = 0;
    for (int64_t p = 0; p < np; ++p) {
      mm[p] = cnt(px[p]);
      nn[p] = cnt(py[p]);
      full[p] = (int32_t)std::min<int64_t>(std::min(mm[p], nn[p]), capmax);
      capv[p] = full[p];
      tot_rows += mm[p] + nn[p];
    }
    if (model) {  // predicted caps
      std::vector<float> feats(8 * np), pred(np);
      for (int64_t p = 0; p < np; ++p)
        pair_features(h, l, px[p], py[p], mm[p], nn[p], feats.data() + 8 * p);
      float *d_f = nullptr, *d_p = nullptr;
      H2D_CK(cudaMalloc(&d_f, 4 * 8 * np));
      H2D_CK(cudaMalloc(&d_p, 4 * np));
      H2D_CK(cudaMemcpy(d_f, feats.data(), 4 * 8 * np, cudaMemcpyHostToDevice));
      H2D_TRY(mlp_predict_device(model, d_f, np, d_p, 0));
      H2D_CK(cudaMemcpy(pred.data(), d_p, 4 * np, cudaMemcpyDeviceToHost));
      cudaFree(d_f);
      cudaFree(d_p);
      for (int64_t p = 0; p < np; ++p) {
        const double y = std::min<double>(std::max<double>(pred[p], 0.0), 20.0);
        const int c = (int)ceil(1.25 * (exp2(y) - 1.0)) + 4;
        capv[p] = std::max(1, std::min(full[p], c));
      }
    }
    int32_t* d_conv = nullptr;
    H2D_CK(cudaMalloc(&d_conv, sizeof(int32_t) * np));
    const int mean_rows = (int)(tot_rows / (2 * np));
    // staging of finished pairs: (buffer, offset) per pair
    std::vector<double*> stage_bufs;
    std::vector<const double*> src_of(np, nullptr);
    std::vector<int64_t> packed(np, 0);
    std::vector<int32_t> conv(np, 0);
    std::vector<int64_t> todo(np);
    for (int64_t p = 0; p < np; ++p) todo[p] = p;
    for (int pass = 0; pass < 2 && !todo.empty(); ++pass) {
      const std::vector<int32_t>& caps = pass == 0 ? capv : full;
      std::vector<int64_t> again;
      size_t b0 = 0;
      while (b0 < todo.size()) {
        size_t b1 = b0;
        int64_t wtot = 0;
        while (b1 < todo.size() &&
               (b1 == b0 || wtot + (mm[todo[b1]] + nn[todo[b1]]) * caps[todo[b1]] <= ws_budget) &&
               b1 - b0 < (1u << 20)) {
          wtot += (mm[todo[b1]] + nn[todo[b1]]) * caps[todo[b1]];
          ++b1;
        }
        const int64_t nbp = (int64_t)(b1 - b0);
        ws_peak = std::max(ws_peak, wtot);
        // pairs for one block each first, then the wide ones
        std::vector<int64_t> order(todo.begin() + b0, todo.begin() + b1);
        auto is_wide = [&](int64_t p) {
          return mm[p] + nn[p] >= kWideRows && caps[p] <= 256;
        };
        std::stable_partition(order.begin(), order.end(), [&](int64_t p) { return !is_wide(p); });
        int64_t nnarrow = 0;
        while (nnarrow < nbp && !is_wide(order[nnarrow])) ++nnarrow;
        std::vector<int64_t> plist(nbp), wsoff(nbp), fgoff(nbp);
        std::vector<int32_t> bcap(nbp);
        int64_t wo = 0, fo = 0;
        for (int64_t i = 0; i < nbp; ++i) {
          const int64_t p = order[i];
          plist[i] = p;
          bcap[i] = caps[p];
          wsoff[i] = wo;
          fgoff[i] = fo;
          wo += (mm[p] + nn[p]) * caps[p];
          fo += mm[p];
        }
        double* d_ws = nullptr;
        uint8_t* d_flags = nullptr;
        int64_t *d_plist = nullptr, *d_wsoff = nullptr, *d_fgoff = nullptr, *d_dst = nullptr;
        int32_t* d_bcap = nullptr;
        H2D_CK(cudaMalloc(&d_ws, sizeof(double) * std::max<int64_t>(wo, 1)));
        H2D_CK(cudaMalloc(&d_flags, std::max<int64_t>(fo, 1)));
        H2D_CK(cudaMalloc(&d_plist, sizeof(int64_t) * nbp));
        H2D_CK(cudaMalloc(&d_wsoff, sizeof(int64_t) * nbp));
        H2D_CK(cudaMalloc(&d_fgoff, sizeof(int64_t) * nbp));
        H2D_CK(cudaMalloc(&d_dst, sizeof(int64_t) * nbp));
        H2D_CK(cudaMalloc(&d_bcap, sizeof(int32_t) * nbp));
        H2D_CK(cudaMemcpyAsync(d_plist, plist.data(), 8 * nbp, cudaMemcpyHostToDevice, s));
        H2D_CK(cudaMemcpyAsync(d_wsoff, wsoff.data(), 8 * nbp, cudaMemcpyHostToDevice, s));
        H2D_CK(cudaMemcpyAsync(d_fgoff, fgoff.data(), 8 * nbp, cudaMemcpyHostToDevice, s));
        H2D_CK(cudaMemcpyAsync(d_bcap, bcap.data(), 4 * nbp, cudaMemcpyHostToDevice, s));
        AcaArgs A;
        A.x = h->d_x;
        A.y = h->d_y;
        A.perm = h->d_perm;
        A.leaf_off = h->d_leaf_off;
        A.kappa = h->kappa;
        A.l = l;
        A.kp = h->kp;
        A.eps = h->eps;
        A.max_rank = capmax;
        A.px = L.d_px;
        A.py = L.d_py;
        A.p0 = 0;
        A.wsoff = d_wsoff;
        A.fgoff = d_fgoff;
        A.ws = d_ws;
        A.flags = d_flags;
        A.rank = L.d_rank;
        A.conv = d_conv;
        A.plist = d_plist;
        A.bcap = d_bcap;
        if (nnarrow > 0) {
          if (mean_rows <= 96)
            k_aca<64><<<(unsigned)nnarrow, 64, smem, s>>>(A);
          else
            k_aca<256><<<(unsigned)nnarrow, 256, smem, s>>>(A);
          H2D_CK(cudaGetLastError());
        }
        if (nnarrow < nbp) {
          std::vector<WideState> wst;
          for (int64_t i = nnarrow; i < nbp; ++i) {
            const int64_t p = plist[i];
            WideState S{};
            S.p = p;
            S.wsoff = wsoff[i];
            S.fgoff = fgoff[i];
            S.xs = h->h_leaf_off[(int64_t)px[p] << sh];
            S.ys = h->h_leaf_off[(int64_t)py[p] << sh];
            S.m = (int32_t)mm[p];
            S.n = (int32_t)nn[p];
            S.kfull = (int32_t)std::min(mm[p], nn[p]);
            S.cap = bcap[i];
            wst.push_back(S);
          }
          H2D_TRY(aca_wide(A, std::move(wst), s));
        }
        std::vector<int32_t> rk(np), cv(np);
        H2D_CK(cudaMemcpyAsync(rk.data(), L.d_rank, 4 * np, cudaMemcpyDeviceToHost, s));
        H2D_CK(cudaMemcpyAsync(cv.data(), d_conv, 4 * np, cudaMemcpyDeviceToHost, s));
        H2D_CK(cudaStreamSynchronize(s));
        // finished pairs go to a staging buffer; capped ones are redone
        std::vector<int64_t> dst(nbp, -1);
        int64_t so = 0;
        for (int64_t i = 0; i < nbp; ++i) {
          const int64_t p = plist[i];
          L.h_rank[p] = rk[p];
          conv[p] = cv[p];
          if (pass == 0 && !cv[p] && rk[p] == caps[p] && caps[p] < full[p]) {
            again.push_back(p);
            continue;
          }
          dst[i] = so;
          packed[p] = (ldpad(mm[p]) + ldpad(nn[p])) * (int64_t)rk[p];
          so += packed[p];
        }
        double* sb = nullptr;
        H2D_CK(cudaMalloc(&sb, sizeof(double) * std::max<int64_t>(so, 1)));
        stage_bufs.push_back(sb);
        for (int64_t i = 0; i < nbp; ++i)
          if (dst[i] >= 0) src_of[plist[i]] = sb + dst[i];
        H2D_CK(cudaMemcpyAsync(d_dst, dst.data(), 8 * nbp, cudaMemcpyHostToDevice, s));
        k_compact<<<(unsigned)nbp, 256, 0, s>>>(d_ws, d_wsoff, h->d_leaf_off, h->kappa, l, L.d_px,
                                                L.d_py, d_plist, L.d_rank, d_bcap, d_dst, sb);
        H2D_CK(cudaGetLastError());
        H2D_CK(cudaStreamSynchronize(s));
        cudaFree(d_ws);
        cudaFree(d_flags);
        cudaFree(d_plist);
        cudaFree(d_wsoff);
        cudaFree(d_fgoff);
        cudaFree(d_dst);
        cudaFree(d_bcap);
        b0 = b1;
      }
      if (pass == 0) fallbacks += (int64_t)again.size();
      todo.swap(again);
    }
    // pack in pair order
    int64_t tot = 0, stored = 0;
    for (int64_t p = 0; p < np; ++p) {
      L.h_foff[p] = tot;
      tot += packed[p];
      stored += (mm[p] + nn[p]) * (int64_t)L.h_rank[p];
    }
    L.h_foff[np] = tot;
    L.nvalues = tot;
    L.nstored = stored;
    // 16 bytes of slack: bulk copies widen each column to 16-byte boundaries
    H2D_CK(cudaMalloc(&L.d_fac, sizeof(double) * (std::max<int64_t>(tot, 1) + 2)));
    H2D_CK(cudaMemcpy(L.d_foff, L.h_foff.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice));
    {
      const double** d_src = nullptr;
      int64_t* d_cnt = nullptr;
      H2D_CK(cudaMalloc(&d_src, sizeof(double*) * np));
      H2D_CK(cudaMalloc(&d_cnt, sizeof(int64_t) * np));
      H2D_CK(cudaMemcpy(d_src, src_of.data(), sizeof(double*) * np, cudaMemcpyHostToDevice));
      H2D_CK(cudaMemcpy(d_cnt, packed.data(), sizeof(int64_t) * np, cudaMemcpyHostToDevice));
      k_pack_pairs<<<(unsigned)np, 256, 0, s>>>(d_src, d_cnt, L.d_foff, L.d_fac);
      H2D_CK(cudaGetLastError());
      H2D_CK(cudaStreamSynchronize(s));
      cudaFree(d_src);
      cudaFree(d_cnt);
    }
    for (double* b : stage_bufs) cudaFree(b);
    cudaFree(d_conv);
    L.max_rank = 0;
    for (int64_t p = 0; p < np; ++p) {
      L.max_rank = std::max(L.max_rank, L.h_rank[p]);
      unconverged += conv[p] ? 0 : 1;
    }
  }
  h->st.unconverged = unconverged;
  h->st.aca_fallbacks = fallbacks;
  h->st.aca_workspace_values = ws_peak;
  return HODLR2D_OK;
}

}  // namespace h2d
