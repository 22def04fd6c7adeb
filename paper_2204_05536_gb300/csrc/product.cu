// The HODLR2D product (Alg. 2), second generation: native FP64 (F64A) or
// float-float (DF32A) arithmetic over the same factor layout.
//
// Far field, levels whose boxes hold <= kFuseRows points ("fused" levels):
// one thread block per row box X reads each stored pair (X,Y), Y > X, once:
//   t1 = V^T x_Y and t2 = U^T x_X      (one warp per column, shuffle sums)
//   y_X += U t1                         (one thread per row, kept on chip)
//   partial_(X,Y) = V t2                (one thread per row of Y, to HBM)
// The pair is staged in shared memory while it is read when it fits, so the
// expansions re-read it from there.  Each box's own sum goes to its level
// slab; the partials are added by the combine pass in a fixed order.
// Coarser levels (huge boxes) use a projection pass over row chunks, a fixed-
// order sum of the chunk partials, and an expansion pass.
// Near field: every leaf against itself and its edge sharers, entries
// evaluated from the points.
// No atomics anywhere: a product is bitwise reproducible.
#include <algorithm>
#include <vector>

#include "arith.cuh"
#include "internal.h"

namespace h2d {

constexpr int kFuseRows = 4096;   // largest box handled by the fused kernel
constexpr int kSmallRows = 256;   // boxes up to this size use small blocks
constexpr int kChunk2 = 2048;     // row chunk of the two-pass levels
constexpr int kNearRhs = 4;       // right-hand sides per near-field pass

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
};

struct ArgsV2 {
  LevelV2 lev[HODLR2D_MAX_LEVELS];
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

// ---------------------------------------------------------------------------
// gather x into tree order
// ---------------------------------------------------------------------------
template <class A>
__global__ void k_gather2(const double* __restrict__ x, const int64_t* __restrict__ perm,
                          int64_t n, int nrhs, typename A::val* __restrict__ xt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t g = perm[i];
  for (int c = 0; c < nrhs; ++c) xt[i + c * n] = A::from_double(x[g + c * n]);
}

// ---------------------------------------------------------------------------
// near field, float-float: one block per leaf, sources staged in shared memory
// ---------------------------------------------------------------------------
constexpr int kNearThreads = 64;
constexpr int kNearStage = 256;

__global__ void __launch_bounds__(kNearThreads)
    k_near_df32(const float2* __restrict__ xf, const float2* __restrict__ yf,
                const int64_t* __restrict__ perm, const int32_t* __restrict__ leaf_off, int kappa,
                KernelFF kp, const float2* __restrict__ xt, int64_t n, int nrhs,
                float2* __restrict__ yout) {
  __shared__ float2 sxy[kNearStage][2];
  __shared__ int64_t sg[kNearStage];
  __shared__ float2 sv[kNearRhs][kNearStage];
  const uint32_t b = blockIdx.x;
  const int32_t s0 = leaf_off[b], m = leaf_off[b + 1] - s0;
  if (m == 0) return;
  int cx, cy;
  morton_decode(b, cx, cy);
  const int side = 1 << kappa;
  uint32_t src[5];
  int ns = 0;
  src[ns++] = b;
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
  for (int i = 0; i < nn; ++i) src[ns++] = nb[i];
  // targets in rounds of kNearThreads, right-hand sides in blocks of kNearRhs
  for (int t0 = 0; t0 < m; t0 += kNearThreads) {
    const int t = t0 + threadIdx.x;
    const bool act = t < m;
    const int64_t it = s0 + (act ? t : 0);
    const float2 xi = xf[it], yi = yf[it];
    const int64_t gi = perm[it];
    for (int c0 = 0; c0 < nrhs; c0 += kNearRhs) {
      const int nc = min(kNearRhs, nrhs - c0);
      float2 acc[kNearRhs];
#pragma unroll
      for (int r = 0; r < kNearRhs; ++r) acc[r] = DF32A::zero();
      for (int q = 0; q < ns; ++q) {
        const int32_t a = leaf_off[src[q]], e = leaf_off[src[q] + 1];
        for (int32_t j0 = a; j0 < e; j0 += kNearStage) {
          const int cnt = min(kNearStage, e - j0);
          __syncthreads();
          for (int u = threadIdx.x; u < cnt; u += kNearThreads) {
            sxy[u][0] = xf[j0 + u];
            sxy[u][1] = yf[j0 + u];
            sg[u] = perm[j0 + u];
            for (int r = 0; r < nc; ++r) sv[r][u] = xt[(int64_t)(c0 + r) * n + j0 + u];
          }
          __syncthreads();
          if (act)
            for (int u = 0; u < cnt; ++u) {
              const float2 kij = entry_ff(kp, xi, yi, gi, sxy[u][0], sxy[u][1], sg[u]);
#pragma unroll
              for (int r = 0; r < kNearRhs; ++r)
                if (r < nc) DF32A::fma(acc[r], kij, sv[r][u]);
            }
        }
      }
      if (act)
        for (int r = 0; r < nc; ++r) yout[(int64_t)(c0 + r) * n + it] = DF32A::fin(acc[r]);
    }
  }
}

// ---------------------------------------------------------------------------
// fused far field (levels >= lfuse): one block per row box
// ---------------------------------------------------------------------------
template <class A, int T>
__global__ void __launch_bounds__(T)
    k_fused(ArgsV2 P, const int2* __restrict__ tasks, int rmax, int kmax, int svals,
            const typename A::val* __restrict__ xt, typename A::val* __restrict__ yl,
            typename A::val* __restrict__ ppart) {
  using V = typename A::val;
  using Acc = typename A::acc;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sx = reinterpret_cast<V*>(smraw);
  V* sy = sx + rmax;
  Acc* yacc = reinterpret_cast<Acc*>(sy + rmax);
  V* t1 = reinterpret_cast<V*>(yacc + rmax);
  V* t2 = t1 + kmax;
  V* stage = t2 + kmax;
  constexpr int NW = T / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int2 task = tasks[blockIdx.x];
  const int l = task.x;
  const uint32_t X = (uint32_t)task.y;
  const LevelV2& L = P.lev[l];
  const int32_t xs = bstart(P.leaf_off, P.kappa, l, X);
  const int32_t m = bsize(P.leaf_off, P.kappa, l, X);
  const int64_t lm = ldpad(m);
  const int64_t p0 = L.prow[X], p1 = L.prow[X + 1];
  const V* fac = reinterpret_cast<const V*>(L.fac);
  for (int c = 0; c < P.nrhs; ++c) {
    const V* xc = xt + (int64_t)c * P.n;
    for (int i = tid; i < m; i += T) {
      sx[i] = xc[xs + i];
      yacc[i] = A::zero();
    }
    for (int64_t p = p0; p < p1; ++p) {
      const int k = L.rank[p];
      const uint32_t Y = (uint32_t)L.py[p];
      const int32_t ys = bstart(P.leaf_off, P.kappa, l, Y);
      const int32_t n = bsize(P.leaf_off, P.kappa, l, Y);
      const int64_t ln = ldpad(n);
      const V* Ug = fac + L.foff[p];
      const V* Vg = Ug + lm * k;
      const bool staged = (lm + ln) * k <= (int64_t)svals;
      for (int j = tid; j < n; j += T) sy[j] = xc[ys + j];
      __syncthreads();
      for (int job = warp; job < 2 * k; job += NW) {
        const bool isV = job < k;
        const int q = isV ? job : job - k;
        const int rows = isV ? n : m;
        const int64_t ld = isV ? ln : lm;
        const V* col = (isV ? Vg : Ug) + q * ld;
        const V* xv = isV ? sy : sx;
        Acc a = A::zero();
        if (staged) {
          V* st = stage + (isV ? lm * k : 0) + q * ld;
          for (int r = lane; r < rows; r += 32) {
            const V v = col[r];
            st[r] = v;
            A::fma(a, v, xv[r]);
          }
        } else {
          for (int r = lane; r < rows; r += 32) A::fma(a, col[r], xv[r]);
        }
        const V s = A::warp_sum(a);
        if (lane == 0) (isV ? t1 : t2)[q] = s;
      }
      __syncthreads();
      const V* Us = staged ? stage : Ug;
      const V* Vs = staged ? stage + lm * k : Vg;
      for (int i = tid; i < m; i += T) {
        Acc a = yacc[i];
        for (int q = 0; q < k; ++q) A::fma(a, Us[q * lm + i], t1[q]);
        yacc[i] = a;
      }
      V* out = ppart + (int64_t)c * P.pstride + L.ppoff[p];
      for (int j = tid; j < n; j += T) {
        Acc a = A::zero();
        for (int q = 0; q < k; ++q) A::fma(a, Vs[q * ln + j], t2[q]);
        out[j] = A::fin(a);
      }
      __syncthreads();
    }
    V* own = yl + ((int64_t)l * P.nrhs + c) * P.n + xs;
    for (int i = tid; i < m; i += T) own[i] = A::fin(yacc[i]);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// two-pass far field (levels < lfuse)
// ---------------------------------------------------------------------------
template <class A>
__global__ void k_proj2(ArgsV2 P, const ProjTask* __restrict__ tasks, int64_t ntasks,
                        const typename A::val* __restrict__ xt, typename A::val* __restrict__ part) {
  using V = typename A::val;
  using Acc = typename A::acc;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= ntasks) return;
  const ProjTask T = tasks[w];
  const LevelV2& L = P.lev[T.level];
  const uint32_t bx = (uint32_t)L.px[T.pair], by = (uint32_t)L.py[T.pair];
  const int32_t m = bsize(P.leaf_off, P.kappa, T.level, bx);
  const int32_t nrow = T.side == 0 ? bsize(P.leaf_off, P.kappa, T.level, by) : m;
  const int32_t base = bstart(P.leaf_off, P.kappa, T.level, T.side == 0 ? by : bx);
  const int k = L.rank[T.pair];
  const V* M = reinterpret_cast<const V*>(L.fac) + L.foff[T.pair] + (T.side == 0 ? ldpad(m) * k : 0);
  const int64_t ld = ldpad(nrow);
  for (int c = 0; c < P.nrhs; ++c) {
    const V* xv = xt + c * P.n + base;
    for (int q = 0; q < k; ++q) {
      const V* col = M + q * ld;
      Acc a = A::zero();
      for (int i = T.r0 + lane; i < T.r0 + T.nr; i += 32) A::fma(a, col[i], xv[i]);
      const V s = A::warp_sum(a);
      if (lane == 0) part[T.out * P.nrhs + (int64_t)c * k + q] = s;
    }
  }
}

template <class A>
__global__ void k_tsum2(ArgsV2 P, const ProjTask* __restrict__ tasks,
                        const int64_t* __restrict__ red, int64_t nsides,
                        const typename A::val* __restrict__ part, typename A::val* __restrict__ t) {
  using V = typename A::val;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nsides) return;
  const int64_t first = red[2 * s], count = red[2 * s + 1];
  if (count == 0) return;
  const ProjTask T0 = tasks[first];
  const LevelV2& L = P.lev[T0.level];
  const int k = L.rank[T0.pair];
  V* out = t + L.toff[T0.pair] * P.nrhs + (int64_t)T0.side * k * P.nrhs;
  for (int c = 0; c < P.nrhs; ++c)
    for (int q = 0; q < k; ++q) {
      V acc = A::vzero();
      for (int64_t j = 0; j < count; ++j)
        acc = A::add(acc, part[tasks[first + j].out * P.nrhs + c * k + q]);
      out[c * k + q] = acc;
    }
}

template <class A>
__global__ void k_exp2(ArgsV2 P, const ExpTask* __restrict__ tasks, int64_t ntasks,
                       const typename A::val* __restrict__ t, typename A::val* __restrict__ yl) {
  using V = typename A::val;
  using Acc = typename A::acc;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= ntasks) return;
  const ExpTask T = tasks[w];
  const LevelV2& L = P.lev[T.level];
  const uint32_t X = (uint32_t)T.box;
  const int32_t base = bstart(P.leaf_off, P.kappa, T.level, X);
  const int32_t nX = bsize(P.leaf_off, P.kappa, T.level, X);
  const int64_t ld = ldpad(nX);
  const int32_t e0 = L.ent_off[X], e1 = L.ent_off[X + 1];
  const V* fac = reinterpret_cast<const V*>(L.fac);
  for (int c = 0; c < P.nrhs; ++c) {
    V* out = yl + ((int64_t)T.level * P.nrhs + c) * P.n + base;
    for (int i = T.r0 + lane; i < T.r0 + T.nr; i += 32) {
      Acc a = A::zero();
      for (int32_t e = e0; e < e1; ++e) {
        const int32_t code = L.ent[e];
        const int64_t p = code >> 1;
        const int side = code & 1;
        const int k = L.rank[p];
        int64_t off = L.foff[p];
        if (side == 1) off += ldpad(bsize(P.leaf_off, P.kappa, T.level, (uint32_t)L.px[p])) * k;
        const V* M = fac + off;
        const V* tv = t + L.toff[p] * P.nrhs + (int64_t)side * k * P.nrhs + (int64_t)c * k;
        for (int q = 0; q < k; ++q) A::fma(a, M[q * ld + i], tv[q]);
      }
      out[i] = A::fin(a);
    }
  }
}

// ---------------------------------------------------------------------------
// combine: y[perm[i]] = near + sum over levels of (own / two-pass result)
// + the partials of the pairs in which the point's box is the column side
// ---------------------------------------------------------------------------
template <class A>
__global__ void k_combine2(ArgsV2 P, const typename A::val* __restrict__ yl,
                           const typename A::val* __restrict__ ppart,
                           const int32_t* __restrict__ leaf_of, const int64_t* __restrict__ perm,
                           double* __restrict__ y) {
  using V = typename A::val;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  const uint32_t leaf = (uint32_t)leaf_of[i];
  const int64_t g = perm[i];
  for (int c = 0; c < P.nrhs; ++c) {
    V acc = yl[(int64_t)c * P.n + i];
    for (int l = 1; l <= P.kappa; ++l) {
      acc = A::add(acc, yl[((int64_t)l * P.nrhs + c) * P.n + i]);
      if (l < P.lfuse) continue;
      const LevelV2& L = P.lev[l];
      const uint32_t B = leaf >> (2 * (P.kappa - l));
      const int64_t loc = i - bstart(P.leaf_off, P.kappa, l, B);
      const V* pc = ppart + (int64_t)c * P.pstride;
      for (int32_t e = L.ent_off[B]; e < L.ent_off[B + 1]; ++e) {
        const int32_t code = L.ent[e];
        if (code & 1) acc = A::add(acc, pc[L.ppoff[code >> 1] + loc]);
      }
    }
    y[g + (int64_t)c * P.n] = A::to_double(acc);
  }
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
// FP64 near field (defined with the first-generation product)
__global__ void k_near_f64(const double* __restrict__ xs, const double* __restrict__ ys,
                           const int64_t* __restrict__ perm, const int32_t* __restrict__ leaf_off,
                           int kappa, KernelParams kp, const double* __restrict__ xt, int64_t n,
                           int nrhs, double* __restrict__ yout);

static ArgsV2 args_v2(const hodlr2d* h, int nrhs, int mode) {
  ArgsV2 P;
  for (int l = 0; l < HODLR2D_MAX_LEVELS; ++l) {
    const Level& L = h->lev[l];
    const void* fac = mode == HODLR2D_MODE_F64 ? (const void*)L.d_fac : L.d_fac_mode[mode];
    P.lev[l] = LevelV2{L.d_px, L.d_py, L.d_rank, L.d_foff, L.d_prow, L.d_ppoff,
                       L.d_toff, L.d_ent_off, L.d_ent, fac};
  }
  P.leaf_off = h->d_leaf_off;
  P.kappa = h->kappa;
  P.lfuse = h->v2.lfuse;
  P.n = h->n;
  P.nrhs = nrhs;
  P.pstride = h->v2.pstride;
  return P;
}

// Plan of the v2 product (once per handle, after the factors exist).
int plan_v2(hodlr2d* h) {
  V2Plan& V = h->v2;
  if (V.ready) return HODLR2D_OK;
  const int kappa = h->kappa;
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
  // two-pass task lists for levels < lfuse
  std::vector<ProjTask> proj;
  std::vector<ExpTask> exps;
  std::vector<int64_t> red;
  int64_t out = 0;
  for (int l = 1; l < V.lfuse; ++l) {
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
          for (int32_t r0 = 0; r0 < rows; r0 += kChunk2) {
            ProjTask T;
            T.level = l;
            T.side = side;
            T.pair = p;
            T.r0 = r0;
            T.nr = std::min(kChunk2, rows - r0);
            T.out = out;
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
  // fused levels: partial offsets (|Y| per pair, absolute) and block tasks
  std::vector<int2> big, small;
  int64_t pbase = 0;
  V.kmax = 1;
  V.rmax_big = 1;
  V.rmax_small = 1;
  for (int l = V.lfuse; l <= kappa; ++l) {
    Level& L = h->lev[l];
    const int64_t np = L.npairs;
    const int sh = 2 * (kappa - l);
    std::vector<int32_t> py(np);
    if (np) H2D_CK(cudaMemcpy(py.data(), L.d_py, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    std::vector<int64_t> pp(np + 1);
    for (int64_t p = 0; p < np; ++p) {
      pp[p] = pbase;
      pbase += h->h_leaf_off[(int64_t)(py[p] + 1) << sh] - h->h_leaf_off[(int64_t)py[p] << sh];
    }
    pp[np] = pbase;
    L.npart = pp[np] - pp[0];
    H2D_CK(cudaMalloc(&L.d_ppoff, sizeof(int64_t) * (np + 1)));
    H2D_CK(cudaMemcpy(L.d_ppoff, pp.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice));
    V.kmax = std::max(V.kmax, L.max_rank);
    const int64_t mc = maxcount(l);
    const bool is_small = mc <= kSmallRows;
    if (is_small) V.rmax_small = std::max<int64_t>(V.rmax_small, mc);
    else V.rmax_big = std::max<int64_t>(V.rmax_big, mc);
    for (int64_t b = 0; b < ((int64_t)1 << (2 * l)); ++b) {
      if (h->h_leaf_off[(b + 1) << sh] == h->h_leaf_off[b << sh]) continue;
      (is_small ? small : big).push_back(make_int2(l, (int)b));
    }
  }
  V.pstride = std::max<int64_t>(pbase, 1);
  V.nbig = (int64_t)big.size();
  V.nsmall = (int64_t)small.size();
  H2D_CK(cudaMalloc(&V.d_big, sizeof(int2) * std::max<int64_t>(V.nbig, 1)));
  H2D_CK(cudaMalloc(&V.d_small, sizeof(int2) * std::max<int64_t>(V.nsmall, 1)));
  if (V.nbig) H2D_CK(cudaMemcpy(V.d_big, big.data(), sizeof(int2) * V.nbig, cudaMemcpyHostToDevice));
  if (V.nsmall)
    H2D_CK(cudaMemcpy(V.d_small, small.data(), sizeof(int2) * V.nsmall, cudaMemcpyHostToDevice));
  // leaf of every tree position
  const int64_t nleaf = (int64_t)1 << (2 * kappa);
  H2D_CK(cudaMalloc(&V.d_leaf_of, sizeof(int32_t) * h->n));
  k_leaf_of<<<(unsigned)((nleaf + 255) / 256), 256>>>(h->d_leaf_off, nleaf, V.d_leaf_of);
  H2D_CK(cudaGetLastError());
  H2D_CK(cudaDeviceSynchronize());
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
  H2D_CK(cudaMalloc(&V.d_xt, 8 * n * nrhs));
  H2D_CK(cudaMalloc(&V.d_yl, 8 * n * nrhs * (h->kappa + 1)));
  H2D_CK(cudaMalloc(&V.d_ppart, 8 * V.pstride * nrhs));
  H2D_CK(cudaMalloc(&V.d_part, 8 * std::max<int64_t>(V.proj_partials, 1) * nrhs));
  H2D_CK(cudaMalloc(&V.d_t, 8 * std::max<int64_t>(h->t_total, 1) * nrhs));
  V.scratch_nrhs = nrhs;
  return HODLR2D_OK;
}

static size_t fused_smem(int rmax, int kmax, int svals) {
  return (size_t)8 * (3 * (size_t)rmax + 2 * (size_t)kmax + (size_t)svals);
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
  const int64_t vb = 8 * n * nrhs;
  {
    PhaseScope ps(h, 0, 1, vb + 8 * n + 8 * n * nrhs);
    k_gather2<A><<<g, 256, 0, s>>>(x, h->d_perm, n, nrhs, xt);
  }
  {
    const unsigned nleaf = (unsigned)(1u << (2 * h->kappa));
    PhaseScope ps(h, 1, 1, (mode == HODLR2D_MODE_F64 ? 24 : 24) * n + 2 * vb);
    if (mode == HODLR2D_MODE_F64)
      k_near_f64<<<nleaf, 64, 0, s>>>(h->d_x, h->d_y, h->d_perm, h->d_leaf_off, h->kappa, h->kp,
                                       reinterpret_cast<const double*>(xt), n, nrhs,
                                       reinterpret_cast<double*>(yl));
    else
      k_near_df32<<<nleaf, kNearThreads, 0, s>>>(
          reinterpret_cast<const float2*>(V.d_xf), reinterpret_cast<const float2*>(V.d_yf),
          h->d_perm, h->d_leaf_off, h->kappa, V.kff, reinterpret_cast<const float2*>(xt), n, nrhs,
          reinterpret_cast<float2*>(yl));
  }
  if (V.nproj) {
    int64_t two_pass_vals = 0;
    for (int l = 1; l < V.lfuse; ++l) two_pass_vals += h->lev[l].nstored;
    {
      PhaseScope ps(h, 2, 1, 8 * two_pass_vals + 8 * V.proj_partials * nrhs);
      const int64_t thr = V.nproj * 32;
      k_proj2<A><<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(P, V.d_proj, V.nproj, xt,
                                                                reinterpret_cast<Val*>(V.d_part));
    }
    {
      PhaseScope ps(h, 3, 1, 8 * (V.proj_partials + h->t_total) * nrhs);
      k_tsum2<A><<<(unsigned)((V.nsides + 255) / 256), 256, 0, s>>>(
          P, V.d_proj, V.d_red, V.nsides, reinterpret_cast<const Val*>(V.d_part),
          reinterpret_cast<Val*>(V.d_t));
    }
    {
      PhaseScope ps(h, 4, 1, 8 * two_pass_vals + vb * (V.lfuse - 1));
      const int64_t thr = V.nexp * 32;
      k_exp2<A><<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(
          P, V.d_exp, V.nexp, reinterpret_cast<const Val*>(V.d_t), yl);
    }
  }
  if (V.nbig || V.nsmall) {
    int64_t fused_vals = 0;
    for (int l = V.lfuse; l <= h->kappa; ++l) fused_vals += h->lev[l].nstored;
    PhaseScope ps(h, 6, (V.nbig ? 1 : 0) + (V.nsmall ? 1 : 0),
                  8 * fused_vals + 8 * V.pstride * nrhs + vb * (h->kappa - V.lfuse + 1));
    if (V.nbig) {
      const int svals = 8192;
      const size_t sm = fused_smem((int)V.rmax_big, V.kmax, svals);
      H2D_CK(cudaFuncSetAttribute(k_fused<A, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm));
      k_fused<A, 256><<<(unsigned)V.nbig, 256, sm, s>>>(P, V.d_big, (int)V.rmax_big, V.kmax, svals,
                                                        xt, yl, ppart);
    }
    if (V.nsmall) {
      const int svals = 2048;
      const size_t sm = fused_smem((int)V.rmax_small, V.kmax, svals);
      H2D_CK(cudaFuncSetAttribute(k_fused<A, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm));
      k_fused<A, 64><<<(unsigned)V.nsmall, 64, sm, s>>>(P, V.d_small, (int)V.rmax_small, V.kmax,
                                                        svals, xt, yl, ppart);
    }
  }
  {
    PhaseScope ps(h, 5, 1, vb * (h->kappa + 1) + 8 * V.pstride * nrhs + 16 * n + 8 * n * nrhs);
    k_combine2<A><<<g, 256, 0, s>>>(P, yl, ppart, V.d_leaf_of, h->d_perm, y);
  }
  H2D_CK(cudaGetLastError());
  return HODLR2D_OK;
}

// The product in a prepared mode (F64 or DF32) with device x and y.
int product_device(hodlr2d* h, const double* x, double* y, int nrhs, int mode) {
  H2D_TRY(plan_v2(h));
  H2D_TRY(scratch_v2(h, nrhs));
  if (mode == HODLR2D_MODE_F64) return run_v2<F64A>(h, x, y, nrhs, mode);
  if (mode == HODLR2D_MODE_DF32) return run_v2<DF32A>(h, x, y, nrhs, mode);
  return HODLR2D_ERR_STATE;
}

// Float-float copies of the factors, the points and the kernel parameters.
int prepare_df32(hodlr2d* h) {
  V2Plan& V = h->v2;
  for (int l = 1; l <= h->kappa; ++l) {
    Level& L = h->lev[l];
    if (L.d_fac_mode[HODLR2D_MODE_DF32]) continue;
    const int64_t nv = std::max<int64_t>(L.nvalues, 1);
    H2D_CK(cudaMalloc(&L.d_fac_mode[HODLR2D_MODE_DF32], 8 * nv));
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
  V.kff.p64 = h->kp;
  return HODLR2D_OK;
}

void free_v2(hodlr2d* h) {
  V2Plan& V = h->v2;
  cudaFree(V.d_proj);
  cudaFree(V.d_exp);
  cudaFree(V.d_red);
  cudaFree(V.d_big);
  cudaFree(V.d_small);
  cudaFree(V.d_leaf_of);
  cudaFree(V.d_xt);
  cudaFree(V.d_yl);
  cudaFree(V.d_ppart);
  cudaFree(V.d_part);
  cudaFree(V.d_t);
  cudaFree(V.d_xf);
  cudaFree(V.d_yf);
  V = V2Plan();
}

}  // namespace h2d
