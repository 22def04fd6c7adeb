// MatVec (Alg. 2) on the GPU, FP64, first generation: kept as the product
// behind hodlr2d_matvec_noalloc (caller-provided scratch) and for its plan
// (projection / expansion task lists and t offsets, shared with product.cu).
//
//   1. x is gathered into tree order.
//   2. Near field: every leaf X adds K(X,X) x_X + sum_{Y in E_X} K(X,Y) x_Y,
//      the entries evaluated from the points (Alg. 2, dense leaf products).
//   3. Projection: for every stored pair (X,Y), t1 = V^T x_Y and t2 = U^T x_X,
//      split into row chunks; chunk sums are added in a fixed order.
//   4. Expansion: every box X of level l sums U t1 (X is the row side) or
//      V t2 (X is the column side) over its list, in ascending partner order.
//   5. y = near + level 1 + ... + level kappa, in that order, scattered back
//      to the caller's order.
// No atomics: the result is bitwise reproducible.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace h2d {

constexpr int kChunkRows = 2048;

__global__ void k_gather_x(const double* __restrict__ x, const int64_t* __restrict__ perm,
                           int64_t n, int nrhs, double* __restrict__ xt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t g = perm[i];
  for (int c = 0; c < nrhs; ++c) xt[i + c * n] = x[g + c * n];
}

// y[perm[i]] = sum_{l=0..kappa} yl[l][i]
__global__ void k_combine(const double* __restrict__ yl, int nlev, const int64_t* __restrict__ perm,
                          int64_t n, int nrhs, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t g = perm[i];
  const int64_t stride = n * nrhs;
  for (int c = 0; c < nrhs; ++c) {
    double s = yl[i + c * n];
    for (int l = 1; l < nlev; ++l) s += yl[l * stride + i + c * n];
    y[g + c * n] = s;
  }
}

// Near field: one block per leaf; sources are the leaf itself, then its edge
// sharers in ascending Morton order (Def. ec).
__global__ void k_near_f64(const double* __restrict__ xs, const double* __restrict__ ys,
                           const int64_t* __restrict__ perm, const int32_t* __restrict__ leaf_off,
                           int kappa, KernelParams kp, const double* __restrict__ xt, int64_t n,
                           int nrhs, double* __restrict__ yout) {
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
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    const int64_t it = s0 + t;
    const double xi = xs[it], yi = ys[it];
    const int64_t gi = perm[it];
    for (int c = 0; c < nrhs; ++c) {
      double acc = 0.0;
      for (int q = 0; q < ns; ++q) {
        const int32_t a = leaf_off[src[q]], e = leaf_off[src[q] + 1];
        for (int32_t j = a; j < e; ++j)
          acc += entry(kp, xi, yi, gi, xs[j], ys[j], perm[j]) * xt[j + c * n];
      }
      yout[it + c * n] = acc;
    }
  }
}

struct LevelView {
  const int32_t* px;
  const int32_t* py;
  const int32_t* rank;
  const int64_t* foff;
  const int64_t* toff;
  const double* fac;
  const int32_t* ent_off;
  const int32_t* ent;
};

struct PlanView {
  LevelView lev[HODLR2D_MAX_LEVELS];
  const int32_t* leaf_off;
  int kappa;
  int64_t n;
  int nrhs;
};

__device__ __forceinline__ int32_t box_start(const int32_t* leaf_off, int kappa, int l, uint32_t b) {
  return leaf_off[(int64_t)b << (2 * (kappa - l))];
}
__device__ __forceinline__ int32_t box_size(const int32_t* leaf_off, int kappa, int l, uint32_t b) {
  const int sh = 2 * (kappa - l);
  return leaf_off[(int64_t)(b + 1) << sh] - leaf_off[(int64_t)b << sh];
}

// Projection: one warp per task.  Side 0: V (rows of Y) against x_Y; side 1:
// U (rows of X) against x_X.  Partial sums go to part[out * nrhs + c k + q].
__global__ void k_proj_f64(PlanView P, const ProjTask* __restrict__ tasks, int64_t ntasks,
                           const double* __restrict__ xt, double* __restrict__ part) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= ntasks) return;
  const ProjTask T = tasks[w];
  const LevelView& L = P.lev[T.level];
  const uint32_t bx = (uint32_t)L.px[T.pair], by = (uint32_t)L.py[T.pair];
  const int32_t m = box_size(P.leaf_off, P.kappa, T.level, bx);
  const int32_t nrow = T.side == 0 ? box_size(P.leaf_off, P.kappa, T.level, by) : m;
  const int32_t base = box_start(P.leaf_off, P.kappa, T.level, T.side == 0 ? by : bx);
  const int k = L.rank[T.pair];
  const double* M = L.fac + L.foff[T.pair] + (T.side == 0 ? ldpad(m) * k : 0);
  const int64_t ld = ldpad(nrow);
  for (int c = 0; c < P.nrhs; ++c) {
    const double* xv = xt + c * P.n + base;
    for (int q = 0; q < k; ++q) {
      const double* col = M + (int64_t)q * ld;
      double acc = 0.0;
      for (int i = T.r0 + lane; i < T.r0 + T.nr; i += 32) acc += col[i] * xv[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) part[T.out * P.nrhs + (int64_t)c * k + q] = acc;
    }
  }
}

// t[pair, side] = sum of its chunks' partial sums, chunks in row order.
// red[2 * gp + side] = {first task, count}; one thread per (pair, side).
__global__ void k_tsum(PlanView P, const ProjTask* __restrict__ tasks,
                       const int64_t* __restrict__ red, int64_t nsides,
                       const double* __restrict__ part, double* __restrict__ t) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= nsides) return;
  const int64_t first = red[2 * s], count = red[2 * s + 1];
  if (count == 0) return;
  const ProjTask T0 = tasks[first];
  const LevelView& L = P.lev[T0.level];
  const int k = L.rank[T0.pair];
  double* out = t + L.toff[T0.pair] * P.nrhs + (int64_t)T0.side * k * P.nrhs;
  for (int c = 0; c < P.nrhs; ++c)
    for (int q = 0; q < k; ++q) {
      double acc = 0.0;
      for (int64_t j = 0; j < count; ++j) acc += part[tasks[first + j].out * P.nrhs + c * k + q];
      out[c * k + q] = acc;
    }
}

// Expansion: one warp per task (rows [r0, r0+nr) of box X at level l).
__global__ void k_exp_f64(PlanView P, const ExpTask* __restrict__ tasks, int64_t ntasks,
                          const double* __restrict__ t, double* __restrict__ yl) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= ntasks) return;
  const ExpTask T = tasks[w];
  const LevelView& L = P.lev[T.level];
  const uint32_t X = (uint32_t)T.box;
  const int32_t base = box_start(P.leaf_off, P.kappa, T.level, X);
  const int32_t nX = box_size(P.leaf_off, P.kappa, T.level, X);
  const int32_t e0 = L.ent_off[X], e1 = L.ent_off[X + 1];
  double* out = yl + (int64_t)T.level * P.n * P.nrhs;
  for (int c = 0; c < P.nrhs; ++c) {
    for (int i = T.r0 + lane; i < T.r0 + T.nr; i += 32) {
      double acc = 0.0;
      for (int32_t e = e0; e < e1; ++e) {
        const int32_t code = L.ent[e];
        const int64_t p = code >> 1;
        const int side = code & 1;
        const int k = L.rank[p];
        int64_t off = L.foff[p];
        if (side == 1)
          off += ldpad(box_size(P.leaf_off, P.kappa, T.level, (uint32_t)L.px[p])) * k;
        const double* M = L.fac + off;
        const double* tv = t + L.toff[p] * P.nrhs + (int64_t)side * k * P.nrhs + (int64_t)c * k;
        const int64_t ld = ldpad(nX);
        for (int q = 0; q < k; ++q) acc += M[(int64_t)q * ld + i] * tv[q];
      }
      out[base + i + c * P.n] = acc;
    }
  }
}

// Host-side plan: projection and expansion task lists, t offsets.
int matvec_plan(hodlr2d* h) {
  std::vector<ProjTask> proj;
  std::vector<ExpTask> exps;
  std::vector<int64_t> red;
  int64_t out = 0, tpos = 0;
  for (int l = 1; l <= h->kappa; ++l) {
    Level& L = h->lev[l];
    const int64_t np = L.npairs;
    const int sh = 2 * (h->kappa - l);
    auto cnt = [&](int32_t b) {
      return (int32_t)(h->h_leaf_off[(int64_t)(b + 1) << sh] - h->h_leaf_off[(int64_t)b << sh]);
    };
    std::vector<int32_t> px(np), py(np);
    if (np) {
      H2D_CK(cudaMemcpy(px.data(), L.d_px, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
      H2D_CK(cudaMemcpy(py.data(), L.d_py, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    }
    std::vector<int64_t> toff(np + 1);
    for (int64_t p = 0; p < np; ++p) {
      const int k = L.h_rank[p];
      toff[p] = tpos;
      tpos += 2 * (int64_t)k;
      for (int side = 0; side < 2; ++side) {
        const int32_t rows = side == 0 ? cnt(py[p]) : cnt(px[p]);
        const int64_t first = (int64_t)proj.size();
        if (k > 0)
          for (int32_t r0 = 0; r0 < rows; r0 += kChunkRows) {
            ProjTask T;
            T.level = l;
            T.side = side;
            T.pair = p;
            T.r0 = r0;
            T.nr = std::min(kChunkRows, rows - r0);
            T.out = out;
            out += k;
            proj.push_back(T);
          }
        red.push_back(first);
        red.push_back((int64_t)proj.size() - first);
      }
    }
    toff[np] = tpos;
    H2D_CK(cudaMalloc(&L.d_toff, sizeof(int64_t) * (np + 1)));
    H2D_CK(cudaMemcpy(L.d_toff, toff.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice));
    const int64_t nb = (int64_t)1 << (2 * l);
    for (int64_t b = 0; b < nb; ++b) {
      const int32_t rows = cnt((int32_t)b);
      for (int32_t r0 = 0; r0 < rows; r0 += kChunkRows) {
        ExpTask T;
        T.level = l;
        T.box = (int32_t)b;
        T.r0 = r0;
        T.nr = std::min(kChunkRows, rows - r0);
        exps.push_back(T);
      }
    }
  }
  h->nproj = (int64_t)proj.size();
  h->nexp = (int64_t)exps.size();
  h->proj_partials = out;
  h->t_total = tpos;
  h->nt_sides = (int64_t)red.size() / 2;
  H2D_CK(cudaMalloc(&h->d_proj, sizeof(ProjTask) * std::max<int64_t>(h->nproj, 1)));
  H2D_CK(cudaMalloc(&h->d_exp, sizeof(ExpTask) * std::max<int64_t>(h->nexp, 1)));
  H2D_CK(cudaMalloc(&h->d_tred, sizeof(int64_t) * std::max<int64_t>((int64_t)red.size(), 2)));
  if (h->nproj)
    H2D_CK(cudaMemcpy(h->d_proj, proj.data(), sizeof(ProjTask) * h->nproj, cudaMemcpyHostToDevice));
  if (h->nexp)
    H2D_CK(cudaMemcpy(h->d_exp, exps.data(), sizeof(ExpTask) * h->nexp, cudaMemcpyHostToDevice));
  if (!red.empty())
    H2D_CK(cudaMemcpy(h->d_tred, red.data(), sizeof(int64_t) * red.size(), cudaMemcpyHostToDevice));
  return HODLR2D_OK;
}

static PlanView plan_view(const hodlr2d* h, int nrhs) {
  PlanView P;
  for (int l = 0; l < HODLR2D_MAX_LEVELS; ++l) {
    const Level& L = h->lev[l];
    P.lev[l] = LevelView{L.d_px, L.d_py, L.d_rank, L.d_foff, L.d_toff, L.d_fac, L.d_ent_off, L.d_ent};
  }
  P.leaf_off = h->d_leaf_off;
  P.kappa = h->kappa;
  P.n = h->n;
  P.nrhs = nrhs;
  return P;
}

}  // namespace h2d

namespace h2d {

// The F64 product with caller-supplied scratch (no allocation): xt n x nrhs,
// yl (kappa + 1) x n x nrhs, part proj_partials x nrhs, t t_total x nrhs.
// First-generation kernels: projection by row chunks, fixed-order chunk sums,
// expansion, all in FP64.
int matvec_f64_scratch(hodlr2d* h, const double* x, double* y, int nrhs, double* xt, double* yl,
                       double* part, double* t) {
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  const unsigned g = (unsigned)((n + 255) / 256);
  k_gather_x<<<g, 256, 0, s>>>(x, h->d_perm, n, nrhs, xt);
  const unsigned nleaf = (unsigned)(1u << (2 * h->kappa));
  k_near_f64<<<nleaf, 64, 0, s>>>(h->d_x, h->d_y, h->d_perm, h->d_leaf_off, h->kappa, h->kp, xt,
                                   n, nrhs, yl);
  const PlanView P = plan_view(h, nrhs);
  if (h->nproj) {
    const int64_t thr = h->nproj * 32;
    k_proj_f64<<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(P, h->d_proj, h->nproj, xt, part);
    k_tsum<<<(unsigned)((h->nt_sides + 255) / 256), 256, 0, s>>>(P, h->d_proj, h->d_tred,
                                                                 h->nt_sides, part, t);
  }
  if (h->nexp) {
    const int64_t thr = h->nexp * 32;
    k_exp_f64<<<(unsigned)((thr + 255) / 256), 256, 0, s>>>(P, h->d_exp, h->nexp, t, yl);
  }
  k_combine<<<g, 256, 0, s>>>(yl, h->kappa + 1, h->d_perm, n, nrhs, y);
  H2D_CK(cudaGetLastError());
  return HODLR2D_OK;
}

}  // namespace h2d
