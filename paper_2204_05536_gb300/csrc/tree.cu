// Quadtree (Sec. 4, Alg. 1) and interaction lists (Defs. ec, vc, wc, cc, ic;
// Eq. ilist) on the GPU.
//
// Tree: every point gets its cell at depth 14, floor((x - x0) / w * 2^14)
// clamped to [0, 2^14 - 1]; the cell at depth l is that index shifted right
// by 14 - l, which equals floor((x - x0) / w * 2^l) clamped.  kappa is the
// smallest depth whose leaves all hold <= N_max points.  Points are ordered
// by leaf Morton key (counting sort), then by ascending original index inside
// each leaf, so every box of every level is a contiguous range.
//
// Lists: the interaction list of box C is derived in closed form from the
// clan of Def. cc (siblings of C and the children of its parent's edge
// sharers), keeping the members that share only a vertex with C or none of
// its boundary.  Each unordered pair is stored once, rows = smaller Morton id.
#include <stdio.h>

#include <algorithm>

#include "internal.h"
#include "scan.cuh"

namespace h2d {

constexpr int kDeepLevel = 14;

// ---------------------------------------------------------------------------
// bounding box
// ---------------------------------------------------------------------------
__global__ void k_bbox_partial(const double* __restrict__ pts, int64_t n, double* out) {
  double mn[2] = {INFINITY, INFINITY}, mx[2] = {-INFINITY, -INFINITY};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int d = 0; d < 2; ++d) {
      const double v = pts[2 * i + d];
      mn[d] = fmin(mn[d], v);
      mx[d] = fmax(mx[d], v);
    }
  }
  __shared__ double s[4][256];
  s[0][threadIdx.x] = mn[0];
  s[1][threadIdx.x] = mn[1];
  s[2][threadIdx.x] = mx[0];
  s[3][threadIdx.x] = mx[1];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s[0][threadIdx.x] = fmin(s[0][threadIdx.x], s[0][threadIdx.x + o]);
      s[1][threadIdx.x] = fmin(s[1][threadIdx.x], s[1][threadIdx.x + o]);
      s[2][threadIdx.x] = fmax(s[2][threadIdx.x], s[2][threadIdx.x + o]);
      s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int d = 0; d < 4; ++d) out[4 * blockIdx.x + d] = s[d][0];
}

// NaN / inf check folded into the cell pass: flag[0] = 1 if any coordinate
// is not finite.
__global__ void k_cells(const double* __restrict__ pts, int64_t n, double x0, double y0,
                        double w, int32_t* __restrict__ cx, int32_t* __restrict__ cy,
                        int* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double px = pts[2 * i], py = pts[2 * i + 1];
  if (!isfinite(px) || !isfinite(py)) flag[0] = 1;
  const double m = (double)(1 << kDeepLevel);
  double fx = floor((px - x0) / w * m), fy = floor((py - y0) / w * m);
  fx = fx < 0.0 ? 0.0 : (fx > m - 1.0 ? m - 1.0 : fx);
  fy = fy < 0.0 ? 0.0 : (fy > m - 1.0 ? m - 1.0 : fy);
  cx[i] = isfinite(fx) ? (int32_t)fx : 0;
  cy[i] = isfinite(fy) ? (int32_t)fy : 0;
}

__global__ void k_hist(const int32_t* __restrict__ cx, const int32_t* __restrict__ cy,
                       int64_t n, int level, int32_t* __restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int sh = kDeepLevel - level;
  const uint32_t key = morton_encode((uint32_t)(cx[i] >> sh), (uint32_t)(cy[i] >> sh));
  atomicAdd(&cnt[key], 1);
}

__global__ void k_max(const int32_t* __restrict__ cnt, int64_t m, int32_t* out) {
  int32_t best = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    best = max(best, cnt[i]);
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

// unstable scatter into leaf slots; the within-leaf order is fixed next
__global__ void k_scatter(const int32_t* __restrict__ cx, const int32_t* __restrict__ cy,
                          int64_t n, int level, int32_t* __restrict__ cursor,
                          int32_t* __restrict__ slot_idx, int32_t* __restrict__ slot_leaf) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int sh = kDeepLevel - level;
  const uint32_t key = morton_encode((uint32_t)(cx[i] >> sh), (uint32_t)(cy[i] >> sh));
  const int32_t pos = atomicAdd(&cursor[key], 1);
  slot_idx[pos] = (int32_t)i;
  slot_leaf[pos] = (int32_t)key;
}

// final position of slot s = leaf start + number of points of the same leaf
// with a smaller original index
__global__ void k_leaf_rank(const int32_t* __restrict__ slot_idx,
                            const int32_t* __restrict__ slot_leaf,
                            const int32_t* __restrict__ leaf_off, int64_t n,
                            const double* __restrict__ pts, int64_t* __restrict__ perm,
                            double* __restrict__ xs, double* __restrict__ ys) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int32_t g = slot_idx[s];
  const int32_t leaf = slot_leaf[s];
  const int32_t b = leaf_off[leaf], e = leaf_off[leaf + 1];
  int32_t r = 0;
  for (int32_t t = b; t < e; ++t) r += slot_idx[t] < g;
  const int64_t pos = b + r;
  perm[pos] = g;
  xs[pos] = pts[2 * (int64_t)g];
  ys[pos] = pts[2 * (int64_t)g + 1];
}

int tree_build(hodlr2d* h, const double* d_pts) {
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  // root box
  if (!(h->opts.root[2] > 0.0)) {
    const int nb = (int)std::min<int64_t>(1024, (n + 255) / 256);
    double* d_part = nullptr;
    H2D_CK(cudaMalloc(&d_part, sizeof(double) * 4 * nb));
    k_bbox_partial<<<nb, 256, 0, s>>>(d_pts, n, d_part);
    std::vector<double> part(4 * nb);
    cudaError_t e = cudaMemcpyAsync(part.data(), d_part, sizeof(double) * 4 * nb,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_part);
    if (e != cudaSuccess) return HODLR2D_ERR_CUDA;
    double xmin = part[0], ymin = part[1], xmax = part[2], ymax = part[3];
    for (int b = 1; b < nb; ++b) {
      xmin = fmin(xmin, part[4 * b]);
      ymin = fmin(ymin, part[4 * b + 1]);
      xmax = fmax(xmax, part[4 * b + 2]);
      ymax = fmax(ymax, part[4 * b + 3]);
    }
    if (!std::isfinite(xmin) || !std::isfinite(xmax) || !std::isfinite(ymin) ||
        !std::isfinite(ymax))
      return HODLR2D_ERR_ARG;
    double w = fmax(xmax - xmin, ymax - ymin);
    if (!(w > 0.0)) w = 1.0;
    h->root[2] = w;
    h->root[0] = 0.5 * (xmin + xmax) - 0.5 * w;
    h->root[1] = 0.5 * (ymin + ymax) - 0.5 * w;
  } else {
    for (int d = 0; d < 3; ++d) h->root[d] = h->opts.root[d];
  }

  int32_t *d_cx = nullptr, *d_cy = nullptr, *d_small = nullptr;
  H2D_CK(cudaMalloc(&d_cx, sizeof(int32_t) * n));
  H2D_CK(cudaMalloc(&d_cy, sizeof(int32_t) * n));
  H2D_CK(cudaMalloc(&d_small, sizeof(int32_t) * 2));
  H2D_CK(cudaMemsetAsync(d_small, 0, sizeof(int32_t) * 2, s));
  const unsigned nblk = (unsigned)((n + 255) / 256);
  k_cells<<<nblk, 256, 0, s>>>(d_pts, n, h->root[0], h->root[1], h->root[2], d_cx, d_cy,
                               d_small);
  int32_t flag = 0;
  H2D_CK(cudaMemcpyAsync(&flag, d_small, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  H2D_CK(cudaStreamSynchronize(s));
  int rc = HODLR2D_OK;
  if (flag) rc = HODLR2D_ERR_ARG;

  // depth: smallest kappa whose leaves hold <= N_max points (Alg. 1).  No depth
  // below ceil(log4(N / N_max)) can satisfy it, so the search starts there.
  int kappa = -1;
  int32_t* d_cnt = nullptr;
  if (rc == HODLR2D_OK) {
    if (h->opts.levels >= 0) {
      if (h->opts.levels > kDeepLevel) rc = HODLR2D_ERR_ARG;
      kappa = h->opts.levels;
    } else {
      int k0 = 0;
      while (k0 < kDeepLevel && ((int64_t)h->leaf_size << (2 * k0)) < n) ++k0;
      for (int k = k0; k <= kDeepLevel && rc == HODLR2D_OK; ++k) {
        const int64_t nb = (int64_t)1 << (2 * k);
        if (cudaMalloc(&d_cnt, sizeof(int32_t) * nb) != cudaSuccess) { rc = HODLR2D_ERR_OOM; break; }
        cudaMemsetAsync(d_cnt, 0, sizeof(int32_t) * nb, s);
        cudaMemsetAsync(d_small, 0, sizeof(int32_t), s);
        k_hist<<<nblk, 256, 0, s>>>(d_cx, d_cy, n, k, d_cnt);
        k_max<<<(unsigned)std::min<int64_t>(4096, (nb + 255) / 256), 256, 0, s>>>(d_cnt, nb,
                                                                                  d_small);
        int32_t mx = 0;
        if (cudaMemcpyAsync(&mx, d_small, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
          rc = HODLR2D_ERR_CUDA;
        cudaFree(d_cnt);
        d_cnt = nullptr;
        if (rc == HODLR2D_OK && mx <= h->leaf_size) { kappa = k; break; }
      }
      if (rc == HODLR2D_OK && kappa < 0) rc = HODLR2D_ERR_DEPTH;
    }
  }
  if (rc == HODLR2D_OK) {
    h->kappa = kappa;
    const int64_t nleaf = (int64_t)1 << (2 * kappa);
    int32_t *d_cursor = nullptr, *d_slot = nullptr, *d_sleaf = nullptr;
    if (cudaMalloc(&h->d_leaf_off, sizeof(int32_t) * (nleaf + 1)) != cudaSuccess ||
        cudaMalloc(&d_cursor, sizeof(int32_t) * (nleaf + 1)) != cudaSuccess ||
        cudaMalloc(&d_slot, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc(&d_sleaf, sizeof(int32_t) * n) != cudaSuccess ||
        cudaMalloc(&h->d_perm, sizeof(int64_t) * n) != cudaSuccess ||
        cudaMalloc(&h->d_x, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&h->d_y, sizeof(double) * n) != cudaSuccess) {
      rc = HODLR2D_ERR_OOM;
    }
    if (rc == HODLR2D_OK) {
      cudaMemsetAsync(d_cursor, 0, sizeof(int32_t) * (nleaf + 1), s);
      k_hist<<<nblk, 256, 0, s>>>(d_cx, d_cy, n, kappa, d_cursor);
      rc = scan_exclusive<int32_t>(d_cursor, h->d_leaf_off, nleaf, s);
    }
    if (rc == HODLR2D_OK) {
      cudaMemcpyAsync(d_cursor, h->d_leaf_off, sizeof(int32_t) * nleaf, cudaMemcpyDeviceToDevice,
                      s);
      k_scatter<<<nblk, 256, 0, s>>>(d_cx, d_cy, n, kappa, d_cursor, d_slot, d_sleaf);
      k_leaf_rank<<<nblk, 256, 0, s>>>(d_slot, d_sleaf, h->d_leaf_off, n, d_pts, h->d_perm,
                                       h->d_x, h->d_y);
      h->h_leaf_off.resize(nleaf + 1);
      if (cudaMemcpyAsync(h->h_leaf_off.data(), h->d_leaf_off, sizeof(int32_t) * (nleaf + 1),
                          cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        rc = HODLR2D_ERR_CUDA;
    }
    cudaFree(d_cursor);
    cudaFree(d_slot);
    cudaFree(d_sleaf);
  }
  cudaFree(d_cx);
  cudaFree(d_cy);
  cudaFree(d_small);
  if (rc == HODLR2D_OK && cudaGetLastError() != cudaSuccess) rc = HODLR2D_ERR_CUDA;
  return rc;
}

// ---------------------------------------------------------------------------
// Interaction lists
// ---------------------------------------------------------------------------

// number of points of box b at level l
__device__ __forceinline__ int32_t box_count(const int32_t* leaf_off, int kappa, int l,
                                             uint32_t b) {
  const int sh = 2 * (kappa - l);
  return leaf_off[(int64_t)(b + 1) << sh] - leaf_off[(int64_t)b << sh];
}

// The interaction list of box (cx, cy) at level l >= 1 (Eq. ilist), as Morton
// ids of non-empty boxes in ascending order.  Returns the count (<= 15).
__device__ int interaction_list(const int32_t* leaf_off, int kappa, int l, int cx, int cy,
                                uint32_t* out) {
  const int m = 1 << l;
  const int px = cx >> 1, py = cy >> 1;
  int c = 0;
  // clan: siblings and children of the parent's edge sharers; the parent
  // itself is included below so that its other children (the siblings) come
  // out of the same loop.
  const int pdx[5] = {0, 1, -1, 0, 0}, pdy[5] = {0, 0, 0, 1, -1};
  for (int e = 0; e < 5; ++e) {
    const int qx = px + pdx[e], qy = py + pdy[e];
    if (qx < 0 || qy < 0 || qx >= (m >> 1) || qy >= (m >> 1)) continue;
    for (int ch = 0; ch < 4; ++ch) {
      const int ox = 2 * qx + (ch & 1), oy = 2 * qy + (ch >> 1);
      const int dx = abs(ox - cx), dy = abs(oy - cy);
      if (dx + dy <= 1) continue;  // self or edge sharer (Def. ec): not admissible
      const uint32_t key = morton_encode((uint32_t)ox, (uint32_t)oy);
      if (box_count(leaf_off, kappa, l, key) == 0) continue;
      out[c++] = key;
    }
  }
  // ascending (insertion sort of <= 15 ids)
  for (int i = 1; i < c; ++i) {
    const uint32_t v = out[i];
    int j = i - 1;
    while (j >= 0 && out[j] > v) { out[j + 1] = out[j]; --j; }
    out[j + 1] = v;
  }
  return c;
}

// per box: number of stored pairs it is the row of, and its list length
__global__ void k_count_pairs(const int32_t* __restrict__ leaf_off, int kappa, int l,
                              int64_t* __restrict__ npair_row, int32_t* __restrict__ nlist) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nb = (int64_t)1 << (2 * l);
  if (b >= nb) return;
  int cnt = 0, len = 0;
  if (box_count(leaf_off, kappa, l, (uint32_t)b) > 0) {
    int cx, cy;
    morton_decode((uint32_t)b, cx, cy);
    uint32_t lst[24];
    len = interaction_list(leaf_off, kappa, l, cx, cy, lst);
    for (int i = 0; i < len; ++i) cnt += lst[i] > (uint32_t)b;
  }
  npair_row[b] = cnt;
  nlist[b] = len;
}

__global__ void k_write_pairs(const int32_t* __restrict__ leaf_off, int kappa, int l,
                              const int64_t* __restrict__ pair_off, int32_t* __restrict__ px,
                              int32_t* __restrict__ py) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nb = (int64_t)1 << (2 * l);
  if (b >= nb) return;
  if (box_count(leaf_off, kappa, l, (uint32_t)b) == 0) return;
  int cx, cy;
  morton_decode((uint32_t)b, cx, cy);
  uint32_t lst[24];
  const int len = interaction_list(leaf_off, kappa, l, cx, cy, lst);
  int64_t o = pair_off[b];
  for (int i = 0; i < len; ++i)
    if (lst[i] > (uint32_t)b) {
      px[o] = (int32_t)b;
      py[o] = (int32_t)lst[i];
      ++o;
    }
}

// entries of every box's list: pair * 2 + side, ascending partner
__global__ void k_write_entries(const int32_t* __restrict__ leaf_off, int kappa, int l,
                                const int64_t* __restrict__ pair_off,
                                const int32_t* __restrict__ py,
                                const int32_t* __restrict__ ent_off, int32_t* __restrict__ ent) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nb = (int64_t)1 << (2 * l);
  if (b >= nb) return;
  if (box_count(leaf_off, kappa, l, (uint32_t)b) == 0) return;
  int cx, cy;
  morton_decode((uint32_t)b, cx, cy);
  uint32_t lst[24];
  const int len = interaction_list(leaf_off, kappa, l, cx, cy, lst);
  int32_t o = ent_off[b];
  int64_t own = pair_off[b];
  for (int i = 0; i < len; ++i) {
    const uint32_t q = lst[i];
    int64_t p = -1;
    int side = 0;
    if (q > (uint32_t)b) {  // b is the row side; pairs of b are in list order
      p = own++;
      side = 0;
    } else {  // b is the column side of pair (q, b)
      for (int64_t t = pair_off[q]; t < pair_off[q + 1]; ++t)
        if (py[t] == (int32_t)b) { p = t; break; }
      side = 1;
    }
    ent[o++] = (int32_t)(2 * p + side);
  }
}

int lists_build(hodlr2d* h) {
  cudaStream_t s = h->stream;
  for (int l = 1; l <= h->kappa; ++l) {
    Level& L = h->lev[l];
    L.l = l;
    const int64_t nb = (int64_t)1 << (2 * l);
    int64_t* d_poff = nullptr;
    int32_t* d_nlist = nullptr;
    H2D_CK(cudaMalloc(&d_poff, sizeof(int64_t) * (nb + 1)));
    H2D_CK(cudaMalloc(&d_nlist, sizeof(int32_t) * (nb + 1)));
    H2D_CK(cudaMalloc(&L.d_ent_off, sizeof(int32_t) * (nb + 1)));
    const unsigned g = (unsigned)((nb + 255) / 256);
    k_count_pairs<<<g, 256, 0, s>>>(h->d_leaf_off, h->kappa, l, d_poff, d_nlist);
    H2D_TRY(scan_exclusive<int64_t>(d_poff, d_poff, nb, s));
    H2D_TRY(scan_exclusive<int32_t>(d_nlist, L.d_ent_off, nb, s));
    int64_t np = 0;
    int32_t ne = 0;
    H2D_CK(cudaMemcpyAsync(&np, d_poff + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    H2D_CK(cudaMemcpyAsync(&ne, L.d_ent_off + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    H2D_CK(cudaStreamSynchronize(s));
    L.npairs = np;
    L.nent = ne;
    H2D_CK(cudaMalloc(&L.d_px, sizeof(int32_t) * (np + 1)));
    H2D_CK(cudaMalloc(&L.d_py, sizeof(int32_t) * (np + 1)));
    H2D_CK(cudaMalloc(&L.d_ent, sizeof(int32_t) * (ne + 1)));
    k_write_pairs<<<g, 256, 0, s>>>(h->d_leaf_off, h->kappa, l, d_poff, L.d_px, L.d_py);
    k_write_entries<<<g, 256, 0, s>>>(h->d_leaf_off, h->kappa, l, d_poff, L.d_py, L.d_ent_off,
                                      L.d_ent);
    H2D_CK(cudaGetLastError());
    H2D_CK(cudaStreamSynchronize(s));
    L.d_prow = d_poff;  // kept: first stored pair of each row box
    cudaFree(d_nlist);
  }
  return HODLR2D_OK;
}

}  // namespace h2d
