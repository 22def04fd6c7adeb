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

  const int64_t p = A.p0 + blockIdx.x;
  const uint32_t bx = (uint32_t)A.px[p], by = (uint32_t)A.py[p];
  const int sh = 2 * (A.kappa - A.l);
  const int32_t xs = A.leaf_off[(int64_t)bx << sh];
  const int32_t m = A.leaf_off[(int64_t)(bx + 1) << sh] - xs;
  const int32_t ys = A.leaf_off[(int64_t)by << sh];
  const int32_t n = A.leaf_off[(int64_t)(by + 1) << sh] - ys;
  const int kfull = min(m, n);
  const int cap = min(kfull, capmax);
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

// copy U[:, :k] and V[:, :k] of each batch pair to the level's packed buffer
__global__ void k_compact(const double* __restrict__ ws, const int64_t* __restrict__ wsoff,
                          const int32_t* __restrict__ leaf_off, int kappa, int l,
                          const int32_t* __restrict__ px, const int32_t* __restrict__ py,
                          int64_t p0, const int32_t* __restrict__ rank, int max_rank,
                          const int64_t* __restrict__ foff, double* __restrict__ fac) {
  const int64_t p = p0 + blockIdx.x;
  const int sh = 2 * (kappa - l);
  const uint32_t bx = (uint32_t)px[p], by = (uint32_t)py[p];
  const int64_t m = leaf_off[(int64_t)(bx + 1) << sh] - leaf_off[(int64_t)bx << sh];
  const int64_t n = leaf_off[(int64_t)(by + 1) << sh] - leaf_off[(int64_t)by << sh];
  const int64_t cap = min(min(m, n), (int64_t)max_rank);
  const int64_t k = rank[p];
  const double* U = ws + wsoff[blockIdx.x];
  const double* V = U + m * cap;
  const int64_t lm = ldpad(m), ln = ldpad(n);
  double* out = fac + foff[p];
  for (int64_t t = threadIdx.x; t < lm * k; t += blockDim.x) {
    const int64_t q = t / lm, i = t - q * lm;
    out[t] = i < m ? U[q * m + i] : 0.0;
  }
  for (int64_t t = threadIdx.x; t < ln * k; t += blockDim.x) {
    const int64_t q = t / ln, j = t - q * ln;
    out[lm * k + t] = j < n ? V[q * n + j] : 0.0;
  }
}

// Compress every pair of every level; fills Level::{d_rank, d_foff, d_fac,
// nvalues, max_rank, h_rank, h_foff} and the unconverged count.
int aca_build(hodlr2d* h) {
  cudaStream_t s = h->stream;
  const int capmax = h->opts.max_rank;
  const size_t smem = sizeof(double) * (4 * (size_t)capmax + 2);
  const int64_t ws_budget = (int64_t)1 << 28;  // values per batch (2 GiB)
  int64_t unconverged = 0;
  for (int l = h->kappa; l >= 1; --l) {  // Alg. 1: levels kappa down to 1
    Level& L = h->lev[l];
    const int64_t np = L.npairs;
    H2D_CK(cudaMalloc(&L.d_rank, sizeof(int32_t) * (np + 1)));
    H2D_CK(cudaMalloc(&L.d_foff, sizeof(int64_t) * (np + 1)));
    L.h_rank.assign(np, 0);
    L.h_foff.assign(np + 1, 0);
    if (np == 0) {
      H2D_CK(cudaMemsetAsync(L.d_foff, 0, sizeof(int64_t), s));
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
    std::vector<int64_t> wsz(np), fsz(np);
    int64_t tot_rows = 0;
    for (int64_t p = 0; p < np; ++p) {
      const int64_t m = cnt(px[p]), n = cnt(py[p]);
      const int64_t cap = std::min<int64_t>(std::min(m, n), capmax);
      wsz[p] = (m + n) * cap;
      fsz[p] = m;
      tot_rows += m + n;
    }
    int32_t* d_conv = nullptr;
    H2D_CK(cudaMalloc(&d_conv, sizeof(int32_t) * np));
    const int64_t mean_rows = tot_rows / (2 * np);
    // packed level buffer, grown as batches finish
    int64_t fac_cap = 0, fac_used = 0, stored = 0;
    double* fac = nullptr;
    int64_t p0 = 0;
    while (p0 < np) {
      int64_t p1 = p0, wtot = 0, ftot = 0;
      while (p1 < np && (p1 == p0 || wtot + wsz[p1] <= ws_budget) && p1 - p0 < (1 << 20)) {
        wtot += wsz[p1];
        ftot += fsz[p1];
        ++p1;
      }
      const int64_t nbp = p1 - p0;
      std::vector<int64_t> wsoff(nbp), fgoff(nbp);
      int64_t wo = 0, fo = 0;
      for (int64_t p = p0; p < p1; ++p) {
        wsoff[p - p0] = wo;
        fgoff[p - p0] = fo;
        wo += wsz[p];
        fo += fsz[p];
      }
      double* d_ws = nullptr;
      uint8_t* d_flags = nullptr;
      int64_t *d_wsoff = nullptr, *d_fgoff = nullptr, *d_foff_b = nullptr;
      H2D_CK(cudaMalloc(&d_ws, sizeof(double) * std::max<int64_t>(wo, 1)));
      H2D_CK(cudaMalloc(&d_flags, std::max<int64_t>(fo, 1)));
      H2D_CK(cudaMalloc(&d_wsoff, sizeof(int64_t) * nbp));
      H2D_CK(cudaMalloc(&d_fgoff, sizeof(int64_t) * nbp));
      H2D_CK(cudaMemcpyAsync(d_wsoff, wsoff.data(), sizeof(int64_t) * nbp,
                             cudaMemcpyHostToDevice, s));
      H2D_CK(cudaMemcpyAsync(d_fgoff, fgoff.data(), sizeof(int64_t) * nbp,
                             cudaMemcpyHostToDevice, s));
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
      A.p0 = p0;
      A.wsoff = d_wsoff;
      A.fgoff = d_fgoff;
      A.ws = d_ws;
      A.flags = d_flags;
      A.rank = L.d_rank;
      A.conv = d_conv;
      if (mean_rows <= 96)
        k_aca<64><<<(unsigned)nbp, 64, smem, s>>>(A);
      else
        k_aca<256><<<(unsigned)nbp, 256, smem, s>>>(A);
      H2D_CK(cudaGetLastError());
      // ranks of the batch -> packed offsets
      H2D_CK(cudaMemcpyAsync(L.h_rank.data() + p0, L.d_rank + p0, sizeof(int32_t) * nbp,
                             cudaMemcpyDeviceToHost, s));
      H2D_CK(cudaStreamSynchronize(s));
      int64_t add = 0;
      for (int64_t p = p0; p < p1; ++p) {
        L.h_foff[p] = fac_used + add;
        add += (ldpad(cnt(px[p])) + ldpad(cnt(py[p]))) * (int64_t)L.h_rank[p];
        stored += (cnt(px[p]) + cnt(py[p])) * (int64_t)L.h_rank[p];
      }
      if (fac_used + add > fac_cap) {
        const int64_t ncap = std::max<int64_t>(fac_used + add, 2 * fac_cap);
        double* nf = nullptr;
        H2D_CK(cudaMalloc(&nf, sizeof(double) * std::max<int64_t>(ncap, 1)));
        if (fac_used > 0)
          H2D_CK(cudaMemcpyAsync(nf, fac, sizeof(double) * fac_used, cudaMemcpyDeviceToDevice, s));
        H2D_CK(cudaStreamSynchronize(s));
        cudaFree(fac);
        fac = nf;
        fac_cap = ncap;
      }
      H2D_CK(cudaMalloc(&d_foff_b, sizeof(int64_t) * np));
      H2D_CK(cudaMemcpyAsync(d_foff_b, L.h_foff.data(), sizeof(int64_t) * p1,
                             cudaMemcpyHostToDevice, s));
      k_compact<<<(unsigned)nbp, 256, 0, s>>>(d_ws, d_wsoff, h->d_leaf_off, h->kappa, l, L.d_px,
                                              L.d_py, p0, L.d_rank, capmax, d_foff_b, fac);
      H2D_CK(cudaGetLastError());
      H2D_CK(cudaStreamSynchronize(s));
      fac_used += add;
      cudaFree(d_ws);
      cudaFree(d_flags);
      cudaFree(d_wsoff);
      cudaFree(d_fgoff);
      cudaFree(d_foff_b);
      p0 = p1;
    }
    L.h_foff[np] = fac_used;
    L.nvalues = fac_used;
    L.nstored = stored;
    L.d_fac = fac;
    if (!L.d_fac) H2D_CK(cudaMalloc(&L.d_fac, sizeof(double)));
    H2D_CK(cudaMemcpyAsync(L.d_foff, L.h_foff.data(), sizeof(int64_t) * (np + 1),
                           cudaMemcpyHostToDevice, s));
    std::vector<int32_t> conv(np);
    H2D_CK(cudaMemcpyAsync(conv.data(), d_conv, sizeof(int32_t) * np, cudaMemcpyDeviceToHost, s));
    H2D_CK(cudaStreamSynchronize(s));
    cudaFree(d_conv);
    L.max_rank = 0;
    for (int64_t p = 0; p < np; ++p) {
      L.max_rank = std::max(L.max_rank, L.h_rank[p]);
      unconverged += conv[p] ? 0 : 1;
    }
  }
  h->st.unconverged = unconverged;
  return HODLR2D_OK;
}

}  // namespace h2d
