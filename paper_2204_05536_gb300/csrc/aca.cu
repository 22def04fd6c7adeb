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
        std::vector<int64_t> plist(nbp), wsoff(nbp), fgoff(nbp);
        std::vector<int32_t> bcap(nbp);
        int64_t wo = 0, fo = 0;
        for (int64_t i = 0; i < nbp; ++i) {
          const int64_t p = todo[b0 + i];
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
        if (mean_rows <= 96)
          k_aca<64><<<(unsigned)nbp, 64, smem, s>>>(A);
        else
          k_aca<256><<<(unsigned)nbp, 256, smem, s>>>(A);
        H2D_CK(cudaGetLastError());
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
