// Restarted GMRES on the GPU (the iterative solver of Sec. 5.2 / 5.3), FP64.
//
// Arnoldi with classical Gram-Schmidt applied twice (CGS2) so that each
// orthogonalisation is two batched dot-product launches; the (restart+1) x
// restart Hessenberg matrix and its Givens rotations live on the host (tiny).
// Dot products reduce in a fixed order (block partials, then one pass), so a
// solve is bitwise reproducible.  Inner modes:
//   F64, DF32   plain GMRES with that product (the float-float product keeps
//               binary64-level accuracy, so it needs no refinement);
//   F32, BF16   iterative refinement: r = b - A x with the F64 product, then
//               a GMRES correction with the inner mode's product to a relative
//               residual a little above that product's own error, until
//               |r| <= tol |b|.
// A product whose input is known to be zero (x0 = 0, each fresh correction)
// is skipped.  The Krylov basis lives in a per-handle workspace that grows
// on demand and is kept for the next solve.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace h2d {

bool is_device_ptr(const void* p);
int matvec_mode_device(hodlr2d* h, const double* x, double* y, int nrhs, int mode);

constexpr int kDotBlocks = 304;  // 2 x 152 SMs
constexpr int kDotThreads = 256;

// partial[b * nvec + i] = sum over this block's rows of V_i . w
__global__ void k_dots(const double* __restrict__ V, int64_t ld, int nvec,
                       const double* __restrict__ w, int64_t n, double* __restrict__ partial) {
  __shared__ double red[kDotThreads / 32];
  for (int i = 0; i < nvec; ++i) {
    const double* v = V + (int64_t)i * ld;
    double acc = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * kDotThreads)
      acc += v[r] * w[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int k = 0; k < kDotThreads / 32; ++k) s += red[k];
      partial[(int64_t)blockIdx.x * nvec + i] = s;
    }
    __syncthreads();
  }
}

__global__ void k_dots_final(const double* __restrict__ partial, int nblk, int nvec,
                             double* __restrict__ out) {
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * nvec + i];
    out[i] = s;
  }
}

// w += sign * sum_i c_i V_i
__global__ void k_combo(const double* __restrict__ V, int64_t ld, int nvec,
                        const double* __restrict__ c, double sign, double* __restrict__ w,
                        int64_t n) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  double acc = 0.0;
  for (int i = 0; i < nvec; ++i) acc += c[i] * V[(int64_t)i * ld + r];
  w[r] += sign * acc;
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, double* __restrict__ out, int64_t n) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n) out[r] = a * x[r] + b * y[r];
}

namespace {

struct Work {
  hodlr2d* h;
  int64_t n;
  cudaStream_t s;
  double* partial = nullptr;
  double* dvec = nullptr;  // device copy of small coefficient vectors
  std::vector<double> hbuf;

  int dots(const double* V, int64_t ld, int nvec, const double* w, double* out_host) {
    k_dots<<<kDotBlocks, kDotThreads, 0, s>>>(V, ld, nvec, w, n, partial);
    k_dots_final<<<1, 64, 0, s>>>(partial, kDotBlocks, nvec, dvec);
    H2D_CK(cudaGetLastError());
    H2D_CK(cudaMemcpyAsync(out_host, dvec, sizeof(double) * nvec, cudaMemcpyDeviceToHost, s));
    H2D_CK(cudaStreamSynchronize(s));
    return HODLR2D_OK;
  }
  int combo(const double* V, int64_t ld, int nvec, const double* c_host, double sign, double* w) {
    H2D_CK(cudaMemcpyAsync(dvec, c_host, sizeof(double) * nvec, cudaMemcpyHostToDevice, s));
    k_combo<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, ld, nvec, dvec, sign, w, n);
    H2D_CK(cudaGetLastError());
    return HODLR2D_OK;
  }
  int matvec(const double* x, double* y, int mode) { return matvec_mode_device(h, x, y, 1, mode); }
  double norm(const double* v) {
    double r = 0.0;
    if (dots(v, 0, 1, v, &r) != HODLR2D_OK) return NAN;
    return sqrt(r);
  }
};

// GMRES(restart) on A z = rhs starting from z (device), product `mode`.
// Stops at |rhs - A z| <= tol_abs or after `budget` products.
int gmres_core(Work& W, const double* rhs, double* z, bool z_zero, double tol_abs, int restart,
               int budget, int mode, double* Vb, double* w, int* used, double* final_res) {
  const int64_t n = W.n;
  cudaStream_t s = W.s;
  const int m = restart;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), hcol(m + 1),
      h2(m + 1);
  int it = 0;
  double beta = 0.0;
  const unsigned gb = (unsigned)((n + 255) / 256);
  if (z_zero) H2D_CK(cudaMemsetAsync(z, 0, sizeof(double) * n, s));
  while (true) {
    // r = rhs - A z, into V_0 (r = rhs while z is still zero)
    if (z_zero) {
      H2D_CK(cudaMemcpyAsync(Vb, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      z_zero = false;
    } else {
      H2D_TRY(W.matvec(z, w, mode));
      ++it;
      k_axpby<<<gb, 256, 0, s>>>(1.0, rhs, -1.0, w, Vb, n);
    }
    beta = W.norm(Vb);
    if (!isfinite(beta)) return HODLR2D_ERR_CUDA;
    if (beta <= tol_abs || it >= budget) break;
    const double inv = 1.0 / beta;
    k_axpby<<<gb, 256, 0, s>>>(inv, Vb, 0.0, Vb, Vb, n);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jend = -1;
    for (int j = 0; j < m; ++j) {
      double* vj = Vb + (int64_t)j * n;
      double* vn = Vb + (int64_t)(j + 1) * n;
      H2D_TRY(W.matvec(vj, vn, mode));
      ++it;
      // CGS2
      H2D_TRY(W.dots(Vb, n, j + 1, vn, hcol.data()));
      H2D_TRY(W.combo(Vb, n, j + 1, hcol.data(), -1.0, vn));
      H2D_TRY(W.dots(Vb, n, j + 1, vn, h2.data()));
      H2D_TRY(W.combo(Vb, n, j + 1, h2.data(), -1.0, vn));
      for (int i = 0; i <= j; ++i) hcol[i] += h2[i];
      const double hn = W.norm(vn);
      if (!isfinite(hn)) return HODLR2D_ERR_CUDA;
      hcol[j + 1] = hn;
      if (hn > 0.0) k_axpby<<<gb, 256, 0, s>>>(1.0 / hn, vn, 0.0, vn, vn, n);
      // previous rotations, then a new one that zeroes H[j+1][j]
      for (int i = 0; i < j; ++i) {
        const double a = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
        const double b = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
        hcol[i] = a;
        hcol[i + 1] = b;
      }
      const double den = hypot(hcol[j], hcol[j + 1]);
      cs[j] = den > 0.0 ? hcol[j] / den : 1.0;
      sn[j] = den > 0.0 ? hcol[j + 1] / den : 0.0;
      hcol[j] = den;
      hcol[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
      jend = j;
      if (fabs(g[j + 1]) <= tol_abs || it >= budget || hn == 0.0) break;
    }
    // back substitution and update z += V y
    for (int i = jend; i >= 0; --i) {
      double acc = g[i];
      for (int k = i + 1; k <= jend; ++k) acc -= H[(size_t)i * m + k] * y[k];
      y[i] = acc / H[(size_t)i * m + i];
    }
    H2D_TRY(W.combo(Vb, n, jend + 1, y.data(), 1.0, z));
  }
  *used = it;
  *final_res = beta;
  return HODLR2D_OK;
}

}  // namespace

int gmres_run(hodlr2d* h, const double* b, double* x, double tol, int restart, int maxit,
              int inner_mode, int* iters, double* relres) {
  const int64_t n = h->n;
  cudaStream_t s = h->stream;
  const bool bd = is_device_ptr(b), xd = is_device_ptr(x);
  Work W;
  W.h = h;
  W.n = n;
  W.s = s;
  const int m = std::min<int>(restart, (int)std::min<int64_t>(n, 1 << 20));
  int rc = HODLR2D_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == HODLR2D_OK) {
      (void)cudaGetLastError();
      rc = e == cudaErrorMemoryAllocation ? HODLR2D_ERR_OOM : HODLR2D_ERR_CUDA;
    }
  };
  // workspace: partials, coefficients, basis (m + 1 vectors), w, r, d, b, x
  const int64_t need = (int64_t)kDotBlocks * (m + 2) + (m + 2) + n * (m + 1) + 5 * n;
  if (h->gm_values < need) {
    cudaFree(h->d_gm);
    h->d_gm = nullptr;
    h->gm_values = 0;
    ck(cudaMalloc(&h->d_gm, sizeof(double) * need));
    if (rc == HODLR2D_OK) h->gm_values = need;
  }
  if (rc != HODLR2D_OK) return rc;
  double* p = h->d_gm;
  auto take = [&](int64_t k) {
    double* q = p;
    p += k;
    return q;
  };
  W.partial = take((int64_t)kDotBlocks * (m + 2));
  W.dvec = take(m + 2);
  double* Vb = take(n * (m + 1));
  double* w = take(n);
  double* r = take(n);
  double* d = take(n);
  double* db = bd ? nullptr : take(n);
  double* dx = xd ? nullptr : take(n);
  if (!bd) ck(cudaMemcpyAsync(db, b, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  if (!xd) ck(cudaMemcpyAsync(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  const double* B = bd ? b : db;
  double* X = xd ? x : dx;
  int used = 0;
  double res = 0.0, bn = 0.0, xn = 0.0;
  if (rc == HODLR2D_OK) {
    bn = W.norm(B);
    xn = W.norm(X);
    if (!isfinite(bn) || !isfinite(xn)) rc = HODLR2D_ERR_ARG;
  }
  if (rc == HODLR2D_OK && bn == 0.0) {
    ck(cudaMemsetAsync(X, 0, sizeof(double) * n, s));
    res = 0.0;
  } else if (rc == HODLR2D_OK) {
    if (inner_mode == HODLR2D_MODE_F64 || inner_mode == HODLR2D_MODE_DF32) {
      rc = gmres_core(W, B, X, xn == 0.0, tol * bn, m, maxit, inner_mode, Vb, w, &used, &res);
    } else {
      // iterative refinement: F64 residual, low-precision correction solved to
      // a relative residual just above the inner product's own error
      const unsigned gb = (unsigned)((n + 255) / 256);
      const double inner_rel = inner_mode == HODLR2D_MODE_F32 ? 1e-5 : 1e-2;
      bool x_zero = xn == 0.0;
      while (rc == HODLR2D_OK) {
        if (x_zero) {
          ck(cudaMemcpyAsync(r, B, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        } else {
          rc = matvec_mode_device(h, X, w, 1, HODLR2D_MODE_F64);
          if (rc) break;
          ++used;
          k_axpby<<<gb, 256, 0, s>>>(1.0, B, -1.0, w, r, n);
        }
        res = W.norm(r);
        if (!isfinite(res)) { rc = HODLR2D_ERR_CUDA; break; }
        if (res <= tol * bn || used >= maxit) break;
        int u2 = 0;
        double r2 = 0.0;
        rc = gmres_core(W, r, d, true, std::max(inner_rel * res, 0.5 * tol * bn), m,
                        std::max(1, maxit - used), inner_mode, Vb, w, &u2, &r2);
        used += u2;
        if (rc) break;
        if (x_zero) {
          ck(cudaMemcpyAsync(X, d, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
          x_zero = false;
        } else {
          k_axpby<<<gb, 256, 0, s>>>(1.0, X, 1.0, d, X, n);
        }
      }
    }
  }
  if (rc == HODLR2D_OK && !xd)
    ck(cudaMemcpyAsync(x, X, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  ck(cudaStreamSynchronize(s));
  if (iters) *iters = used;
  if (relres) *relres = bn > 0.0 ? res / bn : 0.0;
  if (rc == HODLR2D_OK && bn > 0.0 && res > tol * bn) rc = HODLR2D_ERR_NOCONV;
  return rc;
}

}  // namespace h2d
