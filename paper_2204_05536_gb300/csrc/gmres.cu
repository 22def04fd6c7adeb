// Restarted GMRES on the GPU (the iterative solver of Sec. 5.2 / 5.3), FP64.
//
// Arnoldi with classical Gram-Schmidt applied twice (CGS2), so that each
// orthogonalisation is two batched dot-product launches.  Everything of a
// cycle stays on the device: the Gram-Schmidt coefficients, the
// (restart+1) x restart Hessenberg matrix, its Givens rotations, the
// residual estimates |g_{j+1}| and the final triangular solve.  The host
// queues Arnoldi steps without waiting and reads the residual estimate of
// step j-1 (a pinned copy behind an event) while step j runs on the GPU, so
// the GPU never idles on the host; a cycle that converges at step j-1 has
// already queued step j, whose extra basis vector is kept (jend = j).  The
// host synchronises once per restart, for the true residual norm.
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

// out[i] = sum of the block partials in block order; with sq, out[0] is
// replaced by its square root (a norm)
__global__ void k_dots_final(const double* __restrict__ partial, int nblk, int nvec,
                             double* __restrict__ out, int sq) {
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * nvec + i];
    out[i] = sq ? sqrt(s) : s;
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

// v *= 1 / *nrm (unless the norm is zero)
__global__ void k_unit(double* __restrict__ v, const double* __restrict__ nrm, int64_t n) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double s = *nrm;
  if (r < n && s > 0.0) v[r] *= 1.0 / s;
}

// State of one Arnoldi cycle on the device.
struct Cyc {
  double* H;     // (m + 1) x m, row-major: H[i * m + j]
  double* cs;    // m
  double* sn;    // m
  double* g;     // m + 1: the rotated right-hand side beta e_1
  double* hcol;  // m + 1: Gram-Schmidt coefficients, first pass, then the column
  double* h2;    // m + 1: second-pass coefficients
  double* hn;    // 1: |v_{j+1}| before normalisation
  double* beta;  // 1: |r_0|
  double* res;   // m: |g_{j+1}| after step j
  double* y;     // m: the least-squares solution
};

// g = beta e_1 at the start of a cycle
__global__ void k_cycle_start(Cyc C, int m) {
  for (int i = threadIdx.x; i <= m; i += blockDim.x) C.g[i] = i == 0 ? *C.beta : 0.0;
}

// Step j of the Hessenberg QR (one thread): column j = CGS2 coefficients
// (both passes) and |v_{j+1}|; the earlier rotations, then the one that
// zeroes H[j+1][j]; g updated; |g_{j+1}| recorded.
__global__ void k_givens(Cyc C, int j, int m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* hc = C.hcol;
  for (int i = 0; i <= j; ++i) hc[i] += C.h2[i];
  hc[j + 1] = *C.hn;
  for (int i = 0; i < j; ++i) {
    const double a = C.cs[i] * hc[i] + C.sn[i] * hc[i + 1];
    const double b = -C.sn[i] * hc[i] + C.cs[i] * hc[i + 1];
    hc[i] = a;
    hc[i + 1] = b;
  }
  const double den = hypot(hc[j], hc[j + 1]);
  const double c = den > 0.0 ? hc[j] / den : 1.0;
  const double s = den > 0.0 ? hc[j + 1] / den : 0.0;
  C.cs[j] = c;
  C.sn[j] = s;
  hc[j] = den;
  hc[j + 1] = 0.0;
  const double gj = C.g[j];
  C.g[j + 1] = -s * gj;
  C.g[j] = c * gj;
  for (int i = 0; i <= j; ++i) C.H[(size_t)i * m + j] = hc[i];
  // -1 marks a breakdown (|v_{j+1}| = 0: the Krylov space holds the
  // solution, and a further step would divide by zero)
  C.res[j] = *C.hn == 0.0 ? -1.0 : fabs(C.g[j + 1]);
}

// Back substitution H[0:jend, 0:jend] y = g[0:jend] (one thread).
__global__ void k_backsub(Cyc C, int jend, int m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = jend; i >= 0; --i) {
    double acc = C.g[i];
    for (int k = i + 1; k <= jend; ++k) acc -= C.H[(size_t)i * m + k] * C.y[k];
    C.y[i] = acc / C.H[(size_t)i * m + i];
  }
}

namespace {

struct Work {
  hodlr2d* h;
  int64_t n;
  cudaStream_t s;
  double* partial = nullptr;
  double* dvec = nullptr;     // device scratch of small vectors (norms)
  double* pinned = nullptr;   // host-visible copies of residual estimates
  cudaEvent_t* ev = nullptr;  // one per Arnoldi step of a cycle
  Cyc C{};

  // out (device) = V_i . w for i < nvec
  int dots_dev(const double* V, int64_t ld, int nvec, const double* w, double* out,
               bool sqrt_first = false) {
    k_dots<<<kDotBlocks, kDotThreads, 0, s>>>(V, ld, nvec, w, n, partial);
    k_dots_final<<<1, 64, 0, s>>>(partial, kDotBlocks, nvec, out, sqrt_first ? 1 : 0);
    H2D_CK(cudaGetLastError());
    return HODLR2D_OK;
  }
  // w += sign * V c with device coefficients c
  int combo_dev(const double* V, int64_t ld, int nvec, const double* c, double sign, double* w) {
    k_combo<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, ld, nvec, c, sign, w, n);
    H2D_CK(cudaGetLastError());
    return HODLR2D_OK;
  }
  int matvec(const double* x, double* y, int mode) { return matvec_mode_device(h, x, y, 1, mode); }
  // |v| read back to the host (synchronises the stream)
  double norm(const double* v) {
    if (dots_dev(v, 0, 1, v, dvec, true) != HODLR2D_OK) return NAN;
    double r = NAN;
    if (cudaMemcpyAsync(&r, dvec, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      (void)cudaGetLastError();
      return NAN;
    }
    return r;
  }
};

// GMRES(restart) on A z = rhs starting from z (device), product `mode`.
// Stops at |rhs - A z| <= tol_abs or after `budget` products.
int gmres_core(Work& W, const double* rhs, double* z, bool z_zero, double tol_abs, int restart,
               int budget, int mode, double* Vb, double* w, int* used, double* final_res) {
  const int64_t n = W.n;
  cudaStream_t s = W.s;
  const int m = restart;
  const Cyc& C = W.C;
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
    H2D_TRY(W.dots_dev(Vb, 0, 1, Vb, C.beta, true));
    H2D_CK(cudaMemcpyAsync(&beta, C.beta, sizeof(double), cudaMemcpyDeviceToHost, s));
    H2D_CK(cudaStreamSynchronize(s));  // once per cycle
    if (!isfinite(beta)) return HODLR2D_ERR_CUDA;
    if (beta <= tol_abs || it >= budget) break;
    k_unit<<<gb, 256, 0, s>>>(Vb, C.beta, n);
    k_cycle_start<<<1, 64, 0, s>>>(C, m);
    H2D_CK(cudaGetLastError());
    int jend = -1;
    for (int j = 0; j < m; ++j) {
      double* vj = Vb + (int64_t)j * n;
      double* vn = Vb + (int64_t)(j + 1) * n;
      H2D_TRY(W.matvec(vj, vn, mode));
      ++it;
      // CGS2, coefficients on the device
      H2D_TRY(W.dots_dev(Vb, n, j + 1, vn, C.hcol));
      H2D_TRY(W.combo_dev(Vb, n, j + 1, C.hcol, -1.0, vn));
      H2D_TRY(W.dots_dev(Vb, n, j + 1, vn, C.h2));
      H2D_TRY(W.combo_dev(Vb, n, j + 1, C.h2, -1.0, vn));
      H2D_TRY(W.dots_dev(vn, 0, 1, vn, C.hn, true));
      k_unit<<<gb, 256, 0, s>>>(vn, C.hn, n);
      k_givens<<<1, 32, 0, s>>>(C, j, m);
      H2D_CK(cudaGetLastError());
      H2D_CK(cudaMemcpyAsync(W.pinned + j, C.res + j, sizeof(double), cudaMemcpyDeviceToHost, s));
      H2D_CK(cudaEventRecord(W.ev[j], s));
      jend = j;
      if (it >= budget) break;
      // the previous step's estimate, read while this step runs
      if (j >= 1) {
        H2D_CK(cudaEventSynchronize(W.ev[j - 1]));
        const double rj = W.pinned[j - 1];
        if (isnan(rj)) return HODLR2D_ERR_CUDA;
        if (rj < 0.0) {  // breakdown at step j - 1: step j is void
          jend = j - 1;
          break;
        }
        if (rj <= tol_abs) break;  // converged at step j - 1; step j's vector is kept
      }
    }
    if (jend >= 0) {
      H2D_CK(cudaEventSynchronize(W.ev[jend]));
      if (isnan(W.pinned[jend])) return HODLR2D_ERR_CUDA;
    }
    // back substitution and update z += V y
    k_backsub<<<1, 32, 0, s>>>(C, jend, m);
    H2D_CK(cudaGetLastError());
    H2D_TRY(W.combo_dev(Vb, n, jend + 1, C.y, 1.0, z));
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
  // workspace: partials, norm scratch, the cycle state, basis (m + 1
  // vectors), w, r, d, b, x
  const int64_t ncyc = (int64_t)(m + 1) * m + 2 * m + 3 * (m + 1) + 2 + 2 * m;
  const int64_t need = (int64_t)kDotBlocks * (m + 2) + 8 + ncyc + n * (m + 1) + 5 * n;
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
  W.dvec = take(8);
  W.C.H = take((int64_t)(m + 1) * m);
  W.C.cs = take(m);
  W.C.sn = take(m);
  W.C.g = take(m + 1);
  W.C.hcol = take(m + 1);
  W.C.h2 = take(m + 1);
  W.C.hn = take(1);
  W.C.beta = take(1);
  W.C.res = take(m);
  W.C.y = take(m);
  // host-visible residual estimates and one event per Arnoldi step
  std::vector<cudaEvent_t> evs(m, nullptr);
  for (int j = 0; j < m && rc == HODLR2D_OK; ++j)
    ck(cudaEventCreateWithFlags(&evs[j], cudaEventDisableTiming));
  ck(cudaMallocHost(&W.pinned, sizeof(double) * m));
  W.ev = evs.data();
  struct Release {
    Work& W;
    std::vector<cudaEvent_t>& evs;
    cudaStream_t s;
    ~Release() {
      cudaStreamSynchronize(s);
      for (auto e : evs)
        if (e) cudaEventDestroy(e);
      if (W.pinned) cudaFreeHost(W.pinned);
      W.pinned = nullptr;
    }
  } release{W, evs, s};
  if (rc != HODLR2D_OK) return rc;
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
