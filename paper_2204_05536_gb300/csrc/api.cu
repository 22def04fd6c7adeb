// C ABI entry points: argument checks, handle lifetime, host/device staging,
// statistics, factor import/export.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace h2d {
int tree_build(hodlr2d* h, const double* d_pts);
int lists_build(hodlr2d* h);
int aca_build(hodlr2d* h);
int matvec_plan(hodlr2d* h);
int matvec_mode_device(hodlr2d* h, const double* x, double* y, int nrhs, int mode);
int product_status(hodlr2d* h);
int prepare_mode(hodlr2d* h, int mode);
void free_modes(hodlr2d* h);
int gmres_run(hodlr2d* h, const double* b, double* x, double tol, int restart, int maxit,
              int inner_mode, int* iters, double* relres);
void pair_features(const hodlr2d* h, int l, int32_t bx, int32_t by, int64_t m, int64_t n,
                   float* f);

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

static double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

static int make_kernel_params(const hodlr2d_kernel& k, KernelParams* kp) {
  if (k.kind < HODLR2D_IMQ || k.kind > HODLR2D_PHI2) return HODLR2D_ERR_ARG;
  if (!isfinite(k.a) || k.a < 0.0) return HODLR2D_ERR_ARG;
  if ((k.kind == HODLR2D_IMQ || k.kind == HODLR2D_PHI1 || k.kind == HODLR2D_PHI2) && !(k.a > 0.0))
    return HODLR2D_ERR_ARG;
  if (k.kind == HODLR2D_PHI1 && (k.a == 1.0 || k.a * log(k.a) - 1.0 == 0.0)) return HODLR2D_ERR_ARG;
  if (k.diag_mode != 0 && k.diag_mode != 1) return HODLR2D_ERR_ARG;
  if (k.diag_mode == 1 && !isfinite(k.diag_value)) return HODLR2D_ERR_ARG;
  kp->kind = k.kind;
  kp->a = k.a;
  kp->a2 = k.a * k.a;
  kp->log_a = k.a > 0.0 ? log(k.a) : 0.0;
  kp->phi1_den = k.a > 0.0 ? k.a * log(k.a) - 1.0 : -1.0;
  kp->inv_a = k.a > 0.0 ? 1.0 / k.a : 0.0;
  if (k.diag_mode == 1) {
    kp->diag = k.diag_value;
  } else {
    switch (k.kind) {
      case HODLR2D_IMQ: kp->diag = 1.0 / k.a; break;
      case HODLR2D_MQ: kp->diag = k.a; break;
      case HODLR2D_PHI1: kp->diag = -1.0 / (k.a * log(k.a) - 1.0); break;
      default: kp->diag = 0.0;
    }
  }
  return HODLR2D_OK;
}

static void fill_stats(hodlr2d* h) {
  hodlr2d_stats& s = h->st;
  s.n = h->n;
  s.kappa = h->kappa;
  for (int d = 0; d < 3; ++d) s.root[d] = h->root[d];
  s.npairs = 0;
  s.far_values = 0;
  s.max_rank = 0;
  for (int l = 0; l < HODLR2D_MAX_LEVELS; ++l) {
    const Level& L = h->lev[l];
    s.pairs_per_level[l] = L.npairs;
    s.values_per_level[l] = L.nstored;
    s.max_rank_per_level[l] = L.max_rank;
    s.npairs += L.npairs;
    s.far_values += L.nstored;
    s.max_rank = std::max(s.max_rank, L.max_rank);
  }
  // dense leaf entries: |X| (|X| + sum_{Y in E_X} |Y|)
  const int kappa = h->kappa;
  const int side = 1 << kappa;
  int64_t near = 0;
  const int64_t nleaf = (int64_t)1 << (2 * kappa);
  for (int64_t b = 0; b < nleaf; ++b) {
    const int64_t m = h->h_leaf_off[b + 1] - h->h_leaf_off[b];
    if (!m) continue;
    int cx, cy;
    morton_decode((uint32_t)b, cx, cy);
    int64_t cols = m;
    const int dx[4] = {-1, 1, 0, 0}, dy[4] = {0, 0, -1, 1};
    for (int e = 0; e < 4; ++e) {
      const int qx = cx + dx[e], qy = cy + dy[e];
      if (qx < 0 || qy < 0 || qx >= side || qy >= side) continue;
      const uint32_t q = morton_encode((uint32_t)qx, (uint32_t)qy);
      cols += h->h_leaf_off[q + 1] - h->h_leaf_off[q];
    }
    near += m * cols;
  }
  s.near_entries = near;
  s.compression_ratio = ((double)s.far_values + (double)near) / ((double)h->n * (double)h->n);
  const int64_t fb[4] = {8, 8, 4, 2};
  for (int m = 0; m < 4; ++m) s.bytes_per_matvec[m] = fb[m] * s.far_values + 16 * h->n + 16 * h->n;
}

static void free_handle(hodlr2d* h) {
  if (!h) return;
  DeviceGuard g(h->device);
  cudaFree(h->d_x);
  cudaFree(h->d_y);
  cudaFree(h->d_perm);
  cudaFree(h->d_leaf_off);
  cudaFree(h->d_gm);
  free_modes(h);
  for (int l = 0; l < HODLR2D_MAX_LEVELS; ++l) {
    Level& L = h->lev[l];
    cudaFree(L.d_px);
    cudaFree(L.d_py);
    cudaFree(L.d_rank);
    cudaFree(L.d_foff);
    cudaFree(L.d_toff);
    cudaFree(L.d_fac);
    cudaFree(L.d_ent_off);
    cudaFree(L.d_ent);
    cudaFree(L.d_prow);
    cudaFree(L.d_ppoff);
    cudaFree(L.d_entpp);
    cudaFree(L.d_meta);
  }
  cudaFree(h->d_proj);
  cudaFree(h->d_exp);
  cudaFree(h->d_tred);
  cudaFree(h->d_xt);
  cudaFree(h->d_yl);
  cudaFree(h->d_part);
  cudaFree(h->d_t);
  cudaFree(h->d_io);
  delete h;
}

}  // namespace h2d

using namespace h2d;

extern "C" {

void hodlr2d_default_opts(hodlr2d_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->rank_model = nullptr;
  o->root[0] = o->root[1] = o->root[2] = 0.0;
  o->levels = -1;
  o->compress = 1;
  o->max_rank = 256;
  o->mode = HODLR2D_MODE_F64;
}

const char* hodlr2d_strerror(int code) {
  switch (code) {
    case HODLR2D_OK: return "ok";
    case HODLR2D_ERR_ARG: return "invalid argument";
    case HODLR2D_ERR_OOM: return "out of memory";
    case HODLR2D_ERR_CUDA: return "CUDA runtime error";
    case HODLR2D_ERR_NOCONV: return "iteration did not converge";
    case HODLR2D_ERR_TIMEOUT: return "device-side wait timed out";
    case HODLR2D_ERR_DEPTH: return "no tree depth <= 14 meets the leaf size";
    case HODLR2D_ERR_STATE: return "handle not ready for this call";
    default: return "unknown error";
  }
}

int hodlr2d_build(const double* points, int64_t n, hodlr2d_kernel kernel, int leaf_size,
                  double eps, hodlr2d_t* out) {
  return hodlr2d_build_ex(points, n, kernel, leaf_size, eps, nullptr, out);
}

int hodlr2d_build_ex(const double* points, int64_t n, hodlr2d_kernel kernel, int leaf_size,
                     double eps, const hodlr2d_opts* opts, hodlr2d_t* out) {
  if (!points || !out || n < 1 || n > (int64_t)INT32_MAX - 1 || leaf_size < 1 || !(eps > 0.0) ||
      !(eps < 1.0))
    return HODLR2D_ERR_ARG;
  hodlr2d_opts o;
  hodlr2d_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_rank < 1 || o.levels > 14 || o.mode < 0 || o.mode > 3 || !isfinite(o.root[0]) ||
      !isfinite(o.root[1]) || !isfinite(o.root[2]))
    return HODLR2D_ERR_ARG;
  KernelParams kp;
  int rc = make_kernel_params(kernel, &kp);
  if (rc) return rc;
  hodlr2d* h = new (std::nothrow) hodlr2d();
  if (!h) return HODLR2D_ERR_OOM;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete h;
    return HODLR2D_ERR_CUDA;
  }
  h->n = n;
  h->kern = kernel;
  h->kp = kp;
  h->leaf_size = leaf_size;
  h->eps = eps;
  h->opts = o;
  const double t0 = now_ms();
  double* d_pts = nullptr;
  const bool dev = is_device_ptr(points);
  if (dev) {
    d_pts = const_cast<double*>(points);
  } else if (cudaMalloc(&d_pts, sizeof(double) * 2 * n) != cudaSuccess ||
             cudaMemcpy(d_pts, points, sizeof(double) * 2 * n, cudaMemcpyHostToDevice) !=
                 cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(d_pts);
    free_handle(h);
    return HODLR2D_ERR_OOM;
  }
  rc = tree_build(h, d_pts);
  if (!dev) cudaFree(d_pts);
  const double t1 = now_ms();
  if (!rc) rc = lists_build(h);
  const double t2 = now_ms();
  if (!rc && o.compress) rc = aca_build(h);
  const double t3 = now_ms();
  if (!rc && o.compress) {
    rc = matvec_plan(h);
    h->has_factors = true;
  }
  const double t4 = now_ms();
  if (rc) {
    (void)cudaGetLastError();
    free_handle(h);
    return rc;
  }
  h->st.build_ms[0] = t1 - t0;
  h->st.build_ms[1] = t2 - t1;
  h->st.build_ms[2] = t3 - t2;
  h->st.build_ms[3] = t4 - t3;
  fill_stats(h);
  *out = h;
  return HODLR2D_OK;
}

int hodlr2d_set_stream(hodlr2d_t h, void* stream) {
  if (!h) return HODLR2D_ERR_ARG;
  h->stream = (cudaStream_t)stream;
  return HODLR2D_OK;
}

int hodlr2d_prepare(hodlr2d_t h, int mode) {
  if (!h || mode < 0 || mode > 3) return HODLR2D_ERR_ARG;
  if (!h->has_factors) return HODLR2D_ERR_STATE;
  if (h->prepared[mode]) return HODLR2D_OK;
  if (h->f64_released) return HODLR2D_ERR_STATE;  // copies are made from the binary64 factors
  DeviceGuard g(h->device);
  return prepare_mode(h, mode);
}

int hodlr2d_release(hodlr2d_t h, int mode) {
  if (!h || mode < 0 || mode > 3) return HODLR2D_ERR_ARG;
  if (!h->has_factors) return HODLR2D_ERR_STATE;
  DeviceGuard g(h->device);
  H2D_CK(cudaStreamSynchronize(h->stream));
  for (int l = 0; l < HODLR2D_MAX_LEVELS; ++l) {
    Level& L = h->lev[l];
    if (mode == HODLR2D_MODE_F64) {
      cudaFree(L.d_fac);
      L.d_fac = nullptr;
    } else {
      cudaFree(L.d_fac_mode[mode]);
      L.d_fac_mode[mode] = nullptr;
    }
  }
  h->prepared[mode] = false;
  if (mode == HODLR2D_MODE_F64) h->f64_released = true;
  ++h->gen;
  return HODLR2D_OK;
}

int hodlr2d_matvec_ex(hodlr2d_t h, const double* x, double* y, int nrhs, int mode) {
  if (!h || !x || !y || nrhs < 1 || mode < 0 || mode > 3) return HODLR2D_ERR_ARG;
  if (!h->has_factors || !h->prepared[mode]) return HODLR2D_ERR_STATE;
  DeviceGuard g(h->device);
  int rc = HODLR2D_OK;
  const bool xd = is_device_ptr(x), yd = is_device_ptr(y);
  const size_t bytes = sizeof(double) * h->n * nrhs;
  if ((!xd || !yd) && h->io_nrhs < nrhs) {  // staging for host buffers
    cudaFree(h->d_io);
    h->d_io = nullptr;
    h->io_nrhs = 0;
    H2D_CK(cudaMalloc(&h->d_io, 2 * bytes));
    h->io_nrhs = nrhs;
  }
  const double* dx = x;
  double* dy = y;
  if (!xd) {
    H2D_CK(cudaMemcpyAsync(h->d_io, x, bytes, cudaMemcpyHostToDevice, h->stream));
    dx = h->d_io;
  }
  if (!yd) dy = h->d_io + h->n * nrhs;
  rc = matvec_mode_device(h, dx, dy, nrhs, mode);
  if (rc) return rc;
  if (!yd) {
    H2D_CK(cudaMemcpyAsync(y, dy, bytes, cudaMemcpyDeviceToHost, h->stream));
  }
  if (!xd || !yd) H2D_CK(cudaStreamSynchronize(h->stream));
  return HODLR2D_OK;
}

int hodlr2d_matvec(hodlr2d_t h, const double* x, double* y, int nrhs) {
  if (!h) return HODLR2D_ERR_ARG;
  return hodlr2d_matvec_ex(h, x, y, nrhs, h->opts.mode);
}

int hodlr2d_gmres(hodlr2d_t h, const double* b, double* x, double tol) {
  if (!h) return HODLR2D_ERR_ARG;
  const int64_t maxit = std::min<int64_t>(10 * h->n, 100000);
  return hodlr2d_gmres_ex(h, b, x, tol, 50, (int)maxit, HODLR2D_MODE_F64, nullptr, nullptr);
}

int hodlr2d_gmres_ex(hodlr2d_t h, const double* b, double* x, double tol, int restart, int maxit,
                     int inner_mode, int* iters, double* relres) {
  if (!h || !b || !x || !(tol > 0.0) || restart < 1 || maxit < 1 || inner_mode < 0 ||
      inner_mode > 3)
    return HODLR2D_ERR_ARG;
  if (!h->has_factors || !h->prepared[inner_mode]) return HODLR2D_ERR_STATE;
  // refinement computes its residuals with the binary64 product
  if ((inner_mode == HODLR2D_MODE_F32 || inner_mode == HODLR2D_MODE_BF16) &&
      !h->prepared[HODLR2D_MODE_F64])
    return HODLR2D_ERR_STATE;
  DeviceGuard g(h->device);
  return gmres_run(h, b, x, tol, restart, maxit, inner_mode, iters, relres);
}

int hodlr2d_get_stats(hodlr2d_t h, hodlr2d_stats* s) {
  if (!h || !s) return HODLR2D_ERR_ARG;
  *s = h->st;
  return HODLR2D_OK;
}

int hodlr2d_pair_features(hodlr2d_t h, int64_t* npairs, float* feats, float* log2rank) {
  if (!h || !npairs) return HODLR2D_ERR_ARG;
  int64_t tot = 0;
  for (int l = 1; l <= h->kappa; ++l) tot += h->lev[l].npairs;
  *npairs = tot;
  if (!feats && !log2rank) return HODLR2D_OK;
  if (!h->has_factors) return HODLR2D_ERR_STATE;
  DeviceGuard g(h->device);
  int64_t o = 0;
  for (int l = 1; l <= h->kappa; ++l) {
    const Level& L = h->lev[l];
    const int64_t np = L.npairs;
    if (!np) continue;
    std::vector<int32_t> px(np), py(np);
    H2D_CK(cudaMemcpy(px.data(), L.d_px, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    H2D_CK(cudaMemcpy(py.data(), L.d_py, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    const int sh = 2 * (h->kappa - l);
    for (int64_t p = 0; p < np; ++p, ++o) {
      const int64_t m = h->h_leaf_off[(int64_t)(px[p] + 1) << sh] - h->h_leaf_off[(int64_t)px[p] << sh];
      const int64_t n = h->h_leaf_off[(int64_t)(py[p] + 1) << sh] - h->h_leaf_off[(int64_t)py[p] << sh];
      if (feats) pair_features(h, l, px[p], py[p], m, n, feats + 8 * o);
      if (log2rank) log2rank[o] = (float)log2(1.0 + (double)L.h_rank[p]);
    }
  }
  return HODLR2D_OK;
}

int hodlr2d_get_perm(hodlr2d_t h, int64_t* perm) {
  if (!h || !perm) return HODLR2D_ERR_ARG;
  DeviceGuard g(h->device);
  H2D_CK(cudaMemcpy(perm, h->d_perm, sizeof(int64_t) * h->n, cudaMemcpyDeviceToHost));
  return HODLR2D_OK;
}

int hodlr2d_get_pairs(hodlr2d_t h, int64_t* npairs, int32_t* info) {
  if (!h || !npairs) return HODLR2D_ERR_ARG;
  int64_t tot = 0;
  for (int l = 1; l <= h->kappa; ++l) tot += h->lev[l].npairs;
  *npairs = tot;
  if (!info) return HODLR2D_OK;
  DeviceGuard g(h->device);
  int64_t o = 0;
  for (int l = 1; l <= h->kappa; ++l) {
    const Level& L = h->lev[l];
    const int64_t np = L.npairs;
    if (!np) continue;
    std::vector<int32_t> px(np), py(np), rk(np, 0);
    H2D_CK(cudaMemcpy(px.data(), L.d_px, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    H2D_CK(cudaMemcpy(py.data(), L.d_py, sizeof(int32_t) * np, cudaMemcpyDeviceToHost));
    if (h->has_factors) rk = L.h_rank;
    for (int64_t p = 0; p < np; ++p, ++o) {
      int ax, ay, bx, by;
      morton_decode((uint32_t)px[p], ax, ay);
      morton_decode((uint32_t)py[p], bx, by);
      int32_t* r = info + 6 * o;
      r[0] = l; r[1] = ax; r[2] = ay; r[3] = bx; r[4] = by; r[5] = rk[p];
    }
  }
  return HODLR2D_OK;
}

// Row order of box b (level l): canon[r] = the tree row holding the r-th
// point of the box in ascending original index.
static void canonical_rows(const std::vector<int64_t>& perm, int32_t start, int32_t m,
                           std::vector<int32_t>& canon) {
  canon.resize(m);
  std::iota(canon.begin(), canon.end(), 0);
  std::sort(canon.begin(), canon.end(),
            [&](int32_t a, int32_t b) { return perm[start + a] < perm[start + b]; });
}

int hodlr2d_import_factors(hodlr2d_t h, int64_t npairs, const int32_t* info,
                           const int64_t* offsets, const double* values) {
  if (!h || npairs < 0 || (npairs > 0 && (!info || !offsets || !values))) return HODLR2D_ERR_ARG;
  if (h->has_factors) return HODLR2D_ERR_STATE;
  DeviceGuard g(h->device);
  int64_t tot = 0;
  for (int l = 1; l <= h->kappa; ++l) tot += h->lev[l].npairs;
  if (tot != npairs) return HODLR2D_ERR_ARG;
  std::vector<int64_t> perm(h->n);
  H2D_CK(cudaMemcpy(perm.data(), h->d_perm, sizeof(int64_t) * h->n, cudaMemcpyDeviceToHost));
  // level -> (row key, col key) -> local pair index
  std::vector<std::unordered_map<uint64_t, int64_t>> idx(h->kappa + 1);
  std::vector<std::vector<int32_t>> PX(h->kappa + 1), PY(h->kappa + 1);
  for (int l = 1; l <= h->kappa; ++l) {
    Level& L = h->lev[l];
    PX[l].resize(L.npairs);
    PY[l].resize(L.npairs);
    if (L.npairs) {
      H2D_CK(cudaMemcpy(PX[l].data(), L.d_px, sizeof(int32_t) * L.npairs, cudaMemcpyDeviceToHost));
      H2D_CK(cudaMemcpy(PY[l].data(), L.d_py, sizeof(int32_t) * L.npairs, cudaMemcpyDeviceToHost));
    }
    for (int64_t p = 0; p < L.npairs; ++p)
      idx[l][((uint64_t)(uint32_t)PX[l][p] << 32) | (uint32_t)PY[l][p]] = p;
    L.h_rank.assign(L.npairs, -1);
  }
  std::vector<int64_t> src(npairs, -1);
  std::vector<std::vector<int64_t>> where(h->kappa + 1);
  for (int l = 1; l <= h->kappa; ++l) where[l].assign(h->lev[l].npairs, -1);
  for (int64_t q = 0; q < npairs; ++q) {
    const int32_t* r = info + 6 * q;
    const int l = r[0];
    if (l < 1 || l > h->kappa || r[5] < 0) return HODLR2D_ERR_ARG;
    const int side = 1 << l;
    for (int d = 1; d <= 4; ++d)
      if (r[d] < 0 || r[d] >= side) return HODLR2D_ERR_ARG;
    const uint32_t kx = morton_encode(r[1], r[2]), ky = morton_encode(r[3], r[4]);
    auto it = idx[l].find(((uint64_t)kx << 32) | ky);
    if (it == idx[l].end() || where[l][it->second] >= 0) return HODLR2D_ERR_ARG;
    where[l][it->second] = q;
  }
  for (int l = 1; l <= h->kappa; ++l) {
    Level& L = h->lev[l];
    const int sh = 2 * (h->kappa - l);
    auto start = [&](int32_t b) { return h->h_leaf_off[(int64_t)b << sh]; };
    auto cnt = [&](int32_t b) {
      return h->h_leaf_off[(int64_t)(b + 1) << sh] - h->h_leaf_off[(int64_t)b << sh];
    };
    L.h_foff.assign(L.npairs + 1, 0);
    int64_t tot_v = 0, stored_v = 0;
    for (int64_t p = 0; p < L.npairs; ++p) {
      const int64_t q = where[l][p];
      const int k = info[6 * q + 5];
      const int64_t m = cnt(PX[l][p]), nn = cnt(PY[l][p]);
      if (k > std::min(m, nn) || offsets[q + 1] - offsets[q] != (m + nn) * k) return HODLR2D_ERR_ARG;
      L.h_rank[p] = k;
      L.h_foff[p] = tot_v;
      tot_v += (ldpad(m) + ldpad(nn)) * k;
      stored_v += (m + nn) * k;
    }
    L.h_foff[L.npairs] = tot_v;
    L.nvalues = tot_v;
    L.nstored = stored_v;
    std::vector<double> fac(std::max<int64_t>(tot_v, 1), 0.0);
    std::vector<int32_t> cx, cy;
    L.max_rank = 0;
    for (int64_t p = 0; p < L.npairs; ++p) {
      const int64_t q = where[l][p];
      const int k = L.h_rank[p];
      L.max_rank = std::max(L.max_rank, k);
      const int32_t m = cnt(PX[l][p]), nn = cnt(PY[l][p]);
      canonical_rows(perm, start(PX[l][p]), m, cx);
      canonical_rows(perm, start(PY[l][p]), nn, cy);
      const double* U = values + offsets[q];
      const double* V = U + (int64_t)m * k;
      const int64_t lm = ldpad(m), ln = ldpad(nn);
      double* Uo = fac.data() + L.h_foff[p];
      double* Vo = Uo + lm * k;
      for (int c = 0; c < k; ++c) {
        for (int32_t r = 0; r < m; ++r) Uo[c * lm + cx[r]] = U[(int64_t)c * m + r];
        for (int32_t r = 0; r < nn; ++r) Vo[c * ln + cy[r]] = V[(int64_t)c * nn + r];
      }
    }
    H2D_CK(cudaMalloc(&L.d_rank, sizeof(int32_t) * (L.npairs + 1)));
    H2D_CK(cudaMalloc(&L.d_foff, sizeof(int64_t) * (L.npairs + 1)));
    // 16 bytes of slack: bulk copies widen each column to 16-byte boundaries
    H2D_CK(cudaMalloc(&L.d_fac, sizeof(double) * (fac.size() + 2)));
    if (L.npairs)
      H2D_CK(cudaMemcpy(L.d_rank, L.h_rank.data(), sizeof(int32_t) * L.npairs,
                        cudaMemcpyHostToDevice));
    H2D_CK(cudaMemcpy(L.d_foff, L.h_foff.data(), sizeof(int64_t) * (L.npairs + 1),
                      cudaMemcpyHostToDevice));
    H2D_CK(cudaMemcpy(L.d_fac, fac.data(), sizeof(double) * fac.size(), cudaMemcpyHostToDevice));
  }
  int rc = matvec_plan(h);
  if (rc) return rc;
  h->has_factors = true;
  h->st.unconverged = 0;
  fill_stats(h);
  return HODLR2D_OK;
}

int hodlr2d_export_factors(hodlr2d_t h, int64_t* npairs, int64_t* nvalues, int32_t* info,
                           int64_t* offsets, double* values) {
  if (!h || !npairs || !nvalues) return HODLR2D_ERR_ARG;
  if (!h->has_factors) return HODLR2D_ERR_STATE;
  int64_t tp = 0, tv = 0;
  for (int l = 1; l <= h->kappa; ++l) {
    tp += h->lev[l].npairs;
    tv += h->lev[l].nstored;
  }
  *npairs = tp;
  *nvalues = tv;
  if (!values) return HODLR2D_OK;
  if (!info || !offsets) return HODLR2D_ERR_ARG;
  if (h->f64_released) return HODLR2D_ERR_STATE;
  DeviceGuard g(h->device);
  std::vector<int64_t> perm(h->n);
  H2D_CK(cudaMemcpy(perm.data(), h->d_perm, sizeof(int64_t) * h->n, cudaMemcpyDeviceToHost));
  int rc = hodlr2d_get_pairs(h, &tp, info);
  if (rc) return rc;
  int64_t q = 0, o = 0;
  std::vector<int32_t> cx, cy;
  for (int l = 1; l <= h->kappa; ++l) {
    const Level& L = h->lev[l];
    if (!L.npairs) continue;
    const int sh = 2 * (h->kappa - l);
    std::vector<int32_t> px(L.npairs), py(L.npairs);
    H2D_CK(cudaMemcpy(px.data(), L.d_px, sizeof(int32_t) * L.npairs, cudaMemcpyDeviceToHost));
    H2D_CK(cudaMemcpy(py.data(), L.d_py, sizeof(int32_t) * L.npairs, cudaMemcpyDeviceToHost));
    std::vector<double> fac(std::max<int64_t>(L.nvalues, 1));
    H2D_CK(cudaMemcpy(fac.data(), L.d_fac, sizeof(double) * L.nvalues, cudaMemcpyDeviceToHost));
    for (int64_t p = 0; p < L.npairs; ++p, ++q) {
      const int k = L.h_rank[p];
      const int32_t sx = h->h_leaf_off[(int64_t)px[p] << sh];
      const int32_t m = h->h_leaf_off[(int64_t)(px[p] + 1) << sh] - sx;
      const int32_t sy = h->h_leaf_off[(int64_t)py[p] << sh];
      const int32_t nn = h->h_leaf_off[(int64_t)(py[p] + 1) << sh] - sy;
      canonical_rows(perm, sx, m, cx);
      canonical_rows(perm, sy, nn, cy);
      offsets[q] = o;
      const int64_t lm = ldpad(m), ln = ldpad(nn);
      const double* U = fac.data() + L.h_foff[p];
      const double* V = U + lm * k;
      double* Uo = values + o;
      double* Vo = Uo + (int64_t)m * k;
      for (int c = 0; c < k; ++c) {
        for (int32_t r = 0; r < m; ++r) Uo[(int64_t)c * m + r] = U[c * lm + cx[r]];
        for (int32_t r = 0; r < nn; ++r) Vo[(int64_t)c * nn + r] = V[c * ln + cy[r]];
      }
      o += (int64_t)(m + nn) * k;
    }
  }
  offsets[q] = o;
  return HODLR2D_OK;
}

static void prof_clear(hodlr2d* h) {
  for (auto& r : h->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  h->prof.clear();
}

int hodlr2d_profile(hodlr2d_t h, int enable) {
  if (!h) return HODLR2D_ERR_ARG;
  DeviceGuard g(h->device);
  if (enable) {
    H2D_CK(cudaStreamSynchronize(h->stream));
    prof_clear(h);
    for (int p = 0; p < HODLR2D_NPHASE; ++p) {
      h->prof_ms[p] = 0.0;
      h->prof_launches[p] = 0;
      h->prof_bytes[p] = 0;
      h->prof_flops[p] = 0;
    }
  }
  h->prof_on = enable != 0;
  return HODLR2D_OK;
}

int hodlr2d_get_profile(hodlr2d_t h, double* ms, int64_t* launches, int64_t* bytes) {
  if (!h) return HODLR2D_ERR_ARG;
  DeviceGuard g(h->device);
  H2D_CK(cudaStreamSynchronize(h->stream));
  for (auto& r : h->prof) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) h->prof_ms[r.phase] += t;
    else (void)cudaGetLastError();
  }
  prof_clear(h);
  for (int p = 0; p < HODLR2D_NPHASE; ++p) {
    if (ms) ms[p] = h->prof_ms[p];
    if (launches) launches[p] = h->prof_launches[p];
    if (bytes) bytes[p] = h->prof_bytes[p];
  }
  return HODLR2D_OK;
}

int hodlr2d_check(hodlr2d_t h) {
  if (!h) return HODLR2D_ERR_ARG;
  DeviceGuard g(h->device);
  return product_status(h);
}

int hodlr2d_get_profile_flops(hodlr2d_t h, int64_t* flops) {
  if (!h || !flops) return HODLR2D_ERR_ARG;
  for (int p = 0; p < HODLR2D_NPHASE; ++p) flops[p] = h->prof_flops[p];
  return HODLR2D_OK;
}

void hodlr2d_free(hodlr2d_t h) {
  if (h) prof_clear(h);
  free_handle(h);
}

}  // extern "C"
