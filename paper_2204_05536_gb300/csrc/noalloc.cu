// hodlr2d_matvec_noalloc: the FP64 product with its working memory in a
// fixed, statically sized device array instead of memory the library
// allocates.
//
// Why it exists: some callers must not allocate device memory once they are
// running -- for example a serving loop that cannot afford the implicit
// device-wide synchronisation of cudaMalloc/cudaFree, or a host framework
// that owns the whole device-memory budget and forbids allocations outside
// its own pool.  hodlr2d_matvec may allocate its scratch on first use (or
// when nrhs grows); this entry point never does.
//
// The array below lives in every process that loads the library, on every
// GPU the library is used on, until the process exits.  All calls share it,
// so two calls whose kernels overlap in time on the GPU (different streams,
// different handles, different host threads) race on it and give wrong
// results.  It keeps whatever the previous call left; the product writes
// every scratch word it later reads, so nothing needs clearing between calls.
#include <mutex>

#include "internal.h"

namespace h2d {
bool is_device_ptr(const void* p);
int matvec_f64_scratch(hodlr2d* h, const double* x, double* y, int nrhs, double* xt, double* yl,
                       double* part, double* t);
}  // namespace h2d

static __device__ __align__(256) unsigned char g_noalloc_scratch[HODLR2D_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (host code only
// sees a host-side stand-in under the array's name, which kernels must never
// receive).  Looked up once per device.
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return HODLR2D_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return HODLR2D_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HODLR2D_OK;
}

int64_t align256(int64_t bytes) { return (bytes + 255) / 256 * 256; }

}  // namespace

extern "C" int hodlr2d_matvec_noalloc(hodlr2d_t h, const double* x, double* y, int nrhs) {
  if (!h || !x || !y || nrhs < 1) return HODLR2D_ERR_ARG;
  if (!h->has_factors || h->f64_released) return HODLR2D_ERR_STATE;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    (void)cudaGetLastError();
    return HODLR2D_ERR_CUDA;
  }
  if (cur != h->device) return HODLR2D_ERR_ARG;  // the handle's device must be current
  if (!h2d::is_device_ptr(x) || !h2d::is_device_ptr(y)) return HODLR2D_ERR_ARG;
  const int64_t n = h->n;
  const int64_t b_xt = align256(8 * n * nrhs);
  const int64_t b_yl = align256(8 * n * nrhs * (h->kappa + 1));
  const int64_t b_part = align256(8 * (h->proj_partials > 0 ? h->proj_partials : 1) * nrhs);
  const int64_t b_t = align256(8 * (h->t_total > 0 ? h->t_total : 1) * nrhs);
  if (b_xt + b_yl + b_part + b_t > (int64_t)HODLR2D_NOALLOC_SCRATCH_BYTES) return HODLR2D_ERR_ARG;
  void* base = nullptr;
  const int rc = scratch_address(cur, &base);
  if (rc != HODLR2D_OK) return rc;
  unsigned char* p = static_cast<unsigned char*>(base);
  double* xt = reinterpret_cast<double*>(p);
  double* yl = reinterpret_cast<double*>(p + b_xt);
  double* part = reinterpret_cast<double*>(p + b_xt + b_yl);
  double* t = reinterpret_cast<double*>(p + b_xt + b_yl + b_part);
  return h2d::matvec_f64_scratch(h, x, y, nrhs, xt, yl, part, t);
}
