// Shared device helpers of the CUDA library: kernel entries, Morton codes,
// float-float arithmetic, launch bookkeeping.  Nothing here is shared with the
// CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hodlr2d.h"

namespace h2d {

// ---------------------------------------------------------------------------
// Error plumbing: every CUDA call on the host goes through CK(), which turns
// a failure into HODLR2D_ERR_CUDA (or OOM) for the current entry point.
// ---------------------------------------------------------------------------
#define H2D_CK(call)                                                   \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) {                                           \
      (void)cudaGetLastError();                                        \
      return e_ == cudaErrorMemoryAllocation ? HODLR2D_ERR_OOM         \
                                             : HODLR2D_ERR_CUDA;       \
    }                                                                  \
  } while (0)

#define H2D_TRY(expr)              \
  do {                             \
    int rc_ = (expr);              \
    if (rc_ != HODLR2D_OK) return rc_; \
  } while (0)

// ---------------------------------------------------------------------------
// Kernel entries.  phi as a function of the squared distance, as in Sec. 3
// (log r), Eq. 1byr (1/r) and Eq. ker (phi_1, phi_2); IMQ and MQ are the
// radial basis functions of the interpolation workloads.
// ---------------------------------------------------------------------------
struct KernelParams {
  int kind;
  double a;
  double a2;        // a * a
  double log_a;     // log(a)        (phi_1)
  double phi1_den;  // a log a - 1   (phi_1)
  double inv_a;     // 1 / a         (phi_2)
  double diag;      // A_ii
};

__device__ __forceinline__ double phi_r2(const KernelParams& k, double r2) {
  switch (k.kind) {
    case HODLR2D_IMQ: return 1.0 / sqrt(r2 + k.a2);
    case HODLR2D_MQ: return sqrt(r2 + k.a2);
    case HODLR2D_LOG: return 0.5 * log(r2);
    case HODLR2D_INV_R: return 1.0 / sqrt(r2);
    case HODLR2D_PHI1: {
      const double r = sqrt(r2);
      if (r >= k.a) return log(r) / k.log_a;
      return (r * log(r) - 1.0) / k.phi1_den;
    }
    default: {  // HODLR2D_PHI2
      const double r = sqrt(r2);
      if (r >= k.a) return k.a / r;
      return r * k.inv_a;
    }
  }
}

// Entry between points (xi, yi) and (xj, yj) with original indices gi, gj.
__device__ __forceinline__ double entry(const KernelParams& k, double xi, double yi,
                                        int64_t gi, double xj, double yj, int64_t gj) {
  if (gi == gj) return k.diag;
  const double dx = xi - xj, dy = yi - yj;
  return phi_r2(k, dx * dx + dy * dy);
}

// ---------------------------------------------------------------------------
// Morton codes: x bits in even positions, y bits in odd positions.  Boxes of a
// level are contiguous ranges of leaves in Morton order.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}
__host__ __device__ __forceinline__ uint32_t compact_bits(uint32_t v) {
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0F0F0F0Fu;
  v = (v | (v >> 4)) & 0x00FF00FFu;
  v = (v | (v >> 8)) & 0x0000FFFFu;
  return v;
}
__host__ __device__ __forceinline__ uint32_t morton_encode(uint32_t ix, uint32_t iy) {
  return spread_bits(ix) | (spread_bits(iy) << 1);
}
__host__ __device__ __forceinline__ void morton_decode(uint32_t key, int& ix, int& iy) {
  ix = (int)compact_bits(key);
  iy = (int)compact_bits(key >> 1);
}

// ---------------------------------------------------------------------------
// Float-float ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two binary32 numbers with |lo| <= ulp(hi)/2.  Error-free
// transformations: Knuth's TwoSum and the FMA form of Dekker's TwoProduct.
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_from_double(double d) {
  ff r;
  r.hi = __double2float_rn(d);
  r.lo = __double2float_rn(d - (double)r.hi);
  return r;
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Knuth TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Fast TwoSum (|a| >= |b|).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// TwoProduct with FMA: p + e == a * b exactly.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  ff r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// Accumulator without a renormalisation per step: sum hi exactly with
// TwoSum, collect every rounding error and cross term in lo.
struct ffacc {
  float hi, lo;
};
__device__ __forceinline__ void ffacc_fma(ffacc& s, ff a, ff b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float t, err;
  two_sum(s.hi, p, t, err);
  s.hi = t;
  s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
}
__device__ __forceinline__ ff ffacc_result(ffacc s) {
  ff r;
  fast_two_sum(s.hi, s.lo, r.hi, r.lo);
  return r;
}

}  // namespace h2d
