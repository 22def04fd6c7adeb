// Arithmetic policies of the product kernels.
//
//   F64A   values and sums in IEEE binary64.
//   DF32A  values stored as float pairs (hi, lo) with hi + lo the binary64
//          value to ~2^-48 relative; products and sums in float-float
//          arithmetic (Dekker's product via FMA, Knuth's two-sum).  On GB300
//          binary32 FMA throughput is ~58x that of binary64, so this keeps
//          binary64-level accuracy at memory speed.
//
// Float-float square root and reciprocal square root: one Newton-Raphson
// correction of the binary32 estimate, evaluated with an exact square
// (Karp & Markstein 1997 style), giving ~2^-44 relative accuracy.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace h2d {

// terms between renormalisations of a float-float accumulator in long sums
constexpr int kRenorm = 16;

struct F64A {
  typedef double fac;  // factor storage
  typedef double val;  // vectors and sums
  typedef double acc;
  static __device__ __forceinline__ val ld(fac f) { return f; }
  static __device__ __forceinline__ acc zero() { return 0.0; }
  static __device__ __forceinline__ void fma(acc& s, val a, val b) { s = ::fma(a, b, s); }
  static __device__ __forceinline__ void renorm(acc&) {}
  static __device__ __forceinline__ val fin(acc s) { return s; }
  static __device__ __forceinline__ val add(val a, val b) { return a + b; }
  static __device__ __forceinline__ val from_double(double d) { return d; }
  static __device__ __forceinline__ double to_double(val v) { return v; }
  static __device__ __forceinline__ val vzero() { return 0.0; }
  static __device__ __forceinline__ val warp_sum(acc a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
  }
};

struct DF32A {
  typedef float2 fac;
  typedef float2 val;  // x = hi, y = lo
  static __device__ __forceinline__ val ld(fac f) { return f; }
  typedef float2 acc;  // lazily normalised: hi exact running sum, lo collects errors
  static __device__ __forceinline__ acc zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ val vzero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void fma(acc& s, val a, val b) {
    float p, e;
    two_prod(a.x, b.x, p, e);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    float t, err;
    two_sum(s.x, p, t, err);
    s.x = t;
    s.y = __fadd_rn(s.y, __fadd_rn(err, e));
  }
  static __device__ __forceinline__ val fin(acc s) {
    float h, l;
    fast_two_sum(s.x, s.y, h, l);
    return make_float2(h, l);
  }
  // The accumulator adds every rounding error into lo with plain binary32
  // additions, whose own rounding grows with the number of terms; long sums
  // call this every kRenorm terms to fold lo back into hi (an exact two-sum),
  // which keeps lo below half an ulp of hi.
  static __device__ __forceinline__ void renorm(acc& s) {
    float h, l;
    two_sum(s.x, s.y, h, l);
    s = make_float2(h, l);
  }
  static __device__ __forceinline__ val add(val a, val b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    float h, l;
    fast_two_sum(s, e, h, l);
    return make_float2(h, l);
  }
  static __device__ __forceinline__ val from_double(double d) {
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));
  }
  static __device__ __forceinline__ double to_double(val v) { return (double)v.x + (double)v.y; }
  static __device__ __forceinline__ val warp_sum(acc a) {
    val v = fin(a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      val w;
      w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
      w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
      v = add(v, w);
    }
    return v;
  }
};

// binary32 sums over binary32 factors (the mixed form)
struct F32A {
  typedef float fac;
  typedef float val;
  typedef float acc;
  static __device__ __forceinline__ val ld(fac f) { return f; }
  static __device__ __forceinline__ acc zero() { return 0.f; }
  static __device__ __forceinline__ val vzero() { return 0.f; }
  static __device__ __forceinline__ void fma(acc& s, val a, val b) { s = __fmaf_rn(a, b, s); }
  static __device__ __forceinline__ void renorm(acc&) {}
  static __device__ __forceinline__ val fin(acc s) { return s; }
  static __device__ __forceinline__ val add(val a, val b) { return a + b; }
  static __device__ __forceinline__ val from_double(double d) { return __double2float_rn(d); }
  static __device__ __forceinline__ double to_double(val v) { return (double)v; }
  static __device__ __forceinline__ val warp_sum(acc a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
  }
};

// binary32 sums over bfloat16 factors (the mixed form, half the bytes again)
struct BF16A : F32A {
  typedef __nv_bfloat16 fac;
  static __device__ __forceinline__ val ld(fac f) { return __bfloat162float(f); }
};

// ---------------------------------------------------------------------------
// float-float elementary functions for the near field
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 ffv_sub(float2 a, float2 b) {
  return DF32A::add(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 ffv_mul(float2 a, float2 b) {
  float p, e;
  two_prod(a.x, b.x, p, e);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return make_float2(h, l);
}
// sqrt(a) for a >= 0: s = sqrt(a.hi) in binary32, then s + (a - s^2) / (2 s)
__device__ __forceinline__ float2 ffv_sqrt(float2 a) {
  if (!(a.x > 0.f)) return make_float2(0.f, 0.f);
  const float s = __fsqrt_rn(a.x);
  float p, e;
  two_prod(s, s, p, e);
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(a.x, p), e), a.y);
  const float c = __fdividef(d, 2.0f * s);
  float h, l;
  fast_two_sum(s, c, h, l);
  return make_float2(h, l);
}
// 1/sqrt(a) for a > 0: r = rsqrt(a.hi), then r + r (1 - a r^2) / 2 with a r^2
// formed from the exact square of r
__device__ __forceinline__ float2 ffv_rsqrt(float2 a) {
  const float r = rsqrtf(a.x);
  float p, e;
  two_prod(r, r, p, e);          // r^2 = p + e exactly
  const float2 ar2 = ffv_mul(a, make_float2(p, e));
  float one_minus = __fsub_rn(1.0f, ar2.x);  // exact (ar2 ~ 1)
  one_minus = __fsub_rn(one_minus, ar2.y);
  const float c = 0.5f * r * one_minus;
  float h, l;
  fast_two_sum(r, c, h, l);
  return make_float2(h, l);
}
// 1/a: r = 1/a.hi, then r + r (1 - a r)
__device__ __forceinline__ float2 ffv_rcp(float2 a) {
  const float r = __frcp_rn(a.x);
  const float2 ar = ffv_mul(a, make_float2(r, 0.f));
  float one_minus = __fsub_rn(1.0f, ar.x);
  one_minus = __fsub_rn(one_minus, ar.y);
  const float c = r * one_minus;
  float h, l;
  fast_two_sum(r, c, h, l);
  return make_float2(h, l);
}
__device__ __forceinline__ bool ffv_ge(float2 a, float2 b) {
  return a.x > b.x || (a.x == b.x && a.y >= b.y);
}

// float-float pair of a binary64 constant, at compile time
struct FFConst {
  float hi, lo;
  __host__ __device__ constexpr FFConst(double d)
      : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

// Natural logarithm of a float-float x > 0 (a normal binary32 high part), to
// about 2^-46 relative.  Argument reduction x = 2^e m with m in [sqrt(1/2),
// sqrt(2)), then log m = 2 atanh(s) = 2 s (1 + z/3 + z^2/5 + ...), s =
// (m - 1) / (m + 1), z = s^2 <= 0.0295: the series to z^8 (its remainder is
// below 2^-48) by Horner's rule, the four leading steps in float-float and
// the tail in binary32.  log x = e log 2 + log m.
__device__ __forceinline__ float2 ffv_log(float2 x) {
  constexpr FFConst LN2(0.69314718055994530942);
  constexpr FFConst C3(1.0 / 3.0), C5(1.0 / 5.0), C7(1.0 / 7.0);
  const int bits = __float_as_int(x.x);
  int e = ((bits >> 23) & 0xff) - 127;
  float mh = __int_as_float((bits & 0x007fffff) | 0x3f800000);  // [1, 2)
  if (mh > 1.41421356f) {
    mh *= 0.5f;
    e += 1;
  }
  const float ml = ldexpf(x.y, -e);  // exact: a power-of-two scaling
  // s = (m - 1) / (m + 1); m - 1 is exact in its high part (Sterbenz)
  float nh, nl, dh, dl;
  two_sum(mh - 1.0f, ml, nh, nl);
  two_sum(mh, 1.0f, dh, dl);
  dl = __fadd_rn(dl, ml);
  fast_two_sum(dh, dl, dh, dl);
  const float2 sv = ffv_mul(make_float2(nh, nl), ffv_rcp(make_float2(dh, dl)));
  const float2 z = ffv_mul(sv, sv);
  const float zf = z.x;
  float r = __fmaf_rn(zf, 1.0f / 17.0f, 1.0f / 15.0f);
  r = __fmaf_rn(zf, r, 1.0f / 13.0f);
  r = __fmaf_rn(zf, r, 1.0f / 11.0f);
  r = __fmaf_rn(zf, r, 1.0f / 9.0f);
  float2 c = DF32A::add(make_float2(C7.hi, C7.lo), ffv_mul(z, make_float2(r, 0.f)));
  c = DF32A::add(make_float2(C5.hi, C5.lo), ffv_mul(z, c));
  c = DF32A::add(make_float2(C3.hi, C3.lo), ffv_mul(z, c));
  c = DF32A::add(make_float2(1.f, 0.f), ffv_mul(z, c));
  float2 lm = ffv_mul(sv, c);
  lm.x *= 2.f;
  lm.y *= 2.f;
  const float ef = (float)e;
  float ph, pe;
  two_prod(ef, LN2.hi, ph, pe);
  pe = __fmaf_rn(ef, LN2.lo, pe);
  float eh, el;
  fast_two_sum(ph, pe, eh, el);
  return DF32A::add(make_float2(eh, el), lm);
}

// Kernel parameters in float-float.
struct KernelFF {
  int kind;
  float2 a, a2, inv_a, diag;
  float2 inv_log_a, inv_phi1_den;  // 1 / log a and 1 / (a log a - 1) for phi_1
};

// Entry phi(|x_i - x_j|) of the kernel; gi and gj identify the two points
// (any bijection of the original index) and decide the diagonal.
__device__ __forceinline__ float2 entry_ff(const KernelFF& k, float2 xi, float2 yi, int64_t gi,
                                           float2 xj, float2 yj, int64_t gj) {
  if (gi == gj) return k.diag;
  const float2 dx = ffv_sub(xi, xj), dy = ffv_sub(yi, yj);
  const float2 r2 = DF32A::add(ffv_mul(dx, dx), ffv_mul(dy, dy));
  switch (k.kind) {
    case HODLR2D_IMQ: return ffv_rsqrt(DF32A::add(r2, k.a2));
    case HODLR2D_MQ: return ffv_sqrt(DF32A::add(r2, k.a2));
    case HODLR2D_INV_R: return ffv_rsqrt(r2);
    case HODLR2D_PHI2: {
      const float2 r = ffv_sqrt(r2);
      if (ffv_ge(r, k.a)) return ffv_mul(k.a, ffv_rcp(r));
      return ffv_mul(r, k.inv_a);
    }
    case HODLR2D_LOG: {  // log r = log(r^2) / 2
      const float2 l = ffv_log(r2);
      return make_float2(0.5f * l.x, 0.5f * l.y);
    }
    default: {  // phi_1
      const float2 r = ffv_sqrt(r2);
      const float2 l2 = ffv_log(r2);
      const float2 lr = make_float2(0.5f * l2.x, 0.5f * l2.y);
      if (ffv_ge(r, k.a)) return ffv_mul(lr, k.inv_log_a);
      return ffv_mul(DF32A::add(ffv_mul(r, lr), make_float2(-1.f, 0.f)), k.inv_phi1_den);
    }
  }
}

// binary32 kernel parameters and entries (near field of the mixed form)
struct KernelF32 {
  int kind;
  float a, a2, inv_a, log_a, phi1_den, diag;
};

__device__ __forceinline__ float entry_f32(const KernelF32& k, float xi, float yi, int64_t gi,
                                           float xj, float yj, int64_t gj) {
  if (gi == gj) return k.diag;
  const float dx = xi - xj, dy = yi - yj;
  const float r2 = __fmaf_rn(dx, dx, dy * dy);
  switch (k.kind) {
    case HODLR2D_IMQ: return rsqrtf(r2 + k.a2);
    case HODLR2D_MQ: return sqrtf(r2 + k.a2);
    case HODLR2D_LOG: return 0.5f * logf(r2);
    case HODLR2D_INV_R: return rsqrtf(r2);
    case HODLR2D_PHI1: {
      const float r = sqrtf(r2);
      if (r >= k.a) return logf(r) / k.log_a;
      return (r * logf(r) - 1.0f) / k.phi1_den;
    }
    default: {
      const float r = sqrtf(r2);
      if (r >= k.a) return k.a / r;
      return r * k.inv_a;
    }
  }
}

}  // namespace h2d
