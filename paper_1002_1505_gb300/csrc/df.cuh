// Double-float ("float-float") arithmetic for the FP64-accurate product on GB300.
//
// GB300 executes FP64 at 1/64 of its FP32 rate, so a complex128 FFT product is
// bound by the FP64 units while its complex64 twin is not.  A double-float
// number is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2; it
// carries 48 significand bits (unit roundoff about 2^-47, against FP64's
// 2^-53) and needs only FP32 instructions.  The operations below follow the
// error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2,
// TwoSum), combined as in the double-double work of Hida, Li and Bailey
// (2001):
//   two_sum(a, b)       s + e = a + b exactly (6 additions, any magnitudes)
//   quick_two_sum(a, b) the same when |a| >= |b| (3 additions)
//   two_prod(a, b)      p + e = a * b exactly, e = fma(a, b, -p)
// Addition is the "sloppy" variant (the low parts are added in FP32): its error
// is bounded by a small multiple of 2^-47 (|a| + |b|), which is the norm-wise
// bound an FFT needs; cancellation never amplifies it beyond that.
//
// The types live in their own namespace so that their overloads of fma,
// cadd, cmul, ... are found through argument-dependent lookup inside the
// generic FFT and product templates, without hiding the float and double
// overloads those templates use for the other precisions.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>

#include "fft.cuh"

namespace dda {
namespace dfp {

struct __align__(8) df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  // round a double to the nearest double-float (exact for the 48 leading bits); used for constants
  __host__ __device__ explicit constexpr df(double v)
      : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

struct __align__(16) dfc {
  df x, y;
};

#ifdef __CUDACC__
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = a + b;
  return df(s, b - (s - a));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator+(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
// sign factor (the FFT templates multiply by the transform direction +-1)
__device__ __forceinline__ df operator*(int s, df a) { return s >= 0 ? a : -a; }
// a * b + c with the product kept exact before the addition
__device__ __forceinline__ df fma(df a, df b, df c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const df s = two_sum(p, c.hi);
  return quick_two_sum(s.hi, s.lo + (e + c.lo));
}

__device__ __forceinline__ dfc mk(df a, df b) { dfc r; r.x = a; r.y = b; return r; }
__device__ __forceinline__ dfc cadd(dfc a, dfc b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ dfc csub(dfc a, dfc b) { return mk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ dfc cmul(dfc a, dfc b) { return mk(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x)); }
// a * conj(b)
__device__ __forceinline__ dfc cmulc(dfc a, dfc b) { return mk(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -(a.x * b.y))); }

// complex128 storage <-> double-float registers
__device__ __forceinline__ df split(double v) {
  const float h = __double2float_rn(v);
  return df(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ dfc from_c128(double2 v) { return mk(split(v.x), split(v.y)); }
__device__ __forceinline__ double2 to_c128(dfc v) {
  return make_double2((double)v.x.hi + (double)v.x.lo, (double)v.y.hi + (double)v.y.lo);
}
#endif  // __CUDACC__

}  // namespace dfp

#ifdef __CUDACC__
template <> __device__ __forceinline__ dfp::dfc czero<dfp::dfc>() {
  dfp::dfc r;
  r.x = dfp::df(0.0f, 0.0f);
  r.y = dfp::df(0.0f, 0.0f);
  return r;
}
#endif

// Element type of the product's input and output vectors for a compute type:
// the double-float product reads and writes complex128 vectors.
template <typename C> struct Io { using t = C; };
template <> struct Io<dfp::dfc> { using t = double2; };

#ifdef __CUDACC__
template <typename C>
__device__ __forceinline__ C io_get(const typename Io<C>::t& v) {
  if constexpr (std::is_same<C, dfp::dfc>::value) return dfp::from_c128(v);
  else return v;
}
template <typename C>
__device__ __forceinline__ typename Io<C>::t io_put(const C& v) {
  if constexpr (std::is_same<C, dfp::dfc>::value) return dfp::to_c128(v);
  else return v;
}
#endif

}  // namespace dda
