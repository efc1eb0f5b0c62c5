// Arithmetic of the face kernels: FP32, FP64, and float-float ("ff").
//
// The ff form keeps FP64 data in memory (x and y are double) and computes with
// pairs of floats (hi, lo): products through the exact FMA product error, sums
// through the error-free two-sum, renormalised after every operation.  Each
// operation has a relative error of a few units of 2^-48, so the ff operator
// stays well inside the 1e-12 relative accuracy asked of the FP64 operator while
// running on the FP32 pipes (128 lanes/clock/SM on GB300, against 2 for FP64).
//
// Every float operation of the error-free transforms is written with the _rn
// intrinsics, which the compiler never contracts or reorders.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gp {

struct alignas(8) ff64 {
  float hi, lo;
};

template <typename IO_, typename V_>
struct Arith {
  using IO = IO_;  // element type of x and y in memory
  using V = V_;    // value type of the computation and of the face outputs
};
using ArF32 = Arith<float, float>;
using ArF64 = Arith<double, double>;
using ArFF = Arith<double, ff64>;

// ------------------------------------------------------------------ zero --
template <typename V> __host__ __device__ __forceinline__ V vzero();
template <> __host__ __device__ __forceinline__ float vzero<float>() { return 0.f; }
template <> __host__ __device__ __forceinline__ double vzero<double>() { return 0.0; }
template <> __host__ __device__ __forceinline__ ff64 vzero<ff64>() { return ff64{0.f, 0.f}; }

// ------------------------------------------------------- c = a * b + c --
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ ff64 vfma(ff64 a, ff64 b, ff64 c) {
  // product a*b = p + e exactly for the hi parts, plus the two cross terms
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  // two-sum of c.hi + p
  const float s = __fadd_rn(c.hi, p);
  const float bb = __fsub_rn(s, c.hi);
  const float err = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float lo = __fadd_rn(__fadd_rn(c.lo, e), err);
  // renormalise (fast two-sum)
  const float hi = __fadd_rn(s, lo);
  return ff64{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

// ---------------------------------------------------------------- a + b --
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }

__device__ __forceinline__ ff64 vadd(ff64 a, ff64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
  const float hi = __fadd_rn(s, lo);
  return ff64{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

// ---------------------------------------------------------------- a - b --
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ ff64 vsub(ff64 a, ff64 b) { return vadd(a, ff64{-b.hi, -b.lo}); }

// ------------------------------------------------------------ a * b --
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ double vmul(double a, double b) { return a * b; }

__device__ __forceinline__ ff64 vmul(ff64 a, ff64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float hi = __fadd_rn(p, e);
  return ff64{hi, __fsub_rn(e, __fsub_rn(hi, p))};
}

// ------------------------------------------- dot products and sums --
// Dot<V> accumulates sum_i a_i b_i; Sum<V> accumulates sum_i v_i.  For FP32 and
// FP64 they are plain fused multiply-adds / adds.  For float-float they follow the
// compensated dot product and sum of Ogita, Rump and Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, 2005; Dot2 and Sum2): the running sum s is
// kept as one float updated by error-free two-sums, the rounding errors of all
// products and sums are added into one float c, and (s, c) is renormalised once
// at the end.  The result is as accurate as if computed in twice the working
// precision (about 2^-48 relative to sum |a_i b_i|), with 12 float operations per
// term instead of the 15 of a renormalised float-float multiply-add.
template <typename V>
struct Dot {
  V v;
};
template <>
struct Dot<ff64> {
  float s, c;
};
template <typename V>
using Sum = Dot<V>;

__device__ __forceinline__ Dot<float> dot_first(float a, float b) { return Dot<float>{a * b}; }
__device__ __forceinline__ Dot<double> dot_first(double a, double b) { return Dot<double>{a * b}; }
__device__ __forceinline__ void dot_fma(Dot<float>& d, float a, float b) { d.v = fmaf(a, b, d.v); }
__device__ __forceinline__ void dot_fma(Dot<double>& d, double a, double b) { d.v = fma(a, b, d.v); }
__device__ __forceinline__ float dot_value(const Dot<float>& d) { return d.v; }
__device__ __forceinline__ double dot_value(const Dot<double>& d) { return d.v; }

__device__ __forceinline__ Dot<ff64> dot_first(ff64 a, ff64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return Dot<ff64>{p, e};
}
__device__ __forceinline__ void dot_fma(Dot<ff64>& d, ff64 a, ff64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(d.s, p);                       // two-sum of d.s + p
  const float bb = __fsub_rn(s, d.s);
  const float err = __fadd_rn(__fsub_rn(d.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  d.s = s;
  d.c = __fadd_rn(__fadd_rn(d.c, e), err);
}
__device__ __forceinline__ ff64 dot_value(const Dot<ff64>& d) {
  const float hi = __fadd_rn(d.s, d.c);
  return ff64{hi, __fsub_rn(d.c, __fsub_rn(hi, d.s))};
}

// (a + b) and (a - b) for inputs of the compensated dot products: for float-float
// the two-sum of the high parts with the low parts added to its error, left
// unnormalised (the products of the dot product split both parts exactly or carry
// their rounding into the error sum, so the absolute error stays 2^-48 |a|, |b|).
__device__ __forceinline__ float vadd_loose(float a, float b) { return a + b; }
__device__ __forceinline__ double vadd_loose(double a, double b) { return a + b; }
__device__ __forceinline__ ff64 vadd_loose(ff64 a, ff64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return ff64{s, __fadd_rn(__fadd_rn(a.lo, b.lo), err)};
}
__device__ __forceinline__ float vsub_loose(float a, float b) { return a - b; }
__device__ __forceinline__ double vsub_loose(double a, double b) { return a - b; }
__device__ __forceinline__ ff64 vsub_loose(ff64 a, ff64 b) { return vadd_loose(a, ff64{-b.hi, -b.lo}); }

// value of the sum (NEG = false) or difference (NEG = true) of two dot-product
// accumulators: one two-sum of the running sums, the error sums added, one
// renormalisation
template <bool NEG>
__device__ __forceinline__ float dot_merge(const Dot<float>& a, const Dot<float>& b) {
  return NEG ? a.v - b.v : a.v + b.v;
}
template <bool NEG>
__device__ __forceinline__ double dot_merge(const Dot<double>& a, const Dot<double>& b) {
  return NEG ? a.v - b.v : a.v + b.v;
}
template <bool NEG>
__device__ __forceinline__ ff64 dot_merge(const Dot<ff64>& a, const Dot<ff64>& b) {
  const float bs = NEG ? -b.s : b.s, bc = NEG ? -b.c : b.c;
  const float s = __fadd_rn(a.s, bs);
  const float bb = __fsub_rn(s, a.s);
  const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(bs, bb));
  const float c = __fadd_rn(__fadd_rn(a.c, bc), err);
  const float hi = __fadd_rn(s, c);
  return ff64{hi, __fsub_rn(c, __fsub_rn(hi, s))};
}

template <typename V> __device__ __forceinline__ Sum<V> sum_zero() { return Sum<V>{vzero<V>()}; }
template <> __device__ __forceinline__ Sum<ff64> sum_zero<ff64>() { return Sum<ff64>{0.f, 0.f}; }
__device__ __forceinline__ void sum_add(Sum<float>& d, float v) { d.v += v; }
__device__ __forceinline__ void sum_add(Sum<double>& d, double v) { d.v += v; }
__device__ __forceinline__ void sum_add(Sum<ff64>& d, ff64 v) {
  const float s = __fadd_rn(d.s, v.hi);                    // two-sum of d.s + v.hi
  const float bb = __fsub_rn(s, d.s);
  const float err = __fadd_rn(__fsub_rn(d.s, __fsub_rn(s, bb)), __fsub_rn(v.hi, bb));
  d.s = s;
  d.c = __fadd_rn(__fadd_rn(d.c, v.lo), err);
}

// a sum holding exactly v (what sum_add of v to a zero sum gives, without the add)
__device__ __forceinline__ void sum_set(Sum<float>& d, float v) { d.v = v; }
__device__ __forceinline__ void sum_set(Sum<double>& d, double v) { d.v = v; }
__device__ __forceinline__ void sum_set(Sum<ff64>& d, ff64 v) { d.s = v.hi; d.c = v.lo; }

// d += o for two partial sums (the same compensated scheme for float-float)
__device__ __forceinline__ void sum_merge(Sum<float>& d, const Sum<float>& o) { d.v += o.v; }
__device__ __forceinline__ void sum_merge(Sum<double>& d, const Sum<double>& o) { d.v += o.v; }
__device__ __forceinline__ void sum_merge(Sum<ff64>& d, const Sum<ff64>& o) {
  const float s = __fadd_rn(d.s, o.s);                     // two-sum of d.s + o.s
  const float bb = __fsub_rn(s, d.s);
  const float err = __fadd_rn(__fsub_rn(d.s, __fsub_rn(s, bb)), __fsub_rn(o.s, bb));
  d.s = s;
  d.c = __fadd_rn(__fadd_rn(d.c, o.c), err);
}

// ------------------------------------------------ solver inner products --
// IoDot<T> accumulates an inner product of two solver vectors of element type T.
// FP64 vectors use FP64 fused multiply-adds.  FP32 vectors use the compensated
// dot product above on the exact products of float pairs (product p and its
// rounding error fma(a, b, -p)), so that no FP64 instruction runs per element
// (GB300 issues 2 FP64 FMAs per clock per SM against 128 FP32); value() converts
// the (sum, error) pair to double once.
template <typename T>
struct IoDot;
// merge() adds another partial sum (same scheme), shfl_down() reads lane + o's.
template <>
struct IoDot<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ void merge(const IoDot& o) { v += o.v; }
  __device__ __forceinline__ IoDot shfl_down(int o) const {
    IoDot r;
    r.v = __shfl_down_sync(0xffffffffu, v, o);
    return r;
  }
  __device__ __forceinline__ double value() const { return v; }
};
template <>
struct IoDot<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(s, p);                       // two-sum of s + p
    const float bb = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s = t;
    c = __fadd_rn(__fadd_rn(c, e), err);
  }
  __device__ __forceinline__ void merge(const IoDot& o) {
    const float t = __fadd_rn(s, o.s);                     // two-sum of s + o.s
    const float bb = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(o.s, bb));
    s = t;
    c = __fadd_rn(__fadd_rn(c, o.c), err);
  }
  __device__ __forceinline__ IoDot shfl_down(int o) const {
    IoDot r;
    r.s = __shfl_down_sync(0xffffffffu, s, o);
    r.c = __shfl_down_sync(0xffffffffu, c, o);
    return r;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// --------------------------------------------------------- memory <-> V --
__device__ __forceinline__ float from_io(float x, float*) { return x; }
__device__ __forceinline__ double from_io(double x, double*) { return x; }

// Exact-to-2^-47 split of a double into hi + lo floats with integer operations only
// (no FP64 or conversion-unit work): hi is x truncated to 24 significant bits, lo
// the remainder rounded to 24 bits.  |x| below 2^-126 reads as 0; |x| at or above
// 2^128 reads as +-inf.  Inputs of the ff form are expected in that range.
__device__ __forceinline__ ff64 from_io(double x, ff64*) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff);
  const unsigned sign = (unsigned)(bits >> 63) << 31;
  if (e < 897) return ff64{__int_as_float((int)sign), 0.f};
  if (e > 1150) return ff64{__int_as_float((int)(sign | 0x7f800000u)), 0.f};
  const unsigned long long mant = bits & 0xfffffffffffffull;
  const float hi = __int_as_float((int)(sign | ((unsigned)(e - 896) << 23) | (unsigned)(mant >> 29)));
  const unsigned rem = (unsigned)(mant & 0x1fffffffu);
  float lo = 0.f;
  if (rem != 0u && e >= 926) {
    // rem * 2^(e - 1075) = (rem * 2^-29) * 2^(e - 1046), both factors exact powers of two
    const float r = __fmul_rn(__uint2float_rn(rem), 1.862645149230957e-09f);  // 2^-29
    lo = __fmul_rn(r, __int_as_float((e - 1046 + 127) << 23));
    lo = __int_as_float(__float_as_int(lo) | (int)sign);
  }
  return ff64{hi, lo};
}

__device__ __forceinline__ float to_io(float v, float*) { return v; }
__device__ __forceinline__ double to_io(double v, double*) { return v; }
// float -> double by rebiasing the exponent field (IEEE 754 binary32 -> binary64), so
// that the conversion takes integer operations instead of the FP64 pipe; subnormal
// floats (below 2^-126) read as signed zero.
__device__ __forceinline__ double widen_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  unsigned long long d = (unsigned long long)(u & 0x80000000u) << 32;
  if (e != 0u) {
    const unsigned long long ed = (e == 0xffu) ? 0x7ffull : (unsigned long long)(e + 896u);
    d |= (ed << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  }
  return __longlong_as_double((long long)d);
}
__device__ __forceinline__ double to_io(ff64 v, double*) { return widen_bits(v.hi) + widen_bits(v.lo); }

// ---------------------------------------------------------- host consts --
template <typename V> inline V from_host(double x);
template <> inline float from_host<float>(double x) { return (float)x; }
template <> inline double from_host<double>(double x) { return x; }
template <> inline ff64 from_host<ff64>(double x) {
  const float hi = (float)x;
  return ff64{hi, (float)(x - (double)hi)};
}

}  // namespace gp
