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
__device__ __forceinline__ double to_io(ff64 v, double*) { return (double)v.hi + (double)v.lo; }

// ---------------------------------------------------------- host consts --
template <typename V> inline V from_host(double x);
template <> inline float from_host<float>(double x) { return (float)x; }
template <> inline double from_host<double>(double x) { return x; }
template <> inline ff64 from_host<ff64>(double x) {
  const float hi = (float)x;
  return ff64{hi, (float)(x - (double)hi)};
}

}  // namespace gp
