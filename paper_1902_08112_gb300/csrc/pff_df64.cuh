// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two floats
// (|lo| <= ulp(hi)/2), carrying about 48 significant bits.  Built from the error-free
// transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971) and TwoProduct
// via fused multiply-add; the add is the "sloppy" double-double add of Hida, Li and Bailey
// (QD library, 2001).  Every operation uses round-to-nearest intrinsics so the compiler cannot
// contract or reassociate them.
//
// On GB300 FP64 issues at a small fraction of the FP32 rate, so the FP64-accurate operators of
// this library run their arithmetic in df64 on the FP32 pipes.
#pragma once

#include <cuda_runtime.h>

namespace pff {

struct df64 {
    float hi, lo;
};

__device__ __forceinline__ df64 df_make(float h, float l) { df64 r; r.hi = h; r.lo = l; return r; }

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df_make(s, e);
}

__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {   // requires |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// The pairs are kept unnormalised: the high parts combine exactly (TwoSum, TwoProduct) and the low
// parts accumulate in plain FP32, without the FastTwoSum renormalisation after each operation.
// The applies are chains of linear stages whose low parts stay ~2^-24 of the magnitudes involved,
// so each operation still carries a relative error of order 2^-48 of its operands.
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    const df64 s = df_two_sum(a.hi, b.hi);
    return df_make(s.hi, __fadd_rn(__fadd_rn(a.lo, b.lo), s.lo));
}
__device__ __forceinline__ df64 operator-(df64 a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_make(p, __fmaf_rn(a.hi, b.lo, e));
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { a = a + b; return a; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { a = a - b; return a; }

// Conversions without FP64 instructions (on GB300 conversions to and from FP64 issue on the slow
// FP64 unit).  They work on the IEEE-754 fields: a double (1.m) 2^(e-1023) with a 52-bit m splits
// into hi = the double with m truncated to its top 23 bits and lo = the remaining 29 bits of m
// times 2^(e-1075), rounded to a float (48 significant bits in total).  Magnitudes below 2^-126
// become 0; below 2^-104 the lo part is dropped.  Inf and NaN map to Inf and NaN.
__device__ __forceinline__ df64 df_from_double(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return df_make(__uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u)), 0.f);
    const int fe = e - 1023 + 127;               // biased float exponent
    if (fe <= 0) return df_make(0.f, 0.f);
    if (fe >= 255) return df_make(__uint_as_float(sign | 0x7F800000u), 0.f);
    const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)(m >> 29));
    const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);
    const int se = fe - 23;                      // biased exponent of 2^(e - 1046)
    float lo = 0.f;
    if (se > 0 && rem) lo = __fmul_rn(__fmul_rn(__uint2float_rn(rem), 0x1.0p-29f), __uint_as_float((unsigned)se << 23));
    return df_make(hi, sign ? -lo : lo);
}
// double -> df64 with the conversion instructions (which issue on the FP64 pipe): hi = the nearest
// float, lo = the nearest float to the remainder.  Used where few values are converted per thread, so
// that the FP64 pipe (otherwise idle in the df64 kernels) takes the work off the FP32/integer pipes.
__device__ __forceinline__ df64 df_from_double_cvt(double d) {
    const float hi = __double2float_rn(d);
    return df_make(hi, __double2float_rn(d - (double)hi));
}
template <typename S>
__device__ __forceinline__ S load_cvt(double d);
// exact float -> double by field arithmetic (subnormal floats become 0)
__device__ __forceinline__ double f32_to_f64_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const int e = (int)((u >> 23) & 0xFF);
    const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
    if (e == 0) return __longlong_as_double((long long)sign);
    if (e == 0xFF) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull | m));
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896) << 52) | m));
}
// hi + lo rounded to a double: one FP64 addition
__device__ __forceinline__ double df_to_double(df64 a) { return f32_to_f64_bits(a.hi) + f32_to_f64_bits(a.lo); }

// ---- scalar traits so kernels can be written once for float and df64
template <typename S>
struct Scalar;

template <>
struct Scalar<float> {
    using storage = float;      // element type of vectors in global memory
    __device__ static __forceinline__ float load(float v) { return v; }
    __device__ static __forceinline__ float from_double(double v) { return (float)v; }
    __device__ static __forceinline__ float store(float v) { return v; }
    __device__ static __forceinline__ float zero() { return 0.f; }
};

template <> __device__ __forceinline__ float load_cvt<float>(double d) { return (float)d; }
template <> __device__ __forceinline__ df64 load_cvt<df64>(double d) { return df_from_double_cvt(d); }

template <>
struct Scalar<df64> {
    using storage = double;
    __device__ static __forceinline__ df64 load(double v) { return df_from_double(v); }
    __device__ static __forceinline__ df64 from_double(double v) { return df_from_double(v); }
    __device__ static __forceinline__ double store(df64 v) { return df_to_double(v); }
    __device__ static __forceinline__ df64 zero() { return df_make(0.f, 0.f); }
};

}  // namespace pff
