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

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    const df64 s = df_two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { a = a + b; return a; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { a = a - b; return a; }

// exact split of a double into hi + lo (one FP64 subtraction)
__device__ __forceinline__ df64 df_from_double(double d) {
    const float h = __double2float_rn(d);
    return df_make(h, __double2float_rn(d - (double)h));
}
__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

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

template <>
struct Scalar<df64> {
    using storage = double;
    __device__ static __forceinline__ df64 load(double v) { return df_from_double(v); }
    __device__ static __forceinline__ df64 from_double(double v) { return df_from_double(v); }
    __device__ static __forceinline__ double store(df64 v) { return df_to_double(v); }
    __device__ static __forceinline__ df64 zero() { return df_make(0.f, 0.f); }
};

}  // namespace pff
