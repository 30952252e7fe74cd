// Double-float ("double-word") numbers: an unevaluated sum hi + lo of two FP32 values,
// about 48 significant bits.
//
// GB300's FP64 pipes run at about 1/70 of its FP32 rate (1.06 against 76.8 TFLOP/s
// measured with independent FMA chains), so the refinement residual of a mixed solve,
// the one operator application that needs more than FP32 accuracy, is evaluated in
// this format on the FP32 pipes: an addition costs 8 FP32 operations, a product 4, a
// multiply-add 12.  The building blocks are the error-free transformations of Knuth
// (TwoSum) and Dekker (Fast2Sum, and the FMA form of the exact product), combined as
// the double-word algorithms analysed by Joldes, Muller and Popescu (ACM TOMS 44,
// 2017): the "sloppy" sum of two double-words and the product through one FMA chain,
// here without the final renormalisation (Fast2Sum) of each result.  A pair then need
// not satisfy |lo| <= ulp(hi) / 2, but its lo part stays within a few 2^-24 of the
// magnitudes of the operands it came from, so every later rounding of a lo term is a
// few 2^-47 of those magnitudes.  That is the error bound of the whole evaluation: a
// few units of 2^-47 of the operands' magnitudes (not of the result's), exactly what a
// residual needs, whose terms cancel to a small sum.
//
// Every operation spells out its roundings with the _rn intrinsics, so the compiler
// never contracts or reorders them.
#pragma once

#include <cuda_runtime.h>

namespace elas {

struct __align__(8) dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dfloat(int v) : hi((float)v), lo(0.f) {}   // exact for |v| < 2^24
    __host__ __device__ constexpr dfloat(float v) : hi(v), lo(0.f) {}
    // split of a double (constants: folded at compile time; the kernels never convert
    // run-time doubles this way)
    __host__ __device__ constexpr dfloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

// s + e = a + b exactly, s = fl(a + b)  (Knuth's TwoSum, 6 operations)
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfloat(s, e);
}

// the same when |a| >= |b| or a == 0 (Dekker's Fast2Sum, 3 operations)
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
    const dfloat s = df_two_sum(x.hi, y.hi);
    return dfloat(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ dfloat df_neg(dfloat x) { return dfloat(-x.hi, -x.lo); }

__device__ __forceinline__ dfloat df_sub(dfloat x, dfloat y) { return df_add(x, df_neg(y)); }

// x * y: the exact product of the high parts by one FMA, plus the cross terms
__device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return dfloat(p, e);
}

// x * y for an FP32 y
__device__ __forceinline__ dfloat df_mul(dfloat x, float y) {
    const float p = __fmul_rn(x.hi, y);
    float e = __fmaf_rn(x.hi, y, -p);
    e = __fmaf_rn(x.lo, y, e);
    return dfloat(p, e);
}

// a * b + c: the product's pair added to c as one sum
__device__ __forceinline__ dfloat df_fma(dfloat a, dfloat b, dfloat c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const dfloat s = df_two_sum(p, c.hi);
    return dfloat(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// nearest FP32 value (hi + lo rounded once)
__device__ __forceinline__ float df_to_float(dfloat x) { return __fadd_rn(x.hi, x.lo); }

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) { return df_add(a, b); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return df_sub(a, b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) { return df_mul(a, b); }
__device__ __forceinline__ dfloat operator-(dfloat a) { return df_neg(a); }
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = df_add(a, b); }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = df_sub(a, b); }

// all-lane butterfly exchange of the warp
__device__ __forceinline__ float shfl_xor_all(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor_all(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dfloat shfl_xor_all(dfloat v, int o) {
    return dfloat(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

}  // namespace elas
