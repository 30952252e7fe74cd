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
// never contracts or reorders them.  The arithmetic and the bit-level conversions below
// also compile for the host (IEEE binary32 and binary64 with round-to-nearest; host
// builds must not contract a*b+c, e.g. gcc's -ffp-contract=off), where a test checks
// them against exact rational arithmetic.
#pragma once

#include <cuda_runtime.h>
#ifndef __CUDA_ARCH__
#include <cmath>
#include <cstdint>
#include <cstring>
#endif

namespace elas {

// correctly rounded FP32 operations (round to nearest even), and bit reinterpretations
__host__ __device__ __forceinline__ float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
__host__ __device__ __forceinline__ float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
__host__ __device__ __forceinline__ float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
__host__ __device__ __forceinline__ float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}
__host__ __device__ __forceinline__ float u2f(unsigned b) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float x;
    std::memcpy(&x, &b, 4);
    return x;
#endif
}
__host__ __device__ __forceinline__ unsigned f2u(float x) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    unsigned b;
    std::memcpy(&b, &x, 4);
    return b;
#endif
}
__host__ __device__ __forceinline__ unsigned d_hi(double v) {
#ifdef __CUDA_ARCH__
    return (unsigned)__double2hiint(v);
#else
    std::uint64_t b;
    std::memcpy(&b, &v, 8);
    return (unsigned)(b >> 32);
#endif
}
__host__ __device__ __forceinline__ unsigned d_lo(double v) {
#ifdef __CUDA_ARCH__
    return (unsigned)__double2loint(v);
#else
    std::uint64_t b;
    std::memcpy(&b, &v, 8);
    return (unsigned)b;
#endif
}
__host__ __device__ __forceinline__ double d_from(unsigned hi, unsigned lo) {
#ifdef __CUDA_ARCH__
    return __hiloint2double((int)hi, (int)lo);
#else
    const std::uint64_t b = ((std::uint64_t)hi << 32) | lo;
    double v;
    std::memcpy(&v, &b, 8);
    return v;
#endif
}
// the high word of (hi:lo) << 3
__host__ __device__ __forceinline__ unsigned shl3_hi(unsigned lo, unsigned hi) {
#ifdef __CUDA_ARCH__
    return __funnelshift_l(lo, hi, 3);
#else
    return (hi << 3) | (lo >> 29);
#endif
}

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
__host__ __device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = f_add(a, b);
    const float bb = f_sub(s, a);
    const float e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
    return dfloat(s, e);
}

// the same when |a| >= |b| or a == 0 (Dekker's Fast2Sum, 3 operations)
__host__ __device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    const float s = f_add(a, b);
    return dfloat(s, f_sub(b, f_sub(s, a)));
}

__host__ __device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
    const dfloat s = df_two_sum(x.hi, y.hi);
    return dfloat(s.hi, f_add(s.lo, f_add(x.lo, y.lo)));
}

__host__ __device__ __forceinline__ dfloat df_neg(dfloat x) { return dfloat(-x.hi, -x.lo); }

__host__ __device__ __forceinline__ dfloat df_sub(dfloat x, dfloat y) { return df_add(x, df_neg(y)); }

// x * y: the exact product of the high parts by one FMA, plus the cross terms
__host__ __device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y) {
    const float p = f_mul(x.hi, y.hi);
    float e = f_fma(x.hi, y.hi, -p);
    e = f_fma(x.hi, y.lo, e);
    e = f_fma(x.lo, y.hi, e);
    return dfloat(p, e);
}

// x * y for an FP32 y
__host__ __device__ __forceinline__ dfloat df_mul(dfloat x, float y) {
    const float p = f_mul(x.hi, y);
    float e = f_fma(x.hi, y, -p);
    e = f_fma(x.lo, y, e);
    return dfloat(p, e);
}

// a * b + c: the product's pair added to c as one sum
__host__ __device__ __forceinline__ dfloat df_fma(dfloat a, dfloat b, dfloat c) {
    const float p = f_mul(a.hi, b.hi);
    float e = f_fma(a.hi, b.hi, -p);
    e = f_fma(a.hi, b.lo, e);
    e = f_fma(a.lo, b.hi, e);
    const dfloat s = df_two_sum(p, c.hi);
    return dfloat(s.hi, f_add(s.lo, f_add(e, c.lo)));
}

// nearest FP32 value (hi + lo rounded once)
__host__ __device__ __forceinline__ float df_to_float(dfloat x) { return f_add(x.hi, x.lo); }

// A double as a double-float pair from its bits alone (no FP64 or conversion instruction:
// on this GPU those share the narrow FP64 pipe).  IEEE-754 binary64 v = (-1)^s 1.m 2^(e-1023)
// with a 52-bit m: hi keeps the leading 24 significant bits (truncated), re-biased to the
// binary32 exponent e - 896; lo is the rest, the next 23 bits below hi's last one, formed
// as (1.f - 1) 2^(e-896-127-23) by one exact FP32 subtraction.  |v - (hi + lo)| < 2^-46 |v|.
// |v| below 2^-103 keeps lo = 0 and below 2^-126 gives (0, 0): far under any value of the
// fields split here (moduli, displacements, loads).  |v| >= 2^128 (beyond FP32) is out of
// range.
__host__ __device__ __forceinline__ dfloat df_split(double v) {
    const unsigned h32 = d_hi(v), l32 = d_lo(v);
    const int e = (int)((h32 >> 20) & 0x7ffu);
    if (e < 897) return dfloat(0.f, 0.f);
    const unsigned hb = (shl3_hi(l32, h32) - 0xC0000000u) | (h32 & 0x80000000u);
    float lo = 0.f;
    if (e >= 920) {
        const unsigned base = (hb & 0x7f800000u) - (23u << 23);
        const float one = u2f(base);
        const float lf = u2f(base | ((l32 >> 6) & 0x7fffffu));
        lo = f_sub(lf, one);
        if (h32 & 0x80000000u) lo = -lo;
    }
    return dfloat(u2f(hb), lo);
}

// An FP32 value as a double from its bits (exact; FP32 subnormals, far below any
// correction, read as zero), without a conversion instruction.
__host__ __device__ __forceinline__ double f2d_bits(float x) {
    const unsigned b = f2u(x);
    const unsigned ex = (b >> 23) & 0xffu;
    if (ex == 0) return 0.0;
    const unsigned hi = (b & 0x80000000u) | ((ex + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return d_from(hi, b << 29);
}

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
