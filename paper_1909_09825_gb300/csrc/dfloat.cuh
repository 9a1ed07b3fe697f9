// Double-float arithmetic: a value is hi + lo, two floats with |lo| <= ulp(hi)/2, about
// 48 significant bits.  Sums and products use the error-free transformations of Knuth
// (two-sum) and Dekker (two-product through an FMA), followed by renormalisation
// (fast two-sum).  Every operation is written with the _rn intrinsics so that the
// compiler cannot contract or reassociate the error terms away.
//
// On GB300 one FP64 FMA takes the issue slot of 62 FP32 FMAs; a double-float
// multiply-add costs about 15 FP32 operations, so the FP64-accurate recurrences run
// several times faster in this form.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fgt1d {

// keep the float/double overloads visible next to the dfloat one below
using ::fma;

struct dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h) : hi(h), lo(0.f) {}
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ dfloat df_make(float hi, float lo) { return dfloat(hi, lo); }

// s = a + b exactly as s + e
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// renormalise (s, e) with |e| small relative to s
__device__ __forceinline__ dfloat fast_two_sum(float s, float e) {
    const float hi = __fadd_rn(s, e);
    return df_make(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s, e);
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    float s, e;
    two_sum(p, c.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(pe, c.lo));
    return fast_two_sum(s, e);
}

// a * b + c left unnormalised (hi + lo with |lo| up to a few ulp(hi)): an operand for
// the next fma or +, which renormalise
__device__ __forceinline__ dfloat fma_nr(dfloat a, dfloat b, dfloat c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    float s, e;
    two_sum(p, c.hi, s, e);
    return df_make(s, __fadd_rn(e, __fadd_rn(pe, c.lo)));
}
// a * b left unnormalised
__device__ __forceinline__ dfloat mul_nr(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    return df_make(p, pe);
}

__device__ __forceinline__ bool operator==(dfloat a, dfloat b) { return a.hi == b.hi && a.lo == b.lo; }

__device__ __forceinline__ dfloat df_shfl_up(dfloat v, int o) {
    return df_make(__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ dfloat df_shfl_down(dfloat v, int o) {
    return df_make(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}

}  // namespace fgt1d
