// Two-float ("double-float") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2,
// carried in two FP32 registers.  The error-free transformations are Knuth's
// TwoSum and the FMA form of Dekker's TwoProd; every operation uses the _rn
// intrinsics so the compiler cannot contract or reassociate them.  The
// precision form of the sweeps uses these to keep FP32 storage and FP32 issue
// rate while its sums carry about 48 significant bits.
#pragma once

#include <cuda_runtime.h>

namespace esim {

struct f2 {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ f2 fast_renorm(float s, float e) {  // |s| >= |e|
    const float h = __fadd_rn(s, e);
    return f2{h, __fsub_rn(e, __fsub_rn(h, s))};
}

// a + x for a two-float a and a float x
__device__ __forceinline__ f2 f2_add_f(f2 a, float x) {
    float s, e;
    two_sum(a.hi, x, s, e);
    return fast_renorm(s, __fadd_rn(e, a.lo));
}

// a + b for two-floats
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return fast_renorm(s, e);
}

// a * b for a two-float a and a two-float b (products of lo parts dropped)
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fadd_rn(e, __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi)));
    return fast_renorm(p, e);
}

// a * x for a two-float a and a float x
__device__ __forceinline__ f2 f2_mul_f(f2 a, float x) {
    const float p = __fmul_rn(a.hi, x);
    float e = __fmaf_rn(a.hi, x, -p);
    e = __fadd_rn(e, __fmul_rn(a.lo, x));
    return fast_renorm(p, e);
}

// a / d for a two-float a and a positive float d (exact remainder by FMA)
__device__ __forceinline__ f2 f2_div_f(f2 a, float d) {
    const float q = __fdiv_rn(a.hi, d);
    const float r = __fadd_rn(__fmaf_rn(-q, d, a.hi), a.lo);
    return fast_renorm(q, __fdiv_rn(r, d));
}

// a / b for two-floats, b > 0: q1 = a.hi / b.hi, the remainder a - q1 b formed with FMA
// (exact for the hi product), and one correction q2 = remainder / b.hi; a / a gives 1
// exactly.
__device__ __forceinline__ f2 f2_div(f2 a, f2 b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const float p = __fmul_rn(q1, b.hi);
    const float pe = __fmaf_rn(q1, b.hi, -p);
    float r = __fsub_rn(__fsub_rn(a.hi, p), pe);
    r = __fadd_rn(r, a.lo);
    r = __fmaf_rn(-q1, b.lo, r);
    return fast_renorm(q1, __fdiv_rn(r, b.hi));
}

__device__ __forceinline__ f2 f2_from_double(double v) {
    const float h = __double2float_rn(v);
    return f2{h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double f2_to_double(f2 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ f2 f2_shfl_down(f2 a, int offset, int width) {
    return f2{__shfl_down_sync(0xffffffffu, a.hi, offset, width), __shfl_down_sync(0xffffffffu, a.lo, offset, width)};
}

}  // namespace esim
