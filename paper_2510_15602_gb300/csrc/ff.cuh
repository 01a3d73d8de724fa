// ff.cuh -- float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits.  The
// building blocks are the error-free transformations TwoSum (Knuth),
// FastTwoSum (Dekker) and TwoProd via FMA; every operation uses explicitly
// rounded intrinsics so the compiler cannot re-associate or contract them.
// Used where GB300's FP64 pipe (a few DFMA per clock per SM) would be the
// bottleneck and FP32 (128 lanes per clock per SM) is not accurate enough.
#pragma once

#include <cuda_runtime.h>

namespace qfca {
namespace ffa {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff make(float hi, float lo) { return ff{hi, lo}; }
__device__ __forceinline__ ff zero() { return ff{0.0f, 0.0f}; }

// s + e == a + b exactly
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff{s, e};
}

__device__ __forceinline__ ff add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    const float t = __fadd_rn(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t);
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff sub(ff a, ff b) { return add(a, neg(b)); }

__device__ __forceinline__ ff mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return ff{p, __fmaf_rn(a, b, -p)};
}

// a / b (one correction step: ~47 bits)
__device__ __forceinline__ ff div(ff a, ff b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const ff r = sub(a, mul(ff{q1, 0.0f}, b));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}

// sqrt(a) for a >= 0 (one Newton correction)
__device__ __forceinline__ ff sqrt(ff a) {
    if (!(a.hi > 0.0f)) return ff{0.0f, 0.0f};
    const float s = sqrtf(a.hi);
    const ff e = sub(a, two_prod(s, s));
    return fast_two_sum(s, __fdiv_rn(e.hi, __fmul_rn(2.0f, s)));
}

// The same two operations from the hardware's approximate reciprocal and
// reciprocal square root (PTX rcp.approx / rsqrt.approx, about 2^-23
// relative) refined by two Newton corrections in float-float (each squares the
// relative error, down to float-float rounding).  Shorter dependency chains than
// the correctly rounded FP32 divide and square root, for scalar chains on the
// critical path.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ ff div_newton(ff a, ff b) {
    const float y = rcp_approx(b.hi);
    const float q1 = __fmul_rn(a.hi, y);
    const ff r1 = sub(a, mul(ff{q1, 0.0f}, b));
    const ff q = fast_two_sum(q1, __fmul_rn(r1.hi, y));
    const ff r2 = sub(a, mul(q, b));
    return add(q, ff{__fmul_rn(r2.hi, y), 0.0f});
}
__device__ __forceinline__ ff sqrt_newton(ff a) {
    if (!(a.hi > 0.0f)) return ff{0.0f, 0.0f};
    const float hy = __fmul_rn(0.5f, rsqrt_approx(a.hi));  // 1 / (2 sqrt(a))
    const float s0 = __fmul_rn(a.hi, __fmul_rn(2.0f, hy));
    const ff s1 = fast_two_sum(s0, __fmul_rn(sub(a, two_prod(s0, s0)).hi, hy));
    return add(s1, ff{__fmul_rn(sub(a, mul(s1, s1)).hi, hy), 0.0f});
}

__device__ __forceinline__ ff scale(ff a, float p2) { return ff{__fmul_rn(a.hi, p2), __fmul_rn(a.lo, p2)}; }
__device__ __forceinline__ bool less(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ ff fabs_ff(ff a) { return a.hi < 0.0f ? ff{-a.hi, -a.lo} : a; }

// Compensated dot-product accumulator: s carries the running sum of the
// leading products, c the (small) compensation.
struct acc {
    float s, c;
};
__device__ __forceinline__ acc acc_zero() { return acc{0.0f, 0.0f}; }
__device__ __forceinline__ void acc_fma(acc &A, ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const ff t = two_sum(A.s, p);
    A.s = t.hi;
    A.c = __fadd_rn(A.c, __fadd_rn(t.lo, e));
}
__device__ __forceinline__ void acc_add(acc &A, ff a) {
    const ff t = two_sum(A.s, a.hi);
    A.s = t.hi;
    A.c = __fadd_rn(A.c, __fadd_rn(t.lo, a.lo));
}
__device__ __forceinline__ void acc_merge(acc &A, acc B) {
    const ff t = two_sum(A.s, B.s);
    A.s = t.hi;
    A.c = __fadd_rn(A.c, __fadd_rn(t.lo, B.c));
}
__device__ __forceinline__ ff acc_value(acc A) { return two_sum(A.s, A.c); }

__device__ __forceinline__ acc warp_sum(acc A) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc B;
        B.s = __shfl_xor_sync(0xffffffffu, A.s, o);
        B.c = __shfl_xor_sync(0xffffffffu, A.c, o);
        acc_merge(A, B);
    }
    return A;
}

// conversions (FP64 only at the edges)
__device__ __forceinline__ ff from_double(double x) {
    const float h = (float)x;
    return ff{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double to_double(ff a) { return (double)a.hi + (double)a.lo; }

}  // namespace ffa
}  // namespace qfca
