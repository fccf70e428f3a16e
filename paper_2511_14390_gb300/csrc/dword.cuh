// Double-word ("float-float") arithmetic on the FP32 pipes: a value is hi + lo with
// |lo| <= ulp(hi)/2, about 44 significant bits.  Built from two error-free
// transformations: Knuth's TwoSum (a + b = s + e exactly) and the FMA-based
// TwoProduct (a * b = p + e exactly, e = fma(a, b, -p)); the combination rules are
// the usual double-word sum and product (cf. Joldes, Muller, Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic", 2017).
// Used where GB300's narrow FP64 pipe would otherwise serialise the work: the
// per-channel setup of the low-order tables and the serial high-order chunk-state scan.
#pragma once

namespace dfilt {

struct dw {
    float hi, lo;
};

__device__ __forceinline__ dw dw_make(float x) { return {x, 0.f}; }

// s + e == a + b exactly (any ordering of |a|, |b|)
__device__ __forceinline__ dw two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// s + e == a + b exactly when |a| >= |b|
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dw operator+(dw a, dw b) {
    dw s = two_sum(a.hi, b.hi);
    const dw t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dw operator-(dw a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dw operator-(dw a, dw b) { return a + (-b); }
__device__ __forceinline__ dw operator*(dw a, dw b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ float dw_to_float(dw a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ double dw_to_double(dw a) { return (double)a.hi + (double)a.lo; }

}  // namespace dfilt
