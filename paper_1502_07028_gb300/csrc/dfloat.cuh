// dfloat.cuh -- double-float ("double-word") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  On this GPU the FP32 pipe runs 58 times faster
// than the FP64 pipe, so an operation of 10-30 FP32 instructions still beats
// one FP64 instruction several times over.  The building blocks are the
// error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2), Fast2Sum
// (Dekker 1971) and the FMA-based TwoProd; addition, multiplication, division
// and square root follow the double-word algorithms analysed by Joldes,
// Muller and Popescu ("Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic", ACM TOMS 44(2), 2017): relative errors
// of a few u^2, u = 2^-24.  The complex multiply-adds that dominate a
// Householder pass are written as sums of two products with a single
// renormalisation.
#pragma once

#include "device_common.cuh"

namespace ptca {

struct __align__(8) dfl {
    float hi, lo;
    dfl() = default;
    __device__ __forceinline__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // Nearest double-float to x (exact for every double within the float range
    // up to the 48-bit significand).
    __device__ __forceinline__ explicit dfl(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __device__ __forceinline__ explicit dfl(int x) : dfl((double)x) {}
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth's TwoSum, 6 flops).
__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfl(s, e);
}
// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker's Fast2Sum, 3 flops).
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// x + y (the accurate double-word sum: relative error <= 3u^2).
__device__ __forceinline__ dfl operator+(dfl x, dfl y) {
    const dfl s = two_sum(x.hi, y.hi);
    const dfl t = two_sum(x.lo, y.lo);
    const dfl v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ dfl operator-(dfl x) { return dfl(-x.hi, -x.lo); }
__device__ __forceinline__ dfl operator-(dfl x, dfl y) { return x + (-y); }
// x * y (double-word product with FMA: relative error <= 5u^2).
__device__ __forceinline__ dfl operator*(dfl x, dfl y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}
// x / y: quotient of the leading parts, one correction from the double-word
// remainder x - q y (relative error a few u^2).
__device__ __forceinline__ dfl operator/(dfl x, dfl y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const dfl r = x - dfl(q1, 0.f) * y;
    const float q2 = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(q1, q2);
}
__device__ __forceinline__ dfl& operator+=(dfl& x, dfl y) { x = x + y; return x; }
__device__ __forceinline__ dfl& operator*=(dfl& x, dfl y) { x = x * y; return x; }
__device__ __forceinline__ bool operator>(dfl x, dfl y) { return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo); }
__device__ __forceinline__ bool operator<(dfl x, dfl y) { return y > x; }

// sqrt(x): the float square root of the leading part and one Newton
// correction (x - s^2) / (2 s) from the double-word residual.
__device__ __forceinline__ dfl sqroot(dfl x) {
    if (!(x.hi > 0.f)) return dfl(0.f, 0.f);
    const float s = __fsqrt_rn(x.hi);
    const float p = __fmul_rn(s, s);
    const float pe = __fmaf_rn(s, s, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo);
    return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}

// acc + a1 b1 + a2 b2 with one renormalisation: the leading products and
// their rounding errors (TwoProd), the exact sum of the leading parts
// (TwoSum), and every lower-order term accumulated in float.
__device__ __forceinline__ dfl dot2_acc(dfl acc, dfl a1, dfl b1, dfl a2, dfl b2) {
    const float p1 = __fmul_rn(a1.hi, b1.hi);
    const float p2 = __fmul_rn(a2.hi, b2.hi);
    float lo = __fadd_rn(__fmaf_rn(a1.hi, b1.hi, -p1), __fmaf_rn(a2.hi, b2.hi, -p2));
    const dfl s = two_sum(acc.hi, p1);
    const dfl t = two_sum(s.hi, p2);
    lo = __fadd_rn(lo, acc.lo);
    lo = __fadd_rn(lo, s.lo);
    lo = __fadd_rn(lo, t.lo);
    lo = __fmaf_rn(a1.hi, b1.lo, lo);
    lo = __fmaf_rn(a1.lo, b1.hi, lo);
    lo = __fmaf_rn(a2.hi, b2.lo, lo);
    lo = __fmaf_rn(a2.lo, b2.hi, lo);
    return fast_two_sum(t.hi, lo);
}

// Complex double-float.
struct __align__(16) dfl2 { dfl x, y; };
template <> struct Cplx<dfl> { using type = dfl2; };

__device__ __forceinline__ dfl2 mk(dfl x, dfl y) { dfl2 r; r.x = x; r.y = y; return r; }
__device__ __forceinline__ dfl2 cadd(dfl2 a, dfl2 b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ dfl2 csub(dfl2 a, dfl2 b) { return mk(a.x - b.x, a.y - b.y); }
// acc + a * b
__device__ __forceinline__ dfl2 cfma(dfl2 a, dfl2 b, dfl2 acc) {
    return mk(dot2_acc(acc.x, a.x, b.x, -a.y, b.y), dot2_acc(acc.y, a.x, b.y, a.y, b.x));
}
// acc + conj(a) * b
__device__ __forceinline__ dfl2 cfma_conj_a(dfl2 a, dfl2 b, dfl2 acc) {
    return mk(dot2_acc(acc.x, a.x, b.x, a.y, b.y), dot2_acc(acc.y, a.x, b.y, -a.y, b.x));
}
// acc - a * conj(b)
__device__ __forceinline__ dfl2 cfms_conj_b(dfl2 a, dfl2 b, dfl2 acc) {
    return mk(dot2_acc(acc.x, -a.x, b.x, -a.y, b.y), dot2_acc(acc.y, -a.y, b.x, a.x, b.y));
}
__device__ __forceinline__ dfl cabs2(dfl2 a) { return dot2_acc(dfl(0.f, 0.f), a.x, a.x, a.y, a.y); }

__device__ __forceinline__ dfl shfl_xor_dfl(dfl v, int o) {
    return dfl(__shfl_xor_sync(FULL_MASK, v.hi, o), __shfl_xor_sync(FULL_MASK, v.lo, o));
}
__device__ __forceinline__ dfl2 cshfl_xor(dfl2 v, int o) { return mk(shfl_xor_dfl(v.x, o), shfl_xor_dfl(v.y, o)); }
template <> __device__ __forceinline__ dfl warp_sum<dfl>(dfl v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = v + shfl_xor_dfl(v, o);
    return v;
}

}  // namespace ptca
