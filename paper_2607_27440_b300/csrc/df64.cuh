// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two float32 numbers
// with |lo| <= ulp(hi)/2 (Dekker 1971, "A floating-point technique for extending the available
// precision"; Knuth's TwoSum).  Products are formed error-free with fused multiply-add and sums
// are compensated, which keeps about 48 significand bits (unit roundoff ~2^-48 ~ 3.6e-15).
// Everything runs on the float32 pipes, which on the B300 deliver about sixty times the
// float64 rate; a complex df64 value occupies the same 16 bytes as a complex float64.
// Every operation uses the _rn intrinsics so the compiler cannot contract or reassociate them.
#pragma once
#include "common.cuh"

namespace klst {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_from(double d) {
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(__dsub_rn(d, (double)h))};
}
__device__ __forceinline__ double df_to(df a) { return __dadd_rn((double)a.hi, (double)a.lo); }
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// a + b with compensated summation (TwoSum on the high parts, then renormalise)
__device__ __forceinline__ df df_add(df a, df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    t = __fadd_rn(t, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, t);
    return {h, __fsub_rn(t, __fsub_rn(h, s))};
}

// acc += a * b: the product's rounding error comes from one FMA (TwoProd), the cross terms are
// added to it, the lo*lo term (~2^-48 relative) is dropped, and the sum is compensated.
__device__ __forceinline__ void df_fma(df& acc, df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    float t = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    t = __fadd_rn(t, __fadd_rn(acc.lo, e));
    const float h = __fadd_rn(s, t);
    acc.lo = __fsub_rn(t, __fsub_rn(h, s));
    acc.hi = h;
}

// complex df64, stored as float4 {re.hi, re.lo, im.hi, im.lo} (16 bytes like double2)
struct cdf {
    df re, im;
};
__device__ __forceinline__ cdf cdf_from(double2 v) { return {df_from(v.x), df_from(v.y)}; }
__device__ __forceinline__ double2 cdf_to(cdf a) { return make_double2(df_to(a.re), df_to(a.im)); }
__device__ __forceinline__ cdf cdf_load(const float4* p) {
    const float4 v = *p;
    return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void cdf_store(float4* p, cdf a) { *p = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ cdf cdf_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }

// acc += a * b
__device__ __forceinline__ void cdf_fma(cdf& acc, cdf a, cdf b) {
    df_fma(acc.re, a.re, b.re);
    df_fma(acc.re, df_neg(a.im), b.im);
    df_fma(acc.im, a.re, b.im);
    df_fma(acc.im, a.im, b.re);
}
// acc += conj(a) * b
__device__ __forceinline__ void cdf_fma_conj(cdf& acc, cdf a, cdf b) {
    df_fma(acc.re, a.re, b.re);
    df_fma(acc.re, a.im, b.im);
    df_fma(acc.im, a.re, b.im);
    df_fma(acc.im, df_neg(a.im), b.re);
}

__device__ __forceinline__ df df_shfl_xor(df a, int o) {
    return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
// deterministic warp sum (fixed xor tree)
__device__ __forceinline__ cdf cdf_warp_sum(cdf a) {
    for (int o = 16; o > 0; o >>= 1) {
        const cdf b = {df_shfl_xor(a.re, o), df_shfl_xor(a.im, o)};
        a = cdf_add(a, b);
    }
    return a;
}

// float4-typed storage overloads, so the block-solve kernels can be instantiated for df64 factors
__device__ __forceinline__ cdf cdf_unpack(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 cdf_pack(cdf a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ void cfma(float4& acc, float4 a, float4 b) {
    cdf c = cdf_unpack(acc);
    cdf_fma(c, cdf_unpack(a), cdf_unpack(b));
    acc = cdf_pack(c);
}
template <> __device__ __forceinline__ float4 to_c<float4>(double2 v) { return cdf_pack(cdf_from(v)); }
__device__ __forceinline__ double2 to_d(float4 v) { return cdf_to(cdf_unpack(v)); }

}  // namespace klst
