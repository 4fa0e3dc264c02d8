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

// ---------------------------------------------------------------- scalar and complex helpers
// a * b: TwoProd of the high parts by one FMA, plus the cross terms, renormalised (Fast2Sum)
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float h = __fadd_rn(p, e);
    return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
// multiplication by a power of two (exact while no part leaves the float32 range)
__device__ __forceinline__ df df_scale(df a, float p2) { return {__fmul_rn(a.hi, p2), __fmul_rn(a.lo, p2)}; }

// 1 / sqrt(x) for a normal x > 0.  Seed y0 = float32 reciprocal square root (about 22 correct
// bits); with r = 1 - x y0^2 (formed in df64; |r| ~ 2^-22) the exact value is
// y0 (1 - r)^(-1/2) = y0 (1 + r/2 + 3 r^2/8 + O(r^3)), so one step of this series (Halley's
// method) leaves an error of order r^3 ~ 2^-66, below df64 rounding.
__device__ __forceinline__ df df_rsqrt(df x) {
    const float y0 = rsqrtf(x.hi);
    const float q = __fmul_rn(y0, y0);
    const df yy = {q, __fmaf_rn(y0, y0, -q)};                    // y0^2 exactly
    const df r = df_sub(df{1.f, 0.f}, df_mul(x, yy));
    const float h = __fmul_rn(0.5f, y0);
    const float p = __fmul_rn(h, r.hi);
    float e = __fmaf_rn(h, r.hi, -p);                            // y0 r / 2 = p + e (high part exact)
    e = __fmaf_rn(h, r.lo, e);
    e = __fmaf_rn(__fmul_rn(0.75f, p), r.hi, e);                 // + 3 y0 r^2 / 8
    return df_add(df{y0, 0.f}, df{p, e});
}

__device__ __forceinline__ cdf cdf_neg(cdf a) { return {df_neg(a.re), df_neg(a.im)}; }
__device__ __forceinline__ cdf cdf_conj(cdf a) { return {a.re, df_neg(a.im)}; }
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
    cdf r = {df_mul(a.re, b.re), df_mul(a.re, b.im)};
    df_fma(r.re, df_neg(a.im), b.im);
    df_fma(r.im, a.im, b.re);
    return r;
}
__device__ __forceinline__ cdf cdf_rmul(df c, cdf a) { return {df_mul(c, a.re), df_mul(c, a.im)}; }
__device__ __forceinline__ cdf cdf_scale(cdf a, float p2) { return {df_scale(a.re, p2), df_scale(a.im, p2)}; }
__device__ __forceinline__ df cdf_abs2(cdf a) {
    df r = df_mul(a.re, a.re);
    df_fma(r, a.im, a.im);
    return r;
}
// |re| + |im| of the leading parts (float32), for magnitude tests
__device__ __forceinline__ float cdf_abs1f(cdf a) { return fabsf(a.re.hi) + fabsf(a.im.hi); }

// plane rotation x' = c x + s y, y' = c y - conj(s) x with real c.  The terms in y are formed
// first, so a caller that carries x from the previous rotation waits on two df64 FMAs only.
__device__ __forceinline__ void cdf_rot(cdf& x, cdf& y, df c, cdf s) {
    cdf t = {df_mul(s.re, y.re), df_mul(s.re, y.im)};
    df_fma(t.re, df_neg(s.im), y.im);
    df_fma(t.im, s.im, y.re);
    cdf u = {df_mul(c, y.re), df_mul(c, y.im)};
    df_fma(t.re, c, x.re);
    df_fma(t.im, c, x.im);
    df_fma(u.re, df_neg(s.re), x.re);
    df_fma(u.im, df_neg(s.re), x.im);
    df_fma(u.re, df_neg(s.im), x.im);
    df_fma(u.im, s.im, x.re);
    x = t;
    y = u;
}

__device__ __forceinline__ float2 df_pack(df a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ df df_unpack(float2 v) { return {v.x, v.y}; }

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
