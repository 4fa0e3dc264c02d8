// Shared pieces of the float64-accurate tensor-core products (the Ozaki scheme): the error-free
// split of float64 operands into bfloat16 integer slices, and the tcgen05 / bulk-copy plumbing.
#pragma once
#include <cstdint>

#include "factor.cuh"

namespace klst {

constexpr int OZ_S = 8;        // slices per operand
constexpr int OZ_KMAX = 256;   // exactness bound of the float32 accumulation

// ------------------------------------------------------------------ splitting
// biased float64 exponent of x (0 for zero and subnormals)
__device__ __forceinline__ int dexp(double x) {
    return (int)((unsigned)(__double_as_longlong(x) >> 52) & 0x7FFu);
}

// Fixed-point integer F = x 2^(56 - e) for a row whose entries satisfy |x| < 2^e, e = Emax - 1022.
__device__ __forceinline__ long long oz_fixed(double x, int e) {
    const long long b = __double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0) return 0;
    const long long M = (b & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    const int sh = E - 1019 - e;
    long long F;
    if (sh >= 0) F = M << sh;          // sh <= 3 because |x| < 2^e
    else F = (-sh >= 63) ? 0 : (M >> (-sh));
    return b < 0 ? -F : F;
}

// bfloat16 bit pattern of a small integer d (|d| <= 2^22): 1.5 * 2^23 + d is exact in float32, and
// a value with at most 8 significant bits has zero low 16 mantissa bits
__device__ __forceinline__ unsigned short bf16_of_int(int d) {
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
    return (unsigned short)(__float_as_uint(f) >> 16);
}

// the eight balanced base-128 digits of F (most significant first)
__device__ __forceinline__ void oz_digits(long long F, int dig[OZ_S]) {
#pragma unroll
    for (int s = OZ_S - 1; s >= 1; --s) {
        const int d = (int)((F + 64) & 127) - 64;
        dig[s] = d;
        F = (F - d) >> 7;
    }
    dig[0] = (int)F;
}

// Slice writer shared by both operands: one warp per row of the operand (a row of A, or a column
// of B); lane q handles k-chunk q (eight consecutive k), so Kp <= 256 fits one warp.  The warp
// first takes the row's largest exponent (shuffle max), then every lane writes its chunk's eight
// digits of each slice as one 16-byte store.  dst(s, kc) gives the chunk's 8-element destination.
template <class Src, class Out>
__device__ __forceinline__ void oz_split_row(const Src& src, int r, int Kp, Out out, int* e_out) {
    const int lane = threadIdx.x & 31, nkc = Kp / 8;
    double v[8];
    int Emax = 0;
    if (lane < nkc) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v[q] = src(r, lane * 8 + q);
            Emax = max(Emax, dexp(v[q]));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Emax = max(Emax, __shfl_xor_sync(0xffffffffu, Emax, o));
    const int e = Emax - 1022;
    if (lane == 0) *e_out = e;
    if (lane >= nkc) return;
    int dig[8][OZ_S];
#pragma unroll
    for (int q = 0; q < 8; ++q) oz_digits(oz_fixed(v[q], e), dig[q]);
#pragma unroll
    for (int sl = 0; sl < OZ_S; ++sl) {
        uint4 w;
        w.x = bf16_of_int(dig[0][sl]) | ((unsigned)bf16_of_int(dig[1][sl]) << 16);
        w.y = bf16_of_int(dig[2][sl]) | ((unsigned)bf16_of_int(dig[3][sl]) << 16);
        w.z = bf16_of_int(dig[4][sl]) | ((unsigned)bf16_of_int(dig[5][sl]) << 16);
        w.w = bf16_of_int(dig[6][sl]) | ((unsigned)bf16_of_int(dig[7][sl]) << 16);
        *reinterpret_cast<uint4*>(out(sl, lane)) = w;
    }
}

// A operand: rows padded to whole 128-row tiles (zero rows beyond R); four warps per CTA
template <class Src>
__global__ void __launch_bounds__(128) k_oz_split_a(Src src, int R, int Kp, unsigned short* __restrict__ out,
                                                    int* __restrict__ ea, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int r = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int mtile = r >> 7, rr = r & 127;
    if (mtile >= (R + 127) / 128) return;
    const int nkc = Kp / 8;
    auto dst = [&](int sl, int kc) { return out + ((((size_t)mtile * OZ_S + sl) * nkc + kc) * 128 + rr) * 8; };
    oz_split_row(src, r, Kp, dst, ea + r);
}

// 2^(-7 d) exactly, from its exponent bits
__device__ __forceinline__ double exp2_neg7(int d) { return __longlong_as_double((long long)(1023 - 7 * d) << 52); }

// ------------------------------------------------------------------ tcgen05 plumbing
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance between core matrices
// adjacent in K, sbo = between 8-row groups adjacent in M (or N)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: bfloat16 A and B (K-major), float32 D, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// bounded wait for the phase with the given parity; false when the bound ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long long it = 0; it < (1ll << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}
// bulk copy global -> shared (the TMA engine), completion counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(dtmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// x 2^e by integer operations on the exponent field (x a normal float64 or 0; results below the
// normal range become 0)
__device__ __forceinline__ double scale2(double x, int e) {
    const long long b = __double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0) return 0.0;
    const int En = E + e;
    if (En <= 0) return 0.0;
    return __longlong_as_double(b + ((long long)e << 52));
}

// The exact value sum_{d=0..7} blk[d] 2^(-7 (d + 2)) of eight diagonal blocks, each an integer below
// 2^24 held exactly in float32: the four leading and the four trailing blocks are combined exactly
// in two 64-bit integers (below 2^46 each), which float64 holds exactly, and one fused multiply-add
// rounds the sum once.
__device__ __forceinline__ double oz_combine(const float blk[OZ_S]) {
    long long H = 0, L = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) H = H * 128 + (long long)__float2int_rn(blk[d]);
#pragma unroll
    for (int d = 4; d < 8; ++d) L = L * 128 + (long long)__float2int_rn(blk[d]);
    return fma((double)L, exp2_neg7(9), (double)H * exp2_neg7(5));
}

// Leading 24 significand bits of a float64 as a float32 (truncation), by integer operations only:
// the B300 converts float64 at the float64 rate, this stays on the integer and float32 pipes.
// Values below 2^-126 in magnitude become 0 (the basis vectors have unit norm and w = T v_j is
// far inside the float32 range, so nothing else reaches the limits).
__device__ __forceinline__ float trunc_f32(double x) {
    const long long b = __double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int ef = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    const unsigned f = (hi & 0x80000000u) | ((unsigned)ef << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    return (ef > 0 && ef < 255) ? __uint_as_float(f) : 0.0f;
}

// ---- nine-slice variant (63-bit fixed point): x ~= 2^e sum_{s=0..8} d_s 2^(-7 (s + 1)), |x| < 2^e
constexpr int OZ_S9 = 9;

__device__ __forceinline__ long long oz_fixed63(double x, int e) {
    const long long b = __double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0) return 0;
    const long long M = (b & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    const int sh = E - 1012 - e;         // F = x 2^(63 - e): |F| < 2^63 because |x| < 2^e
    long long F;
    if (sh >= 0) F = M << sh;            // sh <= 10
    else F = (-sh >= 63) ? 0 : (M >> (-sh));
    return b < 0 ? -F : F;
}

__device__ __forceinline__ void oz_digits9(long long F, int dig[OZ_S9]) {
#pragma unroll
    for (int s = OZ_S9 - 1; s >= 1; --s) {
        const int d = (int)((F + 64) & 127) - 64;
        dig[s] = d;
        F = (F - d) >> 7;
    }
    dig[0] = (int)F;
}

// the exact sum_{d=0..8} blk[d] 2^(-7 (d + 2)) of nine diagonal blocks (integers below 2^24): the
// leading four and the trailing five are combined exactly in 64-bit integers (below 2^46 and 2^53),
// which float64 holds exactly, and one fused multiply-add rounds the sum once
__device__ __forceinline__ double oz_combine9(const float blk[OZ_S9]) {
    long long H = 0, L = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) H = H * 128 + (long long)__float2int_rn(blk[d]);
#pragma unroll
    for (int d = 4; d < 9; ++d) L = L * 128 + (long long)__float2int_rn(blk[d]);
    return fma((double)L, exp2_neg7(10), (double)H * exp2_neg7(5));
}

// instruction descriptor of kind::f16 with the A operand MN-major (transpose bit 15)
__host__ __device__ constexpr uint32_t idesc_bf16_amn(int M, int N) { return idesc_bf16(M, N) | (1u << 15); }

}  // namespace klst
