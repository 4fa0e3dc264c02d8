// Float64-accurate real GEMM C = A B on the 5th-generation tensor cores (tcgen05), by error-free
// splitting of the operands into small integer slices (the Ozaki scheme: Ozaki, Ogita, Oishi and
// Rump, "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Splitting.  Row r of A (over the reduction index k) is scaled by 2^-ea[r] with |A[r, k]| < 2^ea[r]
// and written as a signed fixed-point integer F = A[r, k] 2^(56 - ea[r]) (|F| < 2^56, truncated below
// 2^-56 of the row's largest entry).  F is cut into eight balanced base-128 digits,
//     A[r, k] ~= 2^ea[r] sum_{s=1..8} a_s[r, k] 2^(-7 s),   |a_1| <= 128, |a_s| <= 64 (s >= 2),
// every digit an integer held exactly by bfloat16.  B is split the same way per column (eb[c]).
// Products.  a_s b_t is an integer product; for a fixed diagonal d = s + t the sum over k of every
// pair on that diagonal stays below 2^24 for K <= 256 (at most 2 pairs reach 128 x 64, the others
// 64 x 64: (2 * 8192 + 6 * 4096) * 256 < 2^24), so a float32 tensor-core accumulator holds it
// exactly.  The eight diagonals d = 2..9 (36 slice pairs; pairs with s + t > 9 are dropped, a
// relative error below 2^-55 of the row and column maxima) are accumulated in eight TMEM blocks:
// one MMA per A-slice s multiplies a_s by the B slices t = 1..9-s stacked along N, whose products
// land in the TMEM blocks s+1..9 -- a sliding window, so every diagonal block receives exactly its
// own pairs.  The epilogue sums the eight exact block values in float64 (one rounding each) and
// scales by 2^(ea[r] + eb[c]).  The result carries float64-level error relative to
// max_k |A[r, k]| max_k |B[k, c]| K.
//
// Layouts (K-major, no swizzle: 8-row x 16-byte core matrices).  A slices: [mtile][s][kchunk]
// [128 rows][8], so one slice of one 128-row tile is a contiguous block of K x 256 bytes (core
// matrices adjacent in K 2 KB apart, 8-row groups 128 B apart).  B slices: [ntile][kchunk][s]
// [NT rows][8]: for each k-chunk the eight slices' rows follow one another, so a contiguous run of
// (9 - s) slices is one N-stacked operand (8-row groups 128 B apart, k-chunks 8 NT 16 B apart).
#include <algorithm>
#include <atomic>
#include <cstring>

#include "factor.cuh"

namespace klst {

constexpr int OZ_S = 8;        // slices per operand
constexpr int OZ_NT = 32;      // output columns per CTA (8 diagonal blocks x 32 = 256 TMEM columns)
constexpr int OZ_KMAX = 256;   // exactness bound of the float32 accumulation (see above)

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

// Element sources: the GEMM's A rows and B columns as functions (row, k) -> double
struct SrcColMajor {    // A: A[k * ld + r]  (column-major M x K);  B: B[c * ld + k] (column-major K x N)
    const double* p;
    int64_t ld;
    int rows_are_k;     // 0: element (r, k) = p[k * ld + r]; 1: element (c, k) = p[c * ld + k]
    int R, K;
    __device__ double operator()(int r, int k) const {
        if (r >= R || k >= K) return 0.0;
        return rows_are_k ? p[(int64_t)r * ld + k] : p[(int64_t)k * ld + r];
    }
};
struct SrcBasisRows {   // rows of [Re V | Im V] for a complex column-major basis V (n x m, ld)
    const double2* V;
    int64_t ld;
    int m, R;
    __device__ double operator()(int r, int k) const {
        if (r >= R || k >= 2 * m) return 0.0;
        const double2 v = V[(int64_t)(k < m ? k : k - m) * ld + r];
        return k < m ? v.x : v.y;
    }
};
struct SrcRotCols {     // columns of [[Qr, Qi], [-Qi, Qr]] (2m x 2 keep) for a complex Q (m x keep, ld)
    const double2* Q;
    int ld, m, keep;
    __device__ double operator()(int c, int k) const {
        if (c >= 2 * keep || k >= 2 * m) return 0.0;
        const int cc = c < keep ? c : c - keep, kk = k < m ? k : k - m;
        const double2 q = Q[(int64_t)cc * ld + kk];
        if (c < keep) return k < m ? q.x : -q.y;
        return k < m ? q.y : q.x;
    }
};

// One thread per A row: exponent, then every k-chunk's eight digits as eight 16-byte rows.
template <class Src>
__global__ void __launch_bounds__(128) k_oz_split_a(Src src, int R, int Kp, unsigned short* __restrict__ out,
                                                    int* __restrict__ ea) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int mtile = r >> 7, rr = r & 127;
    if (mtile >= (R + 127) / 128) return;
    int Emax = 0;
    for (int k = 0; k < Kp; ++k) Emax = max(Emax, dexp(src(r, k)));
    const int e = Emax - 1022;
    ea[r] = e;
    const int nkc = Kp / 8;
    for (int kc = 0; kc < nkc; ++kc) {
        int dig[8][OZ_S];
#pragma unroll
        for (int q = 0; q < 8; ++q) oz_digits(oz_fixed(src(r, kc * 8 + q), e), dig[q]);
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
            uint4 v;
            v.x = bf16_of_int(dig[0][s]) | ((unsigned)bf16_of_int(dig[1][s]) << 16);
            v.y = bf16_of_int(dig[2][s]) | ((unsigned)bf16_of_int(dig[3][s]) << 16);
            v.z = bf16_of_int(dig[4][s]) | ((unsigned)bf16_of_int(dig[5][s]) << 16);
            v.w = bf16_of_int(dig[6][s]) | ((unsigned)bf16_of_int(dig[7][s]) << 16);
            const size_t off = ((((size_t)mtile * OZ_S + s) * nkc + kc) * 128 + rr) * 8;
            *reinterpret_cast<uint4*>(out + off) = v;
        }
    }
}

// One thread per B column c (a row of B^T): exponent and the stacked slice layout of its N-tile.
template <class Src>
__global__ void __launch_bounds__(128) k_oz_split_b(Src src, int N, int Kp, unsigned short* __restrict__ out,
                                                    int* __restrict__ eb) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int ntile = c / OZ_NT, cc = c % OZ_NT;
    if (ntile >= (N + OZ_NT - 1) / OZ_NT) return;
    int Emax = 0;
    for (int k = 0; k < Kp; ++k) Emax = max(Emax, dexp(src(c, k)));
    const int e = Emax - 1022;
    eb[c] = e;
    const int nkc = Kp / 8;
    for (int kc = 0; kc < nkc; ++kc) {
        int dig[8][OZ_S];
#pragma unroll
        for (int q = 0; q < 8; ++q) oz_digits(oz_fixed(src(c, kc * 8 + q), e), dig[q]);
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
            uint4 v;
            v.x = bf16_of_int(dig[0][s]) | ((unsigned)bf16_of_int(dig[1][s]) << 16);
            v.y = bf16_of_int(dig[2][s]) | ((unsigned)bf16_of_int(dig[3][s]) << 16);
            v.z = bf16_of_int(dig[4][s]) | ((unsigned)bf16_of_int(dig[5][s]) << 16);
            v.w = bf16_of_int(dig[6][s]) | ((unsigned)bf16_of_int(dig[7][s]) << 16);
            const size_t off = ((((size_t)ntile * nkc + kc) * OZ_S + s) * OZ_NT + cc) * 8;
            *reinterpret_cast<uint4*>(out + off) = v;
        }
    }
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

// Output sinks: where C[r, c] goes
struct DstColMajor {    // C[c * ld + r]
    double* p;
    int64_t ld;
    int R, N;
    __device__ void operator()(int r, int c, double v) const {
        if (r < R && c < N) p[(int64_t)c * ld + r] = v;
    }
};
struct DstBasis {       // column c < keep -> Re V'[r, c], c >= keep -> Im V'[r, c - keep] (complex, ld)
    double* p;
    int64_t ld;
    int R, keep;
    __device__ void operator()(int r, int c, double v) const {
        if (r < R && c < 2 * keep) p[((int64_t)(c < keep ? c : c - keep) * ld + r) * 2 + (c < keep ? 0 : 1)] = v;
    }
};

// One CTA = one 128-row M tile x OZ_NT output columns; four warps.  Thread 0 loads (bulk copies)
// and issues the MMAs; every warp then drains its 32 TMEM lanes.  smem: the N-tile's stacked B
// slices (K x OZ_NT x 16 B) and one A slice (K x 256 B).  Waits are bounded: on a timeout the CTA
// sets ST_TIMEOUT in *st, skips the remaining work, frees its TMEM and returns.
template <class Dst>
__global__ void __launch_bounds__(128, 1) k_oz_gemm(const unsigned short* __restrict__ As,
                                                    const unsigned short* __restrict__ Bs,
                                                    const int* __restrict__ ea, const int* __restrict__ eb, int Kp,
                                                    Dst dst, Status* st) {
    extern __shared__ __align__(128) unsigned char oz_smem[];
    __shared__ __align__(8) uint64_t bar_ld, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int ntile = blockIdx.x, mtile = blockIdx.y;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int nkc = Kp / 8;
    const uint32_t bytesB = (uint32_t)Kp * OZ_NT * 16;   // nkc x OZ_S x OZ_NT x 16 B
    const uint32_t bytesA = (uint32_t)Kp * 256;          // nkc x 128 x 16 B
    unsigned char* sB = oz_smem;
    unsigned char* sA = oz_smem + bytesB;
    constexpr uint32_t kCols = 256;                      // 8 diagonal blocks x OZ_NT
    if (tid == 0) {
        mbar_init(&bar_ld, 1);
        mbar_init(&bar_mma, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (wid == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)), "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = tmem_base;
    if (tid == 0) {
        const unsigned short* gB = Bs + (size_t)ntile * nkc * OZ_S * OZ_NT * 8;
        uint32_t ph_ld = 0, ph_mma = 0;
        bool ok = true;
        for (int s = 0; s < OZ_S && ok; ++s) {
            const unsigned short* gA = As + (((size_t)mtile * OZ_S + s) * nkc) * 128 * 8;
            mbar_expect_tx(&bar_ld, bytesA + (s == 0 ? bytesB : 0));
            bulk_g2s(sA, gA, bytesA, &bar_ld);
            if (s == 0) bulk_g2s(sB, gB, bytesB, &bar_ld);
            ok = mbar_wait(&bar_ld, ph_ld);
            ph_ld ^= 1;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // a_s x [b_1 .. b_{8-s}] (N = (8 - s) x OZ_NT) into diagonal blocks s+1 .. 8 (0-based d-2)
            const int nst = OZ_S - s;
            const uint32_t idesc = idesc_bf16(128, nst * OZ_NT);
            const uint32_t dcol = tbase + (uint32_t)(s * OZ_NT);
            const uint32_t aBase = smem_u32(sA), bBase = smem_u32(sB);
            for (int kk = 0; kk < Kp / 16; ++kk) {
                const uint64_t ad = sdesc(aBase + kk * 2 * 2048, 2048, 128);
                const uint64_t bd = sdesc(bBase + kk * 2 * (OZ_S * OZ_NT * 16), OZ_S * OZ_NT * 16, 128);
                mma_bf16(dcol, ad, bd, idesc, (s > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&bar_mma);
            ok = mbar_wait(&bar_mma, ph_mma);
            ph_mma ^= 1;
        }
        if (!ok) {
            s_fail = 1;
            atomicOr(&st->flags, ST_TIMEOUT);
            // give any copy or MMA still in flight one more bounded wait before the TMEM is freed
            mbar_wait(&bar_ld, ph_ld);
            mbar_wait(&bar_mma, ph_mma);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail) {
        // C[r, c] = 2^(ea + eb) sum_{d=2..9} block_d 2^(-7 d), each block an exact integer
        const int r = mtile * 128 + wid * 32 + lane;
        const uint32_t lane_off = (uint32_t)(wid * 32) << 16;
        const int era = ea[r];
        for (int c0 = 0; c0 < OZ_NT; c0 += 8) {
            float blk[OZ_S][8];
#pragma unroll
            for (int d = 0; d < OZ_S; ++d) tmem_ld8(tbase + lane_off + (uint32_t)(d * OZ_NT + c0), blk[d]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                double acc = 0.0;
#pragma unroll
                for (int d = OZ_S - 1; d >= 0; --d) acc = fma((double)blk[d][q], exp2_neg7(d + 2), acc);
                const int c = ntile * OZ_NT + c0 + q;
                dst(r, c, ldexp(acc, era + eb[c]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols));
}

// ------------------------------------------------------------------ host side
size_t oz_workspace_bytes(int M, int N, int K) {
    const int Kp = (K + 15) / 16 * 16;
    const size_t mt = (M + 127) / 128, nt = (N + OZ_NT - 1) / OZ_NT;
    const size_t a = mt * 128 * (size_t)Kp * OZ_S * 2, b = nt * OZ_NT * (size_t)Kp * OZ_S * 2;
    return ((a + 255) & ~size_t(255)) + ((b + 255) & ~size_t(255)) + (mt * 128 + nt * OZ_NT) * sizeof(int) + 256;
}

struct OzWork {
    unsigned short *A, *B;
    int *ea, *eb;
};
static OzWork oz_carve(void* ws, int M, int N, int Kp) {
    const size_t mt = (M + 127) / 128, nt = (N + OZ_NT - 1) / OZ_NT;
    char* p = (char*)ws;
    OzWork w;
    w.A = (unsigned short*)p;
    p += ((mt * 128 * (size_t)Kp * OZ_S * 2) + 255) & ~size_t(255);
    w.B = (unsigned short*)p;
    p += ((nt * OZ_NT * (size_t)Kp * OZ_S * 2) + 255) & ~size_t(255);
    w.ea = (int*)p;
    w.eb = w.ea + mt * 128;
    return w;
}

template <class Dst>
static int oz_launch_gemm(const OzWork& w, int M, int N, int Kp, Dst dst, Status* st, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    const size_t smem = (size_t)Kp * OZ_NT * 16 + (size_t)Kp * 256;
    if (once_per_device(attr)) KLST_CK(cudaFuncSetAttribute(k_oz_gemm<Dst>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    dim3 grid((N + OZ_NT - 1) / OZ_NT, (M + 127) / 128);
    k_oz_gemm<Dst><<<grid, 128, smem, s>>>(w.A, w.B, w.ea, w.eb, Kp, dst, st);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

// V'[:, 0:keep] = V[:, 0:m] Q[:, 0:keep] (complex, column-major, ld n for V and V', m for Q)
int oz_rotate(const double2* V, int64_t n, int m, const double2* Q, int keep, double2* Vout, void* ws, Status* st,
              cudaStream_t s) {
    const int K = 2 * m, Kp = (K + 15) / 16 * 16, N = 2 * keep;
    if (Kp > OZ_KMAX || n > (int64_t)0x7FFFFFFF) { set_error("rotation too large for the tensor-core path"); return KLST_EINVAL; }
    OzWork w = oz_carve(ws, (int)n, N, Kp);
    const int R = (int)n;
    SrcBasisRows sa{V, n, m, R};
    SrcRotCols sb{Q, m, m, keep};
    k_oz_split_a<SrcBasisRows><<<(int)(((n + 127) / 128 * 128 + 127) / 128), 128, 0, s>>>(sa, R, Kp, w.A, w.ea);
    note_launch();
    k_oz_split_b<SrcRotCols><<<((N + OZ_NT - 1) / OZ_NT * OZ_NT + 127) / 128, 128, 0, s>>>(sb, N, Kp, w.B, w.eb);
    note_launch();
    KLST_CK_LAUNCH();
    return oz_launch_gemm(w, R, N, Kp, DstBasis{reinterpret_cast<double*>(Vout), n, R, keep}, st, s);
}

int oz_gemm_f64(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int M, int N, int K,
                void* ws, Status* st, cudaStream_t s) {
    const int Kp = (K + 15) / 16 * 16;
    OzWork w = oz_carve(ws, M, N, Kp);
    SrcColMajor sa{A, lda, 0, M, K};
    SrcColMajor sb{B, ldb, 1, N, K};
    k_oz_split_a<SrcColMajor><<<(M + 127) / 128, 128, 0, s>>>(sa, M, Kp, w.A, w.ea);
    note_launch();
    k_oz_split_b<SrcColMajor><<<((N + OZ_NT - 1) / OZ_NT * OZ_NT + 127) / 128, 128, 0, s>>>(sb, N, Kp, w.B, w.eb);
    note_launch();
    KLST_CK_LAUNCH();
    return oz_launch_gemm(w, M, N, Kp, DstColMajor{C, ldc, M, N}, st, s);
}

}  // namespace klst

using namespace klst;

extern "C" int klst_gemm_f64_tc(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                                int32_t M, int32_t N, int32_t K, klst_stream stream) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || K > OZ_KMAX || lda < M || ldb < K || ldc < M) {
        set_error("invalid arguments to klst_gemm_f64_tc (1 <= K <= %d)", OZ_KMAX);
        return KLST_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    void* ws = nullptr;
    Status* st = nullptr;
    cudaError_t e;
    if ((e = dmalloc(&ws, oz_workspace_bytes(M, N, K), s)) != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    if ((e = dmalloc((void**)&st, sizeof(Status), s)) != cudaSuccess) { dfree(ws, s); return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__); }
    cudaMemsetAsync(st, 0, sizeof(Status), s);
    int rc = oz_gemm_f64(A, lda, B, ldb, C, ldc, M, N, K, ws, st, s);
    Status hst;
    memset(&hst, 0, sizeof(hst));
    if (rc == KLST_OK) {
        if ((e = cudaMemcpyAsync(&hst, st, sizeof(Status), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            rc = cuda_fail(e, "gemm sync", __FILE__, __LINE__);
    }
    dfree(ws, s);
    dfree(st, s);
    if (rc == KLST_OK && (hst.flags & ST_TIMEOUT)) { set_error("tensor-core GEMM: a bounded wait gave up"); return KLST_ETIMEOUT; }
    return rc;
}
