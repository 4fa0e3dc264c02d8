// Float64-accurate Gram-Schmidt products on the tensor cores for the float64 Krylov basis
// (Sec. 4.1, classical Gram-Schmidt applied twice).
//
// The basis V (n x (m + 1), complex, unit columns) is also kept as nine bfloat16 integer slices
// with one fixed scale: |V| <= 1 < 2^1, so each real entry is x = 2 sum_{s=0..8} d_s 2^(-7 (s + 1))
// to 2^-62 absolute (oz.cuh, nine-slice variant).  Rows are grouped in tiles of 128 and the real
// index k = 2 c + p (column c, p = 0 real part, 1 imaginary part) in chunks of 8:
//     SL[tile][slice][kchunk (32)][128 rows][8]        (2 KB per k-chunk of a tile and slice)
// One layout serves both products:
//   update  w - V h: A = V tile (M = rows, K = k), K-major: core matrices 8 rows x 16 B, LBO 2 KB
//   dots    V^H w:   A = V tile^T (M = k, K = rows), the same bytes read MN-major (transpose bit):
//                    core matrices 8 k x 8 rows, LBO 128 B along the rows, SBO 2 KB along k
// B operands (coefficients h, or one tile of w) are split per column with their own exponent into
// nine slices stacked along N with seven zero slices ([kchunk][16 slices x 2 columns][8]); slice s
// of A meets slices t = 0..15 (s = 0) or t = 0..7 (s > 0) of B in the TMEM columns 2 (s + t), so
// every diagonal d = s + t <= 8 collects exactly its pairs (the rest land in unread columns).  With
// K <= 256 every diagonal sum stays below 2^24 ((2 x 128 x 64 + 7 x 64 x 64) x 256), exact in
// float32; the epilogue combines the nine diagonals with integer operations and one rounding.
//
// Per Arnoldi step (orth64_step with slices): first-pass coefficients on the float32 pipes from a
// truncated float32 copy of V; w' = w - V h1 (all nine slices); h2 = V^H w' (nine slices, partial
// sums per CTA, then k_reduce_cols64); w'' = w' - V h2 with six A slices: h2 ~ 1e-7 ||w|| after a
// float32 first pass, so V truncated to 2^-41 changes w'' by ~1e-19 ||w|| per entry, far below
// float64 rounding.  (One pass that fused the first update with the second dots, re-reading the
// slices from L2, was measured no faster than the two passes.)
#include <algorithm>
#include <atomic>

#include "tcstream.cuh"

namespace klst {

constexpr int kSlKc = 32;                               // k-chunks per tile and slice (k < 256)
constexpr size_t kSlTileBytes = (size_t)OZ_S9 * kSlKc * 2048;

size_t basis_slices_bytes(int64_t n) { return (size_t)((n + 127) / 128) * kSlTileBytes; }
bool basis_slices_supported(int m) { return 2 * (m + 1) <= 256; }

// nine digits of the real and imaginary parts of a basis entry (fixed exponent 1), written as the
// bfloat16 pair (k = 2c, 2c + 1) of every slice
__device__ __forceinline__ void split_entry(unsigned short* SL, int64_t r, int c, double2 v) {
    int dr[OZ_S9], di[OZ_S9];
    oz_digits9(oz_fixed63(v.x, 1), dr);
    oz_digits9(oz_fixed63(v.y, 1), di);
    const int64_t tile = r >> 7, rr = r & 127;
    const int k = 2 * c, kc = k >> 3, kk = k & 7;
#pragma unroll
    for (int s = 0; s < OZ_S9; ++s) {
        const unsigned pr = bf16_of_int(dr[s]) | ((unsigned)bf16_of_int(di[s]) << 16);
        *reinterpret_cast<unsigned*>(SL + ((((size_t)tile * OZ_S9 + s) * kSlKc + kc) * 128 + rr) * 8 + kk) = pr;
    }
}

// the basis entry truncated to float32 (the first-pass coefficients' operand, half the bytes)
__device__ __forceinline__ float2 trunc_c32(double2 v) { return make_float2(trunc_f32(v.x), trunc_f32(v.y)); }

__global__ void __launch_bounds__(256) k_split_basis(const double2* __restrict__ V, int64_t n, int64_t ldv, int c0,
                                                     int c1, unsigned short* __restrict__ SL, float2* __restrict__ V32) {
    for (int c = c0 + blockIdx.y; c < c1; c += gridDim.y)
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
            const double2 v = V[(int64_t)c * ldv + r];
            split_entry(SL, r, c, v);
            V32[(int64_t)c * ldv + r] = trunc_c32(v);
        }
}

int split_basis(const double2* V, int64_t n, int c0, int c1, unsigned short* SL, float2* V32, cudaStream_t s) {
    if (c1 <= c0) return KLST_OK;
    const int nb = (int)std::min<int64_t>((n + 255) / 256, 4 * device_sm_count());
    k_split_basis<<<dim3(nb, std::min(c1 - c0, 64)), 256, 0, s>>>(V, n, n, c0, c1, SL, V32);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

// The end of an Arnoldi step in one launch (column j = col - 1):
// - every CTA sums the second update's per-CTA partial norms in one fixed order, giving the same
//   beta = ||w''|| in every CTA;
// - CTA 0 writes column j of the Krylov-Schur matrix (S[0..j, j] = h1 + h2, S[j+1, j] = beta),
//   beta_out and the breakdown test;
// - every CTA writes v_{j+1} = w'' / beta into the basis, into vcur and into the slices.
// Launched with 256 threads, so the sums follow the order of a separate 256-thread reduction.
__global__ void __launch_bounds__(256) k_finish_scale64_split(
    const double2* __restrict__ h1, const double2* __restrict__ h2, const double* __restrict__ npart, int nparts,
    double2* __restrict__ S, int lds, double* __restrict__ beta_out, Status* st, const double2* __restrict__ w,
    int64_t n, double2* __restrict__ V, double2* __restrict__ vcopy, int col, unsigned short* __restrict__ SL,
    float2* __restrict__ V32, const int* __restrict__ jdev) {
    if (jdev) col = *jdev + 1;
    const int j = col - 1;
    __shared__ double red[2][32];
    __shared__ double s_inv;
    {
        double sn = 0.0, hn = 0.0;
        for (int b = threadIdx.x; b < nparts; b += blockDim.x) sn += npart[b];
        if (blockIdx.x == 0)
            for (int i = threadIdx.x; i <= j; i += blockDim.x) {
                const double2 hv = h1[i] + h2[i];
                S[(size_t)j * lds + i] = hv;
                hn += abs2(hv);
            }
        sn = warp_sum(sn);
        hn = warp_sum(hn);
        if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = sn; red[1][threadIdx.x >> 5] = hn; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, hs = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += red[0][q]; hs += red[1][q]; }
            const double b = sqrt(a);
            if (blockIdx.x == 0) {
                if (!(b > 1e-13 * sqrt(hs))) atomicOr(&st->flags, ST_BREAKDOWN);
                S[(size_t)j * lds + j + 1] = make_double2(b, 0.0);
                *beta_out = b;
            }
            s_inv = b > 0 ? 1.0 / b : 0.0;
        }
        __syncthreads();
    }
    const double inv = s_inv;
    double2* vcol = V + (int64_t)col * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = w[i];
        const double2 o = make_double2(v.x * inv, v.y * inv);
        vcol[i] = o;
        vcopy[i] = o;
        split_entry(SL, i, col, o);
        V32[(int64_t)col * n + i] = trunc_c32(o);
    }
}

// common sizes of the Gram-Schmidt passes: real columns K = 2 (j + 1) padded to the MMA step
struct GsShape {
    int j, kcu, nh;  // step, k-chunks used (even), K halves of at most 16 k-chunks
    __device__ void set(int jj) {
        j = jj;
        kcu = (2 * (j + 1) + 15) / 16 * 2;
        nh = kcu > 16 ? 2 : 1;
    }
    __device__ int kc_of(int h) const { return nh == 1 ? kcu : (h == 0 ? 16 : kcu - 16); }
};

// B slices of one complex vector split with exponent e into column col of the stacked layout
// [kchunk][16 slices x 2 columns][8]: the 8 values x[0..7] of k-chunk kc
__device__ __forceinline__ void put_b_chunk(unsigned char* sB, int kc, int col, const double x[8], int e) {
    int dig[8][OZ_S9];
#pragma unroll
    for (int q = 0; q < 8; ++q) oz_digits9(oz_fixed63(x[q], e), dig[q]);
#pragma unroll
    for (int s = 0; s < 16; ++s) {
        uint4 wv = make_uint4(0u, 0u, 0u, 0u);
        if (s < OZ_S9) {
            wv.x = bf16_of_int(dig[0][s]) | ((unsigned)bf16_of_int(dig[1][s]) << 16);
            wv.y = bf16_of_int(dig[2][s]) | ((unsigned)bf16_of_int(dig[3][s]) << 16);
            wv.z = bf16_of_int(dig[4][s]) | ((unsigned)bf16_of_int(dig[5][s]) << 16);
            wv.w = bf16_of_int(dig[6][s]) | ((unsigned)bf16_of_int(dig[7][s]) << 16);
        }
        *reinterpret_cast<uint4*>(sB + ((size_t)kc * 32 + s * 2 + col) * 16) = wv;
    }
}

// nine diagonal sums of TMEM column pair (2d + col) of one accumulator lane -> float64 (unscaled)
__device__ __forceinline__ void diag_pair(uint32_t taddr, double& v0, double& v1) {
    float b[3][8];
    tmem_ld8(taddr, b[0]);
    tmem_ld8(taddr + 8, b[1]);
    tmem_ld8(taddr + 16, b[2]);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    float d0[OZ_S9], d1[OZ_S9];
#pragma unroll
    for (int d = 0; d < OZ_S9; ++d) {
        d0[d] = b[(2 * d) >> 3][(2 * d) & 7];
        d1[d] = b[(2 * d + 1) >> 3][(2 * d + 1) & 7];
    }
    v0 = oz_combine9(d0);
    v1 = oz_combine9(d1);
}

// the MMAs of one A load of the update: ksteps K-steps of 16 into TMEM column dc; descriptors advance
// by adding the address step (field = address / 16) to their low bits, so the issuing thread spends
// a few cycles per MMA instead of rebuilding both descriptors
__device__ __forceinline__ void gs_update_mmas(uint32_t aB, uint32_t bB, uint32_t dc, uint32_t idesc, int ksteps,
                                               bool accumulate) {
    uint64_t ad = sdesc(aB, 2048, 128), bd = sdesc(bB, 512, 128);
    mma_bf16(dc, ad, bd, idesc, accumulate ? 1u : 0u);
#pragma unroll 4
    for (int kk = 1; kk < ksteps; ++kk) {
        ad += (2 * 2048) >> 4;
        bd += (2 * 512) >> 4;
        mma_bf16(dc, ad, bd, idesc, 1u);
    }
}

struct GsArgs {
    const unsigned short* SL;
    int64_t n;
    int ntiles;
    const double2* h;       // update: coefficients (j + 1)
    double2* w;             // update: in/out; dots: input
    double* npart;          // update with norm: [G] partial sums of |w|^2
    double2* part;          // dots: [G][ldp] partial coefficients
    int ldp;
    const int* jd;
    int j;
    Status* st;
};

// w <- w - V h over the tiles of this CTA with the first SA slices of V (B = h, prepared once)
template <int SA, bool NORM>
struct UpdPolicy {
    static constexpr int stage_bytes = 32 * 1024;
    static constexpr int nstages = 5;
    static constexpr int NT = 2, NBB = 1;
    static constexpr int b_total = kSlKc * 512;
    static constexpr int x_bytes = 64;
    static constexpr uint32_t tmem_alloc = 64;
    GsArgs a;
    GsShape sh;
    int g, G, ntl;
    double nrm;

    __device__ int tbuf(int i) const { return i & 1; }
    __device__ int tuse(int i) const { return i >> 1; }
    __device__ bool needs_b(int i) const { return i == 0; }  // h: prepared once
    __device__ int bbuf(int) const { return 0; }
    __device__ int buse(int) const { return 0; }
    __device__ uint32_t tcol_off(int tb) const { return (uint32_t)tb * 32; }
    __device__ int b_off(int) const { return 0; }
    __device__ int b_wait_load(int) const { return 0; }
    __device__ int first_prep() const { return 0; }
    __device__ int prep_before(int) const { return -1; }
    __device__ int prep_after(int) const { return -1; }

    __device__ int nunits() const { return ntl; }
    __device__ int nloads(int) const { return SA * sh.nh; }
    __device__ const void* src(int i, int l) const {
        const size_t t = (size_t)g + (size_t)i * G;
        const int s = l / sh.nh, h = l % sh.nh;
        return a.SL + ((t * OZ_S9 + s) * kSlKc + h * 16) * 1024;
    }
    __device__ uint32_t bytes(int, int l) const { return (uint32_t)sh.kc_of(l % sh.nh) * 2048; }
    __device__ void mma(int, int l, uint32_t aB, uint32_t bB, uint32_t tcol) const {
        const int s = l / sh.nh, h = l % sh.nh;
        const uint32_t idesc = idesc_bf16(128, s == 0 ? 32 : 16);
        gs_update_mmas(aB, bB + (uint32_t)(h * 16) * 512, tcol + (uint32_t)(2 * s), idesc, sh.kc_of(h) / 2,
                       s > 0 || h > 0);
    }
    // B: column 0 gives Re(V h) = sum Re V Re h - Im V Im h, column 1 gives Im(V h)
    __device__ void prep(int, unsigned char* sB, unsigned char* sX, int t) const {
        int* em = reinterpret_cast<int*>(sX);
        if (t == 0) *em = 0;
        epi_sync();
        int e = 0;
        for (int c = t; c <= sh.j; c += kTsEpi) e = max(e, max(dexp(a.h[c].x), dexp(a.h[c].y)));
        atomicMax(em, e);
        epi_sync();
        const int eh = *em - 1022;
        for (int item = t; item < sh.kcu * 2; item += kTsEpi) {
            const int kc = item >> 1, col = item & 1;
            double x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = kc * 8 + q, c = k >> 1, p = k & 1;
                double v = 0.0;
                if (c <= sh.j) {
                    const double2 hv = a.h[c];
                    v = col == 0 ? (p == 0 ? hv.x : -hv.y) : (p == 0 ? hv.y : hv.x);
                }
                x[q] = v;
            }
            put_b_chunk(sB, kc, col, x, eh);
        }
    }
    __device__ void epilogue(int i, uint32_t tcol, unsigned char* sX, int quarter, int lane) {
        double v0, v1;
        diag_pair(tcol + ((uint32_t)(quarter * 32) << 16), v0, v1);
        const int e = *reinterpret_cast<const int*>(sX) - 1022 + 1;
        const int64_t r = ((int64_t)g + (int64_t)i * G) * 128 + quarter * 32 + lane;
        if (r >= a.n) return;
        const double2 wv = a.w[r];
        const double2 o = make_double2(wv.x - scale2(v0, e), wv.y - scale2(v1, e));
        a.w[r] = o;
        if (NORM) nrm += abs2(o);
    }
    __device__ void finish(unsigned char* sX, int quarter, int lane) const {
        if (!NORM) return;
        double* red = reinterpret_cast<double*>(sX + 16);
        const double s = warp_sum(nrm);
        if (lane == 0) red[quarter] = s;
        epi_sync();
        if (quarter == 0 && lane == 0) a.npart[g] = ((red[0] + red[1]) + red[2]) + red[3];
    }
};

// part[g][c] = sum over the CTA's tiles of conj(V[r, c]) w[r] (all nine slices; B = one tile of w,
// split per tile by the B/epilogue threads into the other buffer while the current tile multiplies)
struct DotPolicy {
    static constexpr int stage_bytes = 32 * 1024;
    static constexpr int nstages = 5;
    static constexpr int NT = 2, NBB = 2;
    static constexpr int b_total = 2 * 16 * 512;  // two w tiles, K = 128 rows each
    static constexpr int x_bytes = 64;
    static constexpr uint32_t tmem_alloc = 128;   // 2 x (two M halves (k < 128, k >= 128) x 32)
    GsArgs a;
    GsShape sh;
    int g, G, ntl;
    double acc[2][2];  // [M half][B column] running sums of this lane's row k

    __device__ int nunits() const { return ntl; }
    __device__ int nloads(int) const { return OZ_S9 * sh.nh; }
    __device__ const void* src(int i, int l) const {
        const size_t t = (size_t)g + (size_t)i * G;
        const int s = l / sh.nh, h = l % sh.nh;
        return a.SL + ((t * OZ_S9 + s) * kSlKc + h * 16) * 1024;
    }
    __device__ uint32_t bytes(int, int l) const { return (uint32_t)sh.kc_of(l % sh.nh) * 2048; }
    __device__ int tbuf(int i) const { return i & 1; }
    __device__ int tuse(int i) const { return i >> 1; }
    __device__ bool needs_b(int) const { return true; }
    __device__ int bbuf(int i) const { return i & 1; }
    __device__ int buse(int i) const { return i >> 1; }
    __device__ int b_wait_load(int) const { return 0; }
    __device__ uint32_t tcol_off(int tb) const { return (uint32_t)tb * 64; }
    __device__ int b_off(int bb) const { return bb * 16 * 512; }
    __device__ int first_prep() const { return 0; }
    __device__ int prep_before(int i) const { return i + 1 < ntl ? i + 1 : -1; }
    __device__ int prep_after(int) const { return -1; }
    __device__ void mma(int i, int l, uint32_t aB, uint32_t bB, uint32_t tcol) const {
        // M half h holds k = 128 h .. 128 h + 127; rows beyond the loaded k-chunks are stale integer
        // slices or zeros (the stages are cleared first), and their TMEM lanes are not read
        const int s = l / sh.nh, h = l % sh.nh;
        const uint32_t idesc = idesc_bf16_amn(128, s == 0 ? 32 : 16);
        const uint32_t dc = tcol + (uint32_t)(h * 32 + 2 * s);
        uint64_t ad = sdesc(aB, 128, 2048), bd = sdesc(bB + (uint32_t)b_off(i & 1), 512, 128);
        mma_bf16(dc, ad, bd, idesc, s > 0 ? 1u : 0u);
#pragma unroll
        for (int kk = 1; kk < 8; ++kk) {
            ad += 256 >> 4;
            bd += (2 * 512) >> 4;
            mma_bf16(dc, ad, bd, idesc, 1u);
        }
    }
    __device__ void prep(int i, unsigned char* sB, unsigned char* sX, int t) const {
        int* em = reinterpret_cast<int*>(sX) + 2 * (i & 1);
        if (t < 2) em[t] = 0;
        epi_sync();
        const int64_t r = ((int64_t)g + (int64_t)i * G) * 128 + t;
        const double2 v = r < a.n ? a.w[r] : make_double2(0.0, 0.0);
        atomicMax(&em[0], dexp(v.x));
        atomicMax(&em[1], dexp(v.y));
        epi_sync();
        // row t of B: columns (Re w, Im w), K-major [row chunk][16 slices x 2 columns][8 rows]
        int dr[OZ_S9], di[OZ_S9];
        oz_digits9(oz_fixed63(v.x, em[0] - 1022), dr);
        oz_digits9(oz_fixed63(v.y, em[1] - 1022), di);
        unsigned short* b16 = reinterpret_cast<unsigned short*>(sB);
        const int kc = t >> 3, kk = t & 7;
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            b16[((size_t)kc * 32 + s * 2 + 0) * 8 + kk] = s < OZ_S9 ? bf16_of_int(dr[s]) : 0;
            b16[((size_t)kc * 32 + s * 2 + 1) * 8 + kk] = s < OZ_S9 ? bf16_of_int(di[s]) : 0;
        }
    }
    __device__ void epilogue(int i, uint32_t tcol, unsigned char* sX, int quarter, int lane) {
        const int* em = reinterpret_cast<const int*>(sX) + 2 * (i & 1);
        const int e0 = em[0] - 1022 + 1, e1 = em[1] - 1022 + 1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h >= sh.nh) break;  // uniform over the CTA
            double v0, v1;
            diag_pair(tcol + (uint32_t)(h * 32) + ((uint32_t)(quarter * 32) << 16), v0, v1);
            acc[h][0] += scale2(v0, e0);
            acc[h][1] += scale2(v1, e1);
        }
    }
    // lanes k = 2c and 2c + 1 hold (Re V, Im V) x (Re w, Im w): h_c = sum conj(V) w
    __device__ void finish(unsigned char*, int quarter, int lane) const {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double o0 = __shfl_xor_sync(0xffffffffu, acc[h][0], 1);
            const double o1 = __shfl_xor_sync(0xffffffffu, acc[h][1], 1);
            const int k = h * 128 + quarter * 32 + lane, c = k >> 1;
            if ((lane & 1) == 0 && h < sh.nh && c <= sh.j)
                a.part[(size_t)g * a.ldp + c] = make_double2(acc[h][0] + o1, acc[h][1] - o0);
        }
    }
};

// the stages start zeroed so that the dots' stale k-chunks are integers (see DotPolicy::mma)
template <class P>
__device__ __forceinline__ void clear_stages() {
    extern __shared__ __align__(128) unsigned char ts_smem[];
    uint4* p = reinterpret_cast<uint4*>(ts_smem);
    for (int i = threadIdx.x; i < P::nstages * P::stage_bytes / 16; i += blockDim.x) p[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
}

template <int SA, bool NORM>
__global__ void __launch_bounds__(kTsThreads, 1) k_upd_tc(GsArgs a) {
    UpdPolicy<SA, NORM> p;
    p.a = a;
    p.sh.set(a.jd ? *a.jd : a.j);
    p.g = blockIdx.x;
    p.G = gridDim.x;
    p.ntl = (a.ntiles - p.g + p.G - 1) / p.G;
    p.nrm = 0.0;
    tcstream_body(p, a.st);
}

__global__ void __launch_bounds__(kTsThreads, 1) k_dot_tc(GsArgs a) {
    DotPolicy p;
    p.a = a;
    p.sh.set(a.jd ? *a.jd : a.j);
    p.g = blockIdx.x;
    p.G = gridDim.x;
    p.ntl = (a.ntiles - p.g + p.G - 1) / p.G;
    for (int h = 0; h < 2; ++h) p.acc[h][0] = p.acc[h][1] = 0.0;
    clear_stages<DotPolicy>();
    tcstream_body(p, a.st);
}

int gs_tc_groups(int64_t n) { return std::max(1, std::min((int)((n + 127) / 128), device_sm_count())); }

// w <- w - V h with SA = 9 (first pass) or 6 (second pass, with the norm partial sums)
int gs_update_tc(const unsigned short* SL, int64_t n, const double2* h, double2* w, double* npart, bool second,
                 int j, const int* jd, Status* st, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    const size_t sm9 = tcstream_smem<UpdPolicy<9, false>>(), sm6 = tcstream_smem<UpdPolicy<6, true>>();
    KLST_CK(set_once_per_device(attr, [&] {
        cudaError_t e = cudaFuncSetAttribute(k_upd_tc<9, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm9);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_upd_tc<6, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm6);
        return e;
    }));
    GsArgs a{};
    a.SL = SL; a.n = n; a.ntiles = (int)((n + 127) / 128); a.h = h; a.w = w; a.npart = npart; a.jd = jd; a.j = j;
    a.st = st;
    const int G = gs_tc_groups(n);
    if (second) k_upd_tc<6, true><<<G, kTsThreads, sm6, s>>>(a);
    else k_upd_tc<9, false><<<G, kTsThreads, sm9, s>>>(a);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

// part[g][c] = per-CTA partial sums of V^H w over the step's j + 1 columns (reduced by k_reduce_cols64)
int gs_dots_tc(const unsigned short* SL, int64_t n, const double2* w, double2* part, int ldp, int j, const int* jd,
               Status* st, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    const size_t sm = tcstream_smem<DotPolicy>();
    KLST_CK(set_once_per_device(attr, [&] {
        return cudaFuncSetAttribute(k_dot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    }));
    GsArgs a{};
    a.SL = SL; a.n = n; a.ntiles = (int)((n + 127) / 128); a.w = const_cast<double2*>(w); a.part = part; a.ldp = ldp;
    a.jd = jd; a.j = j; a.st = st;
    k_dot_tc<<<gs_tc_groups(n), kTsThreads, sm, s>>>(a);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

void finish_scale64_split(const double2* h1, const double2* h2, const double* npart, int nparts, double2* S, int lds,
                          double* beta, Status* st, const double2* w, int64_t n, double2* V, double2* vcopy, int col,
                          unsigned short* SL, float2* V32, const int* jd, int nblk, cudaStream_t s) {
    k_finish_scale64_split<<<nblk, 256, 0, s>>>(h1, h2, npart, nparts, S, lds, beta, st, w, n, V, vcopy, col, SL, V32, jd);
    note_launch();
}

}  // namespace klst
