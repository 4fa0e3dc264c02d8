// Float64-accurate Woodbury block solves on the tensor cores (Eq. parShiftInvert in the block form
// z_{c,k} = K_k^{-1} b_{c,k}).
//
// On this part a float64 instruction occupies a warp for 64 cycles whatever the number of active
// lanes, so the complex128 matrix-vector products with the stored K_k^{-1} run at the float64
// pipe's rate (0.28 ms per pass at Nx = 128, Nxi = 1,098) rather than at HBM speed.  Here each
// K_k^{-1} is split once per shift into eight bfloat16 integer slices (the Ozaki scheme of
// oz.cuh: per-row power-of-two scale, balanced base-128 digits), and every solve multiplies the
// slices with the equally split right-hand sides on tcgen05.  Each product of two slices is an
// integer, every diagonal s + t of the 36 kept slice pairs is accumulated exactly in float32 TMEM
// (K = 2 Nx <= 256), and the epilogue combines the eight diagonals with integer operations and one
// float64 rounding.  The result has float64-level error relative to max|K_k^{-1}[j, :]| max|b|.
//
// The real form of one complex block product with two right-hand sides b (g and h components):
//   A = [Re K | Im K]  (Nx x 2Nx),   column pair of B per complex vector v: [Re v; -Im v], [Im v; Re v],
// so C = A B holds (Re z, Im z) of every vector (K = 2 Nx padded with zeros to a multiple of 16).
// A CTA holds two right-hand sides: 8 B columns.
//
// Data movement: the slices (32 B per complex entry, twice the complex128 bytes) are streamed from
// HBM by bulk copies, one 64 KB slice of one block at a time, double buffered and prefetched across
// the block boundary; one CTA per SM walks the blocks k = g, g + G, ...
#include <algorithm>
#include <atomic>

#include "tcstream.cuh"

namespace klst {

constexpr int TC_NB = 8;       // B columns per CTA: 2 right-hand sides x (g, h) x (Re z, Im z)

// rows of [Re K_k^{-1} | Im K_k^{-1}] for the stored transposed inverses KinvT[k][m][j]; row r is
// row j = r mod 128 of block k = r / 128 (rows j >= nx are zero)
struct SrcKinvRows {
    const double2* KinvT;
    int nx, nxi;
    __device__ double operator()(int r, int kk) const {
        const int k = r >> 7, j = r & 127;
        if (k >= nxi || j >= nx || kk >= 2 * nx) return 0.0;
        const int m = kk < nx ? kk : kk - nx;
        const double2 v = KinvT[((size_t)k * nx + m) * nx + j];
        return kk < nx ? v.x : v.y;
    }
};

// reduction length of one block product, 2 nx padded to the MMA's K step (zero entries beyond 2 nx)
static inline int tc_kp(int nx) { return (2 * nx + 15) / 16 * 16; }

size_t tc_kinv_bytes(int nx, int nxi) {
    const int Kp = tc_kp(nx);
    return (size_t)nxi * OZ_S * 128 * Kp * 2 + (size_t)nxi * 128 * sizeof(int);
}

bool tc_solve_supported(int nx) { return nx >= 1 && tc_kp(nx) <= OZ_KMAX; }

// A slices of every block, [k][s][kchunk][128 rows][8], then the row exponents [k * 128 + j]
int tc_split_kinv(const double2* KinvT, int nx, int nxi, void* buf, cudaStream_t s) {
    const int Kp = tc_kp(nx);
    unsigned short* A = (unsigned short*)buf;
    int* ea = (int*)((char*)buf + (size_t)nxi * OZ_S * 128 * Kp * 2);
    SrcKinvRows src{KinvT, nx, nxi};
    k_oz_split_a<SrcKinvRows><<<nxi * 32, 128, 0, s>>>(src, nxi * 128, Kp, A, ea, nullptr);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

struct TcSolveArgs {
    int nx, nxi, Kp, nrhs;
    const unsigned short* As;   // slices of K_k^{-1}
    const int* ea;              // their row exponents
    const double* xi_x;
    int mask;                   // 1: zero the inflow boundary rows of b (B x)
    const double2* b;           // right-hand sides, n complex each, stride ldb
    int64_t ldb;
    const double* w;            // pass 1: w^c_a(j, k), [k][c 4 + a][j]
    double2* tpart;             // pass 1: [rhs][group][4 nx] partial t = V^H z
    int ngroups;
    const double* G;            // pass 2: G^c_a(j, k), [k][c 4 + a][j]
    const double2* sv;          // pass 2: s = C^{-1} t, [rhs][4 nx]
    double2* y;                 // pass 2: result, stride ldb
    int accumulate;
    const int* done;            // optional per right-hand side: skip
    Status* st;
};

// The block solves as a tcstream policy: unit = velocity block k = g + i G; its loads are the
// eight slices of K_k^{-1}, each in one or two K halves of at most 16 k-chunks (32 KB); B holds the
// block's two right-hand sides split into eight slices, stacked along N ([kchunk][slice][8 cols]).
// PASS 1: z = K^{-1} (masked b), running t_a(j) += sum_c w^c_a(j, k) z_c(j) per thread.
// PASS 2: y = K^{-1} (masked b + sum_a G^c_a s_a).
template <int PASS>
struct SolvePolicy {
    static constexpr int stage_bytes = 32 * 1024;
    static constexpr int nstages = 4;
    static constexpr int NT = 2, NBB = 2;                           // double-buffered TMEM and B
    static constexpr int b_total = 2 * 256 * 128;                   // Kp <= 256
    static constexpr int x_bytes = 4 * 128 * 16 + 2 * 4 * 4 + 16;  // sV [4][nx] + exponents [2][4]
    static constexpr uint32_t tmem_alloc = 256;                     // 2 x (9 diagonal blocks x 8 columns)
    TcSolveArgs a;
    int g, G, nblk, nh;      // CTA index, CTA count, its blocks, K halves per slice
    int r0;
    bool on0, on1;
    double2 acc[2][4];       // PASS 1 running sums of t (epilogue threads)

    __device__ int nunits() const { return nblk; }
    __device__ int nloads(int) const { return OZ_S * nh; }
    __device__ int kc_of(int h) const {  // k-chunks of half h
        const int nkc = a.Kp / 8;
        return nh == 1 ? nkc : (h == 0 ? 16 : nkc - 16);
    }
    __device__ const void* src(int i, int l) const {
        const size_t k = (size_t)g + (size_t)i * G;
        const int s = l / nh, h = l % nh;
        return a.As + ((k * OZ_S + s) * (a.Kp / 8) + h * 16) * 1024;
    }
    __device__ uint32_t bytes(int, int l) const { return (uint32_t)kc_of(l % nh) * 2048; }
    __device__ int tbuf(int i) const { return i & 1; }
    __device__ int tuse(int i) const { return i >> 1; }
    __device__ bool needs_b(int) const { return true; }
    __device__ int bbuf(int i) const { return i & 1; }
    __device__ int buse(int i) const { return i >> 1; }
    __device__ uint32_t tcol_off(int tb) const { return (uint32_t)tb * 128; }
    __device__ int b_off(int bb) const { return bb * 256 * 128; }
    __device__ int b_wait_load(int) const { return 0; }
    __device__ int first_prep() const { return 0; }
    __device__ int prep_before(int i) const { return i + 1 < nblk ? i + 1 : -1; }
    __device__ int prep_after(int) const { return -1; }
    __device__ void mma(int i, int l, uint32_t aB, uint32_t bB, uint32_t tcol) const {
        const int s = l / nh, h = l % nh;
        const int cnt = OZ_S - s, np = cnt + (cnt & 1);
        const uint32_t idesc = idesc_bf16(128, np * TC_NB);
        const uint32_t dcol = tcol + (uint32_t)(s * TC_NB);
        const int ksteps = kc_of(h) / 2;
        const uint32_t bh = bB + (uint32_t)b_off(i & 1) + (uint32_t)(h * 16) * (OZ_S * TC_NB * 16);
        // descriptors advance by adding the address step (field = address / 16) to their low bits:
        // the issuing thread then spends a few cycles per MMA instead of rebuilding both
        uint64_t ad = sdesc(aB, 2048, 128), bd = sdesc(bh, OZ_S * TC_NB * 16, 128);
        const uint64_t as = (2 * 2048) >> 4, bs = (2 * OZ_S * TC_NB * 16) >> 4;
        mma_bf16(dcol, ad, bd, idesc, (s > 0 || h > 0) ? 1u : 0u);
#pragma unroll 4
        for (int kk = 1; kk < ksteps; ++kk) {
            ad += as;
            bd += bs;
            mma_bf16(dcol, ad, bd, idesc, 1u);
        }
    }
    __device__ int* emax(unsigned char* sX, int b) const { return reinterpret_cast<int*>(sX + 4 * 128 * 16) + b * 4; }
    __device__ void prep(int i, unsigned char* sB, unsigned char* sX, int t) const {
        const int nx = a.nx, nxi = a.nxi, k = g + i * G, nkc = a.Kp / 8;
        double2* sV = reinterpret_cast<double2*>(sX);
        int* em = emax(sX, i & 1);
        if (t < 4) em[t] = 0;
        epi_sync();
        if (t < nx) {
            const bool bc = a.mask && is_bc(t, nx, a.xi_x[k]);
#pragma unroll
            for (int rl = 0; rl < 2; ++rl)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    double2 v = make_double2(0.0, 0.0);
                    if (rl == 0 ? on0 : on1) {
                        const int rhs = r0 + rl;
                        if (!bc) v = a.b[rhs * a.ldb + ((int64_t)c * nxi + k) * nx + t];
                        if (PASS == 2) {
                            const double* Gk = a.G + (size_t)k * 8 * nx + t;
                            const double2* sr = a.sv + (size_t)rhs * 4 * nx;
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const double gv = Gk[(c * 4 + q) * nx];
                                const double2 sq = sr[q * nx + t];
                                v.x = fma(gv, sq.x, v.x);
                                v.y = fma(gv, sq.y, v.y);
                            }
                        }
                    }
                    sV[(rl * 2 + c) * nx + t] = v;
                    atomicMax(&em[rl * 2 + c], max(dexp(v.x), dexp(v.y)));
                }
        }
        epi_sync();
        for (int item = t; item < nkc * TC_NB; item += kTsEpi) {
            const int c = item & 7, kc = item >> 3;
            const int vec = c >> 1, part = c & 1;
            const int e = em[vec] - 1022;
            const double2* vv = sV + vec * nx;
            int dig[8][OZ_S];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int kk = kc * 8 + q;
                double x = 0.0;
                if (kk < nx) x = part == 0 ? vv[kk].x : vv[kk].y;
                else if (kk < 2 * nx) x = part == 0 ? -vv[kk - nx].y : vv[kk - nx].x;
                oz_digits(oz_fixed(x, e), dig[q]);
            }
#pragma unroll
            for (int s = 0; s < OZ_S; ++s) {
                uint4 wv;
                wv.x = bf16_of_int(dig[0][s]) | ((unsigned)bf16_of_int(dig[1][s]) << 16);
                wv.y = bf16_of_int(dig[2][s]) | ((unsigned)bf16_of_int(dig[3][s]) << 16);
                wv.z = bf16_of_int(dig[4][s]) | ((unsigned)bf16_of_int(dig[5][s]) << 16);
                wv.w = bf16_of_int(dig[6][s]) | ((unsigned)bf16_of_int(dig[7][s]) << 16);
                *reinterpret_cast<uint4*>(sB + ((size_t)(kc * OZ_S + s) * TC_NB + c) * 16) = wv;
            }
        }
    }
    __device__ void epilogue(int i, uint32_t tcol, unsigned char* sX, int quarter, int lane) {
        const int nx = a.nx, nxi = a.nxi, k = g + i * G, j = quarter * 32 + lane;
        float blk[OZ_S][8];
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
#pragma unroll
        for (int d = 0; d < OZ_S; ++d) tmem_ld8(tcol + lane_off + (uint32_t)(d * TC_NB), blk[d]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (j >= nx) return;
        const int* em = emax(sX, i & 1);
        const int era = a.ea[(size_t)k * 128 + j];
        double z[TC_NB];
#pragma unroll
        for (int c = 0; c < TC_NB; ++c) {
            float col[OZ_S];
#pragma unroll
            for (int d = 0; d < OZ_S; ++d) col[d] = blk[d][c];
            z[c] = scale2(oz_combine(col), era + em[c >> 1] - 1022);
        }
#pragma unroll
        for (int rl = 0; rl < 2; ++rl) {
            if (!(rl == 0 ? on0 : on1)) continue;
            const double2 zg = make_double2(z[rl * 4 + 0], z[rl * 4 + 1]);
            const double2 zh = make_double2(z[rl * 4 + 2], z[rl * 4 + 3]);
            if (PASS == 1) {
                const double* wk = a.w + (size_t)k * 8 * nx + j;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double wg = wk[q * nx], wh = wk[(4 + q) * nx];
                    acc[rl][q].x += wg * zg.x + wh * zh.x;
                    acc[rl][q].y += wg * zg.y + wh * zh.y;
                }
            } else {
                double2* yr = a.y + (r0 + rl) * a.ldb;
                const size_t ig = (size_t)k * nx + j, ih = ((size_t)nxi + k) * nx + j;
                if (a.accumulate) {
                    yr[ig] = yr[ig] + zg;
                    yr[ih] = yr[ih] + zh;
                } else {
                    yr[ig] = zg;
                    yr[ih] = zh;
                }
            }
        }
    }
    __device__ void finish(unsigned char*, int quarter, int lane) const {
        if constexpr (PASS == 1) {
            const int j = quarter * 32 + lane;
            if (j >= a.nx) return;
#pragma unroll
            for (int rl = 0; rl < 2; ++rl) {
                if (!(rl == 0 ? on0 : on1)) continue;
                double2* tp = a.tpart + ((size_t)(r0 + rl) * a.ngroups + g) * 4 * a.nx + j;
#pragma unroll
                for (int q = 0; q < 4; ++q) tp[q * a.nx] = acc[rl][q];
            }
        }
    }
};

// one CTA per (k-group, right-hand-side pair); the pair's flags decide before anything is allocated
template <int PASS>
__global__ void __launch_bounds__(kTsThreads, 1) k_solve_tc(TcSolveArgs a) {
    const int r0 = blockIdx.y * 2;
    const bool on0 = r0 < a.nrhs && !(a.done && a.done[r0]);
    const bool on1 = r0 + 1 < a.nrhs && !(a.done && a.done[r0 + 1]);
    if (!on0 && !on1) return;
    SolvePolicy<PASS> p;
    p.a = a;
    p.g = blockIdx.x;
    p.G = gridDim.x;
    p.nblk = (a.nxi - p.g + p.G - 1) / p.G;
    p.nh = a.Kp > 128 ? 2 : 1;
    p.r0 = r0;
    p.on0 = on0;
    p.on1 = on1;
#pragma unroll
    for (int rl = 0; rl < 2; ++rl)
#pragma unroll
        for (int q = 0; q < 4; ++q) p.acc[rl][q] = make_double2(0.0, 0.0);
    tcstream_body(p, a.st);
}

// number of CTAs (k-groups) of the tensor-core passes
int tc_solve_groups(int nxi, int ngroups_cap) { return std::max(1, std::min({nxi, device_sm_count(), ngroups_cap})); }

int tc_solve_pass(int pass, klst_factor f, const double2* b, int mask, double2* y, int accumulate, int nrhs,
                  cudaStream_t s, const int* done) {
    static std::atomic<unsigned long long> attr{0};
    const size_t smem = tcstream_smem<SolvePolicy<1>>();
    KLST_CK(set_once_per_device(attr, [&] {
        cudaError_t e = cudaFuncSetAttribute(k_solve_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_solve_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return e;
    }));
    klst_pencil p = f->p;
    TcSolveArgs a;
    a.nx = p->nx; a.nxi = p->nxi; a.Kp = tc_kp(p->nx); a.nrhs = nrhs;
    a.As = (const unsigned short*)f->kslices;
    a.ea = (const int*)((const char*)f->kslices + (size_t)p->nxi * OZ_S * 128 * a.Kp * 2);
    a.xi_x = p->xi_x; a.mask = mask; a.b = b; a.ldb = p->n;
    a.w = p->w; a.tpart = f->tpart; a.ngroups = tc_solve_groups(p->nxi, f->ngroups);
    a.G = p->G; a.sv = f->sv; a.y = y; a.accumulate = accumulate;
    a.done = done; a.st = f->status;
    dim3 grid(a.ngroups, (nrhs + 1) / 2);
    if (pass == 1) k_solve_tc<1><<<grid, kTsThreads, smem, s>>>(a);
    else k_solve_tc<2><<<grid, kTsThreads, smem, s>>>(a);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

}  // namespace klst
