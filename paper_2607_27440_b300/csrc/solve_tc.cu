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

#include "oz.cuh"

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

size_t tc_solve_smem(int nx) {
    const size_t Kp = tc_kp(nx);
    return 2 * Kp * 256 + Kp * 128 + 4 * (size_t)nx * sizeof(double2);
}

// PASS 1: z = K^{-1} (masked b), accumulating t_a(j) += sum_c w^c_a(j, k) z_c(j) per CTA.
// PASS 2: y = K^{-1} (masked b + sum_a G^c_a s_a).
template <int PASS>
__global__ void __launch_bounds__(128, 1) k_solve_tc(TcSolveArgs a) {
    const int r0 = blockIdx.y * 2;
    const bool on0 = r0 < a.nrhs && !(a.done && a.done[r0]);
    const bool on1 = r0 + 1 < a.nrhs && !(a.done && a.done[r0 + 1]);
    if (!on0 && !on1) return;  // uniform over the CTA, before any allocation
    extern __shared__ __align__(128) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar_ld[2], bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail, s_emax[4];
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int nx = a.nx, nxi = a.nxi, Kp = a.Kp, nkc = Kp / 8;
    const int g = blockIdx.x, Gs = gridDim.x;
    const uint32_t bytesA = (uint32_t)Kp * 256;
    unsigned char* sA[2] = {tc_smem, tc_smem + bytesA};
    unsigned char* sB = tc_smem + 2 * (size_t)bytesA;                  // [kchunk][8 slices][8 cols][16 B]
    double2* sV = reinterpret_cast<double2*>(sB + (size_t)Kp * 128);  // [rhs in pair][g, h][nx]
    constexpr uint32_t kCols = 128;                                    // 9 diagonal blocks x 8 columns
    if (tid == 0) {
        mbar_init(&bar_ld[0], 1);
        mbar_init(&bar_ld[1], 1);
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
    const int nblk = (nxi - g + Gs - 1) / Gs;  // blocks k = g + i Gs
    const int nsl = nblk * OZ_S;               // slices streamed by this CTA, in order
    auto slice_src = [&](int q) {
        const size_t k = (size_t)g + (size_t)(q / OZ_S) * Gs;
        return a.As + ((k * OZ_S + (q % OZ_S)) * nkc) * 1024;
    };
    // thread 0's pipeline state: slice q lives in stage q & 1; its barrier phase is (q >> 1) & 1
    int issued = 0, consumed = 0;
    uint32_t ph_mma = 0;
    if (tid == 0)
        for (; issued < 2 && issued < nsl; ++issued) {
            mbar_expect_tx(&bar_ld[issued], bytesA);
            bulk_g2s(sA[issued], slice_src(issued), bytesA, &bar_ld[issued]);
        }
    double2 acc[2][4];
#pragma unroll
    for (int rl = 0; rl < 2; ++rl)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[rl][q] = make_double2(0.0, 0.0);
    const int j = wid * 32 + lane;  // the output row (TMEM lane) of this thread
    for (int i = 0; i < nblk; ++i) {
        const int k = g + i * Gs;
        // 1. the block's right-hand sides in float64 (sV) and their largest exponents
        if (tid < 4) s_emax[tid] = 0;
        __syncthreads();
        if (tid < nx) {
            const bool bc = a.mask && is_bc(tid, nx, a.xi_x[k]);
#pragma unroll
            for (int rl = 0; rl < 2; ++rl)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    double2 v = make_double2(0.0, 0.0);
                    if (rl == 0 ? on0 : on1) {
                        const int rhs = r0 + rl;
                        if (!bc) v = a.b[rhs * a.ldb + ((int64_t)c * nxi + k) * nx + tid];
                        if (PASS == 2) {
                            const double* Gk = a.G + (size_t)k * 8 * nx + tid;
                            const double2* sr = a.sv + (size_t)rhs * 4 * nx;
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const double gv = Gk[(c * 4 + q) * nx];
                                const double2 s = sr[q * nx + tid];
                                v.x = fma(gv, s.x, v.x);
                                v.y = fma(gv, s.y, v.y);
                            }
                        }
                    }
                    sV[(rl * 2 + c) * nx + tid] = v;
                    atomicMax(&s_emax[rl * 2 + c], max(dexp(v.x), dexp(v.y)));
                }
        }
        __syncthreads();
        // 2. split B = [[Re v, Im v], [-Im v, Re v]] per vector into the stacked slice layout
        for (int item = tid; item < nkc * TC_NB; item += 128) {
            const int c = item & 7, kc = item >> 3;
            const int vec = c >> 1, part = c & 1;
            const int e = s_emax[vec] - 1022;
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
            for (int t = 0; t < OZ_S; ++t) {
                uint4 wv;
                wv.x = bf16_of_int(dig[0][t]) | ((unsigned)bf16_of_int(dig[1][t]) << 16);
                wv.y = bf16_of_int(dig[2][t]) | ((unsigned)bf16_of_int(dig[3][t]) << 16);
                wv.z = bf16_of_int(dig[4][t]) | ((unsigned)bf16_of_int(dig[5][t]) << 16);
                wv.w = bf16_of_int(dig[6][t]) | ((unsigned)bf16_of_int(dig[7][t]) << 16);
                *reinterpret_cast<uint4*>(sB + ((size_t)(kc * OZ_S + t) * TC_NB + c) * 16) = wv;
            }
        }
        // the generic-proxy stores above must be visible to the tensor core's (async proxy) reads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // 3. thread 0: slice s of the block times the stacked B slices t = 0..7-s (padded to an even
        // count; the padding's products land in the unused ninth diagonal block) into blocks s..
        if (tid == 0 && !s_fail) {
            bool ok = true;
            for (int s = 0; s < OZ_S && ok; ++s) {
                const int q = i * OZ_S + s, stg = q & 1;
                ok = mbar_wait(&bar_ld[stg], (uint32_t)((q >> 1) & 1));
                if (!ok) break;
                ++consumed;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int cnt = OZ_S - s, np = cnt + (cnt & 1);
                const uint32_t idesc = idesc_bf16(128, np * TC_NB);
                const uint32_t dcol = tbase + (uint32_t)(s * TC_NB);
                const uint32_t aBase = smem_u32(sA[stg]), bBase = smem_u32(sB);
                for (int kk = 0; kk < Kp / 16; ++kk) {
                    const uint64_t ad = sdesc(aBase + kk * 2 * 2048, 2048, 128);
                    const uint64_t bd = sdesc(bBase + kk * 2 * (OZ_S * TC_NB * 16), OZ_S * TC_NB * 16, 128);
                    mma_bf16(dcol, ad, bd, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(&bar_mma);
                ok = mbar_wait(&bar_mma, ph_mma);
                ph_mma ^= 1;
                if (!ok) break;
                if (issued < nsl) {  // refill this stage with slice q + 2 (possibly of the next block)
                    mbar_expect_tx(&bar_ld[stg], bytesA);
                    bulk_g2s(sA[stg], slice_src(issued), bytesA, &bar_ld[stg]);
                    ++issued;
                }
            }
            if (!ok) {
                s_fail = 1;
                atomicOr(&a.st->flags, ST_TIMEOUT);
                // one more bounded wait for every copy and MMA still in flight before TMEM and the
                // shared buffers are released
                for (int q = consumed; q < issued; ++q) mbar_wait(&bar_ld[q & 1], (uint32_t)((q >> 1) & 1));
                mbar_wait(&bar_mma, ph_mma);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (s_fail) break;
        // 4. epilogue: row j of the block's 8 output columns, exact diagonal sums -> float64
        float blk[OZ_S][8];
        const uint32_t lane_off = (uint32_t)(wid * 32) << 16;
#pragma unroll
        for (int d = 0; d < OZ_S; ++d) tmem_ld8(tbase + lane_off + (uint32_t)(d * TC_NB), blk[d]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (j < nx) {
            const int era = a.ea[(size_t)k * 128 + j];
            double z[TC_NB];
#pragma unroll
            for (int c = 0; c < TC_NB; ++c) {
                float col[OZ_S];
#pragma unroll
                for (int d = 0; d < OZ_S; ++d) col[d] = blk[d][c];
                z[c] = scale2(oz_combine(col), era + s_emax[c >> 1] - 1022);
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
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (PASS == 1 && !s_fail && j < nx) {
#pragma unroll
        for (int rl = 0; rl < 2; ++rl) {
            if (!(rl == 0 ? on0 : on1)) continue;
            double2* tp = a.tpart + ((size_t)(r0 + rl) * a.ngroups + g) * 4 * nx + j;
#pragma unroll
            for (int q = 0; q < 4; ++q) tp[q * nx] = acc[rl][q];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols));
}

// number of CTAs (k-groups) of the tensor-core passes
int tc_solve_groups(int nxi, int ngroups_cap) { return std::max(1, std::min({nxi, device_sm_count(), ngroups_cap})); }

int tc_solve_pass(int pass, klst_factor f, const double2* b, int mask, double2* y, int accumulate, int nrhs,
                  cudaStream_t s, const int* done) {
    static std::atomic<unsigned long long> attr{0};
    if (once_per_device(attr)) {
        // the largest request (Nx = 128); the opt-in limit also covers the kernel's static shared memory
        const int cap = (int)tc_solve_smem(128);
        KLST_CK(cudaFuncSetAttribute(k_solve_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
        KLST_CK(cudaFuncSetAttribute(k_solve_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    }
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
    const size_t smem = tc_solve_smem(p->nx);
    if (pass == 1) k_solve_tc<1><<<grid, 128, smem, s>>>(a);
    else k_solve_tc<2><<<grid, 128, smem, s>>>(a);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

}  // namespace klst
