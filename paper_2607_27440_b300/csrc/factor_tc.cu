// The block inverses K_k^{-1} of the shifted factorisation (Eq. parLUfactor, for the block-diagonal
// part K of A - sigma B = K - U V^H) on the tensor cores.
//
// A complex float32 Gauss-Jordan inverse X_0 of every block (on the float32 pipe), then
// Newton-Schulz steps X <- X + X (I - K X).  With R = I - K X the step gives
// I - K X' = R^2 exactly, so the residual squares each step up to the float64 rounding of R.  Both
// products of a step are float64-accurate Ozaki slice GEMMs on tcgen05 (oz_gemm.cuh):
//   P = D_x X    one GEMM over every block at once: A = the pencil's D_x slices, B = the columns
//                (Re, Im) of all X_k; the epilogue forms R = I - xi_k P - diag(lambda_k) X,
//                lambda_k = nu + i beta xi_y,k - sigma, and R_j = e_j - X_j on the inflow rows
//   Y = X R      batched, one product per block: A = rows of [Re X | Im X], B = columns of
//                [[Re R, Im R], [-Im R, Re R]]; the epilogue writes X' = X + Y
// So the float64 pipe only combines and scales the exact integer products (a few operations per
// output) instead of running the O(Nx^3) elimination.  The float32 inverse of a block with
// condition number kappa has |R| ~ kappa 2^-24; two steps bring it to the float64 level for kappa up
// to ~10^4 (the blocks of the paper's shock pencils have kappa <= 3 10^3).  The largest |R| entry of
// every step is recorded: when the last residual of a block range is above the float64 target the
// range takes two more steps, and when the first residual is too large for the iteration to
// converge (|R| Nx >= 1/2) the range is inverted again by float64 Gauss-Jordan.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>

#include "oz_gemm.cuh"

namespace klst {

template <typename C>
int block_gj_range(klst_factor f, int k0, int nk, C* out, cudaStream_t s);

namespace {

constexpr size_t kNsBudget = size_t(768) << 20;  // scratch bytes of one block range
constexpr int kNsMaxSteps = 6;

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct NsShape {
    int nx, Kp1, Kp2, Np;
    explicit NsShape(int n) : nx(n), Kp1(round_up(n, 16)), Kp2(round_up(2 * n, 16)), Np(round_up(2 * n, OZ_NT)) {}
    size_t xbytes() const { return (size_t)nx * nx * sizeof(double2); }
    size_t b1_bytes(int nk) const {   // B slices of P = D_x X: 2 nx nk columns
        const size_t nt = (size_t)(2 * nx * nk + OZ_NT - 1) / OZ_NT;
        return nt * OZ_NT * (size_t)Kp1 * OZ_S * 2 + nt * OZ_NT * sizeof(int);
    }
    size_t b2_bytes(int nk) const {   // B slices of Y = X R: Np columns per block
        return (size_t)nk * Np * Kp2 * OZ_S * 2 + (size_t)nk * Np * sizeof(int);
    }
    size_t a2_bytes(int nk) const {   // A slices of Y = X R: 128 rows per block
        return (size_t)nk * 128 * Kp2 * OZ_S * 2 + (size_t)nk * 128 * sizeof(int);
    }
    size_t per_range(int nk) const {
        return 2 * nk * xbytes() + std::max(b1_bytes(nk), b2_bytes(nk)) + a2_bytes(nk) + 4 * 256;
    }
};

// blocks per range: as many as kNsBudget of scratch holds (KLST_NS_RANGE=n in the environment: n)
int ns_range_blocks(int nx, int nxi) {
    if (const char* env = getenv("KLST_NS_RANGE")) {
        const int v = atoi(env);
        if (v > 0) return std::min(nxi, v);
    }
    const NsShape sh(nx);
    const size_t per = sh.per_range(1);
    return std::max(1, std::min(nxi, (int)std::min<size_t>(kNsBudget / per, (size_t)1 << 20)));
}

// B of P = D_x X: column col = 2 (block column index) + reim, reduction index = row m of X_k
struct SrcXCols {
    const double* x;   // complex interleaved, column-major blocks [k][i][m]
    int nx, N;
    __device__ double operator()(int col, int kk) const {
        if (col >= N || kk >= nx) return 0.0;
        return x[((size_t)(col >> 1) * nx + kk) * 2 + (col & 1)];
    }
};

// A of Y = X R: row r = 128 k + j of [Re X_k | Im X_k] (zero rows j >= nx)
struct SrcXRows {
    const double2* x;
    int nx, nk;
    __device__ double operator()(int r, int kk) const {
        const int k = r >> 7, j = r & 127;
        if (k >= nk || j >= nx || kk >= 2 * nx) return 0.0;
        const int m = kk < nx ? kk : kk - nx;
        const double2 v = x[((size_t)k * nx + m) * nx + j];
        return kk < nx ? v.x : v.y;
    }
};

// B of Y = X R: column cg = Np k + c of [[Re R_k, Im R_k], [-Im R_k, Re R_k]] (zero columns c >= 2 nx)
struct SrcRCols {
    const double2* R;
    int nx, Np, N;
    __device__ double operator()(int cg, int kk) const {
        if (cg >= N) return 0.0;
        const int k = cg / Np, c = cg - k * Np;
        if (c >= 2 * nx || kk >= 2 * nx) return 0.0;
        const bool imcol = c >= nx, low = kk >= nx;
        const int i = imcol ? c - nx : c, m = low ? kk - nx : kk;
        const double2 v = R[((size_t)k * nx + i) * nx + m];
        return imcol ? (low ? v.x : v.y) : (low ? -v.y : v.x);
    }
};

// Epilogue of P = D_x X: R = I - K X, and the largest |R| entry (its upper 32 bits, which order
// like the value) into *rmax
struct DstResid {
    const double2* X;
    double* R;         // complex interleaved, same layout as X
    const double* xi_x;
    const double* xi_y;
    const double* nu;
    double beta;
    double2 sigma;
    int nx, N;
    unsigned* rmax;
    unsigned m = 0;
    __device__ void operator()(int j, int col, double p) {
        if (j >= nx || col >= N) return;
        const int ci = col >> 1, reim = col & 1;
        const int k = ci / nx, i = ci - k * nx;
        const double xix = xi_x[k];
        const double2 xv = X[(size_t)ci * nx + j];
        const double id = (reim == 0 && i == j) ? 1.0 : 0.0;
        double r;
        if (is_bc(j, nx, xix)) {
            r = id - (reim ? xv.y : xv.x);
        } else {
            const double lr = nu[j] - sigma.x, li = beta * xi_y[k] - sigma.y;
            const double t = reim ? fma(lr, xv.y, li * xv.x) : fma(lr, xv.x, -li * xv.y);
            r = id - fma(xix, p, t);
        }
        R[((size_t)ci * nx + j) * 2 + reim] = r;
        m = max(m, (unsigned)((unsigned long long)__double_as_longlong(fabs(r)) >> 32));
    }
    __device__ void done() {
        const unsigned w = __reduce_max_sync(0xffffffffu, m);
        if ((threadIdx.x & 31) == 0 && w) atomicMax(rmax, w);
    }
};

// Epilogue of Y = X R: X' = X + Y
struct DstXUpd {
    const double* X;
    double* Xn;
    int nx, Np;
    __device__ void operator()(int r, int cg, double y) const {
        const int k = r >> 7, j = r & 127, c = cg - k * Np;
        if (j >= nx || c >= 2 * nx) return;
        const int reim = c >= nx ? 1 : 0, i = c - reim * nx;
        const size_t at = (((size_t)k * nx + i) * nx + j) * 2 + reim;
        Xn[at] = X[at] + y;
    }
    __device__ void done() {}
};

// The complex float32 start X_0 = K_k^{-1}: one CTA per block, Gauss-Jordan with the matrix in
// registers.  Thread t holds row i = t / TPR and the column pairs (2 (t % TPR) + 2 TPR q, +1), so
// the TPR threads of a row read consecutive 16-byte pairs of the pivot row (no bank conflicts).
// Pivoting is implicit: step p pivots on the unused row r_p with the largest |T(r, p)|^2 (compared
// on its leading 25 bits, lowest row on ties) without moving rows; every warp repeats the search on
// the pivot column in shared memory (one packed-key max reduction), with the used rows replicated in
// each thread, and the pivot row's threads publish it unscaled.  In-place update at step p,
// inv = 1 / T(r_p, p):
//   row r_p:  T(r_p, c) <- T(r_p, c) inv,  T(r_p, p) <- inv
//   row i:    f = T(i, p) inv,  T(i, c) <- T(i, c) - f T(r_p, c),  T(i, p) <- -f
// after which K^{-1}(step(i), r_c) = T(i, c), step(r_p) = p; the result is staged in shared memory
// in that order and written out widened to complex128, column-major ([k][m][j] = K^{-1}(j, m)).
// A zero or non-finite pivot column sets *poor to the bit pattern of +inf (the range then takes the
// float64 Gauss-Jordan fallback, which reports a truly singular block).
template <int TPR>   // threads per row
__global__ void __launch_bounds__(128 * TPR, 1)
k_gj32_regs(int nx, double beta, double2 sigma, const double* __restrict__ Dx, const double* __restrict__ xi_x,
            const double* __restrict__ xi_y, const double* __restrict__ nu, double2* __restrict__ out,
            unsigned* __restrict__ poor) {
    constexpr int NP = 64 / TPR, NT = 128 * TPR;    // column pairs per thread, threads
    extern __shared__ __align__(16) float2 stage[];   // [nx][nx]: K^{-1}(j, m) at m nx + j
    __shared__ float2 colp[2][128];
    __shared__ __align__(16) float4 prow[2][64];      // pivot row as column pairs
    __shared__ int s_piv[128], s_step[128];
    const int t = threadIdx.x, i = t / TPR, sub = t % TPR, lane = t & 31;
    const int k = blockIdx.x;
    const bool live = i < nx;
    float4 a[NP];   // pair q: columns 2 (sub + TPR q) and 2 (sub + TPR q) + 1
    {
        const double xix = xi_x[k], xiy = xi_y[k];
        const bool bc = live && is_bc(i, nx, xix);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float v[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = 2 * (sub + TPR * q) + h;
                double re = 0.0, im = 0.0;
                if (live && c < nx) {
                    if (bc) {
                        re = c == i ? 1.0 : 0.0;
                    } else {
                        re = xix * Dx[i * nx + c];
                        if (c == i) { re += nu[i] - sigma.x; im = beta * xiy - sigma.y; }
                    }
                }
                v[2 * h] = (float)re;
                v[2 * h + 1] = (float)im;
            }
            a[q] = make_float4(v[0], v[1], v[2], v[3]);
        }
    }
    unsigned used0 = 0u, used1 = 0u, used2 = 0u, used3 = 0u;
    bool bad = false;
#pragma unroll 1
    for (int p = 0; p < nx; ++p) {
        const int b = p & 1;
        const int owner = (p >> 1) % TPR, qp = (p >> 1) / TPR, hp = p & 1;
        if (live && sub == owner) {
            float4 v = a[0];
#pragma unroll
            for (int q = 1; q < NP; ++q)
                if (q == qp) v = a[q];
            colp[b][i] = hp ? mkf(v.z, v.w) : mkf(v.x, v.y);
        }
        __syncthreads();
        // key = leading bits of |T(r, p)|^2 (non-negative floats order as integers) | 127 - r
        unsigned key = 0u;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int r = lane + 32 * h;
            const unsigned u = h == 0 ? used0 : h == 1 ? used1 : h == 2 ? used2 : used3;
            if (r < nx && !((u >> lane) & 1u)) {
                const float m = abs2(colp[b][r]);
                const unsigned bits = (m >= 0.0f && m <= 3.4e38f) ? (__float_as_uint(m) & ~127u) : 0u;
                key = max(key, (bits | (unsigned)(127 - r)) + 128u);   // + 128: a candidate beats "none"
            }
        }
        key = __reduce_max_sync(0xffffffffu, key);
        int r;
        bool ok;
        if (key >= 128u) {
            key -= 128u;
            r = 127 - (int)(key & 127u);
            ok = (key & ~127u) != 0u;
        } else {
            // no unused row compared (cannot happen while p < nx): the lowest unused row
            r = 0;
            ok = false;
#pragma unroll
            for (int h = 3; h >= 0; --h) {
                const int cnt = min(32, max(0, nx - 32 * h));
                const unsigned u = h == 0 ? used0 : h == 1 ? used1 : h == 2 ? used2 : used3;
                const unsigned fr = ~u & (cnt == 32 ? 0xffffffffu : ((1u << cnt) - 1u));
                if (fr) r = 32 * h + __ffs(fr) - 1;
            }
        }
        const unsigned bit = 1u << (r & 31);
        if ((r >> 5) == 0) used0 |= bit; else if ((r >> 5) == 1) used1 |= bit; else if ((r >> 5) == 2) used2 |= bit; else used3 |= bit;
        if (t == 0) { s_piv[p] = r; s_step[r] = p; }
        bad |= !ok;
        const float2 inv = ok ? cinv(colp[b][r]) : mkf(1.0f, 0.0f);
        if (i == r) {
#pragma unroll
            for (int q = 0; q < NP; ++q) prow[b][sub + TPR * q] = a[q];
        }
        __syncthreads();
        if (i == r) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float2 lo = mkf(a[q].x, a[q].y) * inv, hi = mkf(a[q].z, a[q].w) * inv;
                float4 v = make_float4(lo.x, lo.y, hi.x, hi.y);
                if (q == qp && sub == owner) {
                    if (hp) { v.z = inv.x; v.w = inv.y; } else { v.x = inv.x; v.y = inv.y; }
                }
                a[q] = v;
            }
        } else if (live) {
            const float2 f = colp[b][i] * inv;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float4 pr = prow[b][sub + TPR * q];
                float4 v;
                v.x = a[q].x - (f.x * pr.x - f.y * pr.y);
                v.y = a[q].y - (f.x * pr.y + f.y * pr.x);
                v.z = a[q].z - (f.x * pr.z - f.y * pr.w);
                v.w = a[q].w - (f.x * pr.w + f.y * pr.z);
                if (q == qp && sub == owner) {
                    if (hp) { v.z = -f.x; v.w = -f.y; } else { v.x = -f.x; v.y = -f.y; }
                }
                a[q] = v;
            }
        }
    }
    if (bad && t == 0) atomicMax(poor, 0x7FF00000u);
    __syncthreads();
    if (live) {
        const int j = s_step[i];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int c = 2 * (sub + TPR * q);
            if (c < nx) stage[s_piv[c] * nx + j] = mkf(a[q].x, a[q].y);
            if (c + 1 < nx) stage[s_piv[c + 1] * nx + j] = mkf(a[q].z, a[q].w);
        }
    }
    __syncthreads();
    double2* o = out + (size_t)k * nx * nx;
    for (int e = t; e < nx * nx; e += NT) o[e] = to_d(stage[e]);
}

template <int TPR>
int launch_gj32_t(klst_factor f, int k0, int nk, double2* X, unsigned* poor, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    klst_pencil p = f->p;
    const size_t smem = sizeof(float2) * p->nx * p->nx;
    KLST_CK(set_once_per_device(attr, [] {
        return cudaFuncSetAttribute(k_gj32_regs<TPR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(float2) * 128 * 128));
    }));
    k_gj32_regs<TPR><<<nk, 128 * TPR, smem, s>>>(p->nx, p->desc.beta, f->sigma, p->Dx, p->xi_x + k0, p->xi_y + k0, p->nu,
                                                X, poor);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

// threads per row of the float32 Gauss-Jordan: 4 (512 threads, 2.2 ms for 1,098 blocks of 128 on a
// B300), or 8 with KLST_GJ32_TPR=8 (2.6 ms)
int launch_gj32(klst_factor f, int k0, int nk, double2* X, unsigned* poor, cudaStream_t s) {
    const char* env = getenv("KLST_GJ32_TPR");
    if (env && atoi(env) == 8) return launch_gj32_t<8>(f, k0, nk, X, poor, s);
    return launch_gj32_t<4>(f, k0, nk, X, poor, s);
}

// single_a: one A buffer, so that two CTAs fit on an SM when B and A together take <= 113 KB
template <class Dst>
int launch_gemm(const unsigned short* As, const unsigned short* Bs, const int* ea, const int* eb, int Kp, int ntx,
                int nty, int N, int batched, const Dst& dst, Status* st, cudaStream_t s, bool single_a = false) {
    static std::atomic<unsigned long long> attr{0};
    const size_t bytesB = (size_t)Kp * OZ_NT * 16, bytesA = (size_t)Kp * 256;
    const size_t smem = bytesB + (!single_a && bytesB + 2 * bytesA <= kOzSmemCap ? 2 : 1) * bytesA;
    KLST_CK(set_once_per_device(attr, [] {
        return cudaFuncSetAttribute(k_oz_gemm<Dst>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmemCap);
    }));
    k_oz_gemm<Dst><<<dim3(ntx, nty), 128, smem, s>>>(As, Bs, ea, eb, Kp, dst, st, nullptr, 1, N, batched);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

// One Newton-Schulz step on nk blocks starting at block k0: X (column-major blocks) -> Xn
int ns_step(klst_factor f, const NsShape& sh, int k0, int nk, const double2* X, double2* Xn, double2* R,
            void* bslices, void* aslices, unsigned* rmax, cudaStream_t s) {
    klst_pencil p = f->p;
    const int nx = sh.nx;
    // R = I - K X through P = D_x X over all nk blocks
    prof_begin("factor_ns_resid", s);
    {
        const int N = 2 * nx * nk, nt = (N + OZ_NT - 1) / OZ_NT;
        unsigned short* B = (unsigned short*)bslices;
        int* eb = (int*)((char*)bslices + (size_t)nt * OZ_NT * sh.Kp1 * OZ_S * 2);
        SrcXCols src{reinterpret_cast<const double*>(X), nx, N};
        k_oz_split_b<SrcXCols><<<nt * OZ_NT / 4, 128, 0, s>>>(src, N, sh.Kp1, B, eb, nullptr, 1);
        note_launch();
        KLST_CK_LAUNCH();
        const unsigned short* A = (const unsigned short*)p->dx_oz;
        const int* ea = (const int*)((const char*)p->dx_oz + (size_t)128 * sh.Kp1 * OZ_S * 2);
        DstResid dst{X, reinterpret_cast<double*>(R), p->xi_x + k0, p->xi_y + k0, p->nu, p->desc.beta, f->sigma,
                     nx, N, rmax};
        // one A buffer (96 KB at Nx = 128): two CTAs per SM overlap each other's loads, MMAs and
        // float64 epilogues (3.5 against 5.1 ms for the two steps at Nx = 128, Nxi = 1,098)
        int rc = launch_gemm(A, B, ea, eb, sh.Kp1, nt, 1, N, 0, dst, f->status, s, true);
        if (rc) return rc;
    }
    prof_end("factor_ns_resid", s);
    // X' = X + X R, one product per block
    prof_begin("factor_ns_update", s);
    {
        unsigned short* A = (unsigned short*)aslices;
        int* ea = (int*)((char*)aslices + (size_t)nk * 128 * sh.Kp2 * OZ_S * 2);
        SrcXRows sa{X, nx, nk};
        k_oz_split_a<SrcXRows><<<nk * 32, 128, 0, s>>>(sa, nk * 128, sh.Kp2, A, ea, nullptr);
        note_launch();
        const int N = nk * sh.Np;
        unsigned short* B = (unsigned short*)bslices;
        int* eb = (int*)((char*)bslices + (size_t)N * sh.Kp2 * OZ_S * 2);
        SrcRCols sb{R, nx, sh.Np, N};
        k_oz_split_b<SrcRCols><<<N / 4, 128, 0, s>>>(sb, N, sh.Kp2, B, eb, nullptr, 1);
        note_launch();
        KLST_CK_LAUNCH();
        DstXUpd dst{reinterpret_cast<const double*>(X), reinterpret_cast<double*>(Xn), nx, sh.Np};
        const int rc = launch_gemm(A, B, ea, eb, sh.Kp2, sh.Np / OZ_NT, nk, N, 1, dst, f->status, s);
        prof_end("factor_ns_update", s);
        return rc;
    }
}

double rmax_value(unsigned hi) {
    const unsigned long long b = (unsigned long long)hi << 32;
    double v;
    memcpy(&v, &b, sizeof v);
    return v;
}

}  // namespace

bool ns_inverse_supported(int nx) { return nx >= 1 && round_up(2 * nx, 16) <= OZ_KMAX; }

size_t ns_scratch_bytes(int nx, int nxi) {
    const NsShape sh(nx);
    return sh.per_range(ns_range_blocks(nx, nxi));
}

// Every K_k^{-1} into K64 (column-major complex128 blocks).  info[0] = largest Newton-Schulz step
// count of a block range, info[1] = ranges that fell back to float64 Gauss-Jordan; *rlast = the
// largest |R| entry of the last step over all ranges.
int ns_block_inverses(klst_factor f, double2* K64, cudaStream_t s, int info[2], double* rlast) {
    klst_pencil p = f->p;
    const int nx = p->nx, nxi = p->nxi;
    const NsShape sh(nx);
    const int nkmax = ns_range_blocks(nx, nxi);
    info[0] = info[1] = 0;
    *rlast = 0.0;
    char* buf = nullptr;
    const size_t xb = (size_t)nkmax * sh.xbytes();
    const size_t bsz = std::max(sh.b1_bytes(nkmax), sh.b2_bytes(nkmax));
    cudaError_t e;
    if ((e = dmalloc((void**)&buf, sh.per_range(nkmax), s)) != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    double2* Xb = (double2*)buf;
    double2* R = (double2*)(buf + xb);
    const size_t boff = 2 * xb, aoff = boff + ((bsz + 255) & ~size_t(255));
    const size_t roff = aoff + ((sh.a2_bytes(nkmax) + 255) & ~size_t(255));   // <= per_range - 512
    void* bsl = buf + boff;
    void* asl = buf + aoff;
    unsigned* rmax = (unsigned*)(buf + roff);
    int rc = KLST_OK;
    for (int k0 = 0; k0 < nxi && rc == KLST_OK; k0 += nkmax) {
        const int nk = std::min(nkmax, nxi - k0);
        double2* Xa = K64 + (size_t)k0 * nx * nx;
        cudaMemsetAsync(rmax, 0, sizeof(unsigned) * kNsMaxSteps, s);
        // X_0: complex float32 Gauss-Jordan, widened into Xa
        prof_begin("factor_gj32", s);
        if ((rc = launch_gj32(f, k0, nk, Xa, rmax, s)) != KLST_OK) break;
        prof_end("factor_gj32", s);
        int steps = 0;
        unsigned hr[kNsMaxSteps];
        bool fallback = false;
        while (steps < kNsMaxSteps) {
            // two steps at a time, Xa -> Xb -> Xa
            if ((rc = ns_step(f, sh, k0, nk, Xa, Xb, R, bsl, asl, rmax + steps, s)) != KLST_OK) break;
            if ((rc = ns_step(f, sh, k0, nk, Xb, Xa, R, bsl, asl, rmax + steps + 1, s)) != KLST_OK) break;
            steps += 2;
            if ((e = cudaMemcpyAsync(hr, rmax, sizeof(unsigned) * steps, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess) {
                rc = cuda_fail(e, "newton-schulz sync", __FILE__, __LINE__);
                break;
            }
            const double r0 = rmax_value(hr[0]), rl = rmax_value(hr[steps - 1]);
            if (!(r0 * nx < 0.5)) { fallback = true; break; }   // no guaranteed convergence
            // the residual before the last step bounds the one after it by (nx |R|)^2 plus rounding
            if (rl * nx <= 1e-6) break;
            if (steps >= kNsMaxSteps) { fallback = true; break; }
        }
        if (rc) break;
        if (fallback) {
            prof_begin("factor_gj64", s);
            rc = block_gj_range<double2>(f, k0, nk, Xa, s);
            prof_end("factor_gj64", s);
            if (rc != KLST_OK) break;
            info[1] += 1;
        } else {
            *rlast = std::max(*rlast, rmax_value(hr[steps - 1]));
        }
        info[0] = std::max(info[0], steps);
    }
    dfree(buf, s);
    return rc;
}

}  // namespace klst
