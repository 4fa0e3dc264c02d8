// Shifted factorisation for the shift-and-invert transform (Eqs. parShiftInvert, parLUfactor),
// restated for the structure of the kLST pencil: A - sigma B = K - U V^H with one Nx x Nx block
// K_k per micro-velocity node (shared by g^ and h^) and the rank-4-per-point moment coupling.
// K_k^{-1} by batched Gauss-Jordan with partial pivoting, the capacitance C = I - V^H K^{-1} U
// and C^{-1} by Gauss-Jordan over all SMs, one launch per pivot step.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>

#include "df64.cuh"
#include "factor.cuh"

namespace klst {

template <typename C> struct real_of;
template <> struct real_of<double2> { using type = double; };
template <> struct real_of<float2> { using type = float; };

// One CTA per node k.  Builds M_k = xi_x,k D_x + diag(nu + i beta xi_y,k - sigma) with inflow rows
// replaced by unit rows, inverts it in place by Gauss-Jordan with row pivoting, undoes the
// pivoting by column swaps, and stores K_k^{-1} column-major: out[k][m][j] = (K_k^{-1})_{jm}.
// The working matrix lives in shared memory when it fits, otherwise in the output slot.
template <typename C>
__global__ void __launch_bounds__(256) k_block_gj(int nx, int nxi, double beta, double2 sigma,
                                                  const double* __restrict__ Dx, const double* __restrict__ xi_x,
                                                  const double* __restrict__ xi_y, const double* __restrict__ nu,
                                                  C* __restrict__ out, int use_smem, Status* st) {
    using R = typename real_of<C>::type;
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ C prow[128], pcol[128];
    __shared__ R rv[8];
    __shared__ int ri[8];
    __shared__ int perm[128];
    __shared__ int s_piv;
    const int k = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    C* A = use_smem ? (C*)dsm : out + (size_t)k * nx * nx;
    const double xix = xi_x[k], xiy = xi_y[k];
    for (int idx = tid; idx < nx * nx; idx += nt) {
        int j = idx / nx, m = idx % nx;
        double2 v;
        if (is_bc(j, nx, xix)) v = mk(j == m ? 1.0 : 0.0, 0.0);
        else {
            v = mk(xix * Dx[j * nx + m], 0.0);
            if (j == m) { v.x += nu[j] - sigma.x; v.y += beta * xiy - sigma.y; }
        }
        A[idx] = to_c<C>(v);
    }
    __syncthreads();
    for (int p = 0; p < nx; ++p) {
        // pivot search in column p, rows p..nx-1 (largest |a|^2, lowest row on ties)
        R best = -1;
        int bi = nx;
        for (int i = p + tid; i < nx; i += nt) {
            R v = abs2(A[i * nx + p]);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            R ov = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { rv[tid >> 5] = best; ri[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            R b = rv[0];
            int i0 = ri[0];
            for (int w = 1; w < (nt >> 5); ++w)
                if (rv[w] > b || (rv[w] == b && ri[w] < i0)) { b = rv[w]; i0 = ri[w]; }
            if (!(b > 0)) { atomicOr(&st->flags, ST_SINGULAR); }
            s_piv = i0 < nx ? i0 : p;
            perm[p] = s_piv;
        }
        __syncthreads();
        const int r = s_piv;
        if (r != p)
            for (int c = tid; c < nx; c += nt) { C t = A[p * nx + c]; A[p * nx + c] = A[r * nx + c]; A[r * nx + c] = t; }
        __syncthreads();
        for (int c = tid; c < nx; c += nt) { prow[c] = A[p * nx + c]; pcol[c] = A[c * nx + p]; }
        __syncthreads();
        C inv = prow[p];
        if (!(abs2(inv) > 0)) inv.x = 1;
        inv = cinv(inv);
        for (int idx = tid; idx < nx * nx; idx += nt) {
            int i = idx / nx, c = idx % nx;
            C v;
            if (i == p) v = (c == p) ? inv : prow[c] * inv;
            else {
                C f = pcol[i] * inv;
                v = (c == p) ? -f : A[idx] - f * prow[c];
            }
            A[idx] = v;
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, in reverse order
    for (int p = nx - 1; p >= 0; --p) {
        int q = perm[p];
        if (q != p)
            for (int i = tid; i < nx; i += nt) { C t = A[i * nx + p]; A[i * nx + p] = A[i * nx + q]; A[i * nx + q] = t; }
        __syncthreads();
    }
    // store transposed (column-major)
    C* O = out + (size_t)k * nx * nx;
    if (use_smem) {
        for (int idx = tid; idx < nx * nx; idx += nt) {
            int m = idx / nx, j = idx % nx;
            O[idx] = A[j * nx + m];
        }
    } else {
        for (int idx = tid; idx < nx * nx; idx += nt) {
            int j = idx / nx, m = idx % nx;
            if (j < m) { C t = A[j * nx + m]; A[j * nx + m] = A[m * nx + j]; A[m * nx + j] = t; }
        }
    }
}

// Partial capacitance sums over a k range: Cp[s][(a,j)][(b,j')] = sum_k sum_c w^c_a(j,k) (K_k^{-1})_{jj'} G^c_b(j',k)
template <typename C>
__global__ void __launch_bounds__(256) k_cap_partial(int nx, int nxi, const C* __restrict__ KinvT,
                                                     const double* __restrict__ G, const double* __restrict__ w,
                                                     int kper, double2* __restrict__ Cp) {
    const int j = blockIdx.x * 16 + threadIdx.x, jp = blockIdx.y * 16 + threadIdx.y, sp = blockIdx.z;
    const int r = 4 * nx;
    if (j >= nx || jp >= nx) return;
    double2 acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = mk(0, 0);
    const int k0 = sp * kper, k1 = min(nxi, k0 + kper);
    for (int k = k0; k < k1; ++k) {
        const double2 kin = to_d(KinvT[((size_t)k * nx + jp) * nx + j]);
        const double* wk = w + (size_t)k * 8 * nx;
        const double* Gk = G + (size_t)k * 8 * nx;
        double wg[4], Gg[4], Gh[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) { wg[a] = wk[a * nx + j]; Gg[a] = Gk[a * nx + jp]; Gh[a] = Gk[(4 + a) * nx + jp]; }
        const double whE = wk[7 * nx + j];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                double cf = wg[a] * Gg[b] + (a == 3 ? whE * Gh[b] : 0.0);
                acc[a * 4 + b].x = fma(cf, kin.x, acc[a * 4 + b].x);
                acc[a * 4 + b].y = fma(cf, kin.y, acc[a * 4 + b].y);
            }
    }
    double2* o = Cp + (size_t)sp * r * r;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) o[(size_t)(a * nx + j) * r + b * nx + jp] = acc[a * 4 + b];
}

__global__ void k_cap_reduce(int r, int nsplit, const double2* __restrict__ Cp, double2* __restrict__ Cm) {
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)r * r; idx += gridDim.x * (size_t)blockDim.x) {
        double2 s = mk(0, 0);
        for (int q = 0; q < nsplit; ++q) s = s + Cp[(size_t)q * r * r + idx];
        const size_t i = idx / r, l = idx % r;
        Cm[idx] = mk((i == l ? 1.0 : 0.0) - s.x, -s.y);
    }
}

// Gauss-Jordan inverse of an r x r complex128 matrix (row-major), one launch per pivot step.
// Step p reads buffer p%2 and writes buffer (p+1)%2 (every entry is rewritten), so consecutive
// launches on the stream order the steps without any grid-wide barrier.  Every CTA repeats the
// pivot search on the same column, so all agree on the pivot row; CTA 0 records it.
__global__ void __launch_bounds__(256) k_gj_step(int r, int p, const double2* __restrict__ src, double2* __restrict__ dst,
                                                 int* __restrict__ perm, Status* st) {
    extern __shared__ double2 sh[];
    double2* prow = sh;       // pivot row
    double2* rowp = sh + r;   // row p of the source (moves to the pivot row's slot)
    __shared__ double rv[8];
    __shared__ int ri[8];
    __shared__ int s_piv;
    const int tid = threadIdx.x, nt = blockDim.x;
    double best = -1;
    int bi = r;
    for (int i = p + tid; i < r; i += nt) {
        const double v = abs2(src[(size_t)i * r + p]);
        if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { rv[tid >> 5] = best; ri[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
        double b = rv[0];
        int i0 = ri[0];
        for (int w = 1; w < (nt >> 5); ++w)
            if (rv[w] > b || (rv[w] == b && ri[w] < i0)) { b = rv[w]; i0 = ri[w]; }
        if (!(b > 0) && blockIdx.x == 0) atomicOr(&st->flags, ST_SINGULAR);
        s_piv = i0 < r ? i0 : p;
        if (blockIdx.x == 0) perm[p] = s_piv;
    }
    __syncthreads();
    const int piv = s_piv;
    for (int c = tid; c < r; c += nt) { prow[c] = src[(size_t)piv * r + c]; rowp[c] = src[(size_t)p * r + c]; }
    __syncthreads();
    double2 inv = prow[p];
    if (!(abs2(inv) > 0)) inv.x = 1;
    inv = cinv(inv);
    const int rows_per = (r + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * rows_per, r1 = min(r, r0 + rows_per);
    for (int idx = tid; idx < (r1 - r0) * r; idx += nt) {
        const int i = r0 + idx / r, c = idx % r;
        double2 v;
        if (i == p) v = (c == p) ? inv : prow[c] * inv;
        else {
            const double2 sv = (i == piv) ? rowp[c] : src[(size_t)i * r + c];
            const double2 f = ((i == piv) ? rowp[p] : src[(size_t)i * r + p]) * inv;
            v = (c == p) ? -f : sv - f * prow[c];
        }
        dst[(size_t)i * r + c] = v;
    }
}

// Bounded grid-wide barrier for the cooperative Gauss-Jordan (every CTA of the grid is resident):
// the last CTA to arrive resets the counter and advances the generation; the others poll it with a
// limit, after which the barrier returns false.  Thread 0 of each CTA arrives; the result is
// broadcast to the CTA.
__device__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned& my_gen) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned g = my_gen;
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long it = 0;
            while (*(volatile unsigned*)gen == g) {
                if (++it > (1ll << 24)) { ok = 0; break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        my_gen = g + 1;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The per-pivot Gauss-Jordan of k_gj_step with all r pivots in one cooperative launch: step p reads
// buffer p % 2 (through L2: other CTAs wrote it) and writes buffer (p + 1) % 2, and a grid barrier
// separates the steps instead of a kernel boundary.  Same arithmetic, so the same result.  A barrier
// that gives up sets ST_TIMEOUT and ends the CTA's loop.
__global__ void __launch_bounds__(256) k_gj_coop(int r, double2* __restrict__ b0, double2* __restrict__ b1,
                                                 int* __restrict__ perm, unsigned* __restrict__ barw, Status* st) {
    extern __shared__ double2 sh[];
    double2* prow = sh;
    double2* rowp = sh + r;
    double2* fcol = sh + 2 * r;   // [rows_per]
    __shared__ double rv[8];
    __shared__ int ri[8];
    __shared__ int s_piv;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int rows_per = (r + gridDim.x - 1) / gridDim.x;
    const int r0 = min(r, blockIdx.x * rows_per), r1 = min(r, r0 + rows_per);
    unsigned my_gen = *(volatile unsigned*)(barw + 32);
    for (int p = 0; p < r; ++p) {
        const double2* src = (p & 1) ? b1 : b0;
        double2* dst = (p & 1) ? b0 : b1;
        double best = -1;
        int bi = r;
        for (int i = p + tid; i < r; i += nt) {
            const double v = abs2(__ldcg(src + (size_t)i * r + p));
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { rv[tid >> 5] = best; ri[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            double b = rv[0];
            int i0 = ri[0];
            for (int w = 1; w < (nt >> 5); ++w)
                if (rv[w] > b || (rv[w] == b && ri[w] < i0)) { b = rv[w]; i0 = ri[w]; }
            if (!(b > 0) && blockIdx.x == 0) atomicOr(&st->flags, ST_SINGULAR);
            s_piv = i0 < r ? i0 : p;
            if (blockIdx.x == 0) perm[p] = s_piv;
        }
        __syncthreads();
        const int piv = s_piv;
        for (int c = tid; c < r; c += nt) {
            prow[c] = __ldcg(src + (size_t)piv * r + c);
            rowp[c] = __ldcg(src + (size_t)p * r + c);
        }
        __syncthreads();
        double2 inv = prow[p];
        if (!(abs2(inv) > 0)) inv.x = 1;
        inv = cinv(inv);
        // the multipliers of the CTA's rows, once per row
        if (tid < r1 - r0) {
            const int i = r0 + tid;
            fcol[tid] = ((i == piv) ? rowp[p] : __ldcg(src + (size_t)i * r + p)) * inv;
        }
        __syncthreads();
        for (int i = r0; i < r1; ++i) {
            const double2 f = fcol[i - r0];
            const double2* si = (i == piv) ? rowp : nullptr;
            for (int c = tid; c < r; c += nt) {
                double2 v;
                if (i == p) v = (c == p) ? inv : prow[c] * inv;
                else {
                    const double2 sv = si ? si[c] : __ldcg(src + (size_t)i * r + c);
                    v = (c == p) ? -f : sv - f * prow[c];
                }
                dst[(size_t)i * r + c] = v;
            }
        }
        if (!grid_barrier(barw, barw + 32, my_gen)) {
            if (tid == 0) atomicOr(&st->flags, ST_TIMEOUT);
            return;
        }
    }
}

// Launches k_gj_coop on up to one CTA per SM when the device can hold the whole grid at once
// (cooperative launch); returns false (and launches nothing) otherwise.
static bool launch_gj_coop(int r, double2* b0, double2* b1, int* perm, unsigned* barw, Status* st, cudaStream_t s) {
    static std::mutex mu;
    static int per_sm = -1;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (per_sm < 0) {
            int coop = 0, dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
            int nb = 0;
            if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gj_coop, 256, sizeof(double2) * (2 * 512 + 256)) != cudaSuccess)
                nb = 0;
            per_sm = nb;
            cudaGetLastError();
        }
    }
    int nb = std::max(1, std::min(device_sm_count(), (r + 3) / 4));
    if (per_sm < 1 || r > 512 || (r + nb - 1) / nb > 256) return false;
    const size_t smem = sizeof(double2) * (2 * r + (r + nb - 1) / nb);
    void* args[] = {&r, &b0, &b1, &perm, &barw, &st};
    if (cudaLaunchCooperativeKernel((const void*)k_gj_coop, dim3(nb), dim3(256), args, smem, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    klst::note_launch();
    return true;
}

// The same Gauss-Jordan inverse in one launch of one thread-block cluster of NC CTAs, for
// r <= 384: CTA q keeps rows [q rpc, (q+1) rpc) in shared memory; per pivot the CTAs exchange
// their column-maximum candidates and read the pivot row and row p through distributed shared
// memory, with hardware cluster barriers between the phases (no CTA waits on a flag).  Every
// entry follows the arithmetic of k_gj_step, so the result is identical; the column interchanges
// are undone as the rows are written out.
template <int NC>
__global__ void __launch_bounds__(256) k_gj_cluster(int r, const double2* __restrict__ Cin, double2* __restrict__ Cout,
                                                    Status* st) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank(), tid = threadIdx.x, nt = blockDim.x;
    const int rpc = (r + NC - 1) / NC;
    const int i0 = q * rpc, i1 = min(r, i0 + rpc), nown = max(0, i1 - i0);
    extern __shared__ __align__(16) unsigned char gsm[];
    double2* rows = reinterpret_cast<double2*>(gsm);  // [rpc][r]
    double2* prow = rows + (size_t)rpc * r;           // [r] pivot row
    double2* rowp = prow + r;                         // [r] row p (moves to the pivot row's slot)
    double2* fcol = rowp + r;                         // [rpc] multipliers of the own rows
    __shared__ double cand_v;
    __shared__ int cand_i;
    __shared__ double rv[8];
    __shared__ int ri[8];
    __shared__ int s_piv;
    __shared__ int s_perm[512];
    for (int idx = tid; idx < nown * r; idx += nt) rows[idx] = Cin[(size_t)i0 * r + idx];
    __syncthreads();
    for (int p = 0; p < r; ++p) {
        // this CTA's candidate: the largest |C(i, p)|^2 over its rows i >= p (lowest index on ties)
        double best = -1;
        int bi = r;
        for (int i = max(p, i0) + tid; i < i1; i += nt) {
            const double v = abs2(rows[(size_t)(i - i0) * r + p]);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { rv[tid >> 5] = best; ri[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            double b = rv[0];
            int ib = ri[0];
            for (int w = 1; w < (nt >> 5); ++w)
                if (rv[w] > b || (rv[w] == b && ri[w] < ib)) { b = rv[w]; ib = ri[w]; }
            cand_v = b;
            cand_i = ib;
        }
        cl.sync();
        if (tid == 0) {  // every CTA reduces the NC candidates in the same order
            double b = -1;
            int ib = r;
            for (int k = 0; k < NC; ++k) {
                const double vk = *cl.map_shared_rank(&cand_v, k);
                const int ik = *cl.map_shared_rank(&cand_i, k);
                if (vk > b || (vk == b && ik < ib)) { b = vk; ib = ik; }
            }
            if (!(b > 0) && q == 0) atomicOr(&st->flags, ST_SINGULAR);
            s_piv = ib < r ? ib : p;
            s_perm[p] = s_piv;
        }
        __syncthreads();
        const int piv = s_piv;
        {
            const double2* rp = cl.map_shared_rank(rows, piv / rpc) + (size_t)(piv % rpc) * r;
            const double2* rq = cl.map_shared_rank(rows, p / rpc) + (size_t)(p % rpc) * r;
            for (int c = tid; c < r; c += nt) { prow[c] = rp[c]; rowp[c] = rq[c]; }
        }
        cl.sync();  // every CTA holds its copies before any row changes
        double2 inv = prow[p];
        if (!(abs2(inv) > 0)) inv.x = 1;
        inv = cinv(inv);
        for (int li = tid; li < nown; li += nt) {
            const int i = i0 + li;
            fcol[li] = ((i == piv) ? rowp[p] : rows[(size_t)li * r + p]) * inv;
        }
        __syncthreads();
        for (int idx = tid; idx < nown * r; idx += nt) {
            const int li = idx / r, c = idx % r, i = i0 + li;
            double2 v;
            if (i == p) v = (c == p) ? inv : prow[c] * inv;
            else {
                const double2 sv = (i == piv) ? rowp[c] : rows[idx];
                const double2 f = fcol[li];
                v = (c == p) ? -f : sv - f * prow[c];
            }
            rows[idx] = v;
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges: out[:, c] = rows[:, map[c]]
    __shared__ int colmap[512];
    if (tid == 0) {
        for (int c = 0; c < r; ++c) colmap[c] = c;
        for (int p = r - 1; p >= 0; --p) { const int qq = s_perm[p], t = colmap[p]; colmap[p] = colmap[qq]; colmap[qq] = t; }
    }
    __syncthreads();
    for (int idx = tid; idx < nown * r; idx += nt) {
        const int li = idx / r, c = idx % r;
        Cout[(size_t)(i0 + li) * r + c] = rows[(size_t)li * r + colmap[c]];
    }
    cl.sync();  // no CTA leaves while another may still read its rows
}

template <int NC>
static size_t gj_cluster_smem(int r) {
    const int rpc = (r + NC - 1) / NC;
    return sizeof(double2) * ((size_t)rpc * r + 2 * (size_t)r + rpc);
}

// Launches k_gj_cluster<NC> if one cluster of that shape fits on the device; returns false (and
// launches nothing) otherwise.
template <int NC>
static bool launch_gj_cluster(int r, const double2* Cin, double2* Cout, Status* st, cudaStream_t s) {
    static std::mutex mu;
    static int ok = -1;
    const size_t smem = gj_cluster_smem<NC>(r);
    if (smem > 200 * 1024 || r > 512) return false;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = NC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(NC, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (ok < 0) {
            ok = 0;
            if (cudaFuncSetAttribute(k_gj_cluster<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) == cudaSuccess &&
                (NC <= 8 || cudaFuncSetAttribute(k_gj_cluster<NC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess)) {
                cudaLaunchConfig_t probe = cfg;
                probe.dynamicSmemBytes = 200 * 1024;
                int nclusters = 0;
                if (cudaOccupancyMaxActiveClusters(&nclusters, k_gj_cluster<NC>, &probe) == cudaSuccess && nclusters > 0)
                    ok = 1;
            }
            cudaGetLastError();
        }
    }
    if (!ok) return false;
    if (cudaLaunchKernelEx(&cfg, k_gj_cluster<NC>, r, Cin, Cout, st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    klst::note_launch();
    return true;
}

// Undo the row interchanges as column interchanges (p, perm[p]) for p = r-1..0, as a gather.
__global__ void __launch_bounds__(256) k_gj_unpermute(int r, const double2* __restrict__ fin, double2* __restrict__ res,
                                                      const int* __restrict__ perm) {
    extern __shared__ int idxmap[];
    if (threadIdx.x == 0) {
        for (int c = 0; c < r; ++c) idxmap[c] = c;
        for (int p = r - 1; p >= 0; --p) { const int q = perm[p], t = idxmap[p]; idxmap[p] = idxmap[q]; idxmap[q] = t; }
    }
    __syncthreads();
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)r * r; idx += gridDim.x * (size_t)blockDim.x) {
        const size_t i = idx / r, c = idx % r;
        res[idx] = fin[i * r + idxmap[c]];
    }
}

template <typename C>
static int launch_block_gj(klst_factor f, C* out, cudaStream_t s) {
    klst_pencil p = f->p;
    const size_t bytes = sizeof(C) * p->nx * p->nx;
    const int use_smem = bytes <= 200 * 1024 ? 1 : 0;
    static std::atomic<unsigned long long> attr{0};
    KLST_CK(set_once_per_device(attr, [] {
        return cudaFuncSetAttribute(k_block_gj<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }));
    k_block_gj<C><<<p->nxi, 256, use_smem ? bytes : 0, s>>>(p->nx, p->nxi, p->desc.beta, f->sigma, p->Dx, p->xi_x,
                                                           p->xi_y, p->nu, out, use_smem, f->status); klst::note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

// K_k^{-1} for the blocks k0 .. k0 + nk - 1 into out (column-major, [k - k0][m][j]): float64
// (double2) or the complex float32 start of the tensor-core Newton-Schulz inverse (float2)
template <typename C>
int block_gj_range(klst_factor f, int k0, int nk, C* out, cudaStream_t s) {
    klst_pencil p = f->p;
    const size_t bytes = sizeof(C) * p->nx * p->nx;
    const int use_smem = bytes <= 200 * 1024 ? 1 : 0;
    static std::atomic<unsigned long long> attr{0};
    KLST_CK(set_once_per_device(attr, [] {
        return cudaFuncSetAttribute(k_block_gj<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }));
    k_block_gj<C><<<nk, 256, use_smem ? bytes : 0, s>>>(p->nx, nk, p->desc.beta, f->sigma, p->Dx, p->xi_x + k0,
                                                        p->xi_y + k0, p->nu, out, use_smem, f->status); klst::note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}
template int block_gj_range<double2>(klst_factor, int, int, double2*, cudaStream_t);
template int block_gj_range<float2>(klst_factor, int, int, float2*, cudaStream_t);

template <typename C>
static int launch_cap(klst_factor f, const C* Kinv, double2* Cp, int nsplit, cudaStream_t s) {
    klst_pencil p = f->p;
    const int kper = (p->nxi + nsplit - 1) / nsplit;
    dim3 blk(16, 16), grd((p->nx + 15) / 16, (p->nx + 15) / 16, nsplit);
    k_cap_partial<C><<<grd, blk, 0, s>>>(p->nx, p->nxi, Kinv, p->G, p->w, kper, Cp); klst::note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

// complex128 -> double-float pairs of the block inverses (df64 storage, same bytes)
__global__ void k_split_df(const double2* __restrict__ in, float4* __restrict__ out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += gridDim.x * (size_t)blockDim.x)
        out[i] = cdf_pack(cdf_from(in[i]));
}

// complex128 -> complex64 rounding of the block inverses (mixed precision storage)
__global__ void k_round_c64(const double2* __restrict__ in, float2* __restrict__ out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += gridDim.x * (size_t)blockDim.x) {
        const double2 v = in[i];
        out[i] = mkf((float)v.x, (float)v.y);
    }
}

int factor_reserve(klst_factor f, int nrhs, cudaStream_t s) {
    f->stream = s;
    if (nrhs <= f->nrhs_cap) return KLST_OK;
    dfree(f->tpart, s); dfree(f->t, s); dfree(f->sv, s); dfree(f->bwork, s); dfree(f->rwork, s);
    dfree(f->zwork, s); dfree(f->ozws, s);
    f->zwork = nullptr;
    f->ozws = nullptr;
    dfree(f->normpart, s); dfree(f->done, s); dfree(f->sigma_dev, s);
    f->sigma_dev = nullptr;
    f->tpart = f->t = f->sv = f->bwork = f->rwork = nullptr;
    f->normpart = nullptr;
    f->done = nullptr;
    f->nrhs_cap = 0;
    const size_t r = f->r, n = f->n;
    KLST_CK(dmalloc((void**)&f->tpart, sizeof(double2) * nrhs * (size_t)f->ngroups * r, s));
    KLST_CK(dmalloc((void**)&f->t, sizeof(double2) * nrhs * r, s));
    KLST_CK(dmalloc((void**)&f->sv, sizeof(double2) * nrhs * r, s));
    if (f->precision == KLST_MIXED) {
        KLST_CK(dmalloc((void**)&f->bwork, sizeof(double2) * nrhs * n, s));
        KLST_CK(dmalloc((void**)&f->rwork, sizeof(double2) * nrhs * n, s));
        if (f->tc_resid) {
            KLST_CK(dmalloc((void**)&f->zwork, sizeof(double2) * nrhs * n, s));
            KLST_CK(dmalloc(&f->ozws, oz_dx_ws_bytes(f->nx, f->nxi, nrhs), s));
        }
    }
    KLST_CK(dmalloc((void**)&f->normpart, sizeof(double) * nrhs * 2 * 4096, s));
    KLST_CK(dmalloc((void**)&f->done, sizeof(int) * nrhs, s));
    KLST_CK(dmalloc((void**)&f->sigma_dev, sizeof(double2) * nrhs, s));
    {
        std::vector<double2> sg(nrhs, f->sigma);
        KLST_CK(cudaMemcpyAsync(f->sigma_dev, sg.data(), sizeof(double2) * nrhs, cudaMemcpyHostToDevice, s));
        KLST_CK(cudaStreamSynchronize(s));
    }
    f->nrhs_cap = nrhs;
    return KLST_OK;
}

}  // namespace klst

using namespace klst;

extern "C" void klst_factor_destroy(klst_factor f) {
    if (!f) return;
    cudaStream_t s = f->stream;
    void* bufs[] = {f->KinvT, f->kslices, f->Cinv, f->tpart, f->t, f->sv, f->bwork, f->rwork, f->zwork, f->ozws, f->normpart,
                    f->done, f->sigma_dev, f->worst, f->sweeps, f->status};
    for (void* b : bufs) dfree(b, s);
    delete f;
}

extern "C" int klst_factor_shift(klst_pencil p, double sr, double si, int32_t precision, klst_stream stream,
                                 klst_factor* out) {
    if (!out) { set_error("out is NULL"); return KLST_EINVAL; }
    *out = nullptr;
    if (!p || (precision != KLST_FP64 && precision != KLST_MIXED && precision != KLST_DF64)) {
        set_error("invalid factor arguments");
        return KLST_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    klst_factor f = new klst_factor_s();
    memset(f, 0, sizeof(*f));
    f->p = p;
    f->stream = s;
    f->sigma = mk(sr, si);
    f->precision = precision;
    f->nx = p->nx; f->nxi = p->nxi; f->r = 4 * p->nx; f->n = p->n;
    {
        // block-solve pass 1: one CTA per KB velocity blocks, up to four resident CTAs per SM
        const int KB = 256 / ((p->nx + 31) & ~31);
        f->ngroups = std::max(1, std::min((p->nxi + KB - 1) / KB, 4 * device_sm_count()));
    }
    f->max_refine = 4;
    f->refine_tol = 1e-12;
    {
        // the float64 refinement residual forms its D_x products as float64-accurate tensor-core
        // GEMMs (KLST_NO_TC=1: the float64 CUDA-core rows)
        const char* notc = getenv("KLST_NO_TC");
        f->tc_resid = (precision == KLST_MIXED && p->dx_oz && !(notc && notc[0] == '1')) ? 1 : 0;
        // the float64 block solves multiply integer slices of K_k^{-1} on the tensor cores
        // (KLST_NO_TC=1: complex128 products on the float64 pipe)
        f->tc_solve = (precision == KLST_FP64 && tc_solve_supported(p->nx) && !(notc && notc[0] == '1')) ? 1 : 0;
        // the block inverses: float32 Gauss-Jordan + float64-accurate tensor-core Newton-Schulz steps
        // (KLST_NO_TC=1: float64 Gauss-Jordan)
        f->tc_factor = (p->dx_oz && ns_inverse_supported(p->nx) && !(notc && notc[0] == '1')) ? 1 : 0;
    }
    const int r = f->r;
    const size_t esz = precision == KLST_MIXED ? sizeof(float2) : sizeof(double2);
    const int nsplit = std::max(1, std::min(p->nxi, 8));
    double2 *Cp = nullptr, *b0 = nullptr, *b1 = nullptr;
    int* bar = nullptr;
    auto fail = [&](int code) {
        dfree(Cp, s); dfree(b0, s); dfree(b1, s); dfree(bar, s);
        klst_factor_destroy(f);
        return code;
    };
    cudaError_t e;
#define FALLOC(ptr, bytes)                                                                       \
    if ((e = dmalloc((void**)&(ptr), (bytes), s)) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__)); \
    f->footprint += (int64_t)(bytes);
    FALLOC(f->KinvT, esz * (size_t)p->nxi * p->nx * p->nx);
    if (f->tc_solve) { FALLOC(f->kslices, tc_kinv_bytes(p->nx, p->nxi)); }
    FALLOC(f->Cinv, sizeof(double2) * (size_t)r * r);
    FALLOC(f->worst, sizeof(double));
    FALLOC(f->sweeps, sizeof(int));
    FALLOC(f->status, sizeof(Status));
#undef FALLOC
    if ((e = dmalloc((void**)&Cp, sizeof(double2) * (size_t)nsplit * r * r, s)) != cudaSuccess ||
        (e = dmalloc((void**)&b0, sizeof(double2) * (size_t)r * r, s)) != cudaSuccess ||
        (e = dmalloc((void**)&b1, sizeof(double2) * (size_t)r * r, s)) != cudaSuccess ||
        (e = dmalloc((void**)&bar, sizeof(int) * (r + 128), s)) != cudaSuccess)
        return fail(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    cudaMemsetAsync(f->status, 0, sizeof(Status), s);
    cudaMemsetAsync(f->worst, 0, sizeof(double), s);
    cudaMemsetAsync(f->sweeps, 0, sizeof(int), s);
    // The block inverses are always formed in float64 (the capacitance is built from them); the
    // mixed factor then stores them rounded to complex float32, so the float32 solve carries only
    // the rounding of its operands and not the float32 elimination error.
    double2* K64 = (double2*)f->KinvT;
    if (precision != KLST_FP64) {
        if ((e = dmalloc((void**)&K64, sizeof(double2) * (size_t)p->nxi * p->nx * p->nx, s)) != cudaSuccess)
            return fail(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    }
    auto free64 = [&]() { if (precision != KLST_FP64) dfree(K64, s); };
    int rc;
    if (f->tc_factor) {
        int info[2];
        rc = ns_block_inverses(f, K64, s, info, &f->ns_resid);
        f->ns_steps = info[0];
        f->ns_fallback = info[1];
    } else {
        prof_begin("factor_gj64", s);
        rc = launch_block_gj<double2>(f, K64, s);
        prof_end("factor_gj64", s);
    }
    if (rc) { free64(); return fail(rc); }
    rc = launch_cap<double2>(f, K64, Cp, nsplit, s);
    if (rc) { free64(); return fail(rc); }
    if (f->tc_solve && (rc = tc_split_kinv(K64, p->nx, p->nxi, f->kslices, s)) != KLST_OK) { free64(); return fail(rc); }
    if (precision != KLST_FP64) {
        const size_t cnt = (size_t)p->nxi * p->nx * p->nx;
        const int nb = (int)std::min<size_t>((cnt + 255) / 256, 8192);
        if (precision == KLST_MIXED) k_round_c64<<<nb, 256, 0, s>>>(K64, (float2*)f->KinvT, cnt);
        else k_split_df<<<nb, 256, 0, s>>>(K64, (float4*)f->KinvT, cnt);
        klst::note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) { free64(); return fail(cuda_fail(e, "round", __FILE__, __LINE__)); }
        free64();
    }
    k_cap_reduce<<<std::min(1024, (r * r + 255) / 256), 256, 0, s>>>(r, nsplit, Cp, b0); klst::note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_fail(e, "cap reduce", __FILE__, __LINE__));
    // C^{-1}: one cluster launch when r fits the cluster's shared memory (r <= 384), else one
    // launch per pivot
    bool cluster_done = false;
    if (!getenv("KLST_NO_CLUSTER_GJ")) {
        if (gj_cluster_smem<8>(r) <= 200 * 1024) cluster_done = launch_gj_cluster<8>(r, b0, f->Cinv, f->status, s);
        else if (gj_cluster_smem<16>(r) <= 200 * 1024) cluster_done = launch_gj_cluster<16>(r, b0, f->Cinv, f->status, s);
    }
    if (!cluster_done) {
        const int nb = std::max(1, std::min(device_sm_count(), (r + 3) / 4));
        const size_t smem = sizeof(double2) * 2 * r;
        int* perm = (int*)bar;
        // one cooperative launch with grid barriers between the pivots, else one launch per pivot
        // (KLST_NO_COOP_GJ=1: always per pivot); both give the same result
        unsigned* barw = (unsigned*)(bar + r + 32);   // counter, generation 32 words later
        cudaMemsetAsync(barw, 0, sizeof(unsigned) * 64, s);
        const char* nocoop = getenv("KLST_NO_COOP_GJ");
        if (!(nocoop && nocoop[0] == '1') && launch_gj_coop(r, b0, b1, perm, barw, f->status, s)) {
        } else {
            for (int p = 0; p < r; ++p) {
                k_gj_step<<<nb, 256, smem, s>>>(r, p, (p & 1) ? b1 : b0, (p & 1) ? b0 : b1, perm, f->status);
                klst::note_launch();
            }
        }
        k_gj_unpermute<<<std::min(1024, (r * r + 255) / 256), 256, sizeof(int) * r, s>>>(r, (r & 1) ? b1 : b0,
                                                                                        (r & 1) ? b0 : b1, perm); klst::note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_fail(e, "capacitance inverse", __FILE__, __LINE__));
    }
    if (!cluster_done) {
        double2* res = (r & 1) ? b0 : b1;
        if ((e = cudaMemcpyAsync(f->Cinv, res, sizeof(double2) * (size_t)r * r, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return fail(cuda_fail(e, "copy Cinv", __FILE__, __LINE__));
    }
    Status hst;
    if ((e = cudaMemcpyAsync(&hst, f->status, sizeof(Status), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(cuda_fail(e, "factor sync", __FILE__, __LINE__));
    dfree(Cp, s); dfree(b0, s); dfree(b1, s); dfree(bar, s);
    Cp = b0 = b1 = nullptr;
    bar = nullptr;
    if (hst.flags & ST_SINGULAR) {
        set_error("zero pivot: a shifted block K_k - sigma or the capacitance matrix is singular");
        return fail(KLST_ESINGULAR);
    }
    if (hst.flags & ST_TIMEOUT) {
        set_error("factorisation: a bounded wait of a tensor-core product or a grid barrier gave up");
        return fail(KLST_ETIMEOUT);
    }
    if ((rc = factor_reserve(f, 1, s)) != KLST_OK) return fail(rc);
    f->t_factor_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = f;
    return KLST_OK;
}

extern "C" int klst_factor_inverse_info(klst_factor f, int32_t* method, int32_t* steps, int32_t* fallback, double* resid) {
    if (!f) { set_error("factor is NULL"); return KLST_EINVAL; }
    if (method) *method = f->tc_factor;
    if (steps) *steps = f->ns_steps;
    if (fallback) *fallback = f->ns_fallback;
    if (resid) *resid = f->ns_resid;
    return KLST_OK;
}

extern "C" int klst_factor_info(klst_factor f, double* sr, double* si, int32_t* prec, int64_t* fp, double* tms) {
    if (!f) { set_error("factor is NULL"); return KLST_EINVAL; }
    if (sr) *sr = f->sigma.x;
    if (si) *si = f->sigma.y;
    if (prec) *prec = f->precision;
    if (fp) *fp = f->footprint;
    if (tms) *tms = f->t_factor_ms;
    return KLST_OK;
}

extern "C" int klst_factor_check(klst_factor f, klst_stream stream) {
    if (!f) { set_error("factor is NULL"); return KLST_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    Status hst;
    KLST_CK(cudaMemcpyAsync(&hst, f->status, sizeof(Status), cudaMemcpyDeviceToHost, s));
    KLST_CK(cudaStreamSynchronize(s));
    if (hst.flags & ST_REFINE) {
        const int cleared = hst.flags & ~ST_REFINE;
        KLST_CK(cudaMemcpyAsync(&f->status->flags, &cleared, sizeof(int), cudaMemcpyHostToDevice, s));
        KLST_CK(cudaStreamSynchronize(s));
        set_error("a mixed-precision apply ended its %d refinement sweeps above refine_tol = %g", f->max_refine,
                  f->refine_tol);
        return KLST_EREFINE;
    }
    return KLST_OK;
}

extern "C" int klst_factor_set_refine(klst_factor f, int32_t max_refine, double refine_tol) {
    if (!f || max_refine < 0 || !(refine_tol >= 0)) { set_error("invalid refinement settings"); return KLST_EINVAL; }
    f->max_refine = max_refine;
    f->refine_tol = refine_tol;
    return KLST_OK;
}
