// Krylov-Schur restarted Arnoldi on T = (A - sigma B)^{-1} B (Sec. 4.1, Eq. parShiftInvert):
// basis expansion with the shift-invert apply, classical Gram-Schmidt applied twice (the paper's
// -bv_orthog_type cgs plus a reorthogonalisation: orth64.cu for the float64 basis, the df64
// kernels below for the double-float one), the Schur restart (schur.cu), basis rotation,
// purification and explicit residuals.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "df64.cuh"
#include "factor.cuh"

namespace klst {


// column norm partials: npart[col * nblk + b]
__global__ void k_colnorm_part(const double2* __restrict__ X, int64_t ldx, int64_t n, double* __restrict__ npart) {
    const int col = blockIdx.y;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += abs2(X[col * ldx + i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += red[q];
        npart[(size_t)col * gridDim.x + blockIdx.x] = a;
    }
}

__global__ void k_colnorm_fin(const double* __restrict__ npart, int nblk, int ncols, double* __restrict__ nrm) {
    const int lane = threadIdx.x & 31;
    const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (col >= ncols) return;
    double s = 0;
    for (int b = lane; b < nblk; b += 32) s += npart[(size_t)col * nblk + b];
    s = warp_sum(s);
    if (lane == 0) nrm[col] = sqrt(s);
}

// x *= 1 / scale[col] (column-wise)
__global__ void k_scale_cols(double2* __restrict__ X, int64_t ldx, int64_t n, const double* __restrict__ scale) {
    const int col = blockIdx.y;
    const double sc = scale[col];
    const double inv = sc > 0 ? 1.0 / sc : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = X[col * ldx + i];
        X[col * ldx + i] = mk(v.x * inv, v.y * inv);
    }
}

// Vout[:, c] = sum_l V[:, l] Q[l, c] for c < ncol (8 output columns per block.y)
__global__ void __launch_bounds__(256) k_rotate(const double2* __restrict__ V, int64_t ldv, int m,
                                                const double2* __restrict__ Q, int ldq, int ncol,
                                                double2* __restrict__ Vout, int64_t ldo, int64_t n) {
    extern __shared__ double2 sq[];  // [m][8]
    const int c0 = blockIdx.y * 8;
    for (int idx = threadIdx.x; idx < m * 8; idx += blockDim.x) {
        const int l = idx / 8, c = idx % 8;
        sq[idx] = (c0 + c < ncol) ? Q[(size_t)(c0 + c) * ldq + l] : mk(0, 0);
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = mk(0, 0);
        for (int l = 0; l < m; ++l) {
            const double2 v = V[l * ldv + i];
#pragma unroll
            for (int c = 0; c < 8; ++c) cfma(acc[c], v, sq[l * 8 + c]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c0 + c < ncol) Vout[(c0 + c) * ldo + i] = acc[c];
    }
}

// ---------------------------------------------------------------- double-float (df64) basis
// The Krylov basis is stored as complex df64 (float4) and the Gram-Schmidt projections, updates
// and basis rotations run in df64 arithmetic on the float32 pipes (see df64.cuh).

// Gram-Schmidt in df64, three kernels per pass: chunked dots with per-chunk partials, a reduction
// that also takes the DGKS decision, and the update.
// part[chunk * ldp + col] = sum_{i in chunk} conj(V[i, col]) w[i] (df64) and, in column ncols,
// |w|^2 of the chunk.
__global__ void __launch_bounds__(256, 4) k_dots_df(const float4* __restrict__ V, int64_t ldv, int ncols,
                                                    const double2* __restrict__ w, int64_t n, int chunk,
                                                    float4* __restrict__ part, int ldp, const int* __restrict__ jdev) {
    if (jdev) ncols = *jdev + 1;
    extern __shared__ float4 swf[];
    const int64_t r0 = (int64_t)blockIdx.x * chunk;
    const int len = (int)((n - r0) < chunk ? (n - r0) : chunk);
    for (int i = threadIdx.x; i < len; i += blockDim.x) cdf_store(&swf[i], cdf_from(w[r0 + i]));
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // four columns per warp pass, rows lane + 32 u; two rows per iteration: eight loads in flight
    for (int col = 4 * wid; col < ncols; col += 4 * nw) {
        const int nq = min(4, ncols - col);
        const float4* vc = V + col * ldv + r0;
        cdf a[4] = {cdf_zero(), cdf_zero(), cdf_zero(), cdf_zero()};
        int i = lane;
        for (; i + 32 < len; i += 64) {
            float4 x0[4], x1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                x0[q] = (q < nq) ? vc[q * ldv + i] : z4;
                x1[q] = (q < nq) ? vc[q * ldv + i + 32] : z4;
            }
            const cdf w0 = cdf_load(swf + i), w1 = cdf_load(swf + i + 32);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cdf_fma_conj(a[q], cdf_unpack(x0[q]), w0);
                cdf_fma_conj(a[q], cdf_unpack(x1[q]), w1);
            }
        }
        if (i < len) {
            const cdf w0 = cdf_load(swf + i);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nq) cdf_fma_conj(a[q], cdf_load(vc + q * ldv + i), w0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const cdf t = cdf_warp_sum(a[q]);
            if (lane == 0 && q < nq) part[(size_t)blockIdx.x * ldp + col + q] = cdf_pack(t);
        }
    }
    if (wid == nw - 1) {  // |w|^2 of the chunk
        df s2 = df{0.f, 0.f};
        for (int i = lane; i < len; i += 32) s2 = df_add(s2, cdf_abs2(cdf_load(swf + i)));
        for (int o = 16; o > 0; o >>= 1) s2 = df_add(s2, df_shfl_xor(s2, o));
        if (lane == 0) part[(size_t)blockIdx.x * ldp + ncols] = make_float4(s2.hi, s2.lo, 0.f, 0.f);
    }
}

// acc := w_i + sum_c V[i, c] nh[c] (nh = -h in df64 shared memory) for one row i.  The next four
// basis entries are loaded before the multiply-adds of the current four (two accumulators, even
// and odd columns), so eight loads per thread are in flight.
__device__ __forceinline__ double2 update_row_df(const float4* __restrict__ V, int64_t ldv, int ncols,
                                                 const float4* nh, double2 wi, int64_t i) {
    cdf acc0 = cdf_from(wi), acc1 = cdf_zero();
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 xa[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) xa[u] = (u < ncols) ? V[u * ldv + i] : z4;
    int c = 0;
    for (; c + 4 <= ncols; c += 4) {
        float4 xb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xb[u] = (c + 4 + u < ncols) ? V[(c + 4 + u) * ldv + i] : z4;
        cdf_fma(acc0, cdf_unpack(xa[0]), cdf_load(nh + c));
        cdf_fma(acc1, cdf_unpack(xa[1]), cdf_load(nh + c + 1));
        cdf_fma(acc0, cdf_unpack(xa[2]), cdf_load(nh + c + 2));
        cdf_fma(acc1, cdf_unpack(xa[3]), cdf_load(nh + c + 3));
#pragma unroll
        for (int u = 0; u < 4; ++u) xa[u] = xb[u];
    }
    if (c < ncols) cdf_fma(acc0, cdf_unpack(xa[0]), cdf_load(nh + c));
    if (c + 1 < ncols) cdf_fma(acc1, cdf_unpack(xa[1]), cdf_load(nh + c + 1));
    if (c + 2 < ncols) cdf_fma(acc0, cdf_unpack(xa[2]), cdf_load(nh + c + 2));
    return cdf_to(cdf_add(acc0, acc1));
}

// w -= V h (ncols columns, df64 accumulation).  Two accumulators (even and odd columns) halve
// the dependent chain per row and keep two loads in flight.
__global__ void __launch_bounds__(256) k_update_df(const float4* __restrict__ V, int64_t ldv, int ncols,
                                                   const double2* __restrict__ h, double2* __restrict__ w, int64_t n,
                                                   const int* __restrict__ jdev) {
    if (jdev) ncols = *jdev + 1;
    extern __shared__ float4 shf[];
    for (int i = threadIdx.x; i < ncols; i += blockDim.x) {
        const double2 hv = h[i];
        cdf_store(&shf[i], cdf_from(mk(-hv.x, -hv.y)));
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = update_row_df(V, ldv, ncols, shf, w[i], i);
}

// h[c] = sum over CTAs of part[cta][c] for c < nc (one warp per column, df64, fixed order);
// column nc holds |w|^2: stored in nrm[which].  With second = 1 this is the reorthogonalisation
// pass: the DGKS test (reorthogonalise when ||w'||^2 < ||w||^2 / 2) sets *gate.  h2 is written
// whether or not the gate opens; the consumers read it only when it does.
__global__ void __launch_bounds__(128) k_orth_reduce_df(const float4* __restrict__ part, int nparts, int nc, int ldp,
                                                        double2* __restrict__ h, double* __restrict__ nrm, int second,
                                                        int* __restrict__ gate, int* __restrict__ count,
                                                        const int* __restrict__ jdev) {
    // one CTA of 4 warps per column: each thread sums partials tid, tid + 128, ... (two
    // accumulators), then the warps combine in a fixed order
    if (jdev) nc = *jdev + 1;
    const int col = blockIdx.x;
    if (col > nc) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    cdf a0 = cdf_zero(), a1 = cdf_zero();
    int b = tid;
    for (; b + 128 < nparts; b += 256) {
        const float4 u = part[(size_t)b * ldp + col], v = part[(size_t)(b + 128) * ldp + col];
        a0 = cdf_add(a0, cdf_unpack(u));
        a1 = cdf_add(a1, cdf_unpack(v));
    }
    if (b < nparts) a0 = cdf_add(a0, cdf_unpack(part[(size_t)b * ldp + col]));
    const cdf aw = cdf_warp_sum(cdf_add(a0, a1));
    __shared__ float4 red[4];
    if (lane == 0) red[wid] = cdf_pack(aw);
    __syncthreads();
    if (tid != 0) return;
    const cdf a = cdf_add(cdf_add(cdf_add(cdf_unpack(red[0]), cdf_unpack(red[1])), cdf_unpack(red[2])), cdf_unpack(red[3]));
    if (col < nc) {
        h[col] = cdf_to(a);
        return;
    }
    const double nw2 = df_to(a.re);
    nrm[second] = nw2;
    if (second) {
        const int g = nw2 < 0.5 * nrm[0] ? 1 : 0;
        *gate = g;
        if (g) atomicAdd(count, 1);
    }
}

// Second projection w'' = w' - V h2 (only when the gate is open), then the last CTA to finish
// completes Arnoldi column j: S[0..j, j] = h1 (+ h2), S[j+1, j] = beta = ||w||, breakdown test.
__global__ void __launch_bounds__(256) k_update2_finish_df(const float4* __restrict__ V, int64_t ldv, int nc,
                                                           const double2* __restrict__ h2, double2* __restrict__ w,
                                                           int64_t n, double* __restrict__ npart,
                                                           unsigned* __restrict__ counter, const int* __restrict__ gate,
                                                           const double2* __restrict__ h1, const double* __restrict__ nrm,
                                                           int j, double2* __restrict__ S, int lds,
                                                           double* __restrict__ beta_out, Status* st,
                                                           const int* __restrict__ jdev) {
    if (jdev) { j = *jdev; nc = j + 1; }
    extern __shared__ float4 shf2[];
    __shared__ double red[32];
    __shared__ bool last;
    const int g = *gate;
    if (g) {
        for (int i = threadIdx.x; i < nc; i += blockDim.x) {
            const double2 hv = h2[i];
            cdf_store(&shf2[i], cdf_from(mk(-hv.x, -hv.y)));
        }
        __syncthreads();
        double nr = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            const double2 out = update_row_df(V, ldv, nc, shf2, w[i], i);
            w[i] = out;
            nr += abs2(out);
        }
        nr = warp_sum(nr);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nr;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
            npart[blockIdx.x] = s;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double beta2 = 0.0;
    if (g) {
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(npart + b);
        s = warp_sum(s);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) beta2 += red[q];
    } else {
        beta2 = nrm[1];
    }
    double hn = 0.0;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 hv = g ? h1[i] + h2[i] : h1[i];
        S[(size_t)j * lds + i] = hv;
        hn += abs2(hv);
    }
    hn = warp_sum(hn);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = hn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double hs = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) hs += red[q];
        const double beta = sqrt(beta2);
        if (!(beta > 1e-13 * sqrt(hs))) atomicOr(&st->flags, ST_BREAKDOWN);
        S[(size_t)j * lds + j + 1] = mk(beta, 0.0);
        *beta_out = beta;
        *counter = 0u;
    }
}

// step index of a captured Arnoldi step: set before a cycle, advanced after each step
__global__ void k_set_step(int* jdev, int v) { *jdev = v; }
__global__ void k_step_advance(int* jdev) { *jdev += 1; }

// basis column = w / scale (df64) and the float64 copy that feeds the next apply
// (with jdev: vcol is the basis and the column is jdev[0] + 1)
__global__ void k_scale_df(const double2* __restrict__ w, int64_t n, const double* __restrict__ scale,
                           float4* __restrict__ vcol, double2* __restrict__ vcopy, int64_t ldv,
                           const int* __restrict__ jdev) {
    if (jdev) vcol += (int64_t)(*jdev + 1) * ldv;
    __shared__ double s_inv;  // one float64 division per CTA, not per thread
    if (threadIdx.x == 0) {
        const double sc = *scale;
        s_inv = sc > 0 ? 1.0 / sc : 0.0;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = mk(w[i].x * inv, w[i].y * inv);
        cdf_store(vcol + i, cdf_from(v));
        vcopy[i] = v;
    }
}

// Vout[:, c] = sum_l V[:, l] Q[l, c] for c < ncol, V in df64; output df64 (float4) or float64 (double2)
template <typename O>
__global__ void __launch_bounds__(256) k_rotate_df(const float4* __restrict__ V, int64_t ldv, int m,
                                                   const double2* __restrict__ Q, int ldq, int ncol,
                                                   O* __restrict__ Vout, int64_t ldo, int64_t n) {
    extern __shared__ float4 sqf[];  // [m][8]
    const int c0 = blockIdx.y * 8;
    for (int idx = threadIdx.x; idx < m * 8; idx += blockDim.x) {
        const int l = idx / 8, c = idx % 8;
        cdf_store(&sqf[idx], cdf_from((c0 + c < ncol) ? Q[(size_t)(c0 + c) * ldq + l] : mk(0, 0)));
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        cdf acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = cdf_zero();
        for (int l = 0; l < m; ++l) {
            const cdf v = cdf_load(V + l * ldv + i);
#pragma unroll
            for (int c = 0; c < 8; ++c) cdf_fma(acc[c], v, cdf_load(sqf + l * 8 + c));
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (c0 + c >= ncol) continue;
            if constexpr (sizeof(O) == sizeof(float4) && alignof(O) == 16 && std::is_same<O, float4>::value)
                cdf_store(Vout + (c0 + c) * ldo + i, acc[c]);
            else
                Vout[(c0 + c) * ldo + i] = cdf_to(acc[c]);
        }
    }
}

// Seeded complex Gaussian start vector (splitmix64 counter hash + Box-Muller).
__device__ __forceinline__ uint64_t splitmix(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__global__ void k_randn(double2* x, int64_t n, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = splitmix(seed * 0x100000001b3ull + 2 * i), b = splitmix(seed * 0x100000001b3ull + 2 * i + 1);
        const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0), u2 = (b >> 11) * (1.0 / 9007199254740992.0);
        const double r = sqrt(-2.0 * log(u1));
        x[i] = mk(r * cospi(2.0 * u2), r * sinpi(2.0 * u2));
    }
}

// Carves 256-byte-aligned arrays out of one allocation: a first pass (base == NULL) only sums
// the sizes, a second assigns the pointers.
struct SlabCarver {
    char* base = nullptr;
    size_t off = 0;
    template <typename T>
    void take(T*& p, size_t cnt) {
        const size_t bytes = (sizeof(T) * cnt + 255) & ~size_t(255);
        p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += bytes;
    }
};

struct EigsWork {
    double2 *Va = nullptr, *Vb = nullptr, *S = nullptr, *H = nullptr, *Q = nullptr, *Yc = nullptr, *mu = nullptr;
    double2 *Ysel = nullptr, *musel = nullptr, *Vh = nullptr;
    double *estsel = nullptr, *tau = nullptr;
    Rot *rlog = nullptr, *rlog2 = nullptr;
    int *rcount = nullptr, *loff = nullptr, *rdy = nullptr;
    double* npart2 = nullptr;
    int *gate = nullptr, *reorth = nullptr;
    double2 *h = nullptr, *dpart = nullptr, *X = nullptr, *Z = nullptr, *R = nullptr, *om = nullptr;
    double2 *wbuf = nullptr, *vcur = nullptr;
    char* ozws = nullptr;         // float64 basis: workspace of the tensor-core rotation
    unsigned short* sl = nullptr; // float64 basis: its integer slices (tensor-core Gram-Schmidt)
    float2* v32 = nullptr;        // float64 basis truncated to complex float32 (first-pass coefficients)
    double2 *mw = nullptr, *mp = nullptr;
    double *est = nullptr, *npart = nullptr, *beta = nullptr, *nrm = nullptr;
    int* nconv = nullptr;
    float4* opart = nullptr;      // df64 Gram-Schmidt: per-chunk partial dots [nchunks][m + 2]
    double* onrm = nullptr;       // ||w||^2, ||w'||^2
    unsigned* ocnt = nullptr;     // last-CTA counter of k_update2_finish_df
    int* jdev = nullptr;          // graph mode: device step index
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // graph mode: one captured step per basis buffer
    double2* gV[2] = {nullptr, nullptr};
    int gkern[2] = {0, 0};
    std::vector<cudaEvent_t> evs;
    void* slab = nullptr;         // one allocation holding every array above except X, Z, R
    void release(cudaStream_t st) {
        void* b[] = {slab, X, Z, R};
        for (void* p : b) dfree(p, st);
        for (auto& ge : gexec)
            if (ge) { cudaGraphExecDestroy(ge); ge = nullptr; }
        for (auto& ev : evs)
            if (ev) cudaEventDestroy(ev);
        evs.clear();
    }
};

}  // namespace klst

using namespace klst;

namespace klst {
// The option rules of klst_eigs, shared with the batch and serving entry points so that a bad
// request is rejected before any buffer is sized from it.
int validate_eigs_opts(const klst_eigs_opts* o, int64_t n) {
    const int nev = o->nev, m = o->ncv;
    if (nev < 1 || m < nev + 2 || m > 160 || (int64_t)m + 1 > n || o->max_restarts < 0 || o->max_refine < 0 ||
        !(o->tol > 0)) {
        set_error("invalid eigs options nev=%d ncv=%d (need 1 <= nev, nev+2 <= ncv <= min(160, n-1))", nev, m);
        return KLST_EINVAL;
    }
    if (o->keep != 0 && (o->keep < nev || o->keep >= m)) {
        set_error("invalid keep=%d (need nev <= keep < ncv)", o->keep);
        return KLST_EINVAL;
    }
    if (o->arith != KLST_ARITH_F64 && o->arith != KLST_ARITH_DF64) {
        set_error("invalid arith=%d", o->arith);
        return KLST_EINVAL;
    }
    if (o->conv != KLST_CONV_REL && o->conv != KLST_CONV_RESID) {
        set_error("invalid conv=%d", o->conv);
        return KLST_EINVAL;
    }
    return KLST_OK;
}
}  // namespace klst

extern "C" int klst_eigs(klst_factor f, const klst_eigs_opts* o, double* evals_host, void* evecs, double* resid_host,
                         klst_eigs_info* info, klst_stream stream) {
    if (!f || !o || !evals_host) { set_error("invalid arguments to klst_eigs"); return KLST_EINVAL; }
    const int nev = o->nev, m = o->ncv;
    if (int vrc = validate_eigs_opts(o, f->n)) return vrc;
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    klst_pencil p = f->p;
    const int64_t n = f->n;
    const int lds = m + 1;
    const int sms = device_sm_count();
    int chunk = 256;
    while ((n + chunk - 1) / chunk > 4 * sms && chunk < 2048) chunk *= 2;
    const int nchunks = (int)((n + chunk - 1) / chunk);
    const int nblk = std::min<int64_t>((n + 255) / 256, 6 * sms);  // 6 resident 256-thread CTAs per SM
    const int nupd = std::min<int64_t>((n + 255) / 256, 4 * sms);  // df64 updates: 64 registers, 4 CTAs per SM
    const int ng = pencil_work_groups(p);
    const int keep = o->keep ? o->keep : std::min(m - 1, nev + (m - nev) / 2);
    const int prev_refine = f->max_refine, prev_arith = f->arith;
    const double prev_rtol = f->refine_tol;
    f->max_refine = o->max_refine;
    f->arith = o->arith == KLST_ARITH_DF64 ? 1 : 0;
    if (o->refine_tol > 0) f->refine_tol = o->refine_tol;
    EigsWork W;
    cudaError_t e;
    int rc = KLST_OK;
    auto fail = [&](int code) {
        W.release(s);
        f->max_refine = prev_refine;
        f->refine_tol = prev_rtol;
        f->arith = prev_arith;
        return code;
    };
    // the whole workspace is one stream-ordered allocation: concurrent solves on many host
    // threads otherwise queue on the allocator for dozens of small arrays each
    const bool dfm = o->arith == KLST_ARITH_DF64;
    // float64 basis: the basis rotations run as float64-accurate tensor-core GEMMs (2 ncv <= 256;
    // KLST_NO_TC=1 selects the float64 CUDA-core rotation)
    const char* notc = getenv("KLST_NO_TC");
    const bool use_tc = !dfm && 2 * m <= 256 && n <= 0x7FFFFFFF && !(notc && notc[0] == '1');
    // the float64 Gram-Schmidt products on the tensor cores (basis slices, 2 (m + 1) <= 256)
    const bool use_tcgs = use_tc && basis_slices_supported(m);
    const int gs_groups = gs_tc_groups(n);
    const int ldp = m + 2;
    const int log_cap = 31 * m * m;
    {
        SlabCarver sc;
        for (int pass = 0; pass < 2; ++pass) {
            sc.off = 0;
            sc.take(W.Va, n * (m + 1));
            sc.take(W.Vb, n * (m + 1));
            sc.take(W.S, (size_t)lds * m);
            sc.take(W.H, (size_t)m * m);
            sc.take(W.Q, (size_t)m * m);
            sc.take(W.Yc, (size_t)m * m);
            sc.take(W.Ysel, (size_t)m * nev);
            sc.take(W.mu, m);
            sc.take(W.musel, nev);
            sc.take(W.est, m);
            sc.take(W.estsel, nev);
            sc.take(W.Vh, (size_t)m * m);
            sc.take(W.tau, m);
            sc.take(W.rlog, log_cap);
            sc.take(W.rcount, 4);
            if (!dfm) {
                sc.take(W.rlog2, log_cap);
                sc.take(W.loff, (size_t)log_cap + 1);
                sc.take(W.rdy, 256);
            }
            sc.take(W.npart2, std::max({nblk, gs_groups, 1}));
            sc.take(W.gate, 4);
            sc.take(W.reorth, 4);
            sc.take(W.h, 2 * (m + 1));
            sc.take(W.dpart, (size_t)std::max(nchunks, gs_groups) * (m + 1));
            if (use_tcgs) {
                sc.take(W.sl, basis_slices_bytes(n) / sizeof(unsigned short));
                sc.take(W.v32, (size_t)n * (m + 1));
            }
            sc.take(W.npart, (size_t)std::max(nblk, 1) * std::max(nev, 1) + 64);
            sc.take(W.beta, 4);
            sc.take(W.nrm, nev + 4);
            sc.take(W.nconv, 4);
            sc.take(W.om, nev);
            sc.take(W.mw, (size_t)4 * p->nx * nev);
            sc.take(W.mp, (size_t)4 * p->nx * ng * nev);
            sc.take(W.wbuf, n);
            sc.take(W.vcur, n);
            sc.take(W.jdev, 4);
            if (dfm) {
                sc.take(W.opart, (size_t)nchunks * ldp);
                sc.take(W.onrm, 4);
                sc.take(W.ocnt, 4);
            }
            if (use_tc) sc.take(W.ozws, oz_workspace_bytes((int)n, 2 * std::max(keep, nev), 2 * m));
            if (pass == 0) {
                if ((e = dmalloc(&W.slab, sc.off, s)) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
                sc.base = static_cast<char*>(W.slab);
            }
        }
    }
    KLST_CK(cudaMemsetAsync(W.S, 0, sizeof(double2) * lds * m, s));
    KLST_CK(cudaMemsetAsync(W.reorth, 0, sizeof(int) * 4, s));
    KLST_CK(cudaMemsetAsync(W.rcount, 0, sizeof(int) * 4, s));
    KLST_CK(cudaMemsetAsync(f->status, 0, sizeof(Status), s));
    KLST_CK(cudaMemsetAsync(f->worst, 0, sizeof(double), s));
    KLST_CK(cudaMemsetAsync(f->sweeps, 0, sizeof(int), s));
    if ((rc = factor_reserve(f, std::max(nev, 1), s)) != KLST_OK) return fail(rc);
    double2 *V = W.Va, *Valt = W.Vb;
    // df64 mode: the basis is complex df64 (float4, same bytes); the apply works on float64
    // vectors wbuf (output) and vcur (the newest basis vector in float64)
    double2* wbuf = W.wbuf;
    double2* vcur = W.vcur;
    auto V4 = [&](double2* p0) { return reinterpret_cast<float4*>(p0); };
    if (dfm) KLST_CK(cudaMemsetAsync(W.ocnt, 0, sizeof(unsigned) * 4, s));
    // start: v0 (given or seeded), V[:,0] = T v0 / ||T v0|| (range of T: no B-null components)
    double2* v0 = Valt;
    if (o->v0) KLST_CK(cudaMemcpyAsync(v0, o->v0, sizeof(double2) * n, cudaMemcpyDeviceToDevice, s));
    else { k_randn<<<nblk, 256, 0, s>>>(v0, n, o->seed); klst::note_launch(); }
    int applies = 0;
    if ((rc = apply_T(f, v0, wbuf, 1, s)) != KLST_OK) return fail(rc);
    ++applies;
    k_colnorm_part<<<dim3(nblk, 1), 256, 0, s>>>(wbuf, n, n, W.npart); klst::note_launch();
    k_colnorm_fin<<<1, 256, 0, s>>>(W.npart, nblk, 1, W.nrm); klst::note_launch();
    if (dfm) { k_scale_df<<<nblk, 256, 0, s>>>(wbuf, n, W.nrm, V4(V), vcur, n, nullptr); klst::note_launch(); }
    else { k_scale64_ext(wbuf, n, W.nrm, V, vcur, n, nblk, s); }
    KLST_CK_LAUNCH();
    if (use_tcgs) {
        KLST_CK(cudaMemsetAsync(W.sl, 0, basis_slices_bytes(n), s));
        if ((rc = split_basis(V, n, 0, 1, W.sl, W.v32, s)) != KLST_OK) return fail(rc);
    }
    // phase timers: event pairs recorded per step (eager launches) or per cycle (graph mode) and
    // read after each restart synchronisation; created below once the mode is known
    W.evs.assign(3 * (m + 1) + 4, nullptr);
    std::vector<cudaEvent_t>& evs = W.evs;
    double t_apply = 0, t_orth = 0, t_restart = 0, t_schur = 0;
    int k = 0, restarts = 0, nconv = 0;
    const size_t dots_smem = sizeof(double2) * chunk;
    const size_t upd_smem = sizeof(double2) * (m + 1);
    // df64 Gram-Schmidt of step j (jd != NULL: the kernels read j from device memory, the grids
    // are sized for j = m - 1)
    auto df_orth = [&](double2* Vb, int j, const int* jd) -> int {
        const int nc = j + 1;
        const int nred = nc + 1;  // one CTA per column and one for |w|^2
        double2* w = wbuf;
        prof_begin("orth1_df", s);
        k_dots_df<<<nchunks, 256, dots_smem, s>>>(V4(Vb), n, nc, w, n, chunk, W.opart, ldp, jd); klst::note_launch();
        k_orth_reduce_df<<<nred, 128, 0, s>>>(W.opart, nchunks, nc, ldp, W.h, W.onrm, 0, nullptr, nullptr, jd); klst::note_launch();
        k_update_df<<<nupd, 256, upd_smem, s>>>(V4(Vb), n, nc, W.h, w, n, jd); klst::note_launch();
        prof_end("orth1_df", s);
        prof_begin("orth2_dots_df", s);
        k_dots_df<<<nchunks, 256, dots_smem, s>>>(V4(Vb), n, nc, w, n, chunk, W.opart, ldp, jd); klst::note_launch();
        k_orth_reduce_df<<<nred, 128, 0, s>>>(W.opart, nchunks, nc, ldp, W.h + (m + 1), W.onrm, 1, W.gate, W.reorth, jd); klst::note_launch();
        prof_end("orth2_dots_df", s);
        prof_begin("orth2_update_df", s);
        k_update2_finish_df<<<nupd, 256, upd_smem, s>>>(V4(Vb), n, nc, W.h + (m + 1), w, n, W.npart2, W.ocnt, W.gate,
                                                        W.h, W.onrm, j, W.S, lds, W.beta, f->status, jd); klst::note_launch();
        prof_end("orth2_update_df", s);
        prof_begin("orth_scale", s);
        k_scale_df<<<nblk, 256, 0, s>>>(w, n, W.beta, jd ? V4(Vb) : V4(Vb) + (int64_t)(j + 1) * n, vcur, n, jd); klst::note_launch();
        prof_end("orth_scale", s);
        KLST_CK_LAUNCH();
        return KLST_OK;
    };
    // float64 basis: classical Gram-Schmidt twice, first-pass coefficients on the float32 pipes
    Orth64Args oa;
    oa.n = n; oa.m = m; oa.w = wbuf; oa.vcur = vcur; oa.chunk = chunk; oa.nchunks = nchunks; oa.ldp = m + 1;
    oa.part = W.dpart; oa.h1 = W.h; oa.h2 = W.h + (m + 1); oa.nupd = nblk; oa.npart = W.npart2; oa.nscale = nblk;
    oa.S = W.S; oa.lds = lds; oa.beta = W.beta; oa.st = f->status;
    oa.sl = use_tcgs ? W.sl : nullptr; oa.v32 = W.v32; oa.ntc = gs_groups;
    auto f64_orth = [&](double2* Vb, int j, const int* jd) -> int {
        oa.V = Vb;
        return orth64_step(oa, j, jd, s);
    };
    // Graph mode (df64 basis on a capturable stream): one Arnoldi step (apply, Gram-Schmidt, step
    // advance) is captured once per basis buffer and launched as a single graph per step, which
    // removes the host cost of its ~11 kernel launches.  Not used on the legacy default stream, on
    // a stream that is already capturing, or while kernel-group timing is on.
    bool use_graph = false;
    if (!prof_enabled() && s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread) {
        const char* ng = getenv("KLST_NO_GRAPH");
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (!(ng && ng[0] == '1') && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
            use_graph = true;
        cudaGetLastError();
    }
    auto capture_step = [&](double2* Vb, cudaGraphExec_t* ge, int* nkern) -> int {
        cudaGraph_t g = nullptr;
        cudaError_t e1 = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e1 != cudaSuccess) return cuda_fail(e1, "cudaStreamBeginCapture", __FILE__, __LINE__);
        set_capturing(true);
        int rc2 = apply_T(f, vcur, wbuf, 1, s);
        if (rc2 == KLST_OK) rc2 = dfm ? df_orth(Vb, m - 1, W.jdev) : f64_orth(Vb, m - 1, W.jdev);
        if (rc2 == KLST_OK) k_step_advance<<<1, 1, 0, s>>>(W.jdev);
        set_capturing(false);
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (rc2 != KLST_OK || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc2 != KLST_OK ? rc2 : cuda_fail(e2, "cudaStreamEndCapture", __FILE__, __LINE__);
        }
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
        int kern = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kern;
        }
        e2 = cudaGraphInstantiate(ge, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) { *ge = nullptr; return cuda_fail(e2, "cudaGraphInstantiate", __FILE__, __LINE__); }
        *nkern = kern;
        return KLST_OK;
    };
    // graph mode times a whole cycle (events 0, 1); eager mode every step; both time the restart
    for (int i = 0; i < (int)evs.size(); ++i) {
        if (use_graph && i > 1 && i < 3 * (m + 1)) continue;
        if ((e = cudaEventCreate(&evs[i])) != cudaSuccess) return fail(cuda_fail(e, "cudaEventCreate", __FILE__, __LINE__));
    }
    bool converged = false;
    int f64_steps = 0;  // float64 basis: every step runs both Gram-Schmidt passes
    int64_t schur_rot = 0;
    int schur_sweeps = 0, schur_swaps = 0;
    for (;;) {
        const int jfirst = k;
        if (use_graph) {
            // the whole expansion of this cycle: one graph launch per Arnoldi step
            int slot = (V == W.gV[0]) ? 0 : (V == W.gV[1]) ? 1 : -1;
            if (slot < 0) {
                slot = W.gexec[0] ? 1 : 0;
                if ((rc = capture_step(V, &W.gexec[slot], &W.gkern[slot])) != KLST_OK) return fail(rc);
                W.gV[slot] = V;
            }
            cudaEventRecord(evs[0], s);
            k_set_step<<<1, 1, 0, s>>>(W.jdev, k); klst::note_launch();
            for (int j = k; j < m; ++j) {
                KLST_CK(cudaGraphLaunch(W.gexec[slot], s));
                klst::note_launches(W.gkern[slot]);
            }
            cudaEventRecord(evs[1], s);
            applies += m - k;
        }
        for (int j = use_graph ? m : k; j < m; ++j) {
            cudaEventRecord(evs[3 * j], s);
            if ((rc = apply_T(f, vcur, wbuf, 1, s)) != KLST_OK) return fail(rc);
            cudaEventRecord(evs[3 * j + 1], s);
            ++applies;
            // classical Gram-Schmidt twice (df64: the second pass only when the DGKS test asks)
            if ((rc = dfm ? df_orth(V, j, nullptr) : f64_orth(V, j, nullptr)) != KLST_OK) return fail(rc);
            cudaEventRecord(evs[3 * j + 2], s);
        }
        if (!dfm) f64_steps += m - k;
        SchurArgs a;
        a.m = m; a.lds = lds; a.S = W.S; a.H = W.H; a.Q = W.Q; a.Yc = W.Yc; a.mu = W.mu; a.est = W.est;
        a.Ysel = W.Ysel; a.mu_sel = W.musel; a.est_sel = W.estsel;
        a.Vh = (float4*)W.Vh; a.tau = W.tau; a.log = W.rlog; a.log_cap = log_cap; a.log_count = W.rcount;
        a.log2 = W.rlog2; a.loff = W.loff; a.rdy = W.rdy;
        a.nconv = W.nconv; a.keep = keep; a.nev = nev; a.tol = o->tol; a.conv = o->conv; a.st = f->status;
        cudaEventRecord(evs[3 * (m + 1)], s);
        // the small Schur step runs in the basis arithmetic: float64 for the float64 basis
        if ((rc = dfm ? launch_schur(a, s) : launch_schur64(a, s)) != KLST_OK) return fail(rc);
        cudaEventRecord(evs[3 * (m + 1) + 1], s);
        Status hst;
        int hconv = 0, hcnt[4] = {0, 0, 0, 0};
        KLST_CK(cudaMemcpyAsync(&hconv, W.nconv, sizeof(int), cudaMemcpyDeviceToHost, s));
        KLST_CK(cudaMemcpyAsync(hcnt, W.rcount, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
        KLST_CK(cudaMemcpyAsync(&hst, f->status, sizeof(Status), cudaMemcpyDeviceToHost, s));
        KLST_CK(cudaStreamSynchronize(s));
        if (use_graph) {  // graph mode times the whole expansion (apply + orthogonalisation) as t_orth
            float a1 = 0;
            cudaEventElapsedTime(&a1, evs[0], evs[1]);
            t_orth += a1;
        }
        for (int j = use_graph ? m : jfirst; j < m; ++j) {
            float a1 = 0, a2 = 0;
            cudaEventElapsedTime(&a1, evs[3 * j], evs[3 * j + 1]);
            cudaEventElapsedTime(&a2, evs[3 * j + 1], evs[3 * j + 2]);
            t_apply += a1;
            t_orth += a2;
        }
        {
            float a3 = 0;
            cudaEventElapsedTime(&a3, evs[3 * (m + 1)], evs[3 * (m + 1) + 1]);
            t_restart += a3;
            t_schur += a3;
        }
        schur_rot += hcnt[0];
        if (!dfm) { schur_sweeps += hcnt[1]; schur_swaps += hcnt[2]; }
        if (hconv < 0 || (hst.flags & ST_NOCONV_QR)) { set_error("small Schur QR iteration did not converge"); return fail(KLST_ENOCONV); }
        if (hst.flags & ST_BREAKDOWN) { set_error("Arnoldi breakdown (invariant subspace found)"); return fail(KLST_ENOCONV); }
        if (hst.flags & ST_TIMEOUT) { set_error("tensor-core rotation: a bounded device wait gave up"); return fail(KLST_ETIMEOUT); }
        nconv = hconv;
        if (nconv >= nev) { converged = true; break; }
        if (restarts >= o->max_restarts) break;
        // rotate: V'[:, 0:keep] = V[:, 0:m] Q[:, 0:keep], V'[:, keep] = V[:, m]
        {
            cudaEventRecord(evs[3 * (m + 1) + 2], s);
            dim3 grd(std::max(1, nblk / std::max(1, (keep + 7) / 8)), (keep + 7) / 8);
            prof_begin("rotate", s);
            if (dfm) { k_rotate_df<float4><<<grd, 256, sizeof(double2) * m * 8, s>>>(V4(V), n, m, W.Q, m, keep, V4(Valt), n, n); klst::note_launch(); }
            else if (use_tc) { if ((rc = oz_rotate(V, n, m, W.Q, keep, Valt, W.ozws, f->status, s)) != KLST_OK) return fail(rc); }
            else { k_rotate<<<grd, 256, sizeof(double2) * m * 8, s>>>(V, n, m, W.Q, m, keep, Valt, n, n); klst::note_launch(); }
            prof_end("rotate", s);
            KLST_CK_LAUNCH();
            KLST_CK(cudaMemcpyAsync(Valt + (int64_t)keep * n, V + (int64_t)m * n, sizeof(double2) * n,
                                    cudaMemcpyDeviceToDevice, s));
            if (use_tcgs && (rc = split_basis(Valt, n, 0, keep + 1, W.sl, W.v32, s)) != KLST_OK) return fail(rc);
            cudaEventRecord(evs[3 * (m + 1) + 3], s);
            KLST_CK(cudaEventSynchronize(evs[3 * (m + 1) + 3]));
            float a4 = 0;
            cudaEventElapsedTime(&a4, evs[3 * (m + 1) + 2], evs[3 * (m + 1) + 3]);
            t_restart += a4;
            std::swap(V, Valt);
        }
        k = keep;
        ++restarts;
    }
    // Ritz vectors x_i = V Q y_i (nev columns), purification q_i = T x_i / ||T x_i||, residuals
    const int nret = nev;
    double2* X = Valt;                          // n x nev
    double2* Z = Valt + (int64_t)nev * n;        // n x nev (needs 2 nev <= m + 1 columns)
    double2* Rr = nullptr;
    const bool room = 3 * nev <= m + 1;
    if (!room) {
        if ((e = dmalloc((void**)&W.Z, sizeof(double2) * n * nev, s)) != cudaSuccess ||
            (e = dmalloc((void**)&W.R, sizeof(double2) * n * nev, s)) != cudaSuccess)
            return fail(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
        if (2 * nev > m + 1) {
            if ((e = dmalloc((void**)&W.X, sizeof(double2) * n * nev, s)) != cudaSuccess)
                return fail(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
            X = W.X;
        }
        Z = W.Z;
        Rr = W.R;
    } else {
        Rr = Valt + (int64_t)2 * nev * n;
    }
    {
        dim3 grd(std::max(1, nblk / std::max(1, (nret + 7) / 8)), (nret + 7) / 8);
        if (dfm) { k_rotate_df<double2><<<grd, 256, sizeof(double2) * m * 8, s>>>(V4(V), n, m, W.Ysel, m, nret, X, n, n); klst::note_launch(); }
        else if (use_tc) { if ((rc = oz_rotate(V, n, m, W.Ysel, nret, X, W.ozws, f->status, s)) != KLST_OK) return fail(rc); }
        else { k_rotate<<<grd, 256, sizeof(double2) * m * 8, s>>>(V, n, m, W.Ysel, m, nret, X, n, n); klst::note_launch(); }
        KLST_CK_LAUNCH();
    }
    if ((rc = apply_T(f, X, Z, nret, s)) != KLST_OK) return fail(rc);
    applies += nret;
    k_colnorm_part<<<dim3(nblk, nret), 256, 0, s>>>(Z, n, n, W.npart); klst::note_launch();
    k_colnorm_fin<<<(nret + 7) / 8, 256, 0, s>>>(W.npart, nblk, nret, W.nrm); klst::note_launch();
    k_scale_cols<<<dim3(nblk, nret), 256, 0, s>>>(Z, n, n, W.nrm); klst::note_launch();
    KLST_CK_LAUNCH();
    std::vector<double2> mu(m);
    KLST_CK(cudaMemcpyAsync(mu.data(), W.musel, sizeof(double2) * nev, cudaMemcpyDeviceToHost, s));
    KLST_CK(cudaStreamSynchronize(s));
    std::vector<double2> om(nret);
    for (int i = 0; i < nret; ++i) {
        const double d = mu[i].x * mu[i].x + mu[i].y * mu[i].y;
        om[i] = mk(f->sigma.x + mu[i].x / d, f->sigma.y - mu[i].y / d);
    }
    KLST_CK(cudaMemcpyAsync(W.om, om.data(), sizeof(double2) * nret, cudaMemcpyHostToDevice, s));
    if ((rc = apply_pencil_dev(p, Z, Rr, nret, W.om, s, W.mw, W.mp, ng)) != KLST_OK) return fail(rc);
    k_colnorm_part<<<dim3(nblk, nret), 256, 0, s>>>(Rr, n, n, W.npart); klst::note_launch();
    k_colnorm_fin<<<(nret + 7) / 8, 256, 0, s>>>(W.npart, nblk, nret, W.nrm); klst::note_launch();
    KLST_CK_LAUNCH();
    std::vector<double> res(nret);
    double worst = 0;
    int sweeps = 0, reorths = 0;
    Status fst;
    KLST_CK(cudaMemcpyAsync(&fst, f->status, sizeof(Status), cudaMemcpyDeviceToHost, s));
    KLST_CK(cudaMemcpyAsync(res.data(), W.nrm, sizeof(double) * nret, cudaMemcpyDeviceToHost, s));
    KLST_CK(cudaMemcpyAsync(&worst, f->worst, sizeof(double), cudaMemcpyDeviceToHost, s));
    KLST_CK(cudaMemcpyAsync(&sweeps, f->sweeps, sizeof(int), cudaMemcpyDeviceToHost, s));
    KLST_CK(cudaMemcpyAsync(&reorths, W.reorth, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (evecs) KLST_CK(cudaMemcpyAsync(evecs, Z, sizeof(double2) * n * nret, cudaMemcpyDeviceToDevice, s));
    std::vector<double> esth(nret);
    KLST_CK(cudaMemcpyAsync(esth.data(), W.estsel, sizeof(double) * nret, cudaMemcpyDeviceToHost, s));
    KLST_CK(cudaStreamSynchronize(s));
    if (o->est_out) memcpy(o->est_out, esth.data(), sizeof(double) * nret);
    prof_report(s);
    double maxres = 0;
    for (int i = 0; i < nret; ++i) {
        evals_host[2 * i] = om[i].x;
        evals_host[2 * i + 1] = om[i].y;
        if (resid_host) resid_host[i] = res[i];
        maxres = std::max(maxres, res[i]);
    }
    if (info) {
        info->nconv = converged ? nev : nconv;
        info->restarts = restarts;
        info->applies = applies;
        info->refine_sweeps = sweeps;
        info->t_factor_ms = f->t_factor_ms;
        info->t_eigs_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        info->max_resid = maxres;
        info->max_refine_resid = worst;
        info->t_apply_ms = t_apply;
        info->t_orth_ms = t_orth;
        info->t_restart_ms = t_restart;
        info->t_schur_ms = t_schur;
        info->reorths = dfm ? reorths : f64_steps;
        info->schur_sweeps = schur_sweeps;
        info->schur_swaps = schur_swaps;
        info->schur_rotations = schur_rot;
    }
    W.release(s);
    f->max_refine = prev_refine;
    f->refine_tol = prev_rtol;
    f->arith = prev_arith;
    if (!converged) { set_error("only %d of %d eigenpairs converged after %d restarts", nconv, nev, restarts); return KLST_ENOCONV; }
    if (fst.flags & ST_TIMEOUT) {
        set_error("tensor-core rotation: a bounded device wait gave up");
        return KLST_ETIMEOUT;
    }
    if (fst.flags & ST_REFINE) {
        set_error("mixed-precision refinement missed refine_tol in at least one apply (worst %.3g after %d sweeps); "
                  "the eigenpairs and their explicit residuals are returned", worst, o->max_refine);
        return KLST_EREFINE;
    }
    return KLST_OK;
}
