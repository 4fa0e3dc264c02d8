// Classical Gram-Schmidt with one reorthogonalisation for the float64 Krylov basis
// (Sec. 4.1: the paper's -bv_orthog_type cgs, applied twice).  One Arnoldi step j orthogonalises
// w = T v_j against the j + 1 basis columns V[:, 0..j]:
//   pass 1:  h1 = V^H w  (coefficients on the float32 pipes),  w' = w - V h1  (float64)
//   pass 2:  h2 = V^H w' (float64),                            w'' = w' - V h2 (V h2 double-float)
//   column j of the Krylov-Schur matrix: h1 + h2, beta = ||w''||, v_{j+1} = w'' / beta.
// Why the first coefficients may be float32: w' = w - V h1 is formed in float64 with whatever h1
// is, so the Arnoldi relation T v_j = V (h1 + h2) + w'' holds to float64 rounding however rough
// h1 is; h1 only has to remove most of w's component in span(V), and the float64 second pass
// removes the rest (its coefficients are float64, so v_{j+1} is orthogonal to V to float64
// rounding).  The first update and the second projection run in float64; the second update only
// subtracts the small correction V h2, which double-float arithmetic forms well inside float64
// rounding of w (see k_update_corr64): two of the four passes' complex multiply-adds per basis
// entry and step are float64.
// Every kernel reads the step index from device memory when jdev != NULL, so one captured graph
// serves every step.
#include <algorithm>

#include "df64.cuh"
#include "oz.cuh"

namespace klst {

// part[chunk * ldp + col] = sum_{i in chunk} conj(V[i, col]) w[i] in float32 arithmetic on
// truncated operands (first-pass coefficients).  Four columns per warp pass, two rows per lane
// iteration; the per-chunk sums are stored as float64.
// The basis is read in float64 (truncated on the fly) or from its truncated float32 copy.
__device__ __forceinline__ float f32_of(double x) { return trunc_f32(x); }
__device__ __forceinline__ float f32_of(float x) { return x; }
template <typename VT>
__global__ void __launch_bounds__(256) k_dots_f32(const VT* __restrict__ V, int64_t ldv, int ncols,
                                                  const double2* __restrict__ w, int64_t n, int chunk,
                                                  double2* __restrict__ part, int ldp, const int* __restrict__ jdev) {
    if (jdev) ncols = *jdev + 1;
    extern __shared__ float2 sw32[];
    const int64_t r0 = (int64_t)blockIdx.x * chunk;
    const int len = (int)((n - r0) < chunk ? (n - r0) : chunk);
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const double2 v = w[r0 + i];
        sw32[i] = make_float2(trunc_f32(v.x), trunc_f32(v.y));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double2 z2 = make_double2(0.0, 0.0);
    for (int col = 4 * wid; col < ncols; col += 4 * nw) {
        const int nq = min(4, ncols - col);
        const VT* vc = V + col * ldv + r0;
        float2 a[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        int i = lane;
        for (; i + 32 < len; i += 64) {
            VT x0[4], x1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                x0[q] = (q < nq) ? vc[q * ldv + i] : VT{};
                x1[q] = (q < nq) ? vc[q * ldv + i + 32] : VT{};
            }
            const float2 w0 = sw32[i], w1 = sw32[i + 32];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float vr0 = f32_of(x0[q].x), vi0 = f32_of(x0[q].y);
                const float vr1 = f32_of(x1[q].x), vi1 = f32_of(x1[q].y);
                a[q].x = fmaf(vr0, w0.x, a[q].x); a[q].x = fmaf(vi0, w0.y, a[q].x);
                a[q].y = fmaf(vr0, w0.y, a[q].y); a[q].y = fmaf(-vi0, w0.x, a[q].y);
                a[q].x = fmaf(vr1, w1.x, a[q].x); a[q].x = fmaf(vi1, w1.y, a[q].x);
                a[q].y = fmaf(vr1, w1.y, a[q].y); a[q].y = fmaf(-vi1, w1.x, a[q].y);
            }
        }
        if (i < len) {
            const float2 w0 = sw32[i];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nq) {
                    const VT x = vc[q * ldv + i];
                    const float vr = f32_of(x.x), vi = f32_of(x.y);
                    a[q].x = fmaf(vr, w0.x, a[q].x); a[q].x = fmaf(vi, w0.y, a[q].x);
                    a[q].y = fmaf(vr, w0.y, a[q].y); a[q].y = fmaf(-vi, w0.x, a[q].y);
                }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float sx = a[q].x, sy = a[q].y;
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (lane == 0 && q < nq) part[(size_t)blockIdx.x * ldp + col + q] = make_double2(sx, sy);
        }
    }
}

// part[chunk * ldp + col] = sum_{i in chunk} conj(V[i, col]) w[i] in float64 (second-pass
// coefficients).  Four columns per warp pass and two rows per lane iteration keep eight
// independent multiply-add chains per lane.
__global__ void __launch_bounds__(256) k_dots64(const double2* __restrict__ V, int64_t ldv, int ncols,
                                                const double2* __restrict__ w, int64_t n, int chunk,
                                                double2* __restrict__ part, int ldp, const int* __restrict__ jdev) {
    if (jdev) ncols = *jdev + 1;
    extern __shared__ double2 sw64[];
    const int64_t r0 = (int64_t)blockIdx.x * chunk;
    const int len = (int)((n - r0) < chunk ? (n - r0) : chunk);
    for (int i = threadIdx.x; i < len; i += blockDim.x) sw64[i] = w[r0 + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double2 z2 = make_double2(0.0, 0.0);
    for (int col = 4 * wid; col < ncols; col += 4 * nw) {
        const int nq = min(4, ncols - col);
        const double2* vc = V + col * ldv + r0;
        double2 a[4] = {z2, z2, z2, z2}, b[4] = {z2, z2, z2, z2};
        int i = lane;
        for (; i + 32 < len; i += 64) {
            double2 x0[4], x1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                x0[q] = (q < nq) ? vc[q * ldv + i] : z2;
                x1[q] = (q < nq) ? vc[q * ldv + i + 32] : z2;
            }
            const double2 w0 = sw64[i], w1 = sw64[i + 32];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cfma_conj(a[q], x0[q], w0);
                cfma_conj(b[q], x1[q], w1);
            }
        }
        if (i < len) {
            const double2 w0 = sw64[i];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < nq) cfma_conj(a[q], vc[q * ldv + i], w0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double sx = warp_sum(a[q].x + b[q].x), sy = warp_sum(a[q].y + b[q].y);
            if (lane == 0 && q < nq) part[(size_t)blockIdx.x * ldp + col + q] = make_double2(sx, sy);
        }
    }
}

// h[col] = sum over chunks of part[chunk][col], one CTA of four warps per column, float64 in a
// fixed order (each thread strides the chunks with two accumulators, then the warps combine).
__global__ void __launch_bounds__(128) k_reduce_cols64(const double2* __restrict__ part, int nparts, int ncols, int ldp,
                                                       double2* __restrict__ h, const int* __restrict__ jdev) {
    if (jdev) ncols = *jdev + 1;
    const int col = blockIdx.x;
    if (col >= ncols) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double2 a0 = make_double2(0.0, 0.0), a1 = a0;
    int b = tid;
    for (; b + 128 < nparts; b += 256) {
        a0 = a0 + part[(size_t)b * ldp + col];
        a1 = a1 + part[(size_t)(b + 128) * ldp + col];
    }
    if (b < nparts) a0 = a0 + part[(size_t)b * ldp + col];
    const double sx = warp_sum(a0.x + a1.x), sy = warp_sum(a0.y + a1.y);
    __shared__ double2 red[4];
    if (lane == 0) red[wid] = make_double2(sx, sy);
    __syncthreads();
    if (tid == 0) h[col] = ((red[0] + red[1]) + red[2]) + red[3];
}

// w -= V h over ncols columns in float64, one row per thread; the next four basis entries are
// loaded before the multiply-adds of the current four (two accumulators, even and odd columns).
// With npart, each CTA also writes the sum of |w|^2 over its rows (fixed order).
__global__ void __launch_bounds__(256) k_update64(const double2* __restrict__ V, int64_t ldv, int ncols,
                                                  const double2* __restrict__ h, double2* __restrict__ w, int64_t n,
                                                  double* __restrict__ npart, const int* __restrict__ jdev) {
    if (jdev) ncols = *jdev + 1;
    extern __shared__ double2 sh64[];
    for (int i = threadIdx.x; i < ncols; i += blockDim.x) sh64[i] = -h[i];
    __syncthreads();
    const double2 z2 = make_double2(0.0, 0.0);
    double nrm = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 acc0 = w[i], acc1 = z2;
        double2 xa[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xa[u] = (u < ncols) ? V[u * ldv + i] : z2;
        int c = 0;
        for (; c + 4 <= ncols; c += 4) {
            double2 xb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xb[u] = (c + 4 + u < ncols) ? V[(c + 4 + u) * ldv + i] : z2;
            cfma(acc0, xa[0], sh64[c]);
            cfma(acc1, xa[1], sh64[c + 1]);
            cfma(acc0, xa[2], sh64[c + 2]);
            cfma(acc1, xa[3], sh64[c + 3]);
#pragma unroll
            for (int u = 0; u < 4; ++u) xa[u] = xb[u];
        }
        if (c < ncols) cfma(acc0, xa[0], sh64[c]);
        if (c + 1 < ncols) cfma(acc1, xa[1], sh64[c + 1]);
        if (c + 2 < ncols) cfma(acc0, xa[2], sh64[c + 2]);
        const double2 out = acc0 + acc1;
        w[i] = out;
        nrm += abs2(out);
    }
    if (npart) {
        nrm = warp_sum(nrm);
        __shared__ double red[32];
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
            npart[blockIdx.x] = s;
        }
    }
}

// A float64 value as a double-float pair (hi, lo) by integer operations: hi holds the leading 24
// significand bits (truncated), lo the remaining 29 bits rounded to float32 (an error below 2^-48
// of |x|).  Values below 2^-74 in magnitude lose lo and those below 2^-126 become 0.
__device__ __forceinline__ df split_df(double x) {
    const long long b = __double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int e = (int)((hi >> 20) & 0x7FFu);
    const float h = trunc_f32(x);
    const int el = e - 1075 + 127;  // exponent of the unit in the last place of x, biased for float32
    const float scale = el > 0 ? __uint_as_float((unsigned)el << 23) : 0.0f;
    const float l = __uint2float_rn(lo & 0x1FFFFFFFu) * scale;
    return {h, (hi & 0x80000000u) ? -l : l};
}

// Second-pass update w'' = w' - delta with delta = V h2 formed in double-float arithmetic and the
// subtraction in float64.  After a first pass whose coefficients carry float32 rounding, h2 (and
// delta) is about 1e-6 of ||w||, so a double-float delta (relative error 2^-48) changes w'' by far
// less than the float64 rounding of w' itself; w' is never rounded to double-float.
__global__ void __launch_bounds__(256) k_update_corr64(const double2* __restrict__ V, int64_t ldv, int ncols,
                                                       const double2* __restrict__ h, double2* __restrict__ w,
                                                       int64_t n, double* __restrict__ npart,
                                                       const int* __restrict__ jdev) {
    if (jdev) ncols = *jdev + 1;
    extern __shared__ float4 shc[];
    for (int i = threadIdx.x; i < ncols; i += blockDim.x) cdf_store(&shc[i], cdf_from(h[i]));
    __syncthreads();
    const double2 z2 = make_double2(0.0, 0.0);
    double nrm = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        cdf d0 = cdf_zero(), d1 = cdf_zero();
        double2 xa[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) xa[u] = (u < ncols) ? V[u * ldv + i] : z2;
        int c = 0;
        for (; c + 2 <= ncols; c += 2) {
            double2 xb[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) xb[u] = (c + 2 + u < ncols) ? V[(c + 2 + u) * ldv + i] : z2;
            cdf_fma(d0, cdf{split_df(xa[0].x), split_df(xa[0].y)}, cdf_load(shc + c));
            cdf_fma(d1, cdf{split_df(xa[1].x), split_df(xa[1].y)}, cdf_load(shc + c + 1));
            xa[0] = xb[0];
            xa[1] = xb[1];
        }
        if (c < ncols) cdf_fma(d0, cdf{split_df(xa[0].x), split_df(xa[0].y)}, cdf_load(shc + c));
        const double2 dl = cdf_to(cdf_add(d0, d1));
        const double2 out = w[i] - dl;
        w[i] = out;
        nrm += abs2(out);
    }
    nrm = warp_sum(nrm);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sacc = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sacc += red[q];
        npart[blockIdx.x] = sacc;
    }
}

// Column j of the Krylov-Schur matrix: S[0..j, j] = h1 + h2, S[j+1, j] = beta = ||w''|| (from
// the per-CTA partial sums of the second update), and the breakdown test.
__global__ void __launch_bounds__(256) k_finish64(const double2* __restrict__ h1, const double2* __restrict__ h2,
                                                  const double* __restrict__ npart, int nblk, int j,
                                                  double2* __restrict__ S, int lds, double* __restrict__ beta_out,
                                                  Status* st, const int* __restrict__ jdev) {
    if (jdev) j = *jdev;
    __shared__ double red[2][32];
    double s = 0.0, hn = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += npart[b];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 hv = h1[i] + h2[i];
        S[(size_t)j * lds + i] = hv;
        hn += abs2(hv);
    }
    s = warp_sum(s);
    hn = warp_sum(hn);
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = s; red[1][threadIdx.x >> 5] = hn; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, hs = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += red[0][q]; hs += red[1][q]; }
        const double beta = sqrt(a);
        if (!(beta > 1e-13 * sqrt(hs))) atomicOr(&st->flags, ST_BREAKDOWN);
        S[(size_t)j * lds + j + 1] = make_double2(beta, 0.0);
        *beta_out = beta;
    }
}

// v_{j+1} = w'' / beta into the basis and into the float64 vector the next apply reads
// (with jdev the basis column is jdev[0] + 1)
__global__ void k_scale64(const double2* __restrict__ w, int64_t n, const double* __restrict__ beta,
                          double2* __restrict__ vcol, double2* __restrict__ vcopy, int64_t ldv,
                          const int* __restrict__ jdev) {
    if (jdev) vcol += (int64_t)(*jdev + 1) * ldv;
    __shared__ double s_inv;
    if (threadIdx.x == 0) {
        const double b = *beta;
        s_inv = b > 0 ? 1.0 / b : 0.0;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = w[i];
        const double2 o = make_double2(v.x * inv, v.y * inv);
        vcol[i] = o;
        vcopy[i] = o;
    }
}

// The whole orthogonalisation of step j (j read from jd when non-NULL; the grids are sized for the
// largest step).  w is overwritten by w''; the new basis column and vcur receive w'' / beta.
int orth64_step(const Orth64Args& a, int j, const int* jd, cudaStream_t s) {
    const int nc = j + 1, m = a.m;
    const size_t dsm32 = sizeof(float2) * a.chunk, dsm64 = sizeof(double2) * a.chunk;
    const size_t usm = sizeof(double2) * (m + 1);
    const int nred = jd ? m : nc;
    if (a.sl) {
        // the float64 passes as exact integer-slice products on the tensor cores (orth_tc.cu)
        int rc;
        prof_begin("orth1_f32dots", s);
        k_dots_f32<float2><<<a.nchunks, 256, dsm32, s>>>(a.v32, a.n, nc, a.w, a.n, a.chunk, a.part, a.ldp, jd); note_launch();
        k_reduce_cols64<<<nred, 128, 0, s>>>(a.part, a.nchunks, nc, a.ldp, a.h1, jd); note_launch();
        prof_end("orth1_f32dots", s);
        prof_begin("orth_tc_update1", s);
        if ((rc = gs_update_tc(a.sl, a.n, a.h1, a.w, nullptr, false, j, jd, a.st, s)) != KLST_OK) return rc;
        prof_end("orth_tc_update1", s);
        prof_begin("orth_tc_dots2", s);
        if ((rc = gs_dots_tc(a.sl, a.n, a.w, a.part, a.ldp, j, jd, a.st, s)) != KLST_OK) return rc;
        k_reduce_cols64<<<nred, 128, 0, s>>>(a.part, a.ntc, nc, a.ldp, a.h2, jd); note_launch();
        prof_end("orth_tc_dots2", s);
        prof_begin("orth_tc_update2", s);
        if ((rc = gs_update_tc(a.sl, a.n, a.h2, a.w, a.npart, true, j, jd, a.st, s)) != KLST_OK) return rc;
        prof_end("orth_tc_update2", s);
        prof_begin("orth_scale", s);   // column j of S, beta and the new basis column in one launch
        finish_scale64_split(a.h1, a.h2, a.npart, a.ntc, a.S, a.lds, a.beta, a.st, a.w, a.n, a.V, a.vcur, j + 1, a.sl,
                             a.v32, jd, a.nscale, s);
        prof_end("orth_scale", s);
        KLST_CK_LAUNCH();
        return KLST_OK;
    }
    prof_begin("orth1_f32dots_f64update", s);
    k_dots_f32<double2><<<a.nchunks, 256, dsm32, s>>>(a.V, a.n, nc, a.w, a.n, a.chunk, a.part, a.ldp, jd); note_launch();
    k_reduce_cols64<<<nred, 128, 0, s>>>(a.part, a.nchunks, nc, a.ldp, a.h1, jd); note_launch();
    k_update64<<<a.nupd, 256, usm, s>>>(a.V, a.n, nc, a.h1, a.w, a.n, nullptr, jd); note_launch();
    prof_end("orth1_f32dots_f64update", s);
    prof_begin("orth2_f64", s);
    k_dots64<<<a.nchunks, 256, dsm64, s>>>(a.V, a.n, nc, a.w, a.n, a.chunk, a.part, a.ldp, jd); note_launch();
    k_reduce_cols64<<<nred, 128, 0, s>>>(a.part, a.nchunks, nc, a.ldp, a.h2, jd); note_launch();
    k_update_corr64<<<a.nupd, 256, usm, s>>>(a.V, a.n, nc, a.h2, a.w, a.n, a.npart, jd); note_launch();
    k_finish64<<<1, 256, 0, s>>>(a.h1, a.h2, a.npart, a.nupd, j, a.S, a.lds, a.beta, a.st, jd); note_launch();
    prof_end("orth2_f64", s);
    prof_begin("orth_scale", s);
    k_scale64<<<a.nscale, 256, 0, s>>>(a.w, a.n, a.beta, jd ? a.V : a.V + (int64_t)(j + 1) * a.n, a.vcur, a.n, jd);
    note_launch();
    prof_end("orth_scale", s);
    KLST_CK_LAUNCH();
    return KLST_OK;
}

void k_scale64_ext(const double2* w, int64_t n, const double* beta, double2* vcol, double2* vcopy, int64_t ldv,
                   int nblk, cudaStream_t s) {
    k_scale64<<<nblk, 256, 0, s>>>(w, n, beta, vcol, vcopy, ldv, nullptr);
    note_launch();
}

}  // namespace klst
