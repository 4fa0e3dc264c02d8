// Shift-and-invert apply y = (A - sigma B)^{-1} B x (Eq. parShiftInvert) in Woodbury form:
//   b = B x,  z = K^{-1} b,  t = V^H z,  s = C^{-1} t,  y = K^{-1} (b + U s).
// Each block solve is a dense matrix-vector product with the stored K_k^{-1} (column-major)
// for the two components g^, h^ at once.  MIXED factors hold K_k^{-1} in complex float32 and
// the result is refined in float64: y += T~ (b - (A - sigma B) y).
#include <algorithm>
#include <type_traits>

#include "df64.cuh"
#include "factor.cuh"

namespace klst {

static inline int nxp_of(int nx) { return (nx + 31) & ~31; }
int moments_dev(klst_pencil p, const double2* x, int64_t ldx, int nrhs, double2* mwork, double2* mpart,
                int ngroups, cudaStream_t s, const int* done);
int pencil_rows_dev(klst_pencil p, const double2* m, const double2* x, int64_t ldx, int nrhs, const double2* omega,
                    int mode, const double2* b, int mask_b, double2* y, double* normpart, cudaStream_t s,
                    const int* done, int df_arith);
int pencil_rows_blocks(klst_pencil p);

// z_g += K_k^{-1}[j, :] s0, z_h += K_k^{-1}[j, :] s1 for thread row j (Kk points at column 0 of row
// j in the transposed storage, stride nx).  The loads of the next four entries are issued before
// the multiply-adds of the current four, so eight loads per thread are in flight.
// D entries per group: the next group's D loads are issued before the current group's
// multiply-adds, so 2 D loads per thread are in flight.  The 8-byte complex64 entries use D = 8
// (the HBM-bound float32 solves need more bytes in flight per thread), the 16-byte ones D = 4.
template <typename C> struct GemvDepth { static constexpr int D = 4; };
template <> struct GemvDepth<float2> { static constexpr int D = 8; };

template <typename C>
__device__ __forceinline__ void block_gemv2(const C* __restrict__ Kk, int nx, const C* s0, const C* s1, C& zg, C& zh) {
    constexpr int D = GemvDepth<C>::D;
    C ka[D];
#pragma unroll
    for (int u = 0; u < D; ++u) ka[u] = (u < nx) ? Kk[(size_t)u * nx] : czero<C>();
    int m = 0;
    for (; m + D <= nx; m += D) {
        C kb[D];
#pragma unroll
        for (int u = 0; u < D; ++u) kb[u] = (m + D + u < nx) ? Kk[(size_t)(m + D + u) * nx] : czero<C>();
#pragma unroll
        for (int u = 0; u < D; ++u) {
            cfma(zg, ka[u], s0[m + u]);
            cfma(zh, ka[u], s1[m + u]);
        }
#pragma unroll
        for (int u = 0; u < D; ++u) ka[u] = kb[u];
    }
#pragma unroll
    for (int u = 0; u < D - 1; ++u)
        if (m + u < nx) {
            cfma(zg, ka[u], s0[m + u]);
            cfma(zh, ka[u], s1[m + u]);
        }
}

// Pass 1: for each k in the block's group, z_{c,k} = K_k^{-1} b_{c,k} and accumulate
// t_a(j) += sum_c w^c_a(j,k) z_{c,k}(j); tpart[(rhs*ngroups + g)*r + a*nx + j].
template <typename C>
__global__ void __launch_bounds__(256, 4) k_solve_pass1(int nx, int nxi, const C* __restrict__ KinvT, const double* __restrict__ w,
                              const double* __restrict__ xi_x, const double2* __restrict__ b, int64_t ldb, int mask,
                              int ngroups, int kpg, double2* __restrict__ tpart, const int* __restrict__ done) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int NXP = blockDim.x, KB = blockDim.y;
    const int j = threadIdx.x, kk = threadIdx.y, g = blockIdx.x, rhs = blockIdx.y;
    if (done && done[rhs]) return;
    C* sb = (C*)dsm;  // [KB][2][NXP]
    const double2* br = b + rhs * ldb;
    double2 acc[4] = {mk(0, 0), mk(0, 0), mk(0, 0), mk(0, 0)};
    const int k0 = g * kpg, k1 = min(nxi, k0 + kpg);
    for (int kb = k0; kb < k1; kb += KB) {
        const int k = kb + kk;
        const bool valid = (k < k1) && (j < nx);
        if (valid) {
            const bool bc = mask && is_bc(j, nx, xi_x[k]);
            double2 vg = br[(size_t)k * nx + j], vh = br[((size_t)nxi + k) * nx + j];
            if (bc) { vg = mk(0, 0); vh = mk(0, 0); }
            sb[(kk * 2 + 0) * NXP + j] = to_c<C>(vg);
            sb[(kk * 2 + 1) * NXP + j] = to_c<C>(vh);
        }
        __syncthreads();
        if (valid) {
            C zg = czero<C>(), zh = czero<C>();
            block_gemv2<C>(KinvT + (size_t)k * nx * nx + j, nx, sb + (kk * 2 + 0) * NXP, sb + (kk * 2 + 1) * NXP, zg, zh);
            const double2 dg = to_d(zg), dh = to_d(zh);
            const double* wk = w + (size_t)k * 8 * nx + j;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const double wg = wk[a * nx], wh = wk[(4 + a) * nx];
                acc[a].x += wg * dg.x + wh * dh.x;
                acc[a].y += wg * dg.y + wh * dh.y;
            }
        }
        __syncthreads();
    }
    double2* red = (double2*)dsm;
#pragma unroll
    for (int a = 0; a < 4; ++a) red[(kk * 4 + a) * NXP + j] = acc[a];
    __syncthreads();
    if (kk == 0 && j < nx) {
        for (int a = 0; a < 4; ++a) {
            double2 s = mk(0, 0);
            for (int q = 0; q < KB; ++q) s = s + red[(q * 4 + a) * NXP + j];
            tpart[((size_t)rhs * ngroups + g) * 4 * nx + a * nx + j] = s;
        }
    }
}

// s = C^{-1} t : one warp per row of the row-major capacitance inverse; four accumulators per
// lane keep four independent loads and multiply-add chains in flight
__global__ void k_cinv_gemv(int r, const double2* __restrict__ Cinv, const double2* __restrict__ t,
                            double2* __restrict__ sv, const int* __restrict__ done) {
    const int rhs = blockIdx.y;
    if (done && done[rhs]) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= r) return;
    const double2* row = Cinv + (size_t)warp * r;
    const double2* tr = t + (size_t)rhs * r;
    double2 a0 = mk(0, 0), a1 = mk(0, 0), a2 = mk(0, 0), a3 = mk(0, 0);
    int l = lane;
    for (; l + 96 < r; l += 128) {
        const double2 x0 = row[l], x1 = row[l + 32], x2 = row[l + 64], x3 = row[l + 96];
        const double2 y0 = tr[l], y1 = tr[l + 32], y2 = tr[l + 64], y3 = tr[l + 96];
        cfma(a0, x0, y0);
        cfma(a1, x1, y1);
        cfma(a2, x2, y2);
        cfma(a3, x3, y3);
    }
    for (; l < r; l += 32) cfma(a0, row[l], tr[l]);
    double2 a = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) {
        a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
        a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
    }
    if (lane == 0) sv[(size_t)rhs * r + warp] = a;
}

// Pass 2: y_{c,k} (+)= K_k^{-1} (b_{c,k} + sum_a G^c_a(.,k) s_a(.)).
template <typename C>
__global__ void __launch_bounds__(256, 4) k_solve_pass2(int nx, int nxi, const C* __restrict__ KinvT, const double* __restrict__ G,
                              const double* __restrict__ xi_x, const double2* __restrict__ b, int64_t ldb, int mask,
                              const double2* __restrict__ sv, double2* __restrict__ y, int accumulate,
                              const int* __restrict__ done) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int NXP = blockDim.x, KB = blockDim.y;
    const int j = threadIdx.x, kk = threadIdx.y, rhs = blockIdx.y;
    if (done && done[rhs]) return;
    C* sb = (C*)dsm;
    const double2* br = b + rhs * ldb;
    double2* yr = y + rhs * ldb;
    const double2* sr = sv + (size_t)rhs * 4 * nx;
    for (int kb = blockIdx.x * KB; kb < nxi; kb += gridDim.x * KB) {
        const int k = kb + kk;
        const bool valid = (k < nxi) && (j < nx);
        if (valid) {
            const bool bc = mask && is_bc(j, nx, xi_x[k]);
            const double* Gk = G + (size_t)k * 8 * nx + j;
            for (int c = 0; c < 2; ++c) {
                double2 v = br[((size_t)c * nxi + k) * nx + j];
                if (bc) v = mk(0, 0);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const double gv = Gk[(c * 4 + a) * nx];
                    const double2 s = sr[a * nx + j];
                    v.x = fma(gv, s.x, v.x);
                    v.y = fma(gv, s.y, v.y);
                }
                sb[(kk * 2 + c) * NXP + j] = to_c<C>(v);
            }
        }
        __syncthreads();
        if (valid) {
            C zg = czero<C>(), zh = czero<C>();
            block_gemv2<C>(KinvT + (size_t)k * nx * nx + j, nx, sb + (kk * 2 + 0) * NXP, sb + (kk * 2 + 1) * NXP, zg, zh);
            const size_t ig = (size_t)k * nx + j, ih = ((size_t)nxi + k) * nx + j;
            if (accumulate) {
                yr[ig] = yr[ig] + to_d(zg);
                yr[ih] = yr[ih] + to_d(zh);
            } else {
                yr[ig] = to_d(zg);
                yr[ih] = to_d(zh);
            }
        }
        __syncthreads();
    }
}

// Refinement bookkeeping: done[rhs] = ||r|| <= tol ||b||; worst residual; sweep counter.
// One warp per right-hand side sums the per-block norms (fixed order).
__global__ void k_refine_check(int nblk, const double* __restrict__ normpart, double tol, int* done, double* worst,
                               int* sweeps, int last, Status* st) {
    const int rhs = blockIdx.x, lane = threadIdx.x;
    if (done[rhs]) return;
    double rr = 0, bb = 0;
    for (int i = lane; i < nblk; i += 32) {
        rr += normpart[((size_t)rhs * nblk + i) * 2];
        bb += normpart[((size_t)rhs * nblk + i) * 2 + 1];
    }
    rr = warp_sum(rr);
    bb = warp_sum(bb);
    if (lane != 0) return;
    const double rel = bb > 0 ? sqrt(rr / bb) : 0.0;
    const bool ok = rel <= tol;
    if (ok || last) {
        unsigned long long* wp = (unsigned long long*)worst;
        unsigned long long old = *wp, assumed;
        do {
            assumed = old;
            if (__longlong_as_double(assumed) >= rel) break;
            old = atomicCAS(wp, assumed, __double_as_longlong(rel));
        } while (old != assumed);
    }
    if (ok) done[rhs] = 1;
    else if (!last) atomicAdd(sweeps, 1);
    else atomicOr(&st->flags, ST_REFINE);  // max_refine sweeps did not reach refine_tol
}

template <typename C> static const char* pass_name(int pass);
template <> const char* pass_name<double2>(int pass) { return pass == 1 ? "solve_pass1_c128" : "solve_pass2_c128"; }
template <> const char* pass_name<float4>(int pass) { return pass == 1 ? "solve_pass1_df64" : "solve_pass2_df64"; }
template <> const char* pass_name<float2>(int pass) { return pass == 1 ? "solve_pass1_c64" : "solve_pass2_c64"; }

// the float64 Woodbury solve with both block passes on the tensor cores
// kinv_only: y = K^{-1} b, the block inverses alone (s = 0, no first pass)
static int woodbury_solve_tc(klst_factor f, const double2* b, int mask, double2* y, int accumulate, int nrhs,
                             cudaStream_t s, const int* done, int kinv_only = 0) {
    klst_pencil p = f->p;
    const int ng = tc_solve_groups(p->nxi, f->ngroups);
    if (kinv_only) {
        KLST_CK(cudaMemsetAsync(f->sv, 0, sizeof(double2) * f->r * nrhs, s));
        return tc_solve_pass(2, f, b, mask, y, accumulate, nrhs, s, done);
    }
    prof_begin("solve_pass1_tc", s);
    int rc = tc_solve_pass(1, f, b, mask, nullptr, 0, nrhs, s, done);
    prof_end("solve_pass1_tc", s);
    if (rc) return rc;
    prof_begin("cap_solve", s);
    k_reduce_groups_ext(f->r, ng, f->tpart, f->t, done, nrhs, s);
    k_cinv_gemv<<<dim3((f->r * 32 + 255) / 256, nrhs), 256, 0, s>>>(f->r, f->Cinv, f->t, f->sv, done); klst::note_launch();
    prof_end("cap_solve", s);
    prof_begin("solve_pass2_tc", s);
    rc = tc_solve_pass(2, f, b, mask, y, accumulate, nrhs, s, done);
    prof_end("solve_pass2_tc", s);
    return rc;
}

template <typename C>
static int woodbury_solve(klst_factor f, const double2* b, int mask, double2* y, int accumulate, int nrhs,
                          cudaStream_t s, const int* done, int kinv_only = 0) {
    klst_pencil p = f->p;
    if (std::is_same<C, double2>::value && f->tc_solve)
        return woodbury_solve_tc(f, b, mask, y, accumulate, nrhs, s, done, kinv_only);
    const int nx = p->nx, nxi = p->nxi, NXP = nxp_of(nx), KB = 256 / NXP;
    if (kinv_only) {
        KLST_CK(cudaMemsetAsync(f->sv, 0, sizeof(double2) * f->r * nrhs, s));
        const int nb2 = std::min((nxi + KB - 1) / KB, 4 * device_sm_count());
        k_solve_pass2<C><<<dim3(nb2, nrhs), dim3(NXP, KB), sizeof(C) * KB * 2 * NXP, s>>>(
            nx, nxi, (const C*)f->KinvT, p->G, p->xi_x, b, p->n, mask, f->sv, y, accumulate, done);
        klst::note_launch();
        KLST_CK_LAUNCH();
        return KLST_OK;
    }
    const int ng = f->ngroups, kpg = ((nxi + ng - 1) / ng + KB - 1) / KB * KB;
    dim3 blk(NXP, KB);
    const size_t sm1 = std::max(sizeof(C) * KB * 2 * NXP, sizeof(double2) * 4 * KB * NXP);
    prof_begin(pass_name<C>(1), s);
    k_solve_pass1<C><<<dim3(ng, nrhs), blk, sm1, s>>>(nx, nxi, (const C*)f->KinvT, p->w, p->xi_x, b, p->n, mask, ng,
                                                      kpg, f->tpart, done); klst::note_launch();
    prof_end(pass_name<C>(1), s);
    prof_begin("cap_solve", s);
    k_reduce_groups_ext(f->r, ng, f->tpart, f->t, done, nrhs, s);
    k_cinv_gemv<<<dim3((f->r * 32 + 255) / 256, nrhs), 256, 0, s>>>(f->r, f->Cinv, f->t, f->sv, done); klst::note_launch();
    prof_end("cap_solve", s);
    prof_begin(pass_name<C>(2), s);
    const int nb2 = std::min((nxi + KB - 1) / KB, 4 * device_sm_count());
    k_solve_pass2<C><<<dim3(nb2, nrhs), blk, sizeof(C) * KB * 2 * NXP, s>>>(nx, nxi, (const C*)f->KinvT, p->G, p->xi_x,
                                                                           b, p->n, mask, f->sv, y, accumulate, done); klst::note_launch();
    prof_end(pass_name<C>(2), s);
    KLST_CK_LAUNCH();
    return KLST_OK;
}

// The preconditioner of the Jacobi-Davidson correction equation (one vector): mode 0 the exact
// y = (A - sigma B)^{-1} x (the Woodbury solve on x itself, its inflow rows included), mode 1 the
// block inverses alone y = K^{-1} x.  float64 factors.
int apply_inv(klst_factor f, const double2* x, double2* y, int mode, cudaStream_t s) {
    if (f->precision != KLST_FP64) { set_error("apply_inv needs a float64 factor"); return KLST_EINVAL; }
    int rc = factor_reserve(f, 1, s);
    if (rc) return rc;
    return woodbury_solve<double2>(f, x, 0, y, 0, 1, s, nullptr, mode == 1 ? 1 : 0);
}

int apply_T(klst_factor f, const double2* x, double2* y, int nrhs, cudaStream_t s) {
    int rc = factor_reserve(f, nrhs, s);
    if (rc) return rc;
    if (f->precision == KLST_FP64) return woodbury_solve<double2>(f, x, 1, y, 0, nrhs, s, nullptr);
    if (f->precision == KLST_DF64) return woodbury_solve<float4>(f, x, 1, y, 0, nrhs, s, nullptr);
    klst_pencil p = f->p;
    // y0 = T~ x (float32 blocks), then float64 refinement sweeps on r = B x - (A - sigma B) y
    KLST_CK(cudaMemsetAsync(f->done, 0, sizeof(int) * nrhs, s));
    rc = woodbury_solve<float2>(f, x, 1, y, 0, nrhs, s, nullptr);
    if (rc) return rc;
    const int nblk = pencil_rows_blocks(p);
    for (int it = 0; it <= f->max_refine; ++it) {
        const int last = it == f->max_refine;
        prof_begin("refine_residual", s);
        prof_begin("refine_moments", s);
        rc = moments_dev(p, y, p->n, nrhs, f->t, f->tpart, f->ngroups, s, f->done);
        prof_end("refine_moments", s);
        if (rc) return rc;
        if (f->tc_resid && !f->arith) {
            prof_begin("refine_dx_tc", s);
            rc = oz_dx_apply(p->dx_oz, p->nx, p->nxi, y, p->n, nrhs, f->zwork, f->ozws, f->status, s, f->done);
            prof_end("refine_dx_tc", s);
            if (rc) return rc;
            prof_begin("refine_rows", s);
            rc = pencil_rows_z_dev(p, f->t, f->zwork, y, p->n, nrhs, f->sigma_dev, 1, x, 1, f->rwork, f->normpart, s,
                                   f->done);
            prof_end("refine_rows", s);
        } else {
            rc = pencil_rows_dev(p, f->t, y, p->n, nrhs, f->sigma_dev, 1, x, 1, f->rwork, f->normpart, s, f->done,
                                 f->arith);
        }
        if (rc) return rc;
        k_refine_check<<<nrhs, 32, 0, s>>>(nblk, f->normpart, f->refine_tol, f->done, f->worst, f->sweeps, last,
                                            f->status); klst::note_launch();
        prof_end("refine_residual", s);
        KLST_CK_LAUNCH();
        if (last) break;
        rc = woodbury_solve<float2>(f, f->rwork, 0, y, 1, nrhs, s, f->done);
        if (rc) return rc;
    }
    return KLST_OK;
}

}  // namespace klst

using namespace klst;

extern "C" int klst_apply_shift_invert(klst_factor f, const void* x, void* y, int32_t nrhs, klst_stream stream) {
    if (!f || !x || !y || nrhs < 1) { set_error("invalid arguments to klst_apply_shift_invert"); return KLST_EINVAL; }
    if (x == y) { set_error("x and y may not alias"); return KLST_EINVAL; }
    return apply_T(f, (const double2*)x, (double2*)y, nrhs, (cudaStream_t)stream);
}
