// Matrix-free float64 pencil operator y = (A - omega B) x and the refinement residual
// r = b - (A - sigma B) y, from the rows of Eqs. comp_ghat1Dshock / comp_hhat1Dshock.
#include "df64.cuh"
#include "factor.cuh"

namespace klst {

static __host__ __device__ inline int nxp_of(int nx) { return (nx + 31) & ~31; }

// mpart[(rhs*ngroups + g)*4*nx + a*nx + j] = sum_{k in group g, c} w^c_a(j,k) x_{c,k}(j)
__global__ void k_moments_partial(int nx, int nxi, const double* __restrict__ w, const double2* __restrict__ x,
                                  int64_t ldx, int ngroups, int kpg, double2* __restrict__ mpart) {
    extern __shared__ double2 red[];
    const int j = threadIdx.x, kk = threadIdx.y, KB = blockDim.y, g = blockIdx.x, rhs = blockIdx.y;
    const double2* xr = x + rhs * ldx;
    double2 acc[4] = {mk(0, 0), mk(0, 0), mk(0, 0), mk(0, 0)};
    const int k0 = g * kpg, k1 = min(nxi, k0 + kpg);
    if (j < nx) {
        for (int k = k0 + kk; k < k1; k += KB) {
            double2 xg = xr[(size_t)k * nx + j], xh = xr[((size_t)nxi + k) * nx + j];
            const double* wk = w + (size_t)k * 8 * nx + j;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                double wg = wk[a * nx], wh = wk[(4 + a) * nx];
                acc[a].x += wg * xg.x + wh * xh.x;
                acc[a].y += wg * xg.y + wh * xh.y;
            }
        }
    }
    const int NXP = blockDim.x;
#pragma unroll
    for (int a = 0; a < 4; ++a) red[(kk * 4 + a) * NXP + j] = acc[a];
    __syncthreads();
    if (kk == 0 && j < nx) {
        for (int a = 0; a < 4; ++a) {
            double2 s = mk(0, 0);
            for (int q = 0; q < KB; ++q) s = s + red[(q * 4 + a) * NXP + j];
            mpart[((size_t)rhs * ngroups + g) * 4 * nx + a * nx + j] = s;
        }
    }
}

// out[rhs*len + i] = sum_g part[(rhs*ngroups + g)*len + i]: one warp per output, lanes over groups in
// a fixed stride, then a fixed shuffle tree (deterministic, latency-parallel).
__global__ void __launch_bounds__(128) k_reduce_groups(int len, int ngroups, const double2* __restrict__ part,
                                                       double2* __restrict__ out, const int* done) {
    // one CTA of 4 warps per output: each thread sums groups tid, tid + 128, ... (independent
    // loads, two accumulators), then the 4 warps combine in a fixed order
    const int rhs = blockIdx.y, i = blockIdx.x;
    if (done && done[rhs]) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const double2* pr = part + (size_t)rhs * ngroups * len + i;
    double2 a0 = mk(0, 0), a1 = mk(0, 0);
    int g = tid;
    for (; g + 128 < ngroups; g += 256) {
        const double2 u = pr[(size_t)g * len], v = pr[(size_t)(g + 128) * len];
        a0 = a0 + u;
        a1 = a1 + v;
    }
    if (g < ngroups) a0 = a0 + pr[(size_t)g * len];
    double sx = warp_sum(a0.x + a1.x), sy = warp_sum(a0.y + a1.y);
    __shared__ double2 red[4];
    if (lane == 0) red[wid] = mk(sx, sy);
    __syncthreads();
    if (tid == 0) out[(size_t)rhs * len + i] = ((red[0] + red[1]) + red[2]) + red[3];
}

// Rows of (A - omega B) x (mode 0) or the residual b - (A - sigma B) x (mode 1, b masked by B
// when mask_b).  Boundary rows: (A - omega B) x = x.  normpart receives per-block sums of |y|^2
// and |b|^2 (mode 1).
// DF = true forms the D_x product in double-float (df64) arithmetic on the float32 pipes; the
// diagonal, coupling and residual terms stay float64.
template <bool DF>
__global__ void k_pencil_rows(int nx, int nxi, double beta, const double* __restrict__ DxT,
                              const double* __restrict__ xi_x, const double* __restrict__ xi_y,
                              const double* __restrict__ nu, const double* __restrict__ G,
                              const double2* __restrict__ m, const double2* __restrict__ x, int64_t ldx,
                              const double2* __restrict__ omega, int mode, const double2* __restrict__ b,
                              int mask_b, double2* __restrict__ y, double* __restrict__ normpart,
                              const int* __restrict__ done) {
    extern __shared__ double smem[];
    const int NXP = blockDim.x, KB = blockDim.y;
    const int j = threadIdx.x, kk = threadIdx.y, rhs = blockIdx.y;
    if (done && done[rhs]) return;
    double* sD = smem;                                   // nx*nx column-major D_x
    double2* sx = (double2*)(smem + nx * nx + (nx * nx & 1));  // [KB][2][NXP]
    double* sred = (double*)(sx + KB * 2 * NXP);         // [KB*NXP][2]
    const int tid = kk * NXP + j, nthr = NXP * KB;
    df* sDf = reinterpret_cast<df*>(sD);
    float4* sxf = reinterpret_cast<float4*>(sx);
    for (int i = tid; i < nx * nx; i += nthr) {
        if constexpr (DF) sDf[i] = df_from(DxT[i]);
        else sD[i] = DxT[i];
    }
    const double2* xr = x + rhs * ldx;
    const double2* br = b ? b + rhs * ldx : nullptr;
    double2* yr = y + rhs * ldx;
    const double2 om = omega ? omega[rhs] : mk(0, 0);
    const double2* mr = m + (size_t)rhs * 4 * nx;
    double nrm_y = 0.0, nrm_b = 0.0;
    for (int kb = blockIdx.x * KB; kb < nxi; kb += gridDim.x * KB) {
        const int k = kb + kk;
        const bool valid = (k < nxi) && (j < nx);
        __syncthreads();
        if (valid) {
            if constexpr (DF) {
                cdf_store(&sxf[(kk * 2 + 0) * NXP + j], cdf_from(xr[(size_t)k * nx + j]));
                cdf_store(&sxf[(kk * 2 + 1) * NXP + j], cdf_from(xr[((size_t)nxi + k) * nx + j]));
            } else {
                sx[(kk * 2 + 0) * NXP + j] = xr[(size_t)k * nx + j];
                sx[(kk * 2 + 1) * NXP + j] = xr[((size_t)nxi + k) * nx + j];
            }
        }
        __syncthreads();
        if (!valid) continue;
        const double xix = xi_x[k], xiy = xi_y[k];
        const bool bc = is_bc(j, nx, xix);
        for (int c = 0; c < 2; ++c) {
            const double2* xs = sx + (kk * 2 + c) * NXP;
            double2 d = mk(0, 0);
            if constexpr (DF) {
                const float4* xsf = sxf + (kk * 2 + c) * NXP;
                cdf dd = cdf_zero();
                for (int mm = 0; mm < nx; ++mm) {
                    const df dv = sDf[mm * nx + j];
                    const cdf xv = cdf_load(xsf + mm);
                    df_fma(dd.re, dv, xv.re);
                    df_fma(dd.im, dv, xv.im);
                }
                d = cdf_to(dd);
            } else {
                for (int mm = 0; mm < nx; ++mm) {
                    double dv = sD[mm * nx + j];
                    d.x = fma(dv, xs[mm].x, d.x);
                    d.y = fma(dv, xs[mm].y, d.y);
                }
            }
            const double2 xv = xr[((size_t)c * nxi + k) * nx + j];
            double2 val;
            if (bc) {
                val = xv;
            } else {
                const double2 diag = mk(nu[j] - om.x, beta * xiy - om.y);
                val = xix * d + diag * xv;
                const double* Gk = G + ((size_t)k * 2 + c) * 4 * nx + j;
#pragma unroll
                for (int a = 0; a < 4; ++a) val = val - Gk[a * nx] * mr[a * nx + j];
            }
            const size_t idx = ((size_t)c * nxi + k) * nx + j;
            if (mode == 1) {
                double2 bv = br[idx];
                if (mask_b && bc) bv = mk(0, 0);
                val = bv - val;
                nrm_b += abs2(bv);
            }
            nrm_y += abs2(val);
            yr[idx] = val;
        }
    }
    if (normpart) {
        __syncthreads();
        sred[2 * tid] = nrm_y;
        sred[2 * tid + 1] = nrm_b;
        __syncthreads();
        if (tid == 0) {
            double a0 = 0, a1 = 0;
            for (int i = 0; i < nthr; ++i) { a0 += sred[2 * i]; a1 += sred[2 * i + 1]; }
            normpart[((size_t)rhs * gridDim.x + blockIdx.x) * 2 + 0] = a0;
            normpart[((size_t)rhs * gridDim.x + blockIdx.x) * 2 + 1] = a1;
        }
    }
}

// The same rows as k_pencil_rows with the D_x products z (one per velocity block and component,
// layout of x) already formed, one entry per thread: the diagonal, the moment coupling, the inflow
// rows and the residual and norm bookkeeping, all float64.
__global__ void __launch_bounds__(256) k_pencil_rows_z(int nx, int nxi, double beta, const double* __restrict__ xi_x,
                                                       const double* __restrict__ xi_y, const double* __restrict__ nu,
                                                       const double* __restrict__ G, const double2* __restrict__ m,
                                                       const double2* __restrict__ z, const double2* __restrict__ x,
                                                       int64_t ldx, const double2* __restrict__ omega, int mode,
                                                       const double2* __restrict__ b, int mask_b,
                                                       double2* __restrict__ y, double* __restrict__ normpart,
                                                       const int* __restrict__ done) {
    const int rhs = blockIdx.y;
    if (done && done[rhs]) return;
    const int64_t n = 2 * (int64_t)nxi * nx, per = (int64_t)nxi * nx;
    const double2* xr = x + rhs * ldx;
    const double2* zr = z + rhs * ldx;
    const double2* br = b ? b + rhs * ldx : nullptr;
    double2* yr = y + rhs * ldx;
    const double2 om = omega ? omega[rhs] : mk(0, 0);
    const double2* mr = m + (size_t)rhs * 4 * nx;
    double nrm_y = 0.0, nrm_b = 0.0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / per);
        const int64_t rem = idx - c * per;
        const int k = (int)(rem / nx), j = (int)(rem - (int64_t)k * nx);
        const double xix = xi_x[k];
        const bool bc = is_bc(j, nx, xix);
        const double2 xv = xr[idx];
        double2 val;
        if (bc) {
            val = xv;
        } else {
            const double2 diag = mk(nu[j] - om.x, beta * xi_y[k] - om.y);
            val = xix * zr[idx] + diag * xv;
            const double* Gk = G + ((size_t)k * 2 + c) * 4 * nx + j;
#pragma unroll
            for (int a = 0; a < 4; ++a) val = val - Gk[a * nx] * mr[a * nx + j];
        }
        if (mode == 1) {
            double2 bv = br[idx];
            if (mask_b && bc) bv = mk(0, 0);
            val = bv - val;
            nrm_b += abs2(bv);
        }
        nrm_y += abs2(val);
        yr[idx] = val;
    }
    if (normpart) {
        __shared__ double red[2][8];
        nrm_y = warp_sum(nrm_y);
        nrm_b = warp_sum(nrm_b);
        if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = nrm_y; red[1][threadIdx.x >> 5] = nrm_b; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a0 = 0, a1 = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a0 += red[0][q]; a1 += red[1][q]; }
            normpart[((size_t)rhs * gridDim.x + blockIdx.x) * 2 + 0] = a0;
            normpart[((size_t)rhs * gridDim.x + blockIdx.x) * 2 + 1] = a1;
        }
    }
}

int pencil_rows_blocks(klst_pencil p);

int pencil_rows_z_dev(klst_pencil p, const double2* m, const double2* z, const double2* x, int64_t ldx, int nrhs,
                      const double2* omega, int mode, const double2* b, int mask_b, double2* y, double* normpart,
                      cudaStream_t s, const int* done) {
    dim3 grd(pencil_rows_blocks(p), nrhs);
    k_pencil_rows_z<<<grd, 256, 0, s>>>(p->nx, p->nxi, p->desc.beta, p->xi_x, p->xi_y, p->nu, p->G, m, z, x, ldx, omega,
                                        mode, b, mask_b, y, normpart, done);
    note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

void k_reduce_groups_ext(int len, int ngroups, const double2* part, double2* out, const int* done, int nrhs,
                         cudaStream_t s) {
    k_reduce_groups<<<dim3(len, nrhs), 128, 0, s>>>(len, ngroups, part, out, done); klst::note_launch();
}

int pencil_work_groups(klst_pencil p) {
    int sms = device_sm_count();
    int g = std::min(p->nxi, 2 * sms);
    return g < 1 ? 1 : g;
}

int pencil_rows_blocks(klst_pencil p) {
    int KB = 256 / nxp_of(p->nx);
    int nb = (p->nxi + KB - 1) / KB;
    return std::min(nb, 2 * device_sm_count());
}

size_t pencil_rows_smem(klst_pencil p) {
    int NXP = nxp_of(p->nx), KB = 256 / NXP;
    return sizeof(double) * (p->nx * p->nx + 1) + sizeof(double2) * KB * 2 * NXP + sizeof(double) * 2 * KB * NXP;
}

// moments m = V^H x for all rhs (into mwork, layout [rhs][4][nx])
int moments_dev(klst_pencil p, const double2* x, int64_t ldx, int nrhs, double2* mwork, double2* mpart,
                int ngroups, cudaStream_t s, const int* done) {
    const int NXP = nxp_of(p->nx), KB = 256 / NXP;
    const int kpg = (p->nxi + ngroups - 1) / ngroups;
    dim3 blk(NXP, KB), grd(ngroups, nrhs);
    k_moments_partial<<<grd, blk, sizeof(double2) * 4 * KB * NXP, s>>>(p->nx, p->nxi, p->w, x, ldx, ngroups, kpg, mpart); klst::note_launch();
    k_reduce_groups<<<dim3(4 * p->nx, nrhs), 128, 0, s>>>(4 * p->nx, ngroups, mpart, mwork, done); klst::note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

int pencil_rows_dev(klst_pencil p, const double2* m, const double2* x, int64_t ldx, int nrhs, const double2* omega,
                    int mode, const double2* b, int mask_b, double2* y, double* normpart, cudaStream_t s,
                    const int* done, int df_arith) {
    const int NXP = nxp_of(p->nx), KB = 256 / NXP;
    const size_t smem = pencil_rows_smem(p);
    static std::atomic<unsigned long long> attr_set{0};
    set_once_per_device(attr_set, [] {
        cudaError_t e = cudaFuncSetAttribute(k_pencil_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pencil_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return e;
    });
    dim3 blk(NXP, KB), grd(pencil_rows_blocks(p), nrhs);
    if (df_arith)
        k_pencil_rows<true><<<grd, blk, smem, s>>>(p->nx, p->nxi, p->desc.beta, p->DxT, p->xi_x, p->xi_y, p->nu, p->G,
                                                  m, x, ldx, omega, mode, b, mask_b, y, normpart, done);
    else
        k_pencil_rows<false><<<grd, blk, smem, s>>>(p->nx, p->nxi, p->desc.beta, p->DxT, p->xi_x, p->xi_y, p->nu, p->G,
                                                   m, x, ldx, omega, mode, b, mask_b, y, normpart, done); klst::note_launch();
    KLST_CK_LAUNCH();
    return KLST_OK;
}

int apply_pencil_dev(klst_pencil p, const double2* x, double2* y, int nrhs, const double2* omega_dev,
                     cudaStream_t s, double2* mwork, double2* mpart, int ngroups) {
    int rc = moments_dev(p, x, p->n, nrhs, mwork, mpart, ngroups, s, nullptr);
    if (rc) return rc;
    return pencil_rows_dev(p, mwork, x, p->n, nrhs, omega_dev, 0, nullptr, 0, y, nullptr, s, nullptr, 0);
}

}  // namespace klst

using namespace klst;

extern "C" int klst_apply_pencil(klst_pencil p, const void* x, void* y, int32_t nrhs, const double* omega,
                                 klst_stream stream) {
    if (!p || !x || !y || nrhs < 1) { set_error("invalid arguments to klst_apply_pencil"); return KLST_EINVAL; }
    if (x == y) { set_error("x and y may not alias"); return KLST_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int ng = pencil_work_groups(p);
    double2 *mw = nullptr, *mp = nullptr, *om = nullptr;
    cudaError_t e;
    if ((e = dmalloc((void**)&mw, sizeof(double2) * 4 * p->nx * nrhs, s)) != cudaSuccess ||
        (e = dmalloc((void**)&mp, sizeof(double2) * 4 * p->nx * (size_t)ng * nrhs, s)) != cudaSuccess ||
        (e = dmalloc((void**)&om, sizeof(double2) * nrhs, s)) != cudaSuccess) {
        dfree(mw, s);
        dfree(mp, s);
        return cuda_fail(e, "cudaMallocAsync", __FILE__, __LINE__);
    }
    if (omega) e = cudaMemcpyAsync(om, omega, sizeof(double2) * nrhs, cudaMemcpyHostToDevice, s);
    else e = cudaMemsetAsync(om, 0, sizeof(double2) * nrhs, s);
    int rc = e != cudaSuccess ? cuda_fail(e, "copy omega", __FILE__, __LINE__)
                              : apply_pencil_dev(p, (const double2*)x, (double2*)y, nrhs, om, s, mw, mp, ng);
    dfree(mw, s);
    dfree(mp, s);
    dfree(om, s);
    if (rc == KLST_OK && omega) KLST_CK(cudaStreamSynchronize(s));  // host omega buffer must outlive the copy
    return rc;
}
