// Pencil assembly on the device: grids (Sec. 3.1, 3.2), base state, linearisation
// coefficients (Sec. 2.2, Eq. CompBGKtilde) and the dense export used by tests.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "factor.cuh"
#include "kinetic.cuh"

namespace klst {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return e == cudaErrorMemoryAllocation ? KLST_ENOMEM : KLST_ECUDA;
}

// Host-side fault injection for tests: the n-th next device allocation fails as if the device
// were out of memory (n < 0: off).
static std::atomic<long long> g_fail_alloc_after{-1};

cudaError_t dmalloc(void** ptr, size_t bytes, cudaStream_t s) {
    long long v = g_fail_alloc_after.load();
    while (v >= 0 && !g_fail_alloc_after.compare_exchange_weak(v, v - 1)) {}
    if (v == 0) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    static bool pool_ready[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !pool_ready[dev]) {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        pool_ready[dev] = true;
    }
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    return cudaMallocAsync(ptr, bytes, s);
}

void fail_alloc_after(long long n) { g_fail_alloc_after.store(n < 0 ? -1 : n); }

void dfree(void* ptr, cudaStream_t s) {
    if (ptr) cudaFreeAsync(ptr, s);
}

int device_sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// ------------------------------------------------------------------ Gauss-Hermite
// Number of eigenvalues below lam of the symmetric tridiagonal Jacobi matrix of the
// monic Hermite recurrence (zero diagonal, off-diagonal sqrt(i/2)): Sturm sequence count.
__device__ int sturm_count(int Q, double lam) {
    int cnt = 0;
    double q = -lam;
    if (q < 0.0) cnt++;
    for (int i = 1; i < Q; ++i) {
        if (q == 0.0) q = -1e-300;
        q = -lam - (0.5 * i) / q;
        if (q < 0.0) cnt++;
    }
    return cnt;
}

// One thread per positive node: bisection on the Sturm count gives the Golub-Welsch
// eigenvalue; the full-line weight is the Christoffel form 1 / sum_{m<Q} psi_m(x)^2 with
// orthonormal Hermite functions psi_m (Sec. 3.2).  Nodes are mirrored, zero for odd Q.
__global__ void k_gauss_hermite(int Q, double* nodes, double* Wfull) {
    int t = threadIdx.x;
    int half = Q / 2;
    if (t < half) {
        int target = Q - 1 - t;  // ascending index of the positive node
        double lo = 0.0, hi = sqrt(2.0 * Q) + 2.0;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (sturm_count(Q, mid) > target) hi = mid; else lo = mid;
        }
        double x = 0.5 * (lo + hi);
        nodes[target] = x;
        nodes[t] = -x;
    }
    if ((Q & 1) && t == half) nodes[half] = 0.0;
    __syncthreads();
    if (t < Q) {
        double x = nodes[t];
        double p0 = pow(M_PI, -0.25) * exp(-0.5 * x * x), p1 = sqrt(2.0) * x * p0;
        double s = p0 * p0;
        if (Q > 1) s += p1 * p1;
        for (int m = 1; m < Q - 1; ++m) {
            double p2 = sqrt(2.0 / (m + 1)) * x * p1 - sqrt((double)m / (m + 1.0)) * p0;
            p0 = p1; p1 = p2;
            s += p2 * p2;
        }
        Wfull[t] = 1.0 / s;
    }
}

__global__ void k_velocity_grid(int qx, int qy, const double* nx_, const double* Wx, const double* ny_,
                                const double* Wy, double* xi_x, double* xi_y, double* W) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= qx * qy) return;
    int kx = k / qy, ky = k % qy;
    xi_x[k] = nx_[kx];
    xi_y[k] = ny_[ky];
    W[k] = Wx[kx] * Wy[ky];
}

// ------------------------------------------------------------------ Chebyshev + map
// D_y from Eqs. ChebDiag/ChebOffDiag/ChebBC at y_j = cos(j pi / N); x = L y / sqrt(1+s-y^2),
// dy/dx = sqrt(1+s) L^2 / (L^2+x^2)^{3/2}, D_x = diag(dy/dx) D_y (Eq. Chebmapping).
__global__ void k_cheb_map(int nx, double L, double sinf, double* x, double* Dx, double* DxT) {
    int N = nx - 1;
    double s = (L / sinf) * (L / sinf);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nx * nx; idx += gridDim.x * blockDim.x) {
        int j = idx / nx, m = idx % nx;
        double yj = cospi((double)j / N), ym = cospi((double)m / N);
        double xj = L * yj / sqrt(1.0 + s - yj * yj);
        double dydx = sqrt(1.0 + s) * L * L / pow(L * L + xj * xj, 1.5);
        double d;
        if (j != m) {
            double cj = (j == 0 || j == N) ? 2.0 : 1.0, cm = (m == 0 || m == N) ? 2.0 : 1.0;
            d = (cj / cm) * (((j + m) & 1) ? -1.0 : 1.0) / (yj - ym);
        } else if (j == 0) {
            d = (2.0 * N * N + 1.0) / 6.0;
        } else if (j == N) {
            d = -(2.0 * N * N + 1.0) / 6.0;
        } else {
            d = -yj / (2.0 * (1.0 - yj * yj));
        }
        Dx[j * nx + m] = dydx * d;
        DxT[m * nx + j] = dydx * d;
        if (m == 0) x[j] = xj;
    }
}

// ------------------------------------------------------------------ base state + coefficients
struct BaseParams {
    int nx, nxi, base, noneq, conservative;
    double mach, gamma, visc_s, re_delta, width;
    double rho1, u1, T1, rho2, u2, T2, uinf;
};

// One CTA per collocation point j.  Computes the base distributions at the nodes (or takes the
// given ones), their
// discrete moments (rho, u, E; v = 0), the discrete equilibrium (Newton on the Maxwellian
// parameters when conservative), nu = P/mu, the raw equilibrium derivatives C, the moment
// functionals w, the conservative fix C <- C (M C)^{-1}, and G = nu C + (f^e - f) d.
__global__ void k_base_state(BaseParams bp, const double* x, const double* xi_x, const double* xi_y,
                             const double* W, double* gbuf, double* hbuf, double* nu_out, double* macro,
                             double* G, double* w, double* eneq, Status* st, const double* user_g,
                             const double* user_h, const double* gp) {
    __shared__ double sm[32 * 16 + 16];
    __shared__ double s_th[4];
    __shared__ double s_MCinv[16];
    __shared__ double s_d[4];
    const int j = blockIdx.x, nxi = bp.nxi, nx = bp.nx;
    double* g = gbuf + (size_t)j * nxi;
    double* h = hbuf + (size_t)j * nxi;
    const double xj = x[j];
    const double sj = 0.5 * (1.0 + tanh(xj / bp.width));
    double rho_t = 0, u_t = 0, T_t = 0;
    if (bp.base == KLST_BASE_TANH_MAXWELL) {
        u_t = bp.u1 + (bp.u2 - bp.u1) * sj;
        rho_t = bp.rho1 * bp.u1 / u_t;
        double P1 = 0.5 * bp.rho1 * bp.T1;
        T_t = 2.0 * (P1 + bp.rho1 * bp.u1 * bp.u1 - rho_t * u_t * u_t) / rho_t;
    } else if (bp.base == KLST_BASE_GILBARG_PAOLUCCI) {   // the continuum profile at the nodes
        rho_t = gp[j]; u_t = gp[nx + j]; T_t = gp[2 * nx + j];
    }
    // base distributions and their moments
    double mom[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < nxi; k += blockDim.x) {
        double xx = xi_x[k], xy = xi_y[k], gk, hk;
        if (user_g) {  // given base distributions, [j][k]
            gk = user_g[(size_t)j * nxi + k];
            hk = user_h[(size_t)j * nxi + k];
        } else if (bp.base == KLST_BASE_TANH_MAXWELL || bp.base == KLST_BASE_GILBARG_PAOLUCCI) {
            gk = maxw(rho_t, u_t, T_t, xx, xy);
            hk = 0.5 * T_t * gk;
        } else {
            double g1 = maxw(bp.rho1, bp.u1, bp.T1, xx, xy), g2 = maxw(bp.rho2, bp.u2, bp.T2, xx, xy);
            gk = (1.0 - sj) * g1 + sj * g2;
            hk = (1.0 - sj) * (0.5 * bp.T1) * g1 + sj * (0.5 * bp.T2) * g2;
        }
        g[k] = gk;
        h[k] = hk;
        double Wk = W[k];
        mom[0] += Wk * gk;
        mom[1] += Wk * xx * gk;
        mom[2] += Wk * (xx * xx + xy * xy) * gk;
        mom[3] += Wk * hk;
    }
    block_sum<4>(mom, sm);
    const double rho = mom[0], u = mom[1] / rho, E = 0.5 * (mom[2] + mom[3]) / rho;
    const double Tc = (4.0 / 3.0) * (E - 0.5 * u * u);
    // discrete equilibrium parameters theta' = (rho', u', T')
    if (threadIdx.x == 0) { s_th[0] = rho; s_th[1] = u; s_th[2] = Tc; }
    __syncthreads();
    if (bp.conservative) {
        for (int it = 0; it < 60; ++it) {
            const double r_ = s_th[0], u_ = s_th[1], T_ = s_th[2];
            double acc[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) acc[i] = 0.0;
            for (int k = threadIdx.x; k < nxi; k += blockDim.x) {
                double xx = xi_x[k], xy = xi_y[k], Wk = W[k];
                double ge = maxw(r_, u_, T_, xx, xy);
                double dxu = xx - u_, e2 = xx * xx + xy * xy;
                double phi = -1.0 / T_ + (dxu * dxu + xy * xy) / (T_ * T_);
                double dg[3] = {ge / r_, ge * 2.0 * dxu / T_, ge * phi};
                acc[0] += Wk * ge;
                acc[1] += Wk * xx * ge;
                acc[2] += 0.5 * Wk * (e2 * ge + 0.5 * T_ * ge);
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    double dh = 0.5 * T_ * dg[b] + (b == 2 ? 0.5 * ge : 0.0);
                    acc[3 + b] += Wk * dg[b];
                    acc[6 + b] += Wk * xx * dg[b];
                    acc[9 + b] += 0.5 * Wk * (e2 * dg[b] + dh);
                }
            }
            block_sum<12>(acc, sm);
            if (threadIdx.x == 0) {
                double J[9] = {acc[3], acc[4], acc[5], acc[6], acc[7], acc[8], acc[9], acc[10], acc[11]};
                double r[3] = {-(acc[0] - rho), -(acc[1] - rho * u), -(acc[2] - rho * E)};
                small_solve(3, J, r);
                double th[3] = {r_ + r[0], u_ + r[1], T_ + r[2]};
                double mx = fmax(fabs(r[0]) / (fabs(th[0]) + 1.0), fmax(fabs(r[1]) / (fabs(th[1]) + 1.0),
                                                                     fabs(r[2]) / (fabs(th[2]) + 1.0)));
                s_th[0] = th[0]; s_th[1] = th[1]; s_th[2] = th[2];
                s_th[3] = (it >= 1 && mx < 1e-15) ? 1.0 : 0.0;
            }
            __syncthreads();
            if (s_th[3] != 0.0) break;
            __syncthreads();
        }
    }
    const double rp = s_th[0], up = s_th[1], Tp = s_th[2];
    // transport at the base moments
    const double P = 0.5 * rho * Tc;
    const double mu = (bp.uinf / bp.re_delta) * pow(Tc, bp.visc_s);
    const double nu = P / mu;
    // M C (4x4) with raw C at theta' and w at the base moments (v = 0)
    double mc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) mc[i] = 0.0;
    for (int k = threadIdx.x; k < nxi; k += blockDim.x) {
        double xx = xi_x[k], xy = xi_y[k], Wk = W[k];
        double ge = maxw(rp, up, Tp, xx, xy);
        double dxu = xx - up, phi = -1.0 / Tp + (dxu * dxu + xy * xy) / (Tp * Tp);
        double dgT = ge * phi, dhT = 0.5 * ge + 0.5 * Tp * ge * phi;
        double Cg[4] = {ge / rp, ge * 2.0 * dxu / Tp - (4.0 / 3.0) * up * dgT, ge * 2.0 * xy / Tp, (4.0 / 3.0) * dgT};
        double Ch[4] = {0.5 * Tp * ge / rp, 0.5 * Tp * ge * 2.0 * dxu / Tp - (4.0 / 3.0) * up * dhT,
                        0.5 * Tp * ge * 2.0 * xy / Tp, (4.0 / 3.0) * dhT};
        double wg[4] = {Wk, Wk * (xx - u) / rho, Wk * xy / rho, Wk * (xx * xx + xy * xy - 2.0 * E) / (2.0 * rho)};
        double whE = Wk / (2.0 * rho);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) mc[a * 4 + b] += wg[a] * Cg[b] + (a == 3 ? whE * Ch[b] : 0.0);
    }
    block_sum<16>(mc, sm);
    if (threadIdx.x == 0) {
        // inverse of M C by solving against unit vectors
        for (int col = 0; col < 4; ++col) {
            double J[16], r[4] = {0, 0, 0, 0};
            for (int i = 0; i < 16; ++i) J[i] = mc[i];
            r[col] = 1.0;
            small_solve(4, J, r);
            for (int i = 0; i < 4; ++i) s_MCinv[i * 4 + col] = bp.conservative ? r[i] : (i == col ? 1.0 : 0.0);
        }
        // d_a = dP/da / mu - P dmu/da / mu^2 at (rho, u, v = 0, E)
        double dP[4] = {0.5 * Tc, -(2.0 / 3.0) * rho * u, 0.0, (2.0 / 3.0) * rho};
        double dT[4] = {0.0, -(4.0 / 3.0) * u, 0.0, 4.0 / 3.0};
        for (int a = 0; a < 4; ++a) {
            double dmu = bp.visc_s * mu / Tc * dT[a];
            s_d[a] = dP[a] / mu - P * dmu / (mu * mu);
        }
        nu_out[j] = nu;
        macro[0 * nx + j] = rho;
        macro[1 * nx + j] = u;
        macro[2 * nx + j] = E;
        macro[3 * nx + j] = Tc;
    }
    __syncthreads();
    double dev2[1] = {0.0};  // sum_k W_k (g_c - g_c^e)^2 (Eq. L2norm)
    for (int k = threadIdx.x; k < nxi; k += blockDim.x) {
        double xx = xi_x[k], xy = xi_y[k], Wk = W[k];
        double ge = maxw(rp, up, Tp, xx, xy), he = 0.5 * Tp * ge;
        double gk = bp.noneq ? g[k] : ge, hk = bp.noneq ? h[k] : he;
        dev2[0] += Wk * (gk - ge) * (gk - ge);
        double dxu = xx - up, phi = -1.0 / Tp + (dxu * dxu + xy * xy) / (Tp * Tp);
        double dgT = ge * phi, dhT = 0.5 * ge + 0.5 * Tp * ge * phi;
        double Cr[2][4] = {{ge / rp, ge * 2.0 * dxu / Tp - (4.0 / 3.0) * up * dgT, ge * 2.0 * xy / Tp, (4.0 / 3.0) * dgT},
                           {0.5 * Tp * ge / rp, 0.5 * Tp * ge * 2.0 * dxu / Tp - (4.0 / 3.0) * up * dhT,
                            0.5 * Tp * ge * 2.0 * xy / Tp, (4.0 / 3.0) * dhT}};
        double neq[2] = {ge - gk, he - hk};
        bool bc = is_bc(j, nx, xx);
        double wv[2][4] = {{Wk, Wk * (xx - u) / rho, Wk * xy / rho, Wk * (xx * xx + xy * xy - 2.0 * E) / (2.0 * rho)},
                           {0.0, 0.0, 0.0, Wk / (2.0 * rho)}};
        for (int c = 0; c < 2; ++c) {
            for (int a = 0; a < 4; ++a) {
                double cf = 0.0;
                for (int b = 0; b < 4; ++b) cf += Cr[c][b] * s_MCinv[b * 4 + a];
                double Gv = nu * cf + neq[c] * s_d[a];
                size_t off = ((size_t)(k * 2 + c) * 4 + a) * nx + j;
                G[off] = bc ? 0.0 : Gv;
                w[off] = wv[c][a];
            }
        }
    }
    block_sum<1>(dev2, sm);
    if (threadIdx.x == 0) eneq[j] = sqrt(dev2[0]);
}

// ------------------------------------------------------------------ dense export (tests)
// Row (c, k, j) of A - sigma B: streaming xi_x D_x row, diagonal nu + i beta xi_y - sigma,
// coupling -sum_a G^c_a(j,k) w^{c'}_a(j,p) (Eqs. comp_ghat1Dshock / comp_hhat1Dshock);
// inflow rows are unit rows.
__global__ void k_export_rows(int nx, int nxi, int64_t row0, int64_t nrows, double beta, double2 sigma,
                              const double* Dx, const double* xi_x, const double* xi_y, const double* nu,
                              const double* G, const double* w, double2* out) {
    const int64_t n = 2ll * nx * nxi;
    for (int64_t rr = blockIdx.x; rr < nrows; rr += gridDim.x) {
        int64_t row = row0 + rr;
        int c = (int)(row / ((int64_t)nxi * nx));
        int k = (int)((row / nx) % nxi);
        int j = (int)(row % nx);
        double2* o = out + rr * n;
        for (int64_t col = threadIdx.x; col < n; col += blockDim.x) o[col] = mk(0, 0);
        __syncthreads();
        if (is_bc(j, nx, xi_x[k])) {
            if (threadIdx.x == 0) o[row] = mk(1, 0);
            __syncthreads();
            continue;
        }
        for (int m = threadIdx.x; m < nx; m += blockDim.x) {
            double v = xi_x[k] * Dx[j * nx + m];
            o[((int64_t)c * nxi + k) * nx + m].x += v;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < 2 * nxi; q += blockDim.x) {
            int cp = q / nxi, p = q % nxi;
            double s = 0.0;
            for (int a = 0; a < 4; ++a)
                s += G[((size_t)(k * 2 + c) * 4 + a) * nx + j] * w[((size_t)(p * 2 + cp) * 4 + a) * nx + j];
            o[((int64_t)cp * nxi + p) * nx + j].x -= s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double2& d = o[row];
            d.x += nu[j] - sigma.x;
            d.y += beta * xi_y[k] - sigma.y;
        }
        __syncthreads();
    }
}

}  // namespace klst

using namespace klst;

extern "C" const char* klst_status_string(int s) {
    switch (s) {
        case KLST_OK: return "KLST_OK";
        case KLST_EINVAL: return "KLST_EINVAL";
        case KLST_ENOMEM: return "KLST_ENOMEM";
        case KLST_ESINGULAR: return "KLST_ESINGULAR";
        case KLST_ENOCONV: return "KLST_ENOCONV";
        case KLST_EREFINE: return "KLST_EREFINE";
        case KLST_ETIMEOUT: return "KLST_ETIMEOUT";
        case KLST_ECUDA: return "KLST_ECUDA";
        default: return "KLST_UNKNOWN";
    }
}

extern "C" const char* klst_last_error(void) { return g_err; }

extern "C" void klst_pencil_destroy(klst_pencil p) {
    if (!p) return;
    double* bufs[] = {p->x, p->Dx, p->DxT, p->xi_x, p->xi_y, p->W, p->nu, p->macro, p->G, p->w, p->eneq};
    for (double* b : bufs) dfree(b, p->stream);
    dfree(p->status, p->stream);
    dfree(p->dx_oz, p->stream);
    delete p;
}

static int build_pencil(const klst_pencil_desc* d, const double* user_g, const double* user_h, klst_stream stream,
                        klst_pencil* out);

extern "C" int klst_build_pencil(const klst_pencil_desc* d, klst_stream stream, klst_pencil* out) {
    return build_pencil(d, nullptr, nullptr, stream, out);
}

extern "C" int klst_build_pencil_base(const klst_pencil_desc* d, const void* gc, const void* hc, klst_stream stream,
                                      klst_pencil* out) {
    if (!gc || !hc) {
        if (out) *out = nullptr;
        set_error("gc and hc must be device arrays of the base distributions");
        return KLST_EINVAL;
    }
    return build_pencil(d, (const double*)gc, (const double*)hc, stream, out);
}

static int build_pencil(const klst_pencil_desc* d, const double* user_g, const double* user_h, klst_stream stream,
                        klst_pencil* out) {
    if (!out) { set_error("out is NULL"); return KLST_EINVAL; }
    *out = nullptr;
    if (!d) { set_error("desc is NULL"); return KLST_EINVAL; }
    if (d->nx < 4 || d->nx > 128 || d->qx < 1 || d->qx > 256 || d->qy < 1 || d->qy > 256) {
        set_error("unsupported sizes nx=%d qx=%d qy=%d (4<=nx<=128, 1<=q<=256)", d->nx, d->qx, d->qy);
        return KLST_EINVAL;
    }
    if (!(d->mach > 1.0) || !(d->gamma > 1.0) || !(d->re_delta > 0) || !(d->map_L > 0) || !(d->map_sinf > 0) ||
        (d->base != KLST_BASE_TANH_MAXWELL && d->base != KLST_BASE_MOTT_SMITH && d->base != KLST_BASE_GILBARG_PAOLUCCI) ||
        (d->base != KLST_BASE_GILBARG_PAOLUCCI && !(d->width > 0))) {
        set_error("invalid physical parameters");
        return KLST_EINVAL;
    }
    klst_gp_case gpc = {d->mach, d->re_delta, d->visc_s, 1.0};
    if (d->base == KLST_BASE_GILBARG_PAOLUCCI && !user_g && (fabs(d->gamma - 5.0 / 3.0) > 1e-12 || !gp_case_valid(gpc))) {
        set_error("the Gilbarg-Paolucci base needs gamma = 5/3, 1.01 <= mach <= 100 and 0 <= visc_s <= 2");
        return KLST_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    klst_pencil p = new klst_pencil_s();
    memset(p, 0, sizeof(*p));
    p->desc = *d;
    p->nx = d->nx; p->qx = d->qx; p->qy = d->qy; p->nxi = d->qx * d->qy;
    p->n = 2ll * p->nx * p->nxi;
    const int nx = p->nx, nxi = p->nxi;
    double *gh = nullptr, *Wq = nullptr, *gbuf = nullptr;
    p->stream = s;
    auto fail = [&](int code) { dfree(gh, s); dfree(Wq, s); dfree(gbuf, s); klst_pencil_destroy(p); return code; };
#define ALLOC(ptr, cnt)                                                              \
    do {                                                                             \
        cudaError_t e_ = dmalloc((void**)&(ptr), (size_t)(cnt) * sizeof(*(ptr)), s); \
        if (e_ != cudaSuccess) return fail(cuda_fail(e_, "cudaMalloc", __FILE__, __LINE__)); \
        p->footprint += (int64_t)(cnt) * sizeof(*(ptr));                             \
    } while (0)
    ALLOC(p->x, nx);
    ALLOC(p->Dx, nx * nx);
    ALLOC(p->DxT, nx * nx);
    ALLOC(p->xi_x, nxi);
    ALLOC(p->xi_y, nxi);
    ALLOC(p->W, nxi);
    ALLOC(p->nu, nx);
    ALLOC(p->macro, 4 * nx);
    ALLOC(p->G, (size_t)nxi * 8 * nx);
    ALLOC(p->w, (size_t)nxi * 8 * nx);
    ALLOC(p->eneq, nx);
    ALLOC(p->status, 1);
#undef ALLOC
    cudaError_t e;
    if ((e = dmalloc((void**)&gh, sizeof(double) * (2 * 256), s)) != cudaSuccess ||
        (e = dmalloc((void**)&Wq, sizeof(double) * (2 * 256), s)) != cudaSuccess ||
        (e = dmalloc((void**)&gbuf, sizeof(double) * 2 * (size_t)nx * nxi, s)) != cudaSuccess)
        return fail(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    cudaMemsetAsync(p->status, 0, sizeof(Status), s);
    k_gauss_hermite<<<1, 256, 0, s>>>(d->qx, gh, Wq); klst::note_launch();
    k_gauss_hermite<<<1, 256, 0, s>>>(d->qy, gh + 256, Wq + 256); klst::note_launch();
    k_velocity_grid<<<(nxi + 255) / 256, 256, 0, s>>>(d->qx, d->qy, gh, Wq, gh + 256, Wq + 256, p->xi_x, p->xi_y, p->W); klst::note_launch();
    k_cheb_map<<<(nx * nx + 255) / 256, 256, 0, s>>>(nx, d->map_L, d->map_sinf, p->x, p->Dx, p->DxT); klst::note_launch();
    BaseParams bp;
    bp.nx = nx; bp.nxi = nxi; bp.base = d->base; bp.noneq = d->noneq; bp.conservative = d->conservative;
    bp.mach = d->mach; bp.gamma = d->gamma; bp.visc_s = d->visc_s; bp.re_delta = d->re_delta; bp.width = d->width;
    const double g = d->gamma, M = d->mach;
    bp.rho1 = 1.0; bp.T1 = 1.0; bp.u1 = M * sqrt(g / 2.0); bp.uinf = bp.u1;
    const double r = (g + 1.0) * M * M / ((g - 1.0) * M * M + 2.0);
    const double p1 = 0.5, p2 = p1 * (1.0 + 2.0 * g * (M * M - 1.0) / (g + 1.0));
    bp.rho2 = r; bp.u2 = bp.u1 / r; bp.T2 = 2.0 * p2 / bp.rho2;
    double* gp = nullptr;   // the Gilbarg-Paolucci profile at the nodes: rho, u, T, then the case and its result
    if (d->base == KLST_BASE_GILBARG_PAOLUCCI && !user_g) {
        const size_t words = 3 * (size_t)nx + 8 + 8;
        if ((e = dmalloc((void**)&gp, sizeof(double) * words, s)) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
        klst_gp_case* dc = (klst_gp_case*)(gp + 3 * nx);
        klst_gp_result* dr = (klst_gp_result*)(gp + 3 * nx + 8);
        int rc = KLST_OK;
        if ((e = cudaMemcpyAsync(dc, &gpc, sizeof(gpc), cudaMemcpyHostToDevice, s)) != cudaSuccess)
            rc = cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__);
        // the nodes are in decreasing x (node 0 downstream): the order the integration visits them
        if (!rc) rc = gp_shock_device(dc, nullptr, 1, 0.02, 1e-6, 1 << 20, p->x, nullptr, nx, gp, dr, s);
        klst_gp_result r;
        if (!rc && (e = cudaMemcpyAsync(&r, dr, sizeof(r), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            rc = cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__);
        if (!rc && (e = cudaStreamSynchronize(s)) != cudaSuccess) rc = cuda_fail(e, "gp sync", __FILE__, __LINE__);
        if (!rc && r.status != KLST_OK) { set_error("Gilbarg-Paolucci profile did not reach the upstream state"); rc = KLST_ENOCONV; }
        if (rc) { dfree(gp, s); return fail(rc); }
    }
    k_base_state<<<nx, 256, 0, s>>>(bp, p->x, p->xi_x, p->xi_y, p->W, gbuf, gbuf + (size_t)nx * nxi, p->nu,
                                    p->macro, p->G, p->w, p->eneq, p->status, user_g, user_h, gp); klst::note_launch();
    if (gp) dfree(gp, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_fail(e, "pencil kernels", __FILE__, __LINE__));
    // D_x as integer slices for the float64-accurate tensor-core D_x products of the operator
    {
        const size_t bytes = oz_dx_bytes(nx);
        if ((e = dmalloc(&p->dx_oz, bytes, s)) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
        p->footprint += (int64_t)bytes;
        int rc = oz_split_dx(p->Dx, nx, p->dx_oz, s);
        if (rc) return fail(rc);
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(cuda_fail(e, "build sync", __FILE__, __LINE__));
    dfree(gh, s); dfree(Wq, s); dfree(gbuf, s);
    gh = Wq = gbuf = nullptr;
    *out = p;
    return KLST_OK;
}

extern "C" int klst_pencil_dims(klst_pencil p, int64_t* n, int32_t* nx, int32_t* nxi, int64_t* fp) {
    if (!p) { set_error("pencil is NULL"); return KLST_EINVAL; }
    if (n) *n = p->n;
    if (nx) *nx = p->nx;
    if (nxi) *nxi = p->nxi;
    if (fp) *fp = p->footprint;
    return KLST_OK;
}

extern "C" int klst_pencil_tables(klst_pencil p, double* x, double* Dx, double* xi_x, double* xi_y, double* W,
                                  double* nu, double* G, double* w, uint8_t* bc) {
    if (!p) { set_error("pencil is NULL"); return KLST_EINVAL; }
    const int nx = p->nx, nxi = p->nxi;
    if (x) KLST_CK(cudaMemcpy(x, p->x, sizeof(double) * nx, cudaMemcpyDeviceToHost));
    if (Dx) KLST_CK(cudaMemcpy(Dx, p->Dx, sizeof(double) * nx * nx, cudaMemcpyDeviceToHost));
    if (xi_y) KLST_CK(cudaMemcpy(xi_y, p->xi_y, sizeof(double) * nxi, cudaMemcpyDeviceToHost));
    if (W) KLST_CK(cudaMemcpy(W, p->W, sizeof(double) * nxi, cudaMemcpyDeviceToHost));
    if (nu) KLST_CK(cudaMemcpy(nu, p->nu, sizeof(double) * nx, cudaMemcpyDeviceToHost));
    if (G) KLST_CK(cudaMemcpy(G, p->G, sizeof(double) * (size_t)nxi * 8 * nx, cudaMemcpyDeviceToHost));
    if (w) KLST_CK(cudaMemcpy(w, p->w, sizeof(double) * (size_t)nxi * 8 * nx, cudaMemcpyDeviceToHost));
    std::vector<double> xx(nxi);
    KLST_CK(cudaMemcpy(xx.data(), p->xi_x, sizeof(double) * nxi, cudaMemcpyDeviceToHost));
    if (xi_x) memcpy(xi_x, xx.data(), sizeof(double) * nxi);
    if (bc)
        for (int j = 0; j < nx; ++j)
            for (int k = 0; k < nxi; ++k) bc[(size_t)j * nxi + k] = is_bc(j, nx, xx[k]) ? 1 : 0;
    return KLST_OK;
}

extern "C" int klst_export_dense(klst_pencil p, double sr, double si, double* A_host, double* B_host) {
    if (!p) { set_error("pencil is NULL"); return KLST_EINVAL; }
    if (p->n > 16384) { set_error("export_dense supports n <= 16384 (n = %lld)", (long long)p->n); return KLST_EINVAL; }
    const int64_t n = p->n;
    const int nx = p->nx, nxi = p->nxi;
    if (A_host) {
        const int64_t chunk = std::min<int64_t>(n, (int64_t)(512ll << 20) / (n * 16) + 1);
        double2* buf = nullptr;
        KLST_CK(cudaMalloc(&buf, (size_t)chunk * n * sizeof(double2)));
        for (int64_t r0 = 0; r0 < n; r0 += chunk) {
            int64_t nr = std::min(chunk, n - r0);
            k_export_rows<<<(int)std::min<int64_t>(nr, 4096), 256>>>(nx, nxi, r0, nr, p->desc.beta, mk(sr, si), p->Dx,
                                                                     p->xi_x, p->xi_y, p->nu, p->G, p->w, buf); klst::note_launch();
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpy(A_host + 2 * r0 * n, buf, (size_t)nr * n * sizeof(double2), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { cudaFree(buf); return cuda_fail(e, "export", __FILE__, __LINE__); }
        }
        cudaFree(buf);
    }
    if (B_host) {
        std::vector<double> xx(nxi);
        KLST_CK(cudaMemcpy(xx.data(), p->xi_x, sizeof(double) * nxi, cudaMemcpyDeviceToHost));
        for (int c = 0; c < 2; ++c)
            for (int k = 0; k < nxi; ++k)
                for (int j = 0; j < nx; ++j) B_host[((int64_t)c * nxi + k) * nx + j] = is_bc(j, nx, xx[k]) ? 0.0 : 1.0;
    }
    return KLST_OK;
}
