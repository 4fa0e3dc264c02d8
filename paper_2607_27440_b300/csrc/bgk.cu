// The BE-BGK base-flow solver (Sec. 3.3, Eq. BoltzmannBGK_reduced) on the device.
//
//   dq/dt = RHS(q) = nu (q^e - q) - xi_x dq/dx,   q = (g, h) on the mapped Chebyshev nodes
//
// * streaming: second-order finite volumes with MUSCL reconstruction and the minmod limiter in the
//   paper's form (slopes are plain differences of neighbouring node values, minmod(a, b) =
//   (sgn a + sgn b)/2 min(|a|, |b|)), the interface value taken from the upwind side of each node
//   velocity; cell i spans the midpoints to its neighbours; a stencil past an end repeats the end
//   value;
// * relaxation: toward the discrete equilibrium of the node's own moments (the Maxwellian whose
//   discrete moments equal them, by Newton on (rho', u', T'): the equilibrium the pencil
//   linearises), nu = P / mu(T), mu = (u_inf / Re_Delta) T^s;
// * ends: Dirichlet, the upstream Maxwellian and the Rankine-Hugoniot downstream Maxwellian refined
//   so that its discrete fluxes of mass, momentum and energy equal the upstream ones;
// * time: classical RK4, `check_every` steps captured as one CUDA graph;
// * adaptive re-centring: the interval of largest |dU/dx| of the bulk velocity locates the shock;
//   when it has moved more than `recentre_tol` from the map centre the nodes are rebuilt about it and
//   g, h are moved onto them by linear interpolation in x, the ends re-imposed.
// The start is a Mott-Smith profile about x = 0, or the local Maxwellian of the Gilbarg-Paolucci
// continuum profile with its steepest point at x = 0 (gp.cu).  Layout: q[(c Nxi + k) Nx + i], c in (g, h), i the
// node in increasing x (i = 0 upstream).  The result is written in the pencil's node order.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "kinetic.cuh"

namespace klst {
namespace {

struct BgkConst {
    int nx, nxi, qx, qy;               // nodes, velocity nodes (k = kx qy + ky on the tensor grid)
    double uinf, re, s, width;         // u_inf, Re_Delta, viscosity exponent, Mott-Smith width
    double rho1, u1, T1, rho2, u2, T2; // upstream and continuous Rankine-Hugoniot states
};

// Newton on the equilibrium parameters: stop once the update is below kNewtonTol (relative to
// |value| + 1) or after kNewtonMax updates.  Started from the node's previous parameters, a time step
// changes them by far less than 1e-3, so two or three updates reach the tolerance.
constexpr int kNewtonMax = 30;
constexpr double kNewtonTol = 1e-14;

__device__ __forceinline__ double minmod(double a, double b) {
    const double sa = (a > 0.0) - (a < 0.0), sb = (b > 0.0) - (b < 0.0);
    return 0.5 * (sa + sb) * fmin(fabs(a), fabs(b));
}

// the discrete fluxes (mass, momentum, energy) of a Maxwellian and their derivatives with respect
// to (rho, u, T), summed over the CTA; F[3], J[9] row-major
__device__ void maxwellian_fluxes(const double* xi_x, const double* xi_y, const double* W, int nxi, double r, double u,
                                  double T, double* F, double* J, double* sm) {
    double acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = 0.0;
    for (int k = threadIdx.x; k < nxi; k += blockDim.x) {
        const double xx = xi_x[k], xy = xi_y[k], Wk = W[k];
        const double g = maxw(r, u, T, xx, xy), dxu = xx - u, e2 = xx * xx + xy * xy;
        const double phi = -1.0 / T + (dxu * dxu + xy * xy) / (T * T);
        const double dg[3] = {g / r, g * 2.0 * dxu / T, g * phi};
        acc[0] += Wk * xx * g;
        acc[1] += Wk * xx * xx * g;
        acc[2] += 0.5 * Wk * xx * (e2 * g + 0.5 * T * g);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const double dh = 0.5 * T * dg[b] + (b == 2 ? 0.5 * g : 0.0);
            acc[3 + b] += Wk * xx * dg[b];
            acc[6 + b] += Wk * xx * xx * dg[b];
            acc[9 + b] += 0.5 * Wk * xx * (e2 * dg[b] + dh);
        }
    }
    block_sum<12>(acc, sm);
    for (int i = 0; i < 3; ++i) F[i] = acc[i];
    for (int i = 0; i < 9; ++i) J[i] = acc[3 + i];
}

// One CTA: the downstream end state (rho, u, T) whose discrete fluxes equal the upstream
// Maxwellian's, by Newton from the continuous Rankine-Hugoniot state; ends[0..2] upstream,
// ends[3..5] downstream parameters
__global__ void __launch_bounds__(256) k_bgk_ends(BgkConst c, const double* xi_x, const double* xi_y, const double* W,
                                                  double* ends) {
    __shared__ double sm[32 * 12 + 12];
    __shared__ double s_th[4];
    double F0[3], J0[9], F[3], J[9];
    maxwellian_fluxes(xi_x, xi_y, W, c.nxi, c.rho1, c.u1, c.T1, F0, J0, sm);
    if (threadIdx.x == 0) { s_th[0] = c.rho2; s_th[1] = c.u2; s_th[2] = c.T2; s_th[3] = 0.0; }
    __syncthreads();
    for (int it = 0; it < 50; ++it) {
        maxwellian_fluxes(xi_x, xi_y, W, c.nxi, s_th[0], s_th[1], s_th[2], F, J, sm);
        if (threadIdx.x == 0) {
            double r[3] = {F0[0] - F[0], F0[1] - F[1], F0[2] - F[2]};
            small_solve(3, J, r);
            double mx = 0.0;
            for (int i = 0; i < 3; ++i) {
                s_th[i] += r[i];
                mx = fmax(mx, fabs(r[i]) / fabs(s_th[i]));
            }
            s_th[3] = mx < 1e-15 ? 1.0 : 0.0;
        }
        __syncthreads();
        if (s_th[3] != 0.0) break;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ends[0] = c.rho1; ends[1] = c.u1; ends[2] = c.T1;
        ends[3] = s_th[0]; ends[4] = s_th[1]; ends[5] = s_th[2];
    }
}

// Physical-order nodes x_i = x_pencil[nx - 1 - i] + centre and the inverse interior cell widths;
// one CTA (also: the smallest cell width and the largest |xi_x| into lim[0], lim[1])
__global__ void k_bgk_grid(int nx, int nxi, const double* x_pencil, double centre, const double* xi_x, double* x,
                           double* dxinv, double* lim) {
    for (int i = threadIdx.x; i < nx; i += blockDim.x) x[i] = x_pencil[nx - 1 - i] + centre;
    __syncthreads();
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        if (i == 0 || i == nx - 1) { dxinv[i] = 0.0; continue; }
        const double xr = 0.5 * (x[i] + x[i + 1]), xl = 0.5 * (x[i - 1] + x[i]);
        dxinv[i] = 1.0 / (xr - xl);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double dmin = 1e300, xm = 0.0;
        for (int i = 1; i < nx - 1; ++i) dmin = fmin(dmin, 0.5 * (x[i + 1] - x[i - 1]));
        for (int k = 0; k < nxi; ++k) xm = fmax(xm, fabs(xi_x[k]));
        lim[0] = dmin;
        lim[1] = xm;
    }
}

// the Mott-Smith start about x = 0 (continuous end states in the mixture), ends set to the end states
__global__ void k_bgk_init(BgkConst c, const double* x, const double* xi_x, const double* xi_y, const double* ends,
                           const double* gp, double* q) {
    const int nx = c.nx, nxi = c.nxi;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nx * nxi; idx += gridDim.x * blockDim.x) {
        const int k = idx / nx, i = idx - k * nx;
        const double xx = xi_x[k], xy = xi_y[k];
        double g, h;
        if (i == 0 || i == nx - 1) {
            const double* e = ends + (i == 0 ? 0 : 3);
            g = maxw(e[0], e[1], e[2], xx, xy);
            h = 0.5 * e[2] * g;
        } else if (gp) {   // the Gilbarg-Paolucci profile, [3][nx] in the pencil's node order
            const int j = nx - 1 - i;
            g = maxw(gp[j], gp[nx + j], gp[2 * nx + j], xx, xy);
            h = 0.5 * gp[2 * nx + j] * g;
        } else {
            const double sx = 0.5 * (1.0 + tanh(x[i] / c.width));
            const double g1 = maxw(c.rho1, c.u1, c.T1, xx, xy), g2 = maxw(c.rho2, c.u2, c.T2, xx, xy);
            g = (1.0 - sx) * g1 + sx * g2;
            h = (1.0 - sx) * (0.5 * c.T1) * g1 + sx * (0.5 * c.T2) * g2;
        }
        q[(size_t)k * nx + i] = g;
        q[(size_t)(nxi + k) * nx + i] = h;
    }
}

// the ends of a state re-imposed (after a regrid)
__global__ void k_bgk_set_ends(BgkConst c, const double* xi_x, const double* xi_y, const double* ends, double* q) {
    const int nx = c.nx, nxi = c.nxi;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * nxi; idx += gridDim.x * blockDim.x) {
        const int k = idx >> 1, side = idx & 1, i = side ? nx - 1 : 0;
        const double* e = ends + 3 * side;
        const double g = maxw(e[0], e[1], e[2], xi_x[k], xi_y[k]);
        q[(size_t)k * nx + i] = g;
        q[(size_t)(nxi + k) * nx + i] = 0.5 * e[2] * g;
    }
}

// One CTA per interior node i: discrete moments of q(., i), the discrete equilibrium parameters
// (Newton, started from the node's previous parameters, or from the moments the first time),
// nu = P / mu; th[4 i + (0, 1, 2)] = (rho', u', T'), nu[i], ubulk[i]; the largest nu into *numax
// (its bits: non-negative doubles order as integers)
//
// The Maxwellian is separable on the tensor-product velocity grid: g^e(kx, ky) = rho / (pi T)
// exp(-(xi_x,kx - u)^2 / T) exp(-xi_y,ky^2 / T), so a Newton iteration takes qx + qy exponentials
// (kept in shared memory) instead of one per velocity node, and the reciprocals of T and rho once.
// The final parameters' factors go to eqt for the stage kernel: eqt[kx nx + i] = rho / (pi T)
// exp(-(xi_x,kx - u)^2 / T), eqt[(qx + ky) nx + i] = exp(-xi_y,ky^2 / T).
__global__ void __launch_bounds__(128) k_bgk_eq(BgkConst c, const double* __restrict__ q, const double* xi_x,
                                                const double* xi_y, const double* W, double* th, double* nu,
                                                double* ubulk, unsigned long long* numax, unsigned long long* newton,
                                                double* eqt) {
    __shared__ double sm[32 * 12 + 12];
    __shared__ double s_th[4];
    __shared__ double s_ex[256], s_ey[256];
    const int nx = c.nx, nxi = c.nxi, i = blockIdx.x + 1;
    double mom[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < nxi; k += blockDim.x) {
        const double g = q[(size_t)k * nx + i], h = q[(size_t)(nxi + k) * nx + i];
        const double xx = xi_x[k], xy = xi_y[k], Wk = W[k];
        mom[0] += Wk * g;
        mom[1] += Wk * xx * g;
        mom[2] += Wk * (xx * xx + xy * xy) * g;
        mom[3] += Wk * h;
    }
    block_sum<4>(mom, sm);
    const double rho = mom[0], u = mom[1] / rho, E = 0.5 * (mom[2] + mom[3]) / rho;
    const double T = (4.0 / 3.0) * (E - 0.5 * u * u);
    if (threadIdx.x == 0) {
        const bool warm = th[4 * i + 3] != 0.0;
        s_th[0] = warm ? th[4 * i] : rho;
        s_th[1] = warm ? th[4 * i + 1] : u;
        s_th[2] = warm ? th[4 * i + 2] : T;
        s_th[3] = 0.0;
    }
    __syncthreads();
    int its = 0;
    for (int it = 0; it < kNewtonMax; ++it) {
        ++its;
        const double r_ = s_th[0], u_ = s_th[1], T_ = s_th[2];
        const double iT = 1.0 / T_, ir = 1.0 / r_, pref = r_ * iT * (1.0 / M_PI);
        for (int a = threadIdx.x; a < c.qx + c.qy; a += blockDim.x) {
            if (a < c.qx) {
                const double d = xi_x[a * c.qy] - u_;
                s_ex[a] = pref * exp(-(d * d) * iT);
            } else {
                const double y = xi_y[a - c.qx];
                s_ey[a - c.qx] = exp(-(y * y) * iT);
            }
        }
        __syncthreads();
        double acc[12];
#pragma unroll
        for (int a = 0; a < 12; ++a) acc[a] = 0.0;
        for (int k = threadIdx.x; k < nxi; k += blockDim.x) {
            const int kx = k / c.qy, ky = k - kx * c.qy;
            const double xx = xi_x[k], xy = xi_y[k], Wk = W[k];
            const double ge = s_ex[kx] * s_ey[ky], dxu = xx - u_, e2 = xx * xx + xy * xy;
            const double phi = (dxu * dxu + xy * xy) * (iT * iT) - iT;
            const double dg[3] = {ge * ir, ge * 2.0 * dxu * iT, ge * phi};
            acc[0] += Wk * ge;
            acc[1] += Wk * xx * ge;
            acc[2] += 0.5 * Wk * (e2 * ge + 0.5 * T_ * ge);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const double dh = 0.5 * T_ * dg[b] + (b == 2 ? 0.5 * ge : 0.0);
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
            const double t0 = r_ + r[0], t1 = u_ + r[1], t2 = T_ + r[2];
            const double mx = fmax(fabs(r[0]) / (fabs(t0) + 1.0), fmax(fabs(r[1]) / (fabs(t1) + 1.0), fabs(r[2]) / (fabs(t2) + 1.0)));
            s_th[0] = t0; s_th[1] = t1; s_th[2] = t2;
            s_th[3] = mx < kNewtonTol ? 1.0 : 0.0;
        }
        __syncthreads();
        if (s_th[3] != 0.0) break;
        __syncthreads();
    }
    {   // the final parameters' factors for the stage kernel
        const double r_ = s_th[0], u_ = s_th[1], T_ = s_th[2];
        const double iT = 1.0 / T_, pref = r_ * iT * (1.0 / M_PI);
        for (int a = threadIdx.x; a < c.qx + c.qy; a += blockDim.x) {
            double v;
            if (a < c.qx) {
                const double d = xi_x[a * c.qy] - u_;
                v = pref * exp(-(d * d) * iT);
            } else {
                const double y = xi_y[a - c.qx];
                v = exp(-(y * y) * iT);
            }
            eqt[(size_t)a * nx + i] = v;
        }
    }
    if (threadIdx.x == 0) {
        atomicAdd(newton, (unsigned long long)its);
        th[4 * i] = s_th[0];
        th[4 * i + 1] = s_th[1];
        th[4 * i + 2] = s_th[2];
        th[4 * i + 3] = 1.0;
        const double P = 0.5 * rho * T, mu = (c.uinf / c.re) * pow(T, c.s), v = P / mu;
        nu[i] = v;
        ubulk[i] = u;
        atomicMax(numax, (unsigned long long)__double_as_longlong(v));
    }
}

// One RK4 stage for the interior nodes, both components of node velocity k at node i per thread:
// r = nu (q^e - q) - xi_x (phi_{i+1/2} - phi_{i-1/2}) / dx_i on the stage input qs, then
//   stage 0: acc = r;                 qn = q0 + (dt/2) r
//   stage 1: acc += 2 r;              qn = q0 + (dt/2) r
//   stage 2: acc += 2 r;              qn = q0 + dt r
//   stage 3: q0 = q0 + (dt/6)(acc + r)
// track: the largest |r| and |g| of this stage into res[0], res[1] (bits)
__global__ void __launch_bounds__(256) k_bgk_stage(BgkConst c, int stage, const double* __restrict__ qs,
                                                   double* __restrict__ q0, double* __restrict__ qn,
                                                   double* __restrict__ acc, const double* __restrict__ dxinv,
                                                   const double* xi_x, const double* __restrict__ th,
                                                   const double* __restrict__ eqt, const double* __restrict__ nu,
                                                   const double* dtp, int track, unsigned long long* res) {
    const int nx = c.nx, nxi = c.nxi;
    const double dt = *dtp;
    double rmax = 0.0, gmax = 0.0;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nx * nxi; idx += gridDim.x * blockDim.x) {
        const int k = idx / nx, i = idx - k * nx;
        if (i == 0 || i == nx - 1) continue;
        const double xx = xi_x[k];
        const int kx = k / c.qy, ky = k - kx * c.qy;
        const double ge = eqt[(size_t)kx * nx + i] * eqt[(size_t)(c.qx + ky) * nx + i];   // k_bgk_eq's factors
        const double eq[2] = {ge, 0.5 * th[4 * i + 2] * ge};
        const int im2 = max(i - 2, 0), ip2 = min(i + 2, nx - 1);
#pragma unroll
        for (int comp = 0; comp < 2; ++comp) {
            const double* p = qs + (size_t)(comp * nxi + k) * nx;
            const double pm2 = p[im2], pm1 = p[i - 1], p0 = p[i], pp1 = p[i + 1], pp2 = p[ip2];
            double fr, fl;   // phi_{i+1/2}, phi_{i-1/2}
            if (xx >= 0.0) {
                fr = p0 + 0.5 * minmod(p0 - pm1, pp1 - p0);
                fl = pm1 + 0.5 * minmod(pm1 - pm2, p0 - pm1);
            } else {
                fr = pp1 - 0.5 * minmod(pp1 - p0, pp2 - pp1);
                fl = p0 - 0.5 * minmod(p0 - pm1, pp1 - p0);
            }
            const double stream = xx * (fr - fl) * dxinv[i];
            const double r = nu[i] * (eq[comp] - p0) - stream;
            const size_t at = (size_t)(comp * nxi + k) * nx + i;
            if (track) {
                rmax = fmax(rmax, fabs(r));
                if (comp == 0) gmax = fmax(gmax, fabs(p0));
            }
            if (stage == 0) {
                acc[at] = r;
                qn[at] = q0[at] + 0.5 * dt * r;
            } else if (stage < 3) {
                const double a = acc[at] + 2.0 * r;
                acc[at] = a;
                qn[at] = q0[at] + (stage == 1 ? 0.5 * dt : dt) * r;
            } else {
                q0[at] = q0[at] + dt / 6.0 * (acc[at] + r);
            }
        }
    }
    if (track) {
        for (int o = 16; o > 0; o >>= 1) {
            rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMax(res, (unsigned long long)__double_as_longlong(rmax));
            atomicMax(res + 1, (unsigned long long)__double_as_longlong(gmax));
        }
    }
}

// One CTA: the shock location, the midpoint of the interval with the largest |dU/dx| of the
// piecewise-linear bulk velocity (ends: the end states' velocities)
__global__ void k_bgk_shock(int nx, const double* x, const double* ubulk, const double* ends, double* xs) {
    if (threadIdx.x != 0) return;
    double best = -1.0;
    int bi = 0;
    for (int i = 0; i + 1 < nx; ++i) {
        const double ua = i == 0 ? ends[1] : ubulk[i];
        const double ub = i + 1 == nx - 1 ? ends[4] : ubulk[i + 1];
        const double sl = fabs((ub - ua) / (x[i + 1] - x[i]));
        if (sl > best) { best = sl; bi = i; }
    }
    *xs = 0.5 * (x[bi] + x[bi + 1]);
}

// q moved from the nodes xo onto xn by linear interpolation in x (clamped to the end values
// outside), into qo
__global__ void k_bgk_regrid(int nx, int nxi, const double* xo, const double* xn, const double* __restrict__ q,
                             double* __restrict__ out) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * nx * nxi; idx += gridDim.x * blockDim.x) {
        const int row = idx / nx, i = idx - row * nx;
        const double* p = q + (size_t)row * nx;
        const double xv = xn[i];
        double v;
        if (xv <= xo[0]) v = p[0];
        else if (xv >= xo[nx - 1]) v = p[nx - 1];
        else {
            int lo = 0, hi = nx - 1;   // xo[lo] < xv <= xo[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (xo[mid] < xv) lo = mid; else hi = mid;
            }
            const double t = (xv - xo[lo]) / (xo[hi] - xo[lo]);
            v = p[lo] + t * (p[hi] - p[lo]);
        }
        out[idx] = v;
    }
}

// the state in the pencil's node order: g_out[j][k] = q[0][k][nx - 1 - j]
__global__ void k_bgk_out(int nx, int nxi, const double* __restrict__ q, double* __restrict__ g, double* __restrict__ h) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nx * nxi; idx += gridDim.x * blockDim.x) {
        const int j = idx / nxi, k = idx - j * nxi, i = nx - 1 - j;
        g[idx] = q[(size_t)k * nx + i];
        h[idx] = q[(size_t)(nxi + k) * nx + i];
    }
}

double bits_to_double(unsigned long long b) {
    double v;
    memcpy(&v, &b, sizeof v);
    return v;
}

}  // namespace
}  // namespace klst

using namespace klst;

extern "C" int klst_bgk_base_flow(const klst_pencil_desc* d, const klst_bgk_opts* o, void* g_out, void* h_out,
                                  klst_bgk_info* info, klst_stream stream) {
    if (!d || !o || !g_out || !h_out) { set_error("invalid arguments to klst_bgk_base_flow"); return KLST_EINVAL; }
    if (o->max_steps < 0 || !(o->cfl > 0) || o->check_every < 1 || o->recentre_every < 0 ||
        (o->recentre_every > 0 && o->recentre_every % o->check_every != 0) || !(o->tol >= 0) || !(o->dt >= 0) ||
        !(o->recentre_tol > 0) || (o->start != 0 && o->start != 1)) {
        set_error("invalid BE-BGK options (cfl > 0, check_every >= 1, recentre_every a multiple of check_every, start 0 or 1)");
        return KLST_EINVAL;
    }
    const klst_gp_case gpc = {d->mach, d->re_delta, d->visc_s, 1.0};
    if (o->start == 1 && (fabs(d->gamma - 5.0 / 3.0) > 1e-12 || !gp_case_valid(gpc))) {
        set_error("the Gilbarg-Paolucci start needs gamma = 5/3, 1.01 <= mach <= 100 and 0 <= visc_s <= 2");
        return KLST_EINVAL;
    }
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t user = (cudaStream_t)stream;
    klst_pencil p = nullptr;
    int rc = klst_build_pencil(d, stream, &p);   // the nodes and the velocity grid
    if (rc) return rc;
    const int nx = p->nx, nxi = p->nxi;
    const size_t nq = (size_t)2 * nx * nxi;
    cudaStream_t s = nullptr;
    cudaError_t e;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    double* buf = nullptr;
    auto fail = [&](int code) {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (buf) dfree(buf, s ? s : user);
        if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
        if (ev) cudaEventDestroy(ev);
        klst_pencil_destroy(p);
        return code;
    };
    // a private capturable stream, ordered after the caller's stream and before its later work
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventRecord(ev, user)) != cudaSuccess || (e = cudaStreamWaitEvent(s, ev, 0)) != cudaSuccess)
        return fail(cuda_fail(e, "bgk stream", __FILE__, __LINE__));
    // workspace: q0, two stage buffers, acc, a regrid buffer, node arrays, per-node tables
    const size_t nd = 5 * nq + 4 * (size_t)nx + 4 * (size_t)nx + 2 * (size_t)nx + 16 + 3 * (size_t)nx + 16 +
                      (size_t)(d->qx + d->qy) * nx;
    if ((e = dmalloc((void**)&buf, sizeof(double) * nd, s)) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    double *q0 = buf, *qa = q0 + nq, *qb = qa + nq, *acc = qb + nq, *qr = acc + nq;
    double *x = qr + nq, *xnew = x + nx, *dxinv = xnew + nx, *ubulk = dxinv + nx;
    double *th = ubulk + nx, *nu = th + 4 * (size_t)nx, *scratch = nu + 2 * (size_t)nx;
    double* ends = scratch;          // 6
    double* lim = scratch + 6;       // 2
    double* dtd = scratch + 8;       // 1
    double* xs = scratch + 9;        // 1
    unsigned long long* res = (unsigned long long*)(scratch + 10);     // 2: max|r|, max|g|
    unsigned long long* numax = (unsigned long long*)(scratch + 12);   // 1
    unsigned long long* newton = (unsigned long long*)(scratch + 13);  // 1: Newton updates in total
    double* gpb = scratch + 16;      // the Gilbarg-Paolucci start: rho, u, T at the nodes, its case and result
    double* eqt = gpb + 3 * nx + 16; // the equilibrium's separable factors per node ((qx + qy) x nx)
    cudaMemsetAsync(th, 0, sizeof(double) * 4 * nx, s);
    cudaMemsetAsync(nu, 0, sizeof(double) * nx, s);
    cudaMemsetAsync(ubulk, 0, sizeof(double) * nx, s);
    cudaMemsetAsync(acc, 0, sizeof(double) * nq, s);
    cudaMemsetAsync(newton, 0, sizeof(unsigned long long), s);
    BgkConst c;
    c.nx = nx; c.nxi = nxi; c.qx = d->qx; c.qy = d->qy;
    {
        const double g = d->gamma, M = d->mach;
        c.rho1 = 1.0; c.T1 = 1.0; c.u1 = M * sqrt(g / 2.0);
        const double r = (g + 1.0) * M * M / ((g - 1.0) * M * M + 2.0);
        const double p1 = 0.5, p2 = p1 * (1.0 + 2.0 * g * (M * M - 1.0) / (g + 1.0));
        c.rho2 = r; c.u2 = c.u1 / r; c.T2 = 2.0 * p2 / c.rho2;
        c.uinf = c.u1; c.re = d->re_delta; c.s = d->visc_s; c.width = d->width;
    }
    const int nb = (int)std::min<size_t>((nx * (size_t)nxi + 255) / 256, 4096);
    double centre = 0.0;
    k_bgk_grid<<<1, 128, 0, s>>>(nx, nxi, p->x, 0.0, p->xi_x, x, dxinv, lim); note_launch();
    k_bgk_ends<<<1, 256, 0, s>>>(c, p->xi_x, p->xi_y, p->W, ends); note_launch();
    klst_gp_result gpr;
    gpr.status = KLST_OK;
    if (o->start == 1) {   // the pencil's nodes are in decreasing x: the order the integration visits them
        klst_gp_case* dc = (klst_gp_case*)(gpb + 3 * nx);
        klst_gp_result* dr = (klst_gp_result*)(gpb + 3 * nx + 8);
        if ((e = cudaMemcpyAsync(dc, &gpc, sizeof gpc, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return fail(cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__));
        if ((rc = gp_shock_device(dc, nullptr, 1, 0.02, 1e-6, 1 << 20, p->x, nullptr, nx, gpb, dr, s))) return fail(rc);
        if ((e = cudaMemcpyAsync(&gpr, dr, sizeof gpr, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return fail(cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__));
    }
    k_bgk_init<<<nb, 256, 0, s>>>(c, x, p->xi_x, p->xi_y, ends, o->start == 1 ? gpb : nullptr, q0); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_fail(e, "bgk setup", __FILE__, __LINE__));
    // the stage buffers carry the end values too (never written by the stages)
    cudaMemcpyAsync(qa, q0, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(qb, q0, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
    double hlim[2];
    cudaMemsetAsync(numax, 0, sizeof(unsigned long long), s);
    k_bgk_eq<<<nx - 2, 128, 0, s>>>(c, q0, p->xi_x, p->xi_y, p->W, th, nu, ubulk, numax, newton, eqt); note_launch();
    unsigned long long hnu = 0;
    if ((e = cudaMemcpyAsync(hlim, lim, sizeof hlim, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&hnu, numax, sizeof hnu, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(cuda_fail(e, "bgk setup", __FILE__, __LINE__));
    if (gpr.status != KLST_OK) {
        set_error("the Gilbarg-Paolucci start did not reach the upstream state");
        return fail(KLST_ENOCONV);
    }
    auto pick_dt = [&](double numax_v) {
        if (o->dt > 0) return o->dt;
        return std::min(o->cfl * hlim[0] / hlim[1], numax_v > 0 ? 2.0 / numax_v : 1e300);
    };
    double dt = pick_dt(bits_to_double(hnu));
    if ((e = cudaMemcpyAsync(dtd, &dt, sizeof dt, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(cuda_fail(e, "bgk dt", __FILE__, __LINE__));
    // one graph: check_every RK4 steps, the last step's first stage tracking the residual
    const int G = o->check_every;
    auto rk4 = [&](int track) {
        const double* in[4] = {q0, qa, qb, qa};
        double* outb[4] = {qa, qb, qa, nullptr};
        for (int st = 0; st < 4; ++st) {
            k_bgk_eq<<<nx - 2, 128, 0, s>>>(c, in[st], p->xi_x, p->xi_y, p->W, th, nu, ubulk, numax, newton, eqt);
            k_bgk_stage<<<nb, 256, 0, s>>>(c, st, in[st], q0, outb[st] ? outb[st] : qa, acc, dxinv, p->xi_x, th, eqt,
                                           nu, dtd, st == 0 ? track : 0, res);
        }
    };
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return fail(cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__));
    set_capturing(true);
    cudaMemsetAsync(res, 0, 2 * sizeof(unsigned long long), s);
    cudaMemsetAsync(numax, 0, sizeof(unsigned long long), s);
    for (int st = 0; st < G; ++st) rk4(st == G - 1 ? 1 : 0);
    set_capturing(false);
    e = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
    if (e != cudaSuccess) return fail(cuda_fail(e, "bgk graph", __FILE__, __LINE__));
    int steps = 0, recentres = 0;
    double resid = -1.0;
    while (steps + G <= o->max_steps) {
        if ((e = cudaGraphLaunch(gexec, s)) != cudaSuccess) return fail(cuda_fail(e, "cudaGraphLaunch", __FILE__, __LINE__));
        note_launches(8ull * G);
        steps += G;
        unsigned long long hr[2] = {0, 0};
        if ((e = cudaMemcpyAsync(hr, res, sizeof hr, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&hnu, numax, sizeof hnu, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return fail(cuda_fail(e, "bgk check", __FILE__, __LINE__));
        const double rmax = bits_to_double(hr[0]), gmax = bits_to_double(hr[1]);
        resid = gmax > 0 ? rmax / gmax : rmax;
        if (!std::isfinite(resid)) {
            set_error("BE-BGK solve diverged (non-finite residual after %d steps; lower cfl)", steps);
            return fail(KLST_ENOCONV);
        }
        if (o->tol > 0 && resid <= o->tol) break;
        if (o->recentre_every > 0 && steps % o->recentre_every == 0) {
            // the bulk velocity of the current state (the stages' last moments are of a stage input)
            k_bgk_eq<<<nx - 2, 128, 0, s>>>(c, q0, p->xi_x, p->xi_y, p->W, th, nu, ubulk, numax, newton, eqt); note_launch();
            k_bgk_shock<<<1, 32, 0, s>>>(nx, x, ubulk, ends, xs); note_launch();
            double hxs = 0;
            if ((e = cudaMemcpyAsync(&hxs, xs, sizeof hxs, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess)
                return fail(cuda_fail(e, "bgk shock", __FILE__, __LINE__));
            if (fabs(hxs - centre) > o->recentre_tol) {
                k_bgk_grid<<<1, 128, 0, s>>>(nx, nxi, p->x, hxs, p->xi_x, xnew, dxinv, lim); note_launch();
                k_bgk_regrid<<<nb, 256, 0, s>>>(nx, nxi, x, xnew, q0, qr); note_launch();
                cudaMemcpyAsync(q0, qr, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
                cudaMemcpyAsync(x, xnew, sizeof(double) * nx, cudaMemcpyDeviceToDevice, s);
                k_bgk_set_ends<<<(2 * nxi + 255) / 256, 256, 0, s>>>(c, p->xi_x, p->xi_y, ends, q0); note_launch();
                cudaMemcpyAsync(qa, q0, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
                cudaMemcpyAsync(qb, q0, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s);
                cudaMemsetAsync(th, 0, sizeof(double) * 4 * nx, s);   // restart the Newton from the moments
                if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_fail(e, "bgk regrid", __FILE__, __LINE__));
                centre = hxs;
                ++recentres;
            }
        }
        if (o->dt <= 0) {
            const double ndt = pick_dt(bits_to_double(hnu));
            if (ndt != dt) {
                dt = ndt;
                if ((e = cudaMemcpyAsync(dtd, &dt, sizeof dt, cudaMemcpyHostToDevice, s)) != cudaSuccess)
                    return fail(cuda_fail(e, "bgk dt", __FILE__, __LINE__));
            }
        }
    }
    k_bgk_out<<<nb, 256, 0, s>>>(nx, nxi, q0, (double*)g_out, (double*)h_out); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventRecord(ev, s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(user, ev, 0)) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(cuda_fail(e, "bgk output", __FILE__, __LINE__));
    unsigned long long hnewton = 0;
    cudaMemcpy(&hnewton, newton, sizeof hnewton, cudaMemcpyDeviceToHost);
    if (info) {
        info->newton_avg = steps > 0 ? (double)hnewton / ((double)(4 * (size_t)steps + 1) * (nx - 2)) : 0.0;
        info->steps = steps;
        info->recentres = recentres;
        info->resid = resid;
        info->centre = centre;
        info->dt = dt;
        info->t_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    cudaGraphExecDestroy(gexec);
    cudaGraphDestroy(graph);
    dfree(buf, s);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    cudaEventDestroy(ev);
    klst_pencil_destroy(p);
    return KLST_OK;
}
