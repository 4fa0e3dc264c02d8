// The Gilbarg-Paolucci continuum shock structure (Sec. 2.1, Eq. GB1DShockeqn) and its thickness
// Delta = (u_inf - u_2) / max|du/dx| (Eq. ShockThickness), for a batch of cases on the device.
//
// The pair of printed equations is restated from the steady one-dimensional Navier-Stokes balances
// they come from (monatomic gas, R = 1/2, rho_inf = T_inf = 1, u_inf = M sqrt(5/6)):
//     (4/3) mu du/dx          = m u + m T / (2u) - P
//     (5/4) (mu / Pr) dT/dx   = (3/4) m T - m u^2 / 2 + P u - m H
// with m = u_inf, P = 1/2 + m u_inf, H = 5/4 + u_inf^2 / 2 and mu = (u_inf / Re) T^s.  Their ratio in
// Omega = (m/P) u, theta = (m/P)^2 T / 2 is the printed dtheta/dOmega with the constant (4/5) Pr.
//
// One thread integrates one case: classical RK4 in x with a fixed step, from the downstream
// Rankine-Hugoniot state (a saddle) displaced by eps u_2 along its stable eigenvector, backward in x
// until the upstream state is reached to 1e-13 (the state kept with compensated sums, so that the
// approach to the upstream node does not stall at the state's last bit).  The steepest point is the
// sign change of d^2u/dx^2 = grad(du/dx) . (du/dx, dT/dx) next to the largest sampled |du/dx|,
// found by bisection on the length of a partial RK4 step.  A second pass re-integrates the same
// steps and evaluates the profile at given points (measured from the steepest point) by partial RK4
// steps; past the start point it is the saddle's linear solution y_2 + eps u_2 v exp(lambda_s x),
// past the end the upstream state.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace klst {
namespace {

constexpr double kGamma = 5.0 / 3.0;
constexpr double kReach = 1e-13;   // relative distance to the upstream state that ends the integration

struct GpSys {
    double m, P, H, u1, T1, u2, T2, rmu, s, Pr;   // rmu = 1 / mu(T = 1) = Re / u_inf

    __device__ void init(const klst_gp_case& c) {
        const double M = c.mach;
        u1 = M * sqrt(kGamma / 2.0);
        T1 = 1.0;
        const double r = (kGamma + 1.0) * M * M / ((kGamma - 1.0) * M * M + 2.0);
        const double p2 = 0.5 * (1.0 + 2.0 * kGamma * (M * M - 1.0) / (kGamma + 1.0));
        u2 = u1 / r;
        T2 = 2.0 * p2 / r;
        m = u1;
        P = 0.5 + m * u1;
        H = 1.25 + 0.5 * u1 * u1;
        rmu = c.re / u1;
        s = c.visc_s;
        Pr = c.prandtl;
    }
    // 1 / mu(T); FP64 is a narrow pipe on this part, so the common exponents avoid the general power
    __device__ __forceinline__ double inv_mu(double T) const {
        return rmu * (s == 0.5 ? rsqrt(T) : s == 1.0 ? 1.0 / T : pow(T, -s));
    }
    __device__ __forceinline__ void f(double u, double T, double& du, double& dT) const {
        const double im = inv_mu(T);
        du = 0.75 * im * (m * u + 0.5 * m * T / u - P);
        dT = 0.8 * Pr * im * (0.75 * m * T - 0.5 * m * u * u + P * u - m * H);
    }
    // Jacobian of f (the terms from d(1/mu)/dT vanish at the end states, where f = 0)
    __device__ void jac(double u, double T, double J[4]) const {
        const double im = inv_mu(T), a = 0.75 * im, b = 0.8 * Pr * im;
        double du, dT;
        f(u, T, du, dT);
        J[0] = a * (m - 0.5 * m * T / (u * u));
        J[1] = a * (0.5 * m / u) - du * s / T;
        J[2] = b * (P - m * u);
        J[3] = b * 0.75 * m - dT * s / T;
    }
    // d^2u/dx^2 along the solution through (u, T)
    __device__ double curvature(double u, double T) const {
        double J[4], du, dT;
        jac(u, T, J);
        f(u, T, du, dT);
        return J[0] * du + J[1] * dT;
    }
    // the increment of one RK4 step of length h from (u, T), k1 = f(u, T) given
    __device__ void rk4_inc(double u, double T, double k1u, double k1T, double h, double& du, double& dT) const {
        double k2u, k2T, k3u, k3T, k4u, k4T;
        f(u + 0.5 * h * k1u, T + 0.5 * h * k1T, k2u, k2T);
        f(u + 0.5 * h * k2u, T + 0.5 * h * k2T, k3u, k3T);
        f(u + h * k3u, T + h * k3T, k4u, k4T);
        du = h / 6.0 * (k1u + 2.0 * k2u + 2.0 * k3u + k4u);
        dT = h / 6.0 * (k1T + 2.0 * k2T + 2.0 * k3T + k4T);
    }
    __device__ void rk4(double u, double T, double k1u, double k1T, double h, double& un, double& Tn) const {
        double du, dT;
        rk4_inc(u, T, k1u, k1T, h, du, dT);
        un = u + du;
        Tn = T + dT;
    }
    // a full step of the integration: the state advanced with compensated (Kahan) sums, so that near
    // the upstream node the increments, far below the state's last bit, still accumulate
    __device__ void advance(double& u, double& T, double& cu, double& cT, double ku, double kT, double h) const {
        double du, dT;
        rk4_inc(u, T, ku, kT, h, du, dT);
        const double iu = du - cu, iT = dT - cT;
        const double su = u + iu, sT = T + iT;
        cu = (su - u) - iu;
        cT = (sT - T) - iT;
        u = su;
        T = sT;
    }
    __device__ bool reached(double u, double T) const {
        return fabs(u - u1) <= kReach * u1 && fabs(T - T1) <= kReach * T1;
    }
};

// eigenvalues (real parts and moduli bound) of a 2x2 matrix
__device__ void eig2(const double J[4], double& lo, double& hi, double& absmax) {
    const double tr = J[0] + J[3], det = J[0] * J[3] - J[1] * J[2];
    const double disc = 0.25 * tr * tr - det;
    if (disc >= 0.0) {
        const double r = sqrt(disc);
        // the root of larger modulus first, the other from det / it (no cancellation)
        const double big = tr >= 0.0 ? 0.5 * tr + r : 0.5 * tr - r;
        const double small = big != 0.0 ? det / big : 0.0;
        lo = fmin(big, small);
        hi = fmax(big, small);
        absmax = fmax(fabs(big), fabs(small));
    } else {
        lo = hi = 0.5 * tr;
        absmax = sqrt(det);
    }
}

__global__ void k_gp_shock(const klst_gp_case* cases, const int* cidx, int n, double step, double eps, int max_steps,
                           const double* xs, const int* perm, int npts, double* prof, klst_gp_result* res) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int c = cidx ? cidx[t] : t;   // the case's index in the caller's order
    GpSys S;
    S.init(cases[t]);
    klst_gp_result out;
    out.status = KLST_OK;
    // the end states' Jacobians: the stable direction at the saddle and the step length
    double J2[4], J1[4], lo2, hi2, a2, lo1, hi1, a1;
    S.jac(S.u2, S.T2, J2);
    S.jac(S.u1, S.T1, J1);
    eig2(J2, lo2, hi2, a2);
    eig2(J1, lo1, hi1, a1);
    const double lam = lo2;   // < 0 at a saddle
    double vu = J2[1], vT = lam - J2[0];
    {
        const double wu = lam - J2[3], wT = J2[2];   // the other form of the same eigenvector
        if (wu * wu + wT * wT > vu * vu + vT * vT) { vu = wu; vT = wT; }
        const double nv = sqrt(vu * vu + vT * vT);
        vu /= nv; vT /= nv;
        if (vu < 0.0) { vu = -vu; vT = -vT; }
    }
    const double h = -step / fmax(a1, a2);
    const double U0 = S.u2 + eps * S.u2 * vu, T0 = S.T2 + eps * S.u2 * vT;
    // pass 1: integrate, keep the largest |du/dx| sample and its neighbours
    double u = U0, T = T0, cu = 0.0, cT = 0.0, ku, kT;
    S.f(u, T, ku, kT);
    double best = fabs(ku), ub = u, Tb = T, up = u, Tp = T, un = u, Tn = T;
    int kb = 0, k = 0;
    bool want_next = true;
    while (k < max_steps && !S.reached(u, T)) {
        const double uo = u, To = T;
        S.advance(u, T, cu, cT, ku, kT, h);
        S.f(u, T, ku, kT);
        ++k;
        if (fabs(ku) > best) {
            best = fabs(ku); up = uo; Tp = To; ub = u; Tb = T; kb = k; want_next = true;
        } else if (want_next) {
            un = u; Tn = T; want_next = false;
        }
    }
    const int steps = k;
    if (!S.reached(u, T)) out.status = KLST_ENOCONV;
    // the steepest point: the sign change of d^2u/dx^2 on [x_{kb-1}, x_kb] or [x_kb, x_{kb+1}]
    const double cp = kb > 0 ? S.curvature(up, Tp) : 0.0, cb = S.curvature(ub, Tb);
    const double cn = !want_next ? S.curvature(un, Tn) : 0.0;
    double x0 = kb * h, ua = ub, Ta = Tb, cl = cb;   // left end of the bracketing step, in the direction of h
    bool bracket = false;
    if (kb > 0 && cp * cb <= 0.0) { x0 = (kb - 1) * h; ua = up; Ta = Tp; cl = cp; bracket = true; }
    else if (!want_next && cb * cn <= 0.0) { bracket = true; }
    double xshock = kb * h, us = ub, Ts = Tb;
    if (bracket) {
        double ka, kTa;
        S.f(ua, Ta, ka, kTa);
        double t0 = 0.0, t1 = 1.0;
        for (int it = 0; it < 64 && t1 - t0 > 1e-16; ++it) {
            const double tm = 0.5 * (t0 + t1);
            double um, Tm;
            S.rk4(ua, Ta, ka, kTa, tm * h, um, Tm);
            const double cm = S.curvature(um, Tm);
            if (cm * cl > 0.0) t0 = tm; else t1 = tm;
        }
        const double t = 0.5 * (t0 + t1);
        S.rk4(ua, Ta, ka, kTa, t * h, us, Ts);
        xshock = x0 + t * h;
    }
    double dus, dTs;
    S.f(us, Ts, dus, dTs);
    out.delta = (S.u1 - S.u2) / fabs(dus);
    out.x_shock = xshock;
    out.x_up = steps * h;
    out.lambda_s = lam;
    out.steps = steps;
    res[c] = out;
    if (npts <= 0) return;
    // pass 2: the profile at the points, in decreasing x
    auto put = [&](int i, double uu, double TT) {
        const int o = perm ? perm[i] : i;
        prof[((size_t)0 * n + c) * npts + o] = S.m / uu;
        prof[((size_t)1 * n + c) * npts + o] = uu;
        prof[((size_t)2 * n + c) * npts + o] = TT;
    };
    int i = 0;
    for (; i < npts && xshock + xs[i] > 0.0; ++i) {   // past the start point: the linear solution
        const double tail = eps * S.u2 * exp(lam * (xshock + xs[i]));
        put(i, S.u2 + tail * vu, S.T2 + tail * vT);
    }
    u = U0; T = T0; cu = cT = 0.0;
    S.f(u, T, ku, kT);
    for (k = 0; k < steps && i < npts; ++k) {
        const double xk = k * h, xk1 = (k + 1) * h;
        for (; i < npts && xshock + xs[i] > xk1; ++i) {
            double uu, TT;
            S.rk4(u, T, ku, kT, xshock + xs[i] - xk, uu, TT);
            put(i, uu, TT);
        }
        S.advance(u, T, cu, cT, ku, kT, h);
        S.f(u, T, ku, kT);
    }
    for (; i < npts; ++i) put(i, S.u1, S.T1);   // past the integrated range: the upstream state
}

}  // namespace

// Launches the batch: cases, result and profile in device memory; cidx (device, or null for the
// identity) the caller's index of each case (results and profile rows are written there); xs (device)
// sorted in decreasing order, perm (device, or null) the output column of each sorted point.
int gp_shock_device(const klst_gp_case* cases, const int* cidx, int n, double step, double eps, int max_steps,
                    const double* xs, const int* perm, int npts, double* prof, klst_gp_result* res, cudaStream_t s) {
    if (n <= 0) return KLST_OK;
    // one warp per CTA: a batch of a few thousand cases still spreads over every SM
    k_gp_shock<<<(n + 31) / 32, 32, 0, s>>>(cases, cidx, n, step, eps, max_steps, xs, perm, npts, prof, res);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KLST_OK : cuda_fail(e, "k_gp_shock", __FILE__, __LINE__);
}

bool gp_case_valid(const klst_gp_case& c) {
    return c.mach >= 1.01 && c.mach <= 100.0 && c.re > 0.0 && std::isfinite(c.re) && c.visc_s >= 0.0 &&
           c.visc_s <= 2.0 && c.prandtl > 0.0 && c.prandtl <= 10.0;
}

}  // namespace klst

using namespace klst;

extern "C" int klst_gp_shock(const klst_gp_case* cases, int32_t ncases, const klst_gp_opts* opts, const double* x,
                             int32_t npts, void* profile, klst_gp_result* results, klst_stream stream) {
    if (ncases < 0 || (ncases > 0 && (!cases || !results)) || npts < 0 || (npts > 0 && (!x || !profile))) {
        set_error("invalid arguments to klst_gp_shock");
        return KLST_EINVAL;
    }
    double step = 0.02, eps = 1e-6;
    int max_steps = 1 << 20;
    if (opts) {
        if (opts->step != 0.0) step = opts->step;
        if (opts->eps != 0.0) eps = opts->eps;
        if (opts->max_steps != 0) max_steps = opts->max_steps;
    }
    if (!(step > 0.0 && step <= 0.5) || !(eps > 0.0 && eps <= 1e-3) || max_steps < 1 || max_steps > (1 << 26)) {
        set_error("invalid Gilbarg-Paolucci options (0 < step <= 0.5, 0 < eps <= 1e-3, 1 <= max_steps <= 2^26)");
        return KLST_EINVAL;
    }
    for (int i = 0; i < ncases; ++i)
        if (!gp_case_valid(cases[i])) {
            set_error("invalid Gilbarg-Paolucci case %d (1.01 <= mach <= 100, re > 0, 0 <= visc_s <= 2, 0 < prandtl <= 10)", i);
            return KLST_EINVAL;
        }
    for (int i = 0; i < npts; ++i)
        if (!std::isfinite(x[i])) { set_error("x[%d] is not finite", i); return KLST_EINVAL; }
    if (ncases == 0) return KLST_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> order(npts);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return x[a] > x[b]; });
    std::vector<double> xsorted(npts);
    for (int i = 0; i < npts; ++i) xsorted[i] = x[order[i]];
    // cases in decreasing Mach number: the steps a case takes grow as M -> 1, and a warp runs as long
    // as its longest case, so neighbours of similar length keep the lanes busy
    std::vector<int> corder(ncases);
    std::iota(corder.begin(), corder.end(), 0);
    std::stable_sort(corder.begin(), corder.end(), [&](int a, int b) { return cases[a].mach > cases[b].mach; });
    std::vector<klst_gp_case> csorted(ncases);
    for (int i = 0; i < ncases; ++i) csorted[i] = cases[corder[i]];
    const size_t bytes = sizeof(klst_gp_case) * ncases + sizeof(klst_gp_result) * ncases + sizeof(double) * npts +
                         sizeof(int) * npts + sizeof(int) * ncases + 64;
    char* buf = nullptr;
    cudaError_t e = dmalloc((void**)&buf, bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    klst_gp_case* dc = (klst_gp_case*)buf;
    klst_gp_result* dr = (klst_gp_result*)(dc + ncases);
    double* dx = (double*)(((uintptr_t)(dr + ncases) + 15) & ~(uintptr_t)15);
    int* dp = (int*)(dx + npts);
    int* di = dp + npts;
    int rc = KLST_OK;
    if ((e = cudaMemcpyAsync(dc, csorted.data(), sizeof(klst_gp_case) * ncases, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(di, corder.data(), sizeof(int) * ncases, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (npts > 0 && ((e = cudaMemcpyAsync(dx, xsorted.data(), sizeof(double) * npts, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
                      (e = cudaMemcpyAsync(dp, order.data(), sizeof(int) * npts, cudaMemcpyHostToDevice, s)) != cudaSuccess)))
        rc = cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__);
    if (!rc) rc = gp_shock_device(dc, di, ncases, step, eps, max_steps, dx, dp, npts, (double*)profile, dr, s);
    if (!rc && (e = cudaMemcpyAsync(results, dr, sizeof(klst_gp_result) * ncases, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        rc = cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__);
    if (!rc && (e = cudaStreamSynchronize(s)) != cudaSuccess) rc = cuda_fail(e, "gp sync", __FILE__, __LINE__);
    dfree(buf, s);
    if (rc) return rc;
    for (int i = 0; i < ncases; ++i)
        if (results[i].status != KLST_OK) {
            set_error("case %d did not reach the upstream state within max_steps", i);
            return KLST_ENOCONV;
        }
    return KLST_OK;
}
