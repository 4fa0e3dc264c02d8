"""Gilbarg-Paolucci continuum shock structure (oracle; test infrastructure only): Sec. 2.1, Eq.
GB1DShockeqn, and the shock thickness of Eq. ShockThickness.

The printed pair is garbled (its dtheta/dOmega carries 8/15, which its own z-equations give as 2/5,
and beta, delta are not defined), so the equations are restated from the steady one-dimensional
Navier-Stokes balances they come from, for a monatomic gas in the kLST units (R = 1/2,
rho_inf = T_inf = 1, u_inf = M sqrt(gamma/2), c_v = 3R/2, c_p = 5R/2):
    mass         rho u = m
    momentum     (4/3) mu(T) du/dx = m u + m R T / u - P
    energy       (c_p / Pr) mu(T) dT/dx = m c_v T - m u^2 / 2 + P u - m H
with P = p_inf + m u_inf and H = c_p T_inf + u_inf^2 / 2 (the paper's m, P, E), mu = (u_inf / Re) T^s.
In the paper's variables Omega = (m/P) u, theta = (m/P)^2 R T, alpha = 2 H m^2 / P^2 - 1 the ratio of
the two is  dtheta/dOmega = (4/5) Pr Omega (theta - [(1 - Omega)^2 + alpha] / 3) / (Omega^2 - Omega + theta),
the printed relation's form (its 8/15 is Pr = 2/3).  Pr = 1 (the BGK model's Prandtl number) is the
reading taken: with it the thickness Delta = (u_inf - u_2) / max|du/dx| of the computed profile
reproduces Table 1DShockThickness's Re_Delta (test_oracle_gp.py).

The profile is integrated from the downstream Rankine-Hugoniot state (a saddle of the system)
toward the upstream one, along the saddle's stable direction followed backward in x.
"""
import numpy as np
from scipy.integrate import solve_ivp
from scipy.optimize import brentq, minimize_scalar

from . import gas


def constants(M, gamma=5.0 / 3.0):
    """(m, P, H, (rho1, u1, T1), (rho2, u2, T2)) of the shock in the kLST units."""
    r1, u1, T1 = gas.upstream_state(M, gamma)
    st2 = gas.rankine_hugoniot(M, gamma)
    m = r1 * u1
    P = 0.5 * r1 * T1 + m * u1
    H = 1.25 * T1 + 0.5 * u1 * u1
    return m, P, H, (r1, u1, T1), st2


def rhs(u, T, M, Re, s=0.5, Pr=1.0, gamma=5.0 / 3.0):
    """(du/dx, dT/dx) of the Navier-Stokes shock balances above."""
    m, P, H, (r1, u1, T1), _ = constants(M, gamma)
    mu = (u1 / Re) * T ** s
    du = (m * u + m * 0.5 * T / u - P) / ((4.0 / 3.0) * mu)
    dT = (m * 0.75 * T - 0.5 * m * u * u + P * u - m * H) / ((1.25 / Pr) * mu)
    return du, dT


def dtheta_domega(Omega, theta, alpha, Pr=1.0):
    """The printed dtheta/dOmega relation with its Prandtl-number constant (4/5) Pr."""
    return 0.8 * Pr * Omega * (theta - ((1.0 - Omega) ** 2 + alpha) / 3.0) / (Omega * Omega - Omega + theta)


def _jacobian(u, T, M, Re, s, Pr, gamma, rel=1e-7):
    """Central-difference Jacobian of rhs at (u, T)."""
    y = np.array([u, T])
    J = np.zeros((2, 2))
    for b in range(2):
        d = np.zeros(2)
        d[b] = rel * max(1.0, abs(y[b]))
        J[:, b] = (np.array(rhs(*(y + d), M, Re, s, Pr, gamma)) - np.array(rhs(*(y - d), M, Re, s, Pr, gamma))) / (2 * d[b])
    return J


def profile(M, Re, s=0.5, Pr=1.0, gamma=5.0 / 3.0, span=None, eps=1e-6):
    """Integrated profile: dict(x, u, T, rho, Delta, x_shock, lam_s, v, eps) with x increasing from
    upstream and x = 0 the start point y_2 + eps u_2 v on the saddle's stable direction v (eigenvalue
    lam_s < 0); x_shock the location of max|du/dx| on the continuous solution: the zero of d^2u/dx^2
    next to the largest sample (a bounded search for the maximum if it has no sign change there).  The default span is 60 decay lengths of the slowest end-state eigenvalue,
    so that the profile has reached the upstream state to rounding at x = -span."""
    m, P, H, (r1, u1, T1), (r2, u2, T2) = constants(M, gamma)

    def f(x, y):
        return list(rhs(y[0], y[1], M, Re, s, Pr, gamma))

    y2 = np.array([u2, T2])
    w, V = np.linalg.eig(_jacobian(u2, T2, M, Re, s, Pr, gamma))
    k = int(np.argmin(w.real))
    lam_s, v = float(w[k].real), V[:, k].real
    if v[0] < 0:
        v = -v
    if span is None:
        w1 = np.linalg.eigvals(_jacobian(u1, T1, M, Re, s, Pr, gamma))
        span = 60.0 / min(abs(lam_s), float(np.min(np.abs(w1))))
    sol = solve_ivp(f, [0.0, -span], y2 + eps * u2 * v, rtol=1e-12, atol=1e-14, dense_output=True,
                    max_step=span / 4000)
    x, u, T = sol.t[::-1], sol.y[0][::-1], sol.y[1][::-1]
    du = np.array([rhs(a, b, M, Re, s, Pr, gamma)[0] for a, b in zip(u, T)])
    i = int(np.argmax(np.abs(du)))

    def slope(xx):  # |du/dx| on the continuous (dense-output) solution
        y = sol.sol(xx)
        return abs(rhs(y[0], y[1], M, Re, s, Pr, gamma)[0])

    def curvature(xx):  # d^2u/dx^2 = grad(du/dx) . (du/dx, dT/dx), the gradient by central differences
        y = sol.sol(xx)
        gu = _jacobian(y[0], y[1], M, Re, s, Pr, gamma, rel=1e-6)[0]
        return gu @ np.array(rhs(y[0], y[1], M, Re, s, Pr, gamma))

    a, b = x[max(i - 1, 0)], x[min(i + 1, len(x) - 1)]
    if curvature(a) * curvature(b) < 0:     # the maximum is where d^2u/dx^2 changes sign
        xs = brentq(curvature, a, b, xtol=1e-15 * span, rtol=4 * np.finfo(float).eps)
    else:
        xs = minimize_scalar(lambda xx: -slope(xx), bounds=(a, b), method="bounded",
                             options={"xatol": 1e-12 * span}).x
    return dict(x=x, u=u, T=T, rho=m / u, Delta=(u1 - u2) / slope(xs), x_shock=float(xs), sol=sol,
                lam_s=lam_s, v=v, eps=eps)


def re_delta(M, s=0.5, Pr=1.0, gamma=5.0 / 3.0):
    """The self-consistent Re_Delta: the profile's thickness with Re = 1 (x scales as 1/Re)."""
    return profile(M, 1.0, s, Pr, gamma)["Delta"]


def base_at(M, Re, x_nodes, s=0.5, Pr=1.0, gamma=5.0 / 3.0):
    """(rho, u, T) of the profile at x_nodes measured from the shock (max|du/dx|).  Past the start
    point (downstream) the saddle's linear solution y_2 + eps u_2 v exp(lam_s x); past the integrated
    range (upstream) the upstream state."""
    p = profile(M, Re, s, Pr, gamma)
    xq = np.asarray(x_nodes, dtype=np.float64) + p["x_shock"]
    (r1, u1, T1), (r2, u2, T2) = constants(M, gamma)[3:]
    lo = p["x"][0]
    y = p["sol"].sol(np.clip(xq, lo, 0.0))
    tail = p["eps"] * u2 * np.exp(p["lam_s"] * np.maximum(xq, 0.0))
    u = np.where(xq < lo, u1, np.where(xq > 0.0, u2 + tail * p["v"][0], y[0]))
    T = np.where(xq < lo, T1, np.where(xq > 0.0, T2 + tail * p["v"][1], y[1]))
    return constants(M, gamma)[0] / u, u, T
