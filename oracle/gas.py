"""Gas model, base flows and linearisation coefficients (oracle; test infrastructure only).

Nondimensionalisation (Sec. 2.2): T by T_inf, rho by rho_inf, velocities by
u_ref = sqrt(2 R T_inf), so the nondimensional gas constant is R = 1/2,
p = rho T / 2 and the 2-D equilibrium reduced distributions are
    g^e = rho / (pi T) exp(-|xi - u|^2 / T),   h^e = (T/2) g^e      (K = 0, argon).
Moments (Sec. 2.2): rho = sum W g, rho u = sum W xi g,
rho E = (1/2) sum W (|xi|^2 g + h), hence E = |u|^2/2 + 3T/4.
Viscosity mu = (u_inf / Re_Delta) T^s and collision frequency nu = P / mu
(Eq. CompBGKtilde writes the relaxation rate as P_c / mu_c).

All arrays are float64; per-point quantities have shape (Nx,), distribution
values shape (Nx, Nxi); coefficient tables shape (2, 4, Nx, Nxi) indexed
[component c in (g, h)][moment a in (rho, u, v, E)][j][k].
"""
import numpy as np

from . import grids

# Table 1DShockConditions / 1DShockThickness (Sec. 5)
ARGON = dict(T_inf=300.0, P_inf=41.4, gamma=5.0 / 3.0, R=208.0, mu_inf=2.688e-5, s=0.5)
SHOCK_TABLE = {1.2: (2.548e-3, 24.34, 0.081), 3.0: (0.405e-3, 9.68, 0.511), 4.0: (0.346e-3, 11.03, 0.598)}


def _p(spec, key):
    return spec[key] if isinstance(spec, dict) else getattr(spec, key)


# ---------------------------------------------------------------- dimensional pins
def dimensional_reynolds(M, Delta, gas=ARGON):
    """Re_Delta = rho_inf u_inf Delta / mu_inf with rho_inf = P/(R T), u_inf = M sqrt(gamma R T) (Sec. 5)."""
    rho = gas["P_inf"] / (gas["R"] * gas["T_inf"])
    u = M * np.sqrt(gas["gamma"] * gas["R"] * gas["T_inf"])
    return rho * u * Delta / gas["mu_inf"]


def mean_free_path(gas=ARGON, delta=5.0):
    """Upstream mean free path l = (16/delta) mu / (rho sqrt(2 pi R T)) (Sec. 2.1)."""
    rho = gas["P_inf"] / (gas["R"] * gas["T_inf"])
    return (16.0 / delta) * gas["mu_inf"] / (rho * np.sqrt(2.0 * np.pi * gas["R"] * gas["T_inf"]))


def knudsen_from_re(M, Re, gamma=5.0 / 3.0, s=0.5):
    """Kn_Delta = 2(5-2s)(7-2s) Ma / (15 Re_Delta) sqrt(gamma / (2 pi)) (Sec. 2.2)."""
    return 2.0 * (5 - 2 * s) * (7 - 2 * s) * M / (15.0 * Re) * np.sqrt(gamma / (2.0 * np.pi))


# ---------------------------------------------------------------- nondimensional states
def upstream_state(M, gamma):
    """Free stream (rho, u, T) = (1, M sqrt(gamma/2), 1) in the nondimensional units."""
    return 1.0, M * np.sqrt(gamma / 2.0), 1.0


def rankine_hugoniot(M, gamma):
    """Downstream (rho2, u2, T2) from the normal-shock jump relations of a gamma-law gas."""
    rho1, u1, T1 = upstream_state(M, gamma)
    p1 = 0.5 * rho1 * T1
    r = (gamma + 1.0) * M * M / ((gamma - 1.0) * M * M + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma * (M * M - 1.0) / (gamma + 1.0))
    rho2 = rho1 * r
    u2 = u1 / r
    T2 = 2.0 * p2 / rho2
    return rho2, u2, T2


def maxwellian(rho, u, v, T, xi_x, xi_y):
    """g^e = rho/(pi T) exp(-((xi_x-u)^2 + (xi_y-v)^2)/T); per-point args broadcast over nodes."""
    rho, u, v, T = (np.asarray(a, dtype=np.float64)[..., None] for a in (rho, u, v, T))
    return rho / (np.pi * T) * np.exp(-((xi_x - u) ** 2 + (xi_y - v) ** 2) / T)


def base_flow(spec, x, xi_x, xi_y):
    """Synthetic base-flow reduced distributions (g_c, h_c) at points x, shape (Nx, Nxi).

    s(x) = (1 + tanh(x / width)) / 2 goes from 0 upstream (x -> -inf) to 1 downstream.
    * base 'tanh': local Maxwellian with u = u1 + (u2 - u1) s, rho = rho1 u1 / u
      (mass flux) and T = 2 (P1 + rho1 u1^2 - rho u^2) / rho (momentum flux).
    * base 'mott_smith': g_c = (1 - s) g^e_1 + s g^e_2 and h_c likewise with
      (T_i / 2) g^e_i -- a bimodal, non-equilibrium distribution.
    * base 'gilbarg_paolucci': local Maxwellian of the continuum shock profile (gp.base_at with
      Re = re_delta, mu ~ T^visc_s, Pr = 1), max|du/dx| at x = 0; width is not used.
    """
    M, gamma, width = _p(spec, "mach"), _p(spec, "gamma"), _p(spec, "width")
    rho1, u1, T1 = upstream_state(M, gamma)
    rho2, u2, T2 = rankine_hugoniot(M, gamma)
    s = 0.5 * (1.0 + np.tanh(x / width))
    if _p(spec, "base") == "tanh":
        u = u1 + (u2 - u1) * s
        rho = rho1 * u1 / u
        P1 = 0.5 * rho1 * T1
        T = 2.0 * (P1 + rho1 * u1 * u1 - rho * u * u) / rho
        gc = maxwellian(rho, u, 0.0 * u, T, xi_x, xi_y)
        hc = 0.5 * T[:, None] * gc
    elif _p(spec, "base") == "mott_smith":
        z = np.zeros_like(x)
        g1 = maxwellian(rho1 + z, u1 + z, z, T1 + z, xi_x, xi_y)
        g2 = maxwellian(rho2 + z, u2 + z, z, T2 + z, xi_x, xi_y)
        gc = (1.0 - s)[:, None] * g1 + s[:, None] * g2
        hc = (1.0 - s)[:, None] * (0.5 * T1) * g1 + s[:, None] * (0.5 * T2) * g2
    elif _p(spec, "base") == "gilbarg_paolucci":
        from . import gp   # the continuum profile (Pr = 1, mu ~ T^s, Re = Re_Delta), shock at x = 0
        rho, u, T = gp.base_at(M, _p(spec, "re_delta"), x, s=_p(spec, "visc_s"), gamma=gamma)
        gc = maxwellian(rho, u, 0.0 * u, T, xi_x, xi_y)
        hc = 0.5 * T[:, None] * gc
    else:
        raise ValueError("unknown base flow")
    return gc, hc


def moments(g, h, W, xi_x, xi_y):
    """Discrete macroscopic moments (rho, u, v, E) of (g, h) with full-line weights W (Sec. 2.2)."""
    rho = g @ W
    u = (g * xi_x) @ W / rho
    v = (g * xi_y) @ W / rho
    E = 0.5 * ((g * (xi_x ** 2 + xi_y ** 2)) @ W + h @ W) / rho
    return rho, u, v, E


def temperature(u, v, E):
    """T = (4/3)(E - (u^2 + v^2)/2), from E = |u|^2/2 + 3T/4."""
    return (4.0 / 3.0) * (E - 0.5 * (u * u + v * v))


def equilibrium(rho, u, v, E, W, xi_x, xi_y, conservative, fix_v=False, max_iter=60):
    """Discrete equilibrium (g^e, h^e) carrying the moments (rho, u, v, E).

    conservative = 0: the Maxwellian with parameters (rho, u, v, T(u, v, E)).
    conservative = 1: Newton on the Maxwellian parameters (rho', u', v', T') so
    that the DISCRETE moments of (g^e, h^e = T'/2 g^e) equal (rho, u, v, E)
    exactly: the collision term then conserves mass, momentum and energy to
    round-off on the discrete velocity grid.  ``fix_v`` keeps v' = 0 (the 1-D
    base flow, which has no transverse velocity).
    Returns (g^e, h^e, theta') with theta' = (rho', u', v', T') arrays.
    """
    rho, u, v, E = (np.array(a, dtype=np.float64, copy=True) for a in (rho, u, v, E))
    T = temperature(u, v, E)
    th = np.stack([rho, u, v, T], axis=-1)  # (Nx, 4)
    if conservative:
        target = np.stack([rho, rho * u, rho * v, rho * E], axis=-1)
        ex2 = xi_x ** 2 + xi_y ** 2
        for it in range(max_iter):
            r_, u_, v_, T_ = th.T
            ge = maxwellian(r_, u_, v_, T_, xi_x, xi_y)
            phi = -1.0 / T_[:, None] + ((xi_x - u_[:, None]) ** 2 + (xi_y - v_[:, None]) ** 2) / T_[:, None] ** 2
            dge = [ge / r_[:, None], ge * 2.0 * (xi_x - u_[:, None]) / T_[:, None],
                   ge * 2.0 * (xi_y - v_[:, None]) / T_[:, None], ge * phi]
            F = np.stack([ge @ W, (ge * xi_x) @ W, (ge * xi_y) @ W,
                          0.5 * ((ge * ex2) @ W + 0.5 * T_ * (ge @ W))], axis=-1) - target
            Jm = np.zeros(F.shape + (4,))
            for b in range(4):
                dh = 0.5 * T_[:, None] * dge[b] + (0.5 * ge if b == 3 else 0.0)
                Jm[:, 0, b] = dge[b] @ W
                Jm[:, 1, b] = (dge[b] * xi_x) @ W
                Jm[:, 2, b] = (dge[b] * xi_y) @ W
                Jm[:, 3, b] = 0.5 * ((dge[b] * ex2) @ W + dh @ W)
            if fix_v:
                Jm[:, 2, :] = 0.0
                Jm[:, :, 2] = 0.0
                Jm[:, 2, 2] = 1.0
                F[:, 2] = 0.0
            step = np.linalg.solve(Jm, -F[..., None])[..., 0]
            th = th + step
            if it >= 1 and np.max(np.abs(step) / (np.abs(th) + 1.0)) < 1e-15:
                break
    r_, u_, v_, T_ = th.T
    ge = maxwellian(r_, u_, v_, T_, xi_x, xi_y)
    he = 0.5 * T_[:, None] * ge
    return ge, he, (r_, u_, v_, T_)


def equilibrium_derivatives(theta, xi_x, xi_y):
    """Raw coefficients C: derivatives of (g^e, h^e) w.r.t. (rho, u, v, E) at theta = (rho, u, v, T).

    With T = (4/3)(E - (u^2+v^2)/2) and phi = -1/T + |xi-u|^2/T^2:
      C_grho = g^e/rho,  C_gu = g^e [2(xi_x-u)/T - (4/3) u phi],
      C_gv = g^e [2(xi_y-v)/T - (4/3) v phi],  C_gE = (4/3) g^e phi,
    and for h^e = (T/2) g^e (dh^e/dT = g^e/2 + (T/2) g^e phi):
      C_hrho = h^e/rho, C_hu = (T/2) g^e 2(xi_x-u)/T - (4/3) u dh^e/dT,
      C_hv = (T/2) g^e 2(xi_y-v)/T - (4/3) v dh^e/dT, C_hE = (4/3) dh^e/dT.
    """
    r, u, v, T = (np.asarray(a)[:, None] for a in theta)
    ge = maxwellian(theta[0], theta[1], theta[2], theta[3], xi_x, xi_y)
    phi = -1.0 / T + ((xi_x - u) ** 2 + (xi_y - v) ** 2) / T ** 2
    dgdT = ge * phi
    dhdT = 0.5 * ge + 0.5 * T * ge * phi
    C = np.zeros((2, 4) + ge.shape)
    C[0, 0] = ge / r
    C[0, 1] = ge * 2.0 * (xi_x - u) / T - (4.0 / 3.0) * u * dgdT
    C[0, 2] = ge * 2.0 * (xi_y - v) / T - (4.0 / 3.0) * v * dgdT
    C[0, 3] = (4.0 / 3.0) * dgdT
    C[1, 0] = 0.5 * T * ge / r
    C[1, 1] = 0.5 * T * ge * 2.0 * (xi_x - u) / T - (4.0 / 3.0) * u * dhdT
    C[1, 2] = 0.5 * T * ge * 2.0 * (xi_y - v) / T - (4.0 / 3.0) * v * dhdT
    C[1, 3] = (4.0 / 3.0) * dhdT
    return C


def moment_weights(rho, u, v, E, W, xi_x, xi_y):
    """Linearised moment functionals w (2, 4, Nx, Nxi) of Eqs. comp_ghat1Dshock / comp_hhat1Dshock.

    rho^ = sum W g^,  u^ = sum W (xi_x - u) g^ / rho,  v^ = sum W (xi_y - v) g^ / rho,
    E^ = [sum W (|xi|^2 - 2E) g^ + sum W h^] / (2 rho); all other h-weights vanish.
    """
    rho, u, v, E = (np.asarray(a)[:, None] for a in (rho, u, v, E))
    w = np.zeros((2, 4, rho.shape[0], W.size))
    w[0, 0] = W + 0.0 * rho
    w[0, 1] = W * (xi_x - u) / rho
    w[0, 2] = W * (xi_y - v) / rho
    w[0, 3] = W * (xi_x ** 2 + xi_y ** 2 - 2.0 * E) / (2.0 * rho)
    w[1, 3] = W / (2.0 * rho) + 0.0 * u
    return w


def transport(rho, u, v, E, spec):
    """(T, P, mu, nu) with P = rho T/2, mu = (u_inf/Re) T^s, nu = P/mu."""
    u_inf = upstream_state(_p(spec, "mach"), _p(spec, "gamma"))[1]
    T = temperature(u, v, E)
    P = 0.5 * rho * T
    mu = (u_inf / _p(spec, "re_delta")) * T ** _p(spec, "visc_s")
    return T, P, mu, P / mu


def pressure_viscosity_derivatives(rho, u, v, E, spec):
    """d_a = dP/da / mu - P (dmu/da) / mu^2 for a in (rho, u, v, E), shape (4, Nx).

    dP = (T/2, -(2/3) rho u, -(2/3) rho v, (2/3) rho); dmu = s mu / T * dT with
    dT = (0, -(4/3) u, -(4/3) v, 4/3).  These are the P~ and mu~ factors of the
    non-equilibrium terms of Eq. CompBGKtilde.
    """
    T, P, mu, _ = transport(rho, u, v, E, spec)
    s = _p(spec, "visc_s")
    dP = np.stack([0.5 * T, -(2.0 / 3.0) * rho * u, -(2.0 / 3.0) * rho * v, (2.0 / 3.0) * rho + 0.0 * u])
    dT = np.stack([0.0 * T, -(4.0 / 3.0) * u, -(4.0 / 3.0) * v, (4.0 / 3.0) + 0.0 * T])
    dmu = s * mu / T * dT
    return dP / mu - P * dmu / mu ** 2


def collision_map(g, h, W, xi_x, xi_y, spec):
    """Nonlinear discrete BGK collision term R = nu(m) (eq(m) - f) for (g, h), shape (Nx, Nxi) each.

    The right-hand side of the reduced BGK equations (Sec. 3.3 / Sec. 2.2):
    moments m of (g, h), nu = P/mu at those moments, and the discrete equilibrium
    carrying m (``equilibrium``).  Its Jacobian at the base state is the
    collision part of the pencil (Eq. CompBGKtilde); this function exists only
    to pin that linearisation by finite differences.
    """
    rho, u, v, E = moments(g, h, W, xi_x, xi_y)
    _, _, _, nu = transport(rho, u, v, E, spec)
    ge, he, _ = equilibrium(rho, u, v, E, W, xi_x, xi_y, _p(spec, "conservative"))
    return nu[:, None] * (ge - g), nu[:, None] * (he - h)


def pencil_data(spec, base=None):
    """All per-point and per-node tables the pencil is assembled from (``base``: optional (g_c, h_c)
    of shape (Nx, Nxi) in node order, used in place of the synthetic base flow).

    Returns a dict with x, Dx, xi_x, xi_y, W, gc, hc, gce, hce, rho, u, E, T, P,
    mu, nu, C (fixed, 2x4xNxxNxi), w (moment weights), G (collision coupling
    coefficients G/H of Eq. Comp1DHarm), bc (Nx, Nxi) bool mask of inflow
    boundary rows.

    Base state: (rho_c, u_c, E_c) are the discrete moments of (g_c, h_c), v_c = 0.
    Equilibrium (g_c^e, h_c^e) from ``equilibrium`` (Newton-matched when
    conservative).  In EQ mode (noneq = 0) g_c := g_c^e and h_c := h_c^e.
    C_fixed = C_raw (M C_raw)^{-1} with M the moment map (4 x 2Nxi): the exact
    derivative of the discrete equilibrium w.r.t. the discrete moments, so
    M C_fixed = I_4 (for conservative = 0, C_fixed = C_raw).
    G^c_a = nu C^c_a + (f_c^e - f_c) d_a  (Eq. CompBGKtilde), zero on boundary rows.
    Boundary rows (Sec. 2.2, inflow BC): j = N (x = -s_inf) with xi_x > 0 and
    j = 0 (x = +s_inf) with xi_x < 0.
    """
    nx, qx, qy = _p(spec, "nx"), _p(spec, "qx"), _p(spec, "qy")
    x, Dx = grids.mapped_diff(nx, _p(spec, "map_L"), _p(spec, "map_sinf"))
    xi_x, xi_y, W = grids.velocity_grid(qx, qy)
    if base is None:
        gc, hc = base_flow(spec, x, xi_x, xi_y)
    else:  # given base distributions at the nodes (e.g. the BE-BGK steady state of Sec. 3.3)
        gc, hc = (np.array(a, dtype=np.float64) for a in base)
    rho, u, v, E = moments(gc, hc, W, xi_x, xi_y)
    v = np.zeros_like(v)
    cons = _p(spec, "conservative")
    gce, hce, theta = equilibrium(rho, u, v, E, W, xi_x, xi_y, cons, fix_v=True)
    if not _p(spec, "noneq"):
        gc, hc = gce.copy(), hce.copy()
    T, P, mu, nu = transport(rho, u, v, E, spec)
    C = equilibrium_derivatives(theta, xi_x, xi_y)
    w = moment_weights(rho, u, v, E, W, xi_x, xi_y)
    if cons:
        MC = np.einsum("cajk,cbjk->jab", w, C)
        C = np.einsum("cbjk,jba->cajk", C, np.linalg.inv(MC))
    d = pressure_viscosity_derivatives(rho, u, v, E, spec)
    G = nu[None, None, :, None] * C
    G[0] += d[:, :, None] * (gce - gc)[None]
    G[1] += d[:, :, None] * (hce - hc)[None]
    bc = np.zeros((nx, qx * qy), dtype=bool)
    bc[nx - 1, :] = xi_x > 0
    bc[0, :] = xi_x < 0
    G[:, :, bc] = 0.0
    return dict(x=x, Dx=Dx, xi_x=xi_x, xi_y=xi_y, W=W, gc=gc, hc=hc, gce=gce, hce=hce,
                rho=rho, u=u, E=E, T=T, P=P, mu=mu, nu=nu, C=C, w=w, G=G, bc=bc)
