"""BE-BGK base-flow solver (oracle; test infrastructure only): Sec. 3.3 of the paper.

The reduced 1D2V BGK equations (Eq. BoltzmannBGK_reduced)
    dg/dt + xi_x dg/dx = nu (g^e - g),     dh/dt + xi_x dh/dx = nu (h^e - h)
on the mapped Chebyshev nodes of the kLST grid (Sec. 3.1, shifted by a map centre c), written as
dq/dt = RHS(q) with q = (g, h):
  * streaming: second-order finite volumes with MUSCL reconstruction and the minmod limiter, the
    interface value taken from the upwind side of each node velocity xi_x, in the form the paper
    states (slopes are plain differences of neighbouring values; minmod(a, b) =
    (sgn a + sgn b)/2 min(|a|, |b|)); cell i spans the midpoints to its neighbours;
  * relaxation: nu (q^e - q) toward the discrete equilibrium of q's own moments (the one the
    pencil linearises, gas.equilibrium), nu = P / mu(T) (gas.transport);
  * boundaries: the two end nodes hold the upstream and Rankine-Hugoniot Maxwellians (Dirichlet;
    the downstream one with discrete fluxes equal to the upstream ones, see end_states); a stencil
    that reaches past an end repeats the end value;
  * time: the classical fourth-order Runge-Kutta scheme;
  * adaptive shock re-centring: when the location of the largest |dU/dx| of the bulk velocity
    (piecewise-linear between nodes) has drifted from the map centre by more than a threshold,
    the grid is rebuilt about it and g, h are moved onto the new nodes by linear interpolation in
    x, the end values re-imposed.

The start is the Mott-Smith profile or the Gilbarg-Paolucci one (initial_state).

Arrays here are in physical order (index i = 0 at x = c - s_inf upstream, increasing x), shape
(Nx, Nxi); `to_pencil_order` reverses to the pencil's node order (j = 0 at the downstream end).
"""
import numpy as np

from . import gas, grids


def minmod(a, b):
    """(sgn a + sgn b)/2 min(|a|, |b|)."""
    return 0.5 * (np.sign(a) + np.sign(b)) * np.minimum(np.abs(a), np.abs(b))


def grid(spec, centre=0.0):
    """Physical-order nodes x_i (increasing) of the mapped Chebyshev grid shifted by ``centre``."""
    x, _ = grids.mapped_diff(gas._p(spec, "nx"), gas._p(spec, "map_L"), gas._p(spec, "map_sinf"))
    return x[::-1] + centre


def discrete_fluxes(g, h, xi_x, xi_y, W):
    """Mass, momentum and energy fluxes sum W xi_x (g, xi_x g, (|xi|^2 g + h)/2) of (g, h)."""
    e2 = xi_x ** 2 + xi_y ** 2
    return np.array([(g * xi_x) @ W, (g * xi_x ** 2) @ W, 0.5 * ((g * xi_x * e2) @ W + (h * xi_x) @ W)])


def end_states(spec, xi_x, xi_y, W=None):
    """(g, h) of the upstream (i = 0) and downstream (i = N) Maxwellians, shape (Nxi,).

    Upstream: (rho, u, T) = (1, M sqrt(gamma/2), 1).  Downstream: the Rankine-Hugoniot state,
    refined by Newton so that its DISCRETE fluxes on the node set equal the upstream ones (the
    continuous jump conditions hold only up to the quadrature error of the nodes, and that flux
    mismatch would move the shock forever); without W, the continuous Rankine-Hugoniot state."""
    M, gamma = gas._p(spec, "mach"), gas._p(spec, "gamma")
    (r1, u1, T1), (r2, u2, T2) = gas.upstream_state(M, gamma), gas.rankine_hugoniot(M, gamma)

    def state(r, u, T):
        g = gas.maxwellian(r, u, 0.0, T, xi_x, xi_y)
        return g, 0.5 * T * g

    up = state(r1, u1, T1)
    th = np.array([r2, u2, T2], dtype=np.float64)
    if W is not None:
        target = discrete_fluxes(*up, xi_x, xi_y, W)
        for _ in range(50):
            F = discrete_fluxes(*state(*th), xi_x, xi_y, W) - target
            J = np.zeros((3, 3))
            for b in range(3):
                d = np.zeros(3)
                d[b] = 1e-7 * max(1.0, abs(th[b]))
                J[:, b] = (discrete_fluxes(*state(*(th + d)), xi_x, xi_y, W)
                           - discrete_fluxes(*state(*(th - d)), xi_x, xi_y, W)) / (2 * d[b])
            step = np.linalg.solve(J, -F)
            th = th + step
            if np.max(np.abs(step) / np.abs(th)) < 1e-15:
                break
    return [up, state(*th)]


def interface_values(phi, xi_x):
    """phi_{i+1/2} for i = 0..N-1 (shape (N, Nxi)), upwind MUSCL-minmod per node velocity."""
    p = np.concatenate([phi[:1], phi, phi[-1:]], axis=0)   # ghosts: the end values repeated
    # p[i + 1] = phi_i for i = -1..N+1
    N = phi.shape[0] - 1
    i = np.arange(N)
    left = p[i + 1] + 0.5 * minmod(p[i + 1] - p[i], p[i + 2] - p[i + 1])          # from cell i
    right = p[i + 2] - 0.5 * minmod(p[i + 2] - p[i + 1], p[i + 3] - p[i + 2])     # from cell i + 1
    return np.where(xi_x[None, :] >= 0.0, left, right)


def streaming(phi, x, xi_x):
    """xi_x (phi_{i+1/2} - phi_{i-1/2}) / dx_i for the interior cells i = 1..N-1 (zero at the ends)."""
    xm = 0.5 * (x[1:] + x[:-1])                 # x_{i+1/2}, i = 0..N-1
    f = interface_values(phi, xi_x)             # phi_{i+1/2}
    out = np.zeros_like(phi)
    dx = xm[1:] - xm[:-1]                       # cell widths of i = 1..N-1
    out[1:-1] = xi_x[None, :] * (f[1:] - f[:-1]) / dx[:, None]
    return out


def relaxation(g, h, xi_x, xi_y, W, spec):
    """nu (g^e - g), nu (h^e - h) per node, the discrete equilibrium of (g, h)'s own moments."""
    rho, u, v, E = gas.moments(g, h, W, xi_x, xi_y)
    v = np.zeros_like(v)
    ge, he, _ = gas.equilibrium(rho, u, v, E, W, xi_x, xi_y, 1, fix_v=True)
    nu = gas.transport(rho, u, v, E, spec)[3]
    return nu[:, None] * (ge - g), nu[:, None] * (he - h)


def rhs(g, h, x, xi_x, xi_y, W, spec):
    """(RHS_g, RHS_h) of Sec. 3.3; zero at the two Dirichlet end nodes."""
    cg, ch = relaxation(g, h, xi_x, xi_y, W, spec)
    rg = cg - streaming(g, x, xi_x)
    rh = ch - streaming(h, x, xi_x)
    rg[0] = rg[-1] = 0.0
    rh[0] = rh[-1] = 0.0
    return rg, rh


def rk4_step(g, h, dt, x, xi_x, xi_y, W, spec):
    """One classical RK4 step of dq/dt = RHS(q)."""
    k1 = rhs(g, h, x, xi_x, xi_y, W, spec)
    k2 = rhs(g + 0.5 * dt * k1[0], h + 0.5 * dt * k1[1], x, xi_x, xi_y, W, spec)
    k3 = rhs(g + 0.5 * dt * k2[0], h + 0.5 * dt * k2[1], x, xi_x, xi_y, W, spec)
    k4 = rhs(g + dt * k3[0], h + dt * k3[1], x, xi_x, xi_y, W, spec)
    return (g + dt / 6.0 * (k1[0] + 2.0 * k2[0] + 2.0 * k3[0] + k4[0]),
            h + dt / 6.0 * (k1[1] + 2.0 * k2[1] + 2.0 * k3[1] + k4[1]))


def time_step(x, xi_x, nu_max, cfl):
    """dt = cfl min(dx) / max|xi_x|, and at most 2 / max(nu) (RK4 on the relaxation)."""
    xm = 0.5 * (x[1:] + x[:-1])
    dx = np.min(xm[1:] - xm[:-1])
    return min(cfl * dx / np.max(np.abs(xi_x)), 2.0 / nu_max)


def shock_location(u, x):
    """Midpoint of the interval with the largest |dU/dx| of the piecewise-linear bulk velocity."""
    s = np.abs(np.diff(u) / np.diff(x))
    i = int(np.argmax(s))
    return 0.5 * (x[i] + x[i + 1])


def regrid(g, h, x_old, x_new, ends):
    """g, h moved onto x_new by linear interpolation in x (per node velocity), ends re-imposed."""
    gn = np.empty((len(x_new), g.shape[1]))
    hn = np.empty_like(gn)
    for k in range(g.shape[1]):
        gn[:, k] = np.interp(x_new, x_old, g[:, k])
        hn[:, k] = np.interp(x_new, x_old, h[:, k])
    (gu, hu), (gd, hd) = ends
    gn[0], hn[0], gn[-1], hn[-1] = gu, hu, gd, hd
    return gn, hn


def initial_state(spec, x, xi_x, xi_y, W, start="mott_smith"):
    """The start (gas.base_flow): the Mott-Smith profile about x = 0, or ('gilbarg_paolucci') the local
    Maxwellian of the continuum profile with its steepest point at x = 0 (the paper aligns the grid
    with the peak slope of an initial Gilbarg-Paolucci profile); the ends set to the end states."""
    s2 = dict(spec.as_dict() if hasattr(spec, "as_dict") else spec)
    s2["base"] = start
    g, h = gas.base_flow(s2, x, xi_x, xi_y)
    (gu, hu), (gd, hd) = end_states(spec, xi_x, xi_y, W)
    g[0], h[0], g[-1], h[-1] = gu, hu, gd, hd
    return g, h


def steady(spec, steps, cfl=0.5, recentre_every=0, recentre_tol=0.25, tol=0.0, dt=0.0, start="mott_smith"):
    """Integrate from the start (initial_state) for at most ``steps`` RK4 steps (stopping once
    max|RHS| <= tol max|g|; dt > 0: a fixed time step); returns dict(g, h (pencil order), centre,
    steps, resid, recentres)."""
    xi_x, xi_y, W = grids.velocity_grid(gas._p(spec, "qx"), gas._p(spec, "qy"))
    c = 0.0
    x = grid(spec, c)
    g, h = initial_state(spec, x, xi_x, xi_y, W, start)
    ends = end_states(spec, xi_x, xi_y, W)
    resid = np.inf
    n = recentres = 0
    for n in range(1, steps + 1):
        if dt > 0:
            step = dt
        else:
            rho, u, v, E = gas.moments(g, h, W, xi_x, xi_y)
            nu = gas.transport(rho, u, np.zeros_like(v), E, spec)[3]
            step = time_step(x, xi_x, np.max(nu), cfl)
        g, h = rk4_step(g, h, step, x, xi_x, xi_y, W, spec)
        if recentre_every and n % recentre_every == 0:
            rho, u, v, E = gas.moments(g, h, W, xi_x, xi_y)
            xs = shock_location(u, x)
            if abs(xs - c) > recentre_tol:
                x_new = grid(spec, xs)
                g, h = regrid(g, h, x, x_new, ends)
                x, c = x_new, xs
                recentres += 1
        if tol > 0:
            rg, rh = rhs(g, h, x, xi_x, xi_y, W, spec)
            resid = max(np.max(np.abs(rg)), np.max(np.abs(rh))) / np.max(np.abs(g))
            if resid <= tol:
                break
    return dict(g=to_pencil_order(g), h=to_pencil_order(h), centre=c, steps=n, resid=resid, recentres=recentres)


def to_pencil_order(a):
    """Physical order (upstream first) -> the pencil's node order (j = 0 downstream)."""
    return np.ascontiguousarray(a[::-1])
