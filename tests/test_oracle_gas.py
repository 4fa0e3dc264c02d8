"""Pins for the oracle's gas model and linearisation (Sec. 2.2, Eq. CompBGKtilde, Table 1DShockThickness)."""
import numpy as np
import pytest

from oracle import gas, grids, pencil
from paper_2607_27440_b300 import workloads as wl


@pytest.mark.parametrize("M", [1.2, 3.0, 4.0])
def test_nondimensional_numbers_match_table(M):
    """Re_Delta, Kn_Delta and lambda_inf recomputed from Table 1DShockConditions (Sec. 5)."""
    Delta, Re_tab, Kn_tab = gas.SHOCK_TABLE[M]
    # Delta is printed to 3 significant figures (+-0.0005 mm), which bounds the recomputation
    rel = 0.0005e-3 / Delta + 0.0005 / Re_tab
    assert gas.dimensional_reynolds(M, Delta) == pytest.approx(Re_tab, rel=rel)
    lam = gas.mean_free_path()
    assert lam == pytest.approx(0.207e-3, rel=2e-3)
    assert lam / Delta == pytest.approx(Kn_tab, abs=0.0015)
    assert gas.knudsen_from_re(M, Re_tab) == pytest.approx(Kn_tab, abs=0.0015)


@pytest.mark.parametrize("M", [1.2, 2.0, 3.0, 4.0])
def test_rankine_hugoniot_conserves_fluxes(M):
    g = 5.0 / 3.0
    r1, u1, T1 = gas.upstream_state(M, g)
    r2, u2, T2 = gas.rankine_hugoniot(M, g)
    assert r1 * u1 == pytest.approx(r2 * u2, rel=1e-14)
    assert 0.5 * r1 * T1 + r1 * u1 ** 2 == pytest.approx(0.5 * r2 * T2 + r2 * u2 ** 2, rel=1e-14)
    # energy flux: rho u (E + p/rho), E = u^2/2 + 3T/4, p/rho = T/2
    f1 = r1 * u1 * (0.5 * u1 ** 2 + 0.75 * T1 + 0.5 * T1)
    f2 = r2 * u2 * (0.5 * u2 ** 2 + 0.75 * T2 + 0.5 * T2)
    assert f1 == pytest.approx(f2, rel=1e-14)
    assert u1 / np.sqrt(g * T1 / 2) == pytest.approx(M)


def test_maxwellian_moments_converge():
    """Discrete moments of g^e(rho, u, T) (with h^e = T/2 g^e) reproduce (rho, u, 0, E) to quadrature error."""
    xi_x, xi_y, W = grids.velocity_grid(40, 40)
    rho, u, T = np.array([1.3]), np.array([0.7]), np.array([1.8])
    g = gas.maxwellian(rho, u, 0 * u, T, xi_x, xi_y)
    r, uu, v, E = gas.moments(g, 0.5 * T[:, None] * g, W, xi_x, xi_y)
    assert r[0] == pytest.approx(1.3, rel=1e-9)
    assert uu[0] == pytest.approx(0.7, rel=1e-9)
    assert abs(v[0]) < 1e-12
    assert E[0] == pytest.approx(0.5 * 0.7 ** 2 + 0.75 * 1.8, rel=1e-9)


def test_discrete_equilibrium_matches_moments_exactly():
    """Newton-matched equilibrium carries the target discrete moments to round-off (coarse grid)."""
    xi_x, xi_y, W = grids.velocity_grid(6, 4)
    rho, u, v, E = np.array([1.3, 2.0]), np.array([0.7, 0.2]), np.array([0.0, 0.1]), np.array([2.0, 1.5])
    ge, he, th = gas.equilibrium(rho, u, v, E, W, xi_x, xi_y, conservative=1)
    r2, u2, v2, E2 = gas.moments(ge, he, W, xi_x, xi_y)
    assert np.allclose([r2, u2, v2, E2], [rho, u, v, E], rtol=1e-14, atol=1e-15)
    ge0, he0, _ = gas.equilibrium(rho, u, v, E, W, xi_x, xi_y, conservative=0)
    r0, *_ = gas.moments(ge0, he0, W, xi_x, xi_y)
    assert np.max(np.abs(r0 - rho)) > 1e-6  # the raw Maxwellian is not discretely conservative here


def _fd_jacobian(d, spec, j, eps=1e-6):
    g, h = d["gc"], d["hc"]
    nxi = d["W"].size
    J = np.zeros((2 * nxi, 2 * nxi))
    for c in range(2):
        for p in range(nxi):
            sc = abs((g if c == 0 else h)[j, p]) + 1e-3
            out = []
            for sgn in (1, -1):
                gg, hh = g.copy(), h.copy()
                (gg if c == 0 else hh)[j, p] += sgn * eps * sc
                out.append(gas.collision_map(gg, hh, d["W"], d["xi_x"], d["xi_y"], spec))
            J[:nxi, c * nxi + p] = (out[0][0][j] - out[1][0][j]) / (2 * eps * sc)
            J[nxi:, c * nxi + p] = (out[0][1][j] - out[1][1][j]) / (2 * eps * sc)
    return J


@pytest.mark.parametrize("kw", [dict(mach=3.0, base="mott_smith", noneq=1, conservative=1),
                                dict(mach=4.0, base="mott_smith", noneq=1, conservative=0),
                                dict(mach=1.2, base="tanh", noneq=0, conservative=1, width=0.4),
                                dict(mach=2.0, base="mott_smith", noneq=0, conservative=1)])
def test_collision_block_is_jacobian_of_bgk_map(kw):
    """The collision part of the ASSEMBLED A at an interior point equals minus the Jacobian of the
    nonlinear discrete BGK term nu(m)(f^e(m) - f) (Eq. CompBGKtilde), by central differences."""
    spec = wl.tiny(nx=7, qx=4, qy=3, beta=0.7, **kw).as_dict()
    d = gas.pencil_data(spec)
    A, _ = pencil.assemble_dense(spec, d)
    nx, nxi = 7, 12
    for j in (2, 3):
        idx = np.array([pencil.index(c, k, j, nxi, nx) for c in range(2) for k in range(nxi)])
        blk = A[np.ix_(idx, idx)].copy()
        stream = np.concatenate([d["xi_x"] * d["Dx"][j, j] + 1j * 0.7 * d["xi_y"]] * 2)
        blk -= np.diag(stream)
        J = _fd_jacobian(d, spec, j)
        assert np.abs(blk.imag).max() == 0.0
        assert np.max(np.abs(blk.real + J)) < 2e-7 * np.max(np.abs(J)), j


@pytest.mark.parametrize("noneq,base", [(0, "tanh"), (1, "mott_smith"), (0, "mott_smith")])
def test_collision_invariants_annihilate(noneq, base):
    """Mass, momentum and energy are collisional invariants: psi^T (collision block) = 0 (Sec. 2.2)."""
    spec = wl.tiny(nx=6, qx=5, qy=4, base=base, noneq=noneq, width=0.5).as_dict()
    d = gas.pencil_data(spec)
    nxi = d["W"].size
    W, xx, xy = d["W"], d["xi_x"], d["xi_y"]
    psi = np.zeros((4, 2 * nxi))
    psi[0, :nxi] = W
    psi[1, :nxi] = W * xx
    psi[2, :nxi] = W * xy
    psi[3, :nxi] = 0.5 * W * (xx ** 2 + xy ** 2)
    psi[3, nxi:] = 0.5 * W
    for j in range(1, 5):
        cpl = np.block([[np.einsum("ak,ap->kp", d["G"][c, :, j, :], d["w"][cp, :, j, :]) for cp in range(2)]
                        for c in range(2)])
        coll = d["nu"][j] * np.eye(2 * nxi) - cpl
        assert np.max(np.abs(psi @ coll)) < 1e-12 * np.max(np.abs(psi)) * np.max(np.abs(coll))


def test_eq_collision_spectrum():
    """EQ mode: per point the collision block nu (I - C M) has eigenvalues {0 (x4), nu (x 2Nxi-4)}."""
    spec = wl.tiny(nx=6, qx=6, qy=4, base="tanh", noneq=0, width=0.4, mach=1.2).as_dict()
    d = gas.pencil_data(spec)
    nxi = d["W"].size
    for j in range(1, 5):
        cpl = np.block([[np.einsum("ak,ap->kp", d["G"][c, :, j, :], d["w"][cp, :, j, :]) for cp in range(2)]
                        for c in range(2)])
        ev = np.sort(np.abs(np.linalg.eigvals(d["nu"][j] * np.eye(2 * nxi) - cpl)))
        assert np.max(ev[:4]) < 1e-10 * d["nu"][j]
        assert np.allclose(ev[4:], d["nu"][j], rtol=1e-10)


def test_base_flow_limits():
    """Far upstream/downstream the synthetic bases are the Rankine-Hugoniot Maxwellians."""
    for base in ("tanh", "mott_smith"):
        spec = wl.tiny(nx=16, qx=30, qy=20, mach=3.0, base=base, width=0.5).as_dict()
        d = gas.pencil_data(spec)
        r2, u2, T2 = gas.rankine_hugoniot(3.0, 5.0 / 3.0)
        assert d["rho"][0] == pytest.approx(r2, rel=2e-3)
        assert d["u"][0] == pytest.approx(u2, rel=2e-3)
        assert d["rho"][-1] == pytest.approx(1.0, rel=2e-3)
        assert np.all(d["nu"] > 0)


@pytest.mark.parametrize("M", [1.2, 3.0, 4.0])
def test_nondimensional_viscosity_reproduces_table_knudsen(M):
    """gas.transport's mu at the free-stream state, put into the mean-free-path definition of Sec. 2.1
    (l = (16/5) mu / (rho sqrt(2 pi R T)), here in shock-thickness units with rho = T = 1, R = 1/2),
    is Kn_Delta = l / Delta of Table 1DShockThickness (0.081 / 0.511 / 0.598, printed to 3 decimals).
    A wrong u_inf factor or Re_Delta in mu would miss the table."""
    spec = wl.tiny(mach=M).as_dict()
    u_inf = M * np.sqrt(spec["gamma"] / 2.0)
    T, P, mu, nu = gas.transport(np.array([1.0]), np.array([u_inf]), np.array([0.0]),
                                 np.array([0.5 * u_inf ** 2 + 0.75]), spec)
    assert T[0] == pytest.approx(1.0, rel=1e-15)
    kn = (16.0 / 5.0) * mu[0] / (1.0 * np.sqrt(2.0 * np.pi * 0.5 * 1.0))
    assert kn == pytest.approx(gas.SHOCK_TABLE[M][2], abs=0.0015)


@pytest.mark.parametrize("M", [1.2, 3.0, 4.0])
def test_collision_frequency_matches_dimensional_gas(M):
    """nu = P / mu in the nondimensional units equals the SI collision frequency p / mu(T) with
    mu(T) = mu_inf (T / T_inf)^s (the power law of Eq. GB1DShockeqn, Table 1DShockConditions), scaled
    by the time unit Delta / u_ref, at the downstream Rankine-Hugoniot state where T != 1.  This pins
    P = rho T / 2, the u_inf / Re_Delta factor and the exponent s together (to the table's 3 figures)."""
    spec = wl.tiny(mach=M).as_dict()
    g = gas.ARGON
    rho2, u2, T2 = gas.rankine_hugoniot(M, spec["gamma"])
    _, _, _, nu = gas.transport(np.array([rho2]), np.array([u2]), np.array([0.0]),
                                np.array([0.5 * u2 ** 2 + 0.75 * T2]), spec)
    rho_si = g["P_inf"] / (g["R"] * g["T_inf"]) * rho2
    T_si = g["T_inf"] * T2
    mu_si = g["mu_inf"] * (T_si / g["T_inf"]) ** g["s"]
    nu_si = rho_si * g["R"] * T_si / mu_si
    Delta = gas.SHOCK_TABLE[M][0]
    u_ref = np.sqrt(2.0 * g["R"] * g["T_inf"])
    rel = 0.0005e-3 / Delta + 0.0005 / gas.SHOCK_TABLE[M][1]  # the table's rounding of Delta and Re
    assert nu[0] == pytest.approx(nu_si * Delta / u_ref, rel=rel)


@pytest.mark.parametrize("M", [1.2, 3.0])
def test_tanh_base_conserves_mass_and_momentum_flux(M):
    """The tanh local-Maxwellian base flow: at every collocation point the discrete moments of
    (g_c, h_c) carry the upstream mass flux rho u and momentum flux rho u^2 + P (P = rho T / 2, T from
    the moments) to quadrature error, and both ends reach the Rankine-Hugoniot temperatures (Sec. 2.1:
    the shock joins the two Rankine-Hugoniot states).  A wrong base temperature fails pointwise."""
    spec = wl.tiny(nx=24, qx=48, qy=24, mach=M, base="tanh", noneq=0, width=0.5).as_dict()
    x, _ = grids.mapped_diff(24, spec["map_L"], spec["map_sinf"])
    xi_x, xi_y, W = grids.velocity_grid(48, 24)
    gc, hc = gas.base_flow(spec, x, xi_x, xi_y)
    rho, u, v, E = gas.moments(gc, hc, W, xi_x, xi_y)
    T = gas.temperature(u, v, E)
    r1, u1, T1 = gas.upstream_state(M, spec["gamma"])
    r2, u2, T2 = gas.rankine_hugoniot(M, spec["gamma"])
    mass = rho * u
    mom = rho * u ** 2 + 0.5 * rho * T
    # the unscaled 48 x 24 Gauss-Hermite rule integrates the hot downstream Maxwellian (T2 = 3.7 at
    # M = 3) to ~5e-6; a wrong temperature formula is off by O(1), so 1e-4 separates the two
    tol = 1e-4
    assert np.max(np.abs(mass / (r1 * u1) - 1.0)) < tol
    assert np.max(np.abs(mom / (r1 * u1 ** 2 + 0.5 * r1 * T1) - 1.0)) < tol
    assert T[-1] == pytest.approx(T1, rel=tol)  # x = -s_inf: upstream
    assert T[0] == pytest.approx(T2, rel=tol)   # x = +s_inf: downstream
