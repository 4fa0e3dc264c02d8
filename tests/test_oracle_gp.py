"""Pins of the Gilbarg-Paolucci shock-structure oracle (paper Sec. 2.1, Eq. GB1DShockeqn, Eq.
ShockThickness, Table 1DShockThickness)."""
import numpy as np
import pytest

from oracle import gas, gp


@pytest.mark.parametrize("M", [1.2, 3.0, 4.0])
def test_end_states_are_fixed_points(M):
    """The upstream and Rankine-Hugoniot states annul both balances (the shock connects them)."""
    m, P, H, st1, st2 = gp.constants(M)
    for rho, u, T in (st1, st2):
        du, dT = gp.rhs(u, T, M, 10.0)
        assert abs(du) < 1e-12 * u and abs(dT) < 1e-12 * T


def test_thickness_reproduces_the_paper_table():
    """With Pr = 1 (the BGK model's) and mu ~ T^0.5 the profile's Delta = (u_inf - u_2)/max|du/dx|,
    measured in the units the table's Re_Delta defines, is 1: the computed Re_Delta equals Table
    1DShockThickness's 24.34, 9.68, 11.03 at M = 1.2, 3, 4 (the table's four digits)."""
    for M, (_, Re, _) in gas.SHOCK_TABLE.items():
        assert abs(gp.re_delta(M) / Re - 1.0) < 2e-3, (M, gp.re_delta(M), Re)


@pytest.mark.parametrize("M", [1.2, 4.0])
def test_profile_obeys_the_printed_dtheta_domega_relation(M):
    """Along the profile the ratio of the two balances in the paper's variables Omega = (m/P) u,
    theta = (m/P)^2 R T is the printed dtheta/dOmega with its constant (4/5) Pr."""
    m, P, H, _, _ = gp.constants(M)
    alpha = 2.0 * H * m * m / (P * P) - 1.0
    p = gp.profile(M, 10.0)
    dmax = max(abs(gp.rhs(u, T, M, 10.0)[0]) for u, T in zip(p["u"], p["T"]))
    checked = 0
    for u, T in zip(p["u"][::50], p["T"][::50]):
        du, dT = gp.rhs(u, T, M, 10.0)
        if abs(du) < 1e-2 * dmax:   # near the end states both balances vanish: the ratio is noise
            continue
        Om, th = m / P * u, (m / P) ** 2 * 0.5 * T
        ratio = ((m / P) ** 2 * 0.5 * dT) / (m / P * du)
        assert abs(ratio - gp.dtheta_domega(Om, th, alpha)) <= 1e-9 * max(1.0, abs(ratio))
        checked += 1
    assert checked >= 5


def test_thickness_scales_with_one_over_re_and_the_profile_is_monotone():
    p1, p2 = gp.profile(3.0, 1.0), gp.profile(3.0, 9.68)
    assert abs(p2["Delta"] * 9.68 / p1["Delta"] - 1.0) < 1e-7
    assert np.all(np.diff(p2["u"]) <= 0.0)
    (r1, u1, T1), (r2, u2, T2) = gp.constants(3.0)[3:]
    assert abs(p2["u"][0] - u1) < 1e-6 * u1 and abs(p2["u"][-1] - u2) < 1e-5 * u2


def test_base_at_is_centred_on_the_steepest_point_and_continuous():
    """base_at places max|du/dx| at x = 0: there the finite-difference slope is -(u_inf - u_2)/Delta
    and it is a maximum; the saddle's linear tail past the start point joins the integrated profile."""
    M, Re = 3.0, 9.68
    p = gp.profile(M, Re)
    (r1, u1, T1), (r2, u2, T2) = gp.constants(M)[3:]
    h = 1e-4
    _, u, _ = gp.base_at(M, Re, np.array([-h, h, -50 * h, 50 * h, -0.3 - h, -0.3 + h]))
    slope = (u[1] - u[0]) / (2 * h)
    assert abs(slope * p["Delta"] / (u2 - u1) - 1.0) < 1e-6
    assert abs((u[3] - u[2]) / (100 * h)) < abs(slope)
    assert abs((u[5] - u[4]) / (2 * h)) < abs(slope)
    x0 = -p["x_shock"]   # the start point, in coordinates centred on the shock
    _, ua, Ta = gp.base_at(M, Re, np.array([x0 - 1e-9, x0 + 1e-9]))
    assert abs(ua[1] - ua[0]) < 1e-12 * u2 and abs(Ta[1] - Ta[0]) < 1e-11 * T2
    _, uf, Tf = gp.base_at(M, Re, np.array([-1e4, 1e4]))
    assert uf[0] == u1 and abs(uf[1] - u2) < 1e-14 * u2


@pytest.mark.parametrize("M", [1.05, 10.0])
def test_weak_and_strong_shocks_reach_both_end_states(M):
    """The default span follows the slowest end-state eigenvalue: the profile reaches the upstream
    state to rounding for a weak shock (whose thickness grows like 1/(M - 1)) and a strong one."""
    p = gp.profile(M, 1.0)
    (r1, u1, T1), (r2, u2, T2) = gp.constants(M)[3:]
    assert abs(p["u"][0] - u1) < 1e-12 * u1 and abs(p["T"][0] - T1) < 1e-12 * T1
    assert abs(p["u"][-1] - u2) <= 2e-6 * u2
    assert p["Delta"] > 0 and np.all(np.diff(p["u"]) <= 0.0) and np.all(np.diff(p["T"]) >= 0.0)


def test_gp_base_is_a_local_maxwellian_of_the_profile():
    """The pencil base 'gilbarg_paolucci': at every node the discrete moments of g_c are the profile's
    (rho, u, T) up to the velocity grid's quadrature error (about 1e-8 in rho, 1e-7 in T for the hot downstream state
    on 64 x 32 Gauss-Hermite nodes, rounding upstream), and h_c = (T/2) g_c."""
    from oracle import grids
    from paper_2607_27440_b300 import workloads as wl
    spec = wl.tiny(nx=16, qx=64, qy=32, mach=3.0, base="gilbarg_paolucci", noneq=0).as_dict()
    x, _ = grids.mapped_diff(spec["nx"], spec["map_L"], spec["map_sinf"])
    xi_x, xi_y, W = grids.velocity_grid(spec["qx"], spec["qy"])
    g, h = gas.base_flow(spec, x, xi_x, xi_y)
    rho_p, u_p, T_p = gp.base_at(3.0, spec["re_delta"], x, s=spec["visc_s"])
    rho, u, v, E = gas.moments(g, h, W, xi_x, xi_y)
    assert np.max(np.abs(rho / rho_p - 1)) < 1e-7 and np.max(np.abs(u / u_p - 1)) < 1e-7
    assert np.max(np.abs(gas.temperature(u, v, E) / T_p - 1)) < 3e-7
    up = x < -3.0
    assert np.max(np.abs(rho[up] / rho_p[up] - 1)) < 1e-12 and np.max(np.abs(u[up] / u_p[up] - 1)) < 1e-12
    assert np.allclose(h, 0.5 * T_p[:, None] * g, rtol=1e-14, atol=0)


def test_prandtl_number_enters_as_the_printed_constant():
    """The energy balance carries 1/Pr: at Pr = 2/3 the ratio of the balances in (Omega, theta) is the
    printed dtheta/dOmega with its 8/15 = (4/5)(2/3), and at Pr = 1/2 the 2/5 of the printed
    z-equations; the momentum balance does not depend on Pr."""
    M = 3.0
    m, P, H, _, (r2, u2, T2) = gp.constants(M)
    alpha = 2.0 * H * m * m / (P * P) - 1.0
    u, T = 0.5 * (gp.constants(M)[3][1] + u2), 0.5 * (1.0 + T2)   # a state inside the shock
    for Pr, const in ((2.0 / 3.0, 8.0 / 15.0), (0.5, 0.4)):
        du, dT = gp.rhs(u, T, M, 10.0, Pr=Pr)
        du1, _ = gp.rhs(u, T, M, 10.0, Pr=1.0)
        assert du == du1
        Om, th = m / P * u, (m / P) ** 2 * 0.5 * T
        ratio = ((m / P) ** 2 * 0.5 * dT) / (m / P * du)
        printed = const * Om * (th - ((1.0 - Om) ** 2 + alpha) / 3.0) / (Om * Om - Om + th)
        assert abs(ratio / printed - 1.0) < 1e-12
