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
