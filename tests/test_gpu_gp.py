"""GPU Gilbarg-Paolucci shock structure (paper Sec. 2.1, Eqs. GB1DShockeqn and ShockThickness) vs the
oracle's adaptive integration (oracle/gp.py).

Tolerances: the device integrates with classical RK4 at a fixed step of 0.02 / max|eigenvalue| of the
two end states, the oracle with an adaptive Runge-Kutta at rtol 1e-12.  RK4's global error at that
step is about 1e-10 of the jump, so the thickness agrees to 1e-9; the steepest point is a flat
maximum located by the zero of d^2u/dx^2 on both sides (to ~1e-8 Delta), and the profile at a point
moves with it, by the slope times that shift: 2e-8 of the jump."""
import numpy as np
import pytest

from oracle import gas, gp
from paper_2607_27440_b300 import workloads as wl

pytestmark = pytest.mark.gpu

CASES = [  # (mach, re, visc_s, prandtl)
    (1.05, 1.0, 0.5, 1.0), (1.2, 1.0, 0.5, 1.0), (2.0, 1.0, 0.72, 1.0), (3.0, 9.68, 0.5, 1.0),
    (4.0, 1.0, 1.0, 1.0), (6.0, 1.0, 0.5, 2.0 / 3.0), (10.0, 1.0, 0.5, 1.0), (3.0, 1.0, 0.5, 0.75),
]


@pytest.fixture(scope="module")
def klst():
    from paper_2607_27440_b300 import klst as k
    k.load()
    return k


@pytest.fixture(scope="module")
def oracle_profiles():
    return {c: gp.profile(c[0], c[1], s=c[2], Pr=c[3]) for c in CASES}


def test_thickness_and_steepest_point_match_the_oracle(klst, oracle_profiles):
    M, Re, s, Pr = (np.array(v) for v in zip(*CASES))
    res, prof = klst.gp_shock(M, Re, s, Pr)
    assert prof is None and np.all(res["status"] == klst.KLST_OK)
    for i, c in enumerate(CASES):
        p = oracle_profiles[c]
        assert abs(res["delta"][i] / p["Delta"] - 1.0) <= 1e-9, (c, res["delta"][i], p["Delta"])
        assert abs(res["x_shock"][i] - p["x_shock"]) <= 2e-8 * p["Delta"], (c, res["x_shock"][i], p["x_shock"])
        assert abs(res["lambda_s"][i] / p["lam_s"] - 1.0) <= 1e-7
        assert res["x_up"][i] < res["x_shock"][i] < 0.0 and res["steps"][i] > 100


def test_table_reynolds_numbers(klst):
    """With Re = 1 the thickness is the self-consistent Re_Delta: Table 1DShockThickness's values at
    M = 1.2, 3, 4 to its printed digits (the Pr = 1 reading)."""
    Ms = sorted(gas.SHOCK_TABLE)
    res, _ = klst.gp_shock(Ms)
    for M, d in zip(Ms, res["delta"]):
        assert abs(d / gas.SHOCK_TABLE[M][1] - 1.0) < 2e-3


@pytest.mark.parametrize("c", [CASES[1], CASES[3], CASES[5], CASES[6]], ids=lambda c: f"M{c[0]}Pr{c[3]:.2f}")
def test_profile_at_points_matches_the_oracle(klst, oracle_profiles, c):
    """rho, u, T at points in any order: through the shock, past the start point (the saddle's
    linear solution) and past the upstream end."""
    p = oracle_profiles[c]
    D = p["Delta"]
    rng = np.random.default_rng(7)
    x = np.concatenate([np.linspace(-6 * D, 6 * D, 61), [-1e4, 1e4, -p["x_shock"] + 0.3 * D, 0.0],
                        rng.uniform(-20 * D, 20 * D, 40)])
    rng.shuffle(x)
    res, prof = klst.gp_shock(c[0], c[1], c[2], c[3], x=x)
    got = prof.cpu().numpy()[:, 0, :]
    rho, u, T = gp.base_at(c[0], c[1], x, s=c[2], Pr=c[3])
    (r1, u1, T1), (r2, u2, T2) = gp.constants(c[0])[3:]
    assert np.max(np.abs(got[1] - u)) <= 2e-8 * (u1 - u2)
    assert np.max(np.abs(got[2] - T)) <= 2e-8 * (T2 - T1)
    assert np.max(np.abs(got[0] - rho)) <= 2e-8 * (r2 - r1)
    assert np.array_equal(got[0], gp.constants(c[0])[0] / got[1])
    far = np.abs(x) == 1e4
    assert np.all(got[1][far & (x < 0)] == u1)


def test_large_batch_is_case_independent(klst):
    """2048 cases in one launch: every case converges, sampled cases equal the one-case launches bit
    for bit (one thread per case) and the oracle within the thickness tolerance."""
    rng = np.random.default_rng(11)
    n = 2048
    M = rng.uniform(1.1, 10.0, n)
    s = rng.uniform(0.5, 1.0, n)
    res, _ = klst.gp_shock(M, 1.0, s, 1.0)
    assert np.all(res["status"] == 0) and np.all(res["delta"] > 0)
    for i in rng.choice(n, 4, replace=False):
        one, _ = klst.gp_shock(M[i], 1.0, s[i], 1.0)
        assert one["delta"][0] == res["delta"][i] and one["x_shock"][0] == res["x_shock"][i]
        p = gp.profile(M[i], 1.0, s=s[i])
        assert abs(res["delta"][i] / p["Delta"] - 1.0) <= 1e-9


def test_pencil_on_the_gilbarg_paolucci_base(klst):
    """base = gilbarg_paolucci: the pencil's tables equal the oracle's on the same base (the profile at
    the nodes agrees to ~1e-8, so nu, G, w agree to that), and the eigenvalues nearest sigma of the
    device pencil are those of the oracle's dense pencil."""
    from oracle import eig, pencil
    from tests.helpers import to_dev
    spec = wl.tiny(nx=12, qx=6, qy=4, mach=3.0, base="gilbarg_paolucci", noneq=0)
    d = gas.pencil_data(spec.as_dict())
    P = klst.Pencil(spec)
    t = P.tables()
    assert np.allclose(t["nu"], d["nu"], rtol=1e-7, atol=0)
    G = np.transpose(t["G"], (1, 2, 3, 0))
    w = np.transpose(t["w"], (1, 2, 3, 0))
    assert np.max(np.abs(G - d["G"])) <= 1e-7 * np.max(np.abs(d["G"]))
    assert np.max(np.abs(w - d["w"])) <= 1e-7 * np.max(np.abs(d["w"]))
    A, B = pencil.assemble_dense(spec.as_dict(), d)
    lam, _, kap = eig.interior(A, pencil.boundary_rows(d))
    sigma = 0.1 + 0.1j
    idx = eig.nearest(lam, sigma, 6)
    F = P.factor(sigma, precision=klst.FP64)
    om, _, res, info = F.eigs(6, 24, tol=1e-12, v0=to_dev(wl.start_vector(P.n, 2)))
    perm = eig.match(lam[idx], om)
    assert np.max(np.abs(om[perm] - lam[idx]) / np.abs(lam[idx])) <= 1e-5


def test_invalid_cases_and_options(klst):
    for kw in ({"mach": 1.0}, {"mach": 3.0, "re": 0.0}, {"mach": 3.0, "visc_s": 2.5}, {"mach": 3.0, "prandtl": 0.0},
               {"mach": 3.0, "step": 0.6}, {"mach": 3.0, "eps": 1e-2}, {"mach": 3.0, "max_steps": -1},
               {"mach": 3.0, "x": [0.0, np.nan]}):
        with pytest.raises(klst.KlstError) as ei:
            klst.gp_shock(**kw)
        assert ei.value.code == klst.KLST_EINVAL
    with pytest.raises(klst.KlstError) as ei:   # stops after 10 steps: the result says so
        klst.gp_shock(3.0, max_steps=10)
    assert ei.value.code == klst.KLST_ENOCONV
    with pytest.raises(klst.KlstError) as ei:
        klst.Pencil(wl.tiny(nx=9, qx=4, qy=2, mach=3.0, base="gilbarg_paolucci", gamma=1.4))
    assert ei.value.code == klst.KLST_EINVAL


def test_several_cases_with_points_keep_the_callers_order(klst, oracle_profiles):
    """Cases given out of Mach order (the launch sorts them) with points: row c of the profile and
    result c belong to case c."""
    cases = [CASES[6], CASES[1], CASES[3]]   # M = 10, 1.2, 3
    M, Re, s, Pr = (np.array(v) for v in zip(*cases))
    x = np.linspace(-40.0, 40.0, 23)
    res, prof = klst.gp_shock(M, Re, s, Pr, x=x)
    got = prof.cpu().numpy()
    for c, case in enumerate(cases):
        p = oracle_profiles[case]
        assert abs(res["delta"][c] / p["Delta"] - 1.0) <= 1e-9
        rho, u, T = gp.base_at(case[0], case[1], x, s=case[2], Pr=case[3])
        (r1, u1, T1), (r2, u2, T2) = gp.constants(case[0])[3:]
        assert np.max(np.abs(got[1, c] - u)) <= 2e-8 * (u1 - u2)
        assert np.max(np.abs(got[2, c] - T)) <= 2e-8 * (T2 - T1)
