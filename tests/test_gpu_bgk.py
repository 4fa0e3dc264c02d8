"""GPU BE-BGK base-flow solver (paper Sec. 3.3) against the oracle's scheme, and pencils on its base."""
import numpy as np
import pytest

from oracle import bgk, eig, gas, grids, pencil, post
from paper_2607_27440_b300 import workloads as wl
from tests.helpers import cond1, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def klst():
    from paper_2607_27440_b300 import klst as k
    k.load()
    return k


def _host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("spec", [wl.tiny(nx=12, qx=8, qy=6, mach=1.5), wl.tiny(nx=17, qx=7, qy=4, mach=3.0)],
                         ids=["12x8x6", "17x7x4-oddq"])
def test_rk4_steps_match_oracle(klst, spec):
    """60 RK4 steps at a fixed time step from the Mott-Smith start: node by node equal to the oracle's
    scheme (MUSCL-minmod streaming, relaxation to the discrete equilibrium, Dirichlet ends)."""
    dt = 0.02
    g, h, info = klst.bgk_base_flow(spec, max_steps=60, dt=dt, check_every=20)
    assert info["steps"] == 60
    ref = bgk.steady(spec, steps=60, dt=dt)
    scale = np.abs(ref["g"]).max()
    assert np.abs(_host(g) - ref["g"]).max() <= 1e-11 * scale
    assert np.abs(_host(h) - ref["h"]).max() <= 1e-11 * np.abs(ref["h"]).max()


@pytest.mark.parametrize("steps", [0, 60])
def test_gilbarg_paolucci_start_matches_oracle(klst, steps):
    """The Gilbarg-Paolucci start (the continuum profile's local Maxwellian, steepest point at x = 0)
    and 60 RK4 steps from it equal the oracle's; the start's profile agrees to ~2e-8 of the jump
    (fixed-step RK4 on the device, adaptive integration in the oracle), hence the tolerance."""
    spec = wl.tiny(nx=16, qx=8, qy=6, mach=3.0, re_delta=9.68)
    g, h, info = klst.bgk_base_flow(spec, max_steps=steps, dt=0.02, check_every=20, start="gilbarg_paolucci")
    assert info["steps"] == steps
    ref = bgk.steady(spec, steps=steps, dt=0.02, start="gilbarg_paolucci")
    assert np.abs(_host(g) - ref["g"]).max() <= 1e-7 * np.abs(ref["g"]).max()
    assert np.abs(_host(h) - ref["h"]).max() <= 1e-7 * np.abs(ref["h"]).max()


def test_recentring_matches_oracle(klst):
    """With re-centring every 20 steps and a tight threshold the grid is rebuilt about the shock and
    the state moved by linear interpolation; the same rebuilds and the same state as the oracle."""
    spec = wl.tiny(nx=16, qx=8, qy=6, mach=2.0, width=1.5)
    kw = dict(dt=0.02, recentre_every=20, recentre_tol=1e-3)
    g, h, info = klst.bgk_base_flow(spec, max_steps=200, check_every=20, **kw)
    ref = bgk.steady(spec, steps=200, **kw)
    assert info["recentres"] >= 1 and info["recentres"] == ref["recentres"], (info, ref["recentres"])
    assert abs(info["centre"] - ref["centre"]) <= 1e-12
    assert np.abs(_host(g) - ref["g"]).max() <= 1e-10 * np.abs(ref["g"]).max()


def test_steady_state_conserves_fluxes(klst):
    """After 20,000 steps (t = 100 shock thicknesses of flow time at this grid's dt) the residual is
    at the limiter's floor (~1e-7 of max g: minmod switching keeps a steady TVD scheme from
    converging further) and the state is steady and conservative: the interface fluxes of mass,
    momentum and energy (the oracle's reconstruction and flux sums on the GPU state) agree across
    every interface and with the upstream state's to 1e-6."""
    spec = wl.tiny(nx=32, qx=8, qy=6, mach=2.0)
    g, h, info = klst.bgk_base_flow(spec, max_steps=20000, cfl=0.5, check_every=500)
    assert info["resid"] <= 1e-6, info
    xi_x, xi_y, W = grids.velocity_grid(spec.qx, spec.qy)
    gp, hp = _host(g)[::-1], _host(h)[::-1]
    fg, fh = bgk.interface_values(gp, xi_x), bgk.interface_values(hp, xi_x)
    F = np.stack([bgk.discrete_fluxes(fg[i], fh[i], xi_x, xi_y, W) for i in range(len(fg))])
    up = bgk.discrete_fluxes(gp[0], hp[0], xi_x, xi_y, W)
    assert np.max(np.abs(F - up[None]) / np.abs(up)[None]) < 1e-6
    # a shock: the bulk velocity falls monotonically from u1 to u2
    rho, u, v, E = gas.moments(gp, hp, W, xi_x, xi_y)
    assert np.all(np.diff(u) <= 1e-9) and u[0] > u[-1]


def test_pencil_on_the_bgk_base_matches_dense_lu(klst):
    """A pencil built on the BE-BGK base (klst_build_pencil_base) against the oracle's dense pencil on
    the same base: the shift-and-invert apply element by element."""
    spec = wl.tiny(nx=16, qx=6, qy=4, mach=2.0, beta=0.5)
    g, h, info = klst.bgk_base_flow(spec, max_steps=4000, cfl=0.5, check_every=200)
    base = (_host(g), _host(h))
    d = gas.pencil_data(spec.as_dict(), base=base)
    A, B = pencil.assemble_dense(spec.as_dict(), d)
    sigma = 0.1j
    si = eig.ShiftInvert(A, B, sigma)
    X = wl.random_vectors(A.shape[0], 2, 29)
    ref = np.stack([si.apply(x) for x in X])
    tol = max(1e-12, 64 * cond1(A - sigma * B, si.lu) * 2.220446049250313e-16)
    P = klst.Pencil(spec, base=(g, h))
    F = P.factor(sigma, precision=klst.FP64)
    Y = to_host(F.apply(to_dev(X)))
    err = np.abs(Y - ref).max(axis=1) / np.abs(ref).max(axis=1)
    assert np.all(err <= tol), (err, tol)
    # and the base's non-equilibrium measure is what the oracle computes from it
    ne = P.base_noneq()
    assert np.allclose(ne, post.eneq(d), rtol=1e-10, atol=1e-14)


def test_bgk_invalid_options(klst):
    spec = wl.tiny(nx=12, qx=6, qy=4, mach=1.5)
    for kw in ({"cfl": 0.0}, {"check_every": 0}, {"recentre_every": 150, "check_every": 100}, {"max_steps": -1}):
        with pytest.raises(klst.KlstError) as ei:
            klst.bgk_base_flow(spec, **kw)
        assert ei.value.code == klst.KLST_EINVAL
    with pytest.raises(klst.KlstError) as ei:   # the continuum profile is monatomic
        klst.bgk_base_flow(wl.tiny(nx=12, qx=6, qy=4, mach=1.5, gamma=1.4), start="gilbarg_paolucci")
    assert ei.value.code == klst.KLST_EINVAL
