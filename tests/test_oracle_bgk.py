"""Pins of the BE-BGK base-flow oracle (paper Sec. 3.3) against what the scheme fixes exactly."""
import numpy as np
import pytest

from oracle import bgk, gas, grids
from paper_2607_27440_b300 import workloads as wl

SPEC = wl.tiny(nx=12, qx=8, qy=6, mach=1.5)


def _setup(spec=SPEC):
    xi_x, xi_y, W = grids.velocity_grid(spec.qx, spec.qy)
    x = bgk.grid(spec)
    return x, xi_x, xi_y, W


def test_minmod():
    a = np.array([1.0, -2.0, 3.0, 0.0, -1.0])
    b = np.array([2.0, -1.0, -3.0, 5.0, -4.0])
    assert np.array_equal(bgk.minmod(a, b), np.array([1.0, -1.0, 0.0, 0.0, -1.0]))


def test_muscl_is_exact_on_linear_profiles():
    """On a uniform grid a linear profile has equal slopes, minmod returns them, and the interface
    values are the exact midpoint values: streaming = xi_x * slope / h away from the ends."""
    N, h = 20, 0.3
    x = h * np.arange(N + 1)
    xi_x = np.array([-1.7, -0.4, 0.0, 0.6, 2.2])
    phi = 2.0 + 0.75 * x[:, None] * np.ones((1, len(xi_x)))
    s = bgk.streaming(phi, x, xi_x)
    assert np.allclose(s[2:-2], (0.75 * xi_x)[None, :] * np.ones((N - 3, 1)), rtol=0, atol=1e-13)
    f = bgk.interface_values(phi, xi_x)
    assert np.allclose(f[1:-1], 2.0 + 0.75 * 0.5 * (x[1:-2] + x[2:-1])[:, None], rtol=0, atol=1e-13)


def test_limiter_keeps_a_step_within_its_bounds():
    """Minmod reconstruction of a step creates no new extrema: every interface value lies between
    the values of the two cells it separates (the TVD property of the limiter)."""
    xi_x = np.array([-1.0, 1.0])
    phi = np.where(np.arange(15)[:, None] < 7, 1.0, 3.0) * np.ones((1, 2))
    f = bgk.interface_values(phi, xi_x)
    lo = np.minimum(phi[:-1], phi[1:])
    hi = np.maximum(phi[:-1], phi[1:])
    assert np.all(f >= lo - 1e-15) and np.all(f <= hi + 1e-15)


def test_streaming_telescopes():
    """Finite volumes: sum_i dx_i (streaming)_i over the interior = xi_x (phi_{N-1/2} - phi_{1/2})."""
    x, xi_x, xi_y, W = _setup()
    rng = np.random.default_rng(3)
    phi = rng.standard_normal((len(x), len(xi_x)))
    s = bgk.streaming(phi, x, xi_x)
    xm = 0.5 * (x[1:] + x[:-1])
    dx = xm[1:] - xm[:-1]
    f = bgk.interface_values(phi, xi_x)
    assert np.allclose((dx[:, None] * s[1:-1]).sum(axis=0), xi_x * (f[-1] - f[0]), rtol=1e-12, atol=1e-12)


def test_relaxation_conserves_mass_momentum_energy():
    """The discrete equilibrium carries the discrete moments, so the relaxation term has zero mass,
    momentum and energy moments at every node to round-off (Sec. 2.2 moments, Sec. 3.3)."""
    x, xi_x, xi_y, W = _setup()
    g, h = bgk.initial_state(SPEC, x, xi_x, xi_y, W)
    cg, ch = bgk.relaxation(g, h, xi_x, xi_y, W, SPEC)
    e2 = xi_x ** 2 + xi_y ** 2
    scale = np.abs(g) @ W
    for m in (cg @ W, (cg * xi_x) @ W, (cg * xi_y) @ W, 0.5 * ((cg * e2) @ W + ch @ W)):
        assert np.max(np.abs(m) / scale) < 1e-12


def test_end_states_and_uniform_maxwellians_are_fixed_points():
    """A Maxwellian is the discrete equilibrium of its own moments, so a uniform Maxwellian state has
    RHS = 0 (no streaming, no relaxation); the Rankine-Hugoniot end states are Maxwellians."""
    x, xi_x, xi_y, W = _setup()
    for g0, h0 in bgk.end_states(SPEC, xi_x, xi_y, W):
        g = np.repeat(g0[None], len(x), axis=0)
        h = np.repeat(h0[None], len(x), axis=0)
        rg, rh = bgk.rhs(g, h, x, xi_x, xi_y, W, SPEC)
        assert np.max(np.abs(rg)) < 1e-12 * np.max(g) and np.max(np.abs(rh)) < 1e-12 * np.max(h)


def test_end_states_satisfy_rankine_hugoniot_on_the_grid():
    """The downstream end state carries exactly the upstream discrete fluxes, and it converges to the
    continuous Rankine-Hugoniot state as the node set resolves the Maxwellians."""
    for qx, qy, tol in ((8, 6, 5e-2), (24, 12, 1e-5)):
        spec = wl.tiny(nx=12, qx=qx, qy=qy, mach=1.5)
        xi_x, xi_y, W = grids.velocity_grid(spec.qx, spec.qy)
        (gu, hu), (gd, hd) = bgk.end_states(spec, xi_x, xi_y, W)
        fu, fd = bgk.discrete_fluxes(gu, hu, xi_x, xi_y, W), bgk.discrete_fluxes(gd, hd, xi_x, xi_y, W)
        assert np.max(np.abs(fu - fd) / np.abs(fu)) < 1e-12
        (_, _), (gc, hc) = bgk.end_states(spec, xi_x, xi_y)
        assert np.max(np.abs(gd - gc)) / np.max(gc) < tol


def test_rhs_changes_moments_only_through_the_end_fluxes():
    """Finite-volume conservation: the interior cells' mass, momentum and energy (sum_i dx_i sum_k
    W psi q_i) change at the rate F(1/2) - F(N - 1/2) of the interface fluxes next to the ends,
    because the streaming telescopes and the relaxation conserves every moment at every node."""
    x, xi_x, xi_y, W = _setup()
    g, h = bgk.initial_state(SPEC, x, xi_x, xi_y, W)
    rng = np.random.default_rng(7)
    g[1:-1] *= 1.0 + 0.05 * rng.standard_normal(g[1:-1].shape)
    rg, rh = bgk.rhs(g, h, x, xi_x, xi_y, W, SPEC)
    xm = 0.5 * (x[1:] + x[:-1])
    dx = (xm[1:] - xm[:-1])[:, None]
    e2 = xi_x ** 2 + xi_y ** 2
    rate = np.array([((dx * rg[1:-1]).sum(0)) @ W, ((dx * rg[1:-1]).sum(0) * xi_x) @ W,
                     0.5 * (((dx * rg[1:-1]).sum(0) * e2) @ W + ((dx * rh[1:-1]).sum(0)) @ W)])
    fg, fh = bgk.interface_values(g, xi_x), bgk.interface_values(h, xi_x)
    F = np.stack([bgk.discrete_fluxes(fg[i], fh[i], xi_x, xi_y, W) for i in (0, len(fg) - 1)])
    assert np.allclose(rate, F[0] - F[1], rtol=1e-11, atol=1e-12 * np.abs(F).max())
