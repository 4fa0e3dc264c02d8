"""Pins for the oracle's grids: Chebyshev D (Sec. 3.1), the algebraic map, Gauss-Hermite (Sec. 3.2)."""
import math

import numpy as np
import pytest
import scipy.special as ssp

from oracle import grids


@pytest.mark.parametrize("N", [4, 7, 16, 31, 63, 127])
def test_cheb_diff_exact_on_polynomials(N):
    """D_y differentiates every polynomial of degree <= N exactly (collocation property)."""
    y = grids.cheb_points(N)
    D = grids.cheb_diff(N)
    rng = np.random.default_rng(N)
    for deg in (0, 1, N // 2, N):
        coef = rng.standard_normal(deg + 1)
        p = np.polynomial.chebyshev.Chebyshev(coef)
        dp = p.deriv()(y) if deg > 0 else np.zeros_like(y)
        err = np.max(np.abs(D @ p(y) - dp))
        assert err <= 1e-10 * max(1.0, np.max(np.abs(dp))) * N, (deg, err)


def test_cheb_points_and_corners():
    N = 10
    y = grids.cheb_points(N)
    assert y[0] == 1.0 and y[N] == -1.0
    D = grids.cheb_diff(N)
    assert D[0, 0] == pytest.approx((2 * N * N + 1) / 6.0)
    assert D[N, N] == pytest.approx(-(2 * N * N + 1) / 6.0)
    # rows of a differentiation matrix annihilate constants
    assert np.max(np.abs(D.sum(axis=1))) < 1e-12 * N * N


@pytest.mark.parametrize("L,sinf", [(1.0, 30.0), (0.5, 10.0), (2.0, 100.0)])
def test_map_derivatives_against_complex_step(L, sinf):
    """dy/dx and d2y/dx2 printed beside Eq. Chebmapping vs complex-step differentiation of y(x)."""
    s = (L / sinf) ** 2
    y = grids.cheb_points(20)[1:-1]
    x, dydx, d2 = grids.algebraic_map(y, L, sinf)
    # inverse map y(x) = x sqrt(1+s) / sqrt(L^2 + x^2), written from x = L y / sqrt(1+s-y^2)
    inv = lambda xx: xx * np.sqrt(1.0 + s) / np.sqrt(L * L + xx * xx)
    h = 1e-30
    cs = np.imag(inv(x + 1j * h)) / h
    assert np.allclose(cs, dydx, rtol=1e-13, atol=0)
    hh = 1e-4 * (1 + np.abs(x))
    fd2 = (inv(x + hh) - 2 * inv(x) + inv(x - hh)) / hh ** 2
    assert np.allclose(fd2, d2, rtol=1e-5, atol=1e-9)
    assert np.allclose(inv(x), y, rtol=0, atol=1e-14)
    xe, _, _ = grids.algebraic_map(np.array([1.0, -1.0]), L, sinf)
    assert np.allclose(xe, [sinf, -sinf], rtol=1e-14)


def test_mapped_diff_on_mapped_polynomial():
    """D_x f(x_j) = f'(x) for f(x) = p(y(x)), p a polynomial of degree <= N."""
    nx = 24
    x, Dx = grids.mapped_diff(nx, 1.0, 30.0)
    y = grids.cheb_points(nx - 1)
    p = np.polynomial.chebyshev.Chebyshev(np.random.default_rng(0).standard_normal(nx))
    _, dydx, _ = grids.algebraic_map(y, 1.0, 30.0)
    assert np.allclose(Dx @ p(y), p.deriv()(y) * dydx, rtol=1e-10, atol=1e-9)
    assert x[0] > 0 and x[-1] < 0


@pytest.mark.parametrize("Q", [2, 3, 4, 6, 8, 12, 18, 24, 48, 61])
def test_gauss_hermite_moments(Q):
    """sum w_i x_i^{2m} = Gamma(m + 1/2) exactly for 2m <= 2Q - 1; odd moments vanish (Sec. 3.2)."""
    x, w, W = grids.gauss_hermite(Q)
    assert np.all(np.diff(x) > 0)
    assert np.array_equal(x, -x[::-1])
    for m in range(0, Q):
        exact = math.gamma(m + 0.5)
        got = np.sum(W * np.exp(-x * x) * x ** (2 * m))
        assert got == pytest.approx(exact, rel=1e-10), m
        assert abs(np.sum(W * np.exp(-x * x) * x ** (2 * m + 1))) < 1e-10 * exact


@pytest.mark.parametrize("Q", [4, 10, 20, 40, 61, 100])
def test_gauss_hermite_against_numpy_and_printed_formula(Q):
    """Nodes/weights vs numpy's hermgauss; W_i vs the printed weight formula in log space."""
    x, w, W = grids.gauss_hermite(Q)
    xr, wr = np.polynomial.hermite.hermgauss(Q)
    assert np.allclose(x, xr, rtol=0, atol=1e-12 * max(1, np.abs(xr).max()))
    mask = wr > 1e-250
    assert np.allclose(W[mask] * np.exp(-x[mask] ** 2), wr[mask], rtol=1e-9, atol=0)
    # printed: w_i = 2^{n-1} n! sqrt(pi) / (n^2 H_{n-1}(x_i)^2), evaluated as log via the
    # physicists' Hermite recurrence in scaled form H_m(x) / sqrt(2^m m!) to avoid overflow
    n = Q
    logH = np.zeros_like(x)
    for i, xi in enumerate(x):
        a, b, lscale = 1.0, 0.0, 0.0  # a = H_m/scale, b = H_{m-1}/scale
        for m in range(0, n - 1):
            a, b = 2 * xi * a - 2 * m * b, a
            big = max(abs(a), abs(b))
            if big > 1e100:
                a, b, lscale = a / big, b / big, lscale + math.log(big)
        logH[i] = lscale + math.log(abs(a))
    logw = (n - 1) * math.log(2) + ssp.gammaln(n + 1) + 0.5 * math.log(math.pi) - 2 * math.log(n) - 2 * logH
    logW = logw + x * x
    assert np.allclose(np.log(W), logW, rtol=0, atol=1e-9)


def test_hermite_functions_against_scipy():
    xs = np.linspace(-4, 4, 17)
    psi = grids.hermite_functions(xs, 12)
    for m in range(12):
        ref = ssp.eval_hermite(m, xs) * np.exp(-xs * xs / 2) / math.sqrt(2 ** m * math.factorial(m) * math.sqrt(math.pi))
        assert np.allclose(psi[m], ref, rtol=1e-12, atol=1e-14)


def test_velocity_grid_tensor_order():
    xi_x, xi_y, W = grids.velocity_grid(3, 2)
    nx_, _, Wx = grids.gauss_hermite(3)
    ny_, _, Wy = grids.gauss_hermite(2)
    assert xi_x[2 * 1 + 0] == nx_[1] and xi_y[2 * 1 + 1] == ny_[1]
    assert W[2 * 2 + 1] == pytest.approx(Wx[2] * Wy[1])
    assert xi_x[2] == 0.0 and xi_x[3] == 0.0  # odd qx has an exact zero node
