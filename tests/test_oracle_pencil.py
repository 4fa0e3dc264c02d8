"""Pins for the oracle's assembled pencil (Eqs. comp_ghat1Dshock / comp_hhat1Dshock, Table benchmark_cases)."""
import numpy as np
import pytest

from oracle import gas, grids, pencil
from paper_2607_27440_b300 import workloads as wl


@pytest.mark.parametrize("nx,q,nnz", [(81, 20, 56_320_800), (81, 24, 113_542_272), (81, 32, 348_653_568)])
def test_nnz_formula_matches_paper_table_exactly(nx, q, nnz):
    """Table benchmark_cases prints nnz(A) for N = 80 (81 points), Q = 20/24/32."""
    assert pencil.nnz_formula(nx, q, q) == nnz
    assert 2 * nx * q * q == {20: 64_800, 24: 93_312, 32: 165_888}[q]


@pytest.mark.parametrize("nx,q,nnz_m", [(61, 24, 83.8), (101, 18, 48.5), (121, 16, 38.8)])
def test_nnz_formula_matches_paper_sweep(nx, q, nnz_m):
    """Table m12_nq_comparison prints nnz(A) in millions to 3 significant figures."""
    assert round(pencil.nnz_formula(nx, q, q) / 1e6, 1) == nnz_m


@pytest.mark.slow
@pytest.mark.parametrize("q", [20, 24, 32])
def test_assembled_nnz_equals_paper_table(q):
    """The oracle's assembled rows have exactly the paper's nonzero count at N = 80."""
    spec = wl.tiny(nx=81, qx=q, qy=q, mach=1.2, beta=16.0).as_dict()
    assert pencil.nnz_numerical(spec) == pencil.nnz_formula(81, q, q)


@pytest.mark.parametrize("nx,qx,qy", [(9, 4, 2), (7, 6, 4), (6, 5, 3)])
def test_dense_nnz_and_row_counter_agree(nx, qx, qy):
    spec = wl.tiny(nx=nx, qx=qx, qy=qy).as_dict()
    d = gas.pencil_data(spec)
    A, B = pencil.assemble_dense(spec, d)
    assert np.count_nonzero(A) == pencil.nnz_numerical(spec, d)
    if qx % 2 == 0:
        assert np.count_nonzero(A) == pencil.nnz_formula(nx, qx, qy)
    nbc = 4 * (qx // 2) * qy
    assert np.count_nonzero(np.diag(B) == 0) == nbc


def test_boundary_rows_are_inflow():
    """Boundary rows: x = -s_inf (j = N) with xi_x > 0 and x = +s_inf (j = 0) with xi_x < 0 (Sec. 2.2)."""
    spec = wl.tiny(nx=8, qx=5, qy=2).as_dict()
    d = gas.pencil_data(spec)
    assert d["x"][-1] < 0 < d["x"][0]
    assert np.array_equal(d["bc"][-1], d["xi_x"] > 0)
    assert np.array_equal(d["bc"][0], d["xi_x"] < 0)
    assert not d["bc"][1:-1].any()
    A, B = pencil.assemble_dense(spec, d)
    for r in pencil.boundary_rows(d):
        e = np.zeros(A.shape[0])
        e[r] = 1
        assert np.array_equal(A[r], e) and B[r, r] == 0


def test_streaming_rows_differentiate_manufactured_solution():
    """Row (c=0, k0, j) of A applied to q = p(y(x)) on block (0, k0) gives xi_x p'(y) dy/dx plus
    (nu + i beta xi_y) p minus the moment coupling of that single block (Eq. comp_ghat1Dshock)."""
    nx, qx, qy, beta = 12, 4, 2, 1.3
    spec = wl.tiny(nx=nx, qx=qx, qy=qy, beta=beta).as_dict()
    d = gas.pencil_data(spec)
    A, _ = pencil.assemble_dense(spec, d)
    nxi = qx * qy
    y = grids.cheb_points(nx - 1)
    _, dydx, _ = grids.algebraic_map(y, 1.0, 30.0)
    p = np.polynomial.chebyshev.Chebyshev(np.random.default_rng(1).standard_normal(nx))
    k0 = 5
    q = np.zeros(A.shape[0], dtype=complex)
    q[pencil.index(0, k0, np.arange(nx), nxi, nx)] = p(y)
    Aq = A @ q
    for j in range(1, nx - 1):
        cpl = np.sum(d["G"][0, :, j, k0] * d["w"][0, :, j, k0])
        want = d["xi_x"][k0] * p.deriv()(y[j]) * dydx[j] + (d["nu"][j] + 1j * beta * d["xi_y"][k0] - cpl) * p(y[j])
        assert Aq[pencil.index(0, k0, j, nxi, nx)] == pytest.approx(want, rel=1e-10, abs=1e-10)


@pytest.mark.parametrize("nx,qx,qy", [(9, 4, 2), (7, 5, 3)])
def test_matrix_free_equals_dense(nx, qx, qy):
    spec = wl.tiny(nx=nx, qx=qx, qy=qy, beta=0.9).as_dict()
    d = gas.pencil_data(spec)
    A, B = pencil.assemble_dense(spec, d)
    X = wl.random_vectors(A.shape[0], 3, 7).T
    assert np.allclose(pencil.apply_A(spec, d, X), A @ X, rtol=1e-13, atol=1e-13 * np.abs(A).max())
    assert np.array_equal(pencil.apply_B(d, X), B @ X)


def test_conjugation_symmetry():
    """Symmetric xi_y nodes: conj(A(beta)) = P A(beta) P with P : xi_y -> -xi_y (real beta)."""
    nx, qx, qy = 7, 4, 4
    spec = wl.tiny(nx=nx, qx=qx, qy=qy, beta=1.7).as_dict()
    d = gas.pencil_data(spec)
    A, _ = pencil.assemble_dense(spec, d)
    nxi = qx * qy
    perm = np.empty(A.shape[0], dtype=int)
    for c in range(2):
        for kx in range(qx):
            for ky in range(qy):
                for j in range(nx):
                    perm[pencil.index(c, kx * qy + ky, j, nxi, nx)] = pencil.index(c, kx * qy + (qy - 1 - ky), j, nxi, nx)
    assert np.allclose(A.conj(), A[np.ix_(perm, perm)], rtol=0, atol=1e-13 * np.abs(A).max())
    spec0 = dict(spec, beta=0.0)
    A0, _ = pencil.assemble_dense(spec0, gas.pencil_data(spec0))
    assert np.abs(A0.imag).max() == 0.0
