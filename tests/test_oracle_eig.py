"""Pins for the oracle's eigen-solutions (Sec. 4: QZ, shift-and-invert, Eq. parShiftInvert)."""
import numpy as np
import pytest

from oracle import eig, gas, pencil
from paper_2607_27440_b300 import workloads as wl


@pytest.fixture(scope="module")
def small():
    spec = wl.tiny(nx=9, qx=4, qy=3, beta=1.0, mach=3.0).as_dict()
    d = gas.pencil_data(spec)
    A, B = pencil.assemble_dense(spec, d)
    return spec, d, A, B


def test_qz_matches_interior_reduction(small):
    """Finite spectrum of (A, B): QZ equals the interior standard problem; infinite ones are the boundary rows."""
    spec, d, A, B = small
    lq, Xq, kq = eig.qz(A, B)
    li, Xi, ki = eig.interior(A, pencil.boundary_rows(d))
    assert lq.size == li.size == A.shape[0] - pencil.boundary_rows(d).size
    perm = eig.match(lq, li)
    assert np.max(np.abs(lq - li[perm]) / np.maximum(1, np.abs(lq))) < 1e-10
    assert np.max(eig.residuals(spec, d, li, Xi)) < 1e-12 * np.abs(A).max()
    assert np.max(eig.residuals(spec, d, lq, Xq)) < 1e-11 * np.abs(A).max()


def test_spectrum_closed_under_conjugation(small):
    spec, d, A, B = small
    li, _, _ = eig.interior(A, pencil.boundary_rows(d))
    perm = eig.match(li, li.conj())
    assert np.max(np.abs(li - li.conj()[perm])) < 1e-10 * np.abs(li).max()


def test_shift_invert_arpack_matches_interior(small):
    """ARPACK on T = (A - sigma B)^{-1} B returns the eigenvalues nearest sigma with omega = sigma + 1/mu."""
    spec, d, A, B = small
    sigma = 0.3 + 0.2j
    li, _, kap = eig.interior(A, pencil.boundary_rows(d))
    ref = li[eig.nearest(li, sigma, 8)]
    si = eig.ShiftInvert(A, B, sigma)
    om, X = si.eigs(8, ncv=30, v0=wl.start_vector(A.shape[0], 3))
    perm = eig.match(om, ref)
    assert np.max(np.abs(om - ref[perm]) / np.abs(ref[perm])) < 1e-9
    assert np.max(eig.residuals(spec, d, om, X)) < 1e-10


def test_shift_invert_apply_is_linear_solve(small):
    """T x solves (A - sigma B) y = B x; range of T excludes the boundary null space of B."""
    spec, d, A, B = small
    sigma = 0.1j
    si = eig.ShiftInvert(A, B, sigma)
    x = wl.start_vector(A.shape[0], 11)
    y = si.apply(x)
    assert np.linalg.norm((A - sigma * B) @ y - B @ x) < 1e-12 * np.linalg.norm(B @ x) * np.abs(A).max()
    br = pencil.boundary_rows(d)
    assert np.max(np.abs(y[br])) < 1e-14 * np.linalg.norm(y)


def test_match_is_one_to_one():
    a = np.array([1.0, 1.0 + 1e-9, 5.0])
    b = np.array([5.0, 1.0 + 2e-9, 1.0 - 1e-9])
    perm = eig.match(a, b)
    assert sorted(perm) == [0, 1, 2]
    assert np.max(np.abs(a - b[perm])) < 3e-9
