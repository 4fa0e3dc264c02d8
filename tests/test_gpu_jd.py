"""GPU Jacobi-Davidson with harmonic Ritz extraction (paper Sec. 4.2) vs the oracle's eigenvalues."""
import numpy as np
import pytest

from oracle import eig, gas, pencil
from paper_2607_27440_b300 import workloads as wl
from tests.helpers import eig_gate, pencil_norm2_est, read_golden, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def klst():
    from paper_2607_27440_b300 import klst as k
    k.load()
    return k


def _check_against(omega, ref, kappa, normA, rel=1e-8):
    perm = eig.match(ref, omega)
    got = omega[perm]
    gate = eig_gate(ref, kappa, normA)
    err = np.abs(got - ref) / np.abs(ref)
    assert gate.sum() >= max(1, len(ref) // 2), "too few well-conditioned eigenvalues to gate"
    assert np.all(err[gate] <= rel), (err[gate].max(), ref[gate][np.argmax(err[gate])])


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_jd_against_golden(klst, name):
    """The nev eigenvalues nearest sigma at C1 (vs QZ) and C2 (vs dense LU + ARPACK) within 1e-8, with
    explicit residuals <= 1e-10 by the library and by the oracle's own operator."""
    spec, es = getattr(wl, name)()
    ref, kap, _ = read_golden(f"{name}_eigs.txt")
    d = gas.pencil_data(spec.as_dict())
    P = klst.Pencil(spec)
    F = P.factor(es.sigma, precision=klst.FP64)
    om, vec, res, info = F.jd_eigs(es.nev, ncv=min(64, es.nev + 20), kmin=6, tol=1e-11,
                                   v0=to_dev(wl.start_vector(P.n, es.seed)), vectors=True)
    assert info["nconv"] == es.nev and len(om) == es.nev
    _check_against(om, ref, kap, pencil_norm2_est(d, spec.beta))
    assert np.max(res) <= 1e-10
    r = eig.residuals(spec.as_dict(), d, om, to_host(vec).T)
    assert np.max(r) <= 1e-10
    assert np.all(np.diff(np.abs(1.0 / (om - es.sigma))) <= 1e-9 * np.abs(1.0 / (om - es.sigma))[:-1])


def test_jd_matches_krylov_schur_tiny(klst):
    """A tiny pencil: the 8 eigenvalues nearest sigma of the interior problem (oracle) by JD and by
    Krylov-Schur agree."""
    spec = wl.tiny(nx=9, qx=4, qy=3, beta=1.0, mach=3.0)
    d = gas.pencil_data(spec.as_dict())
    A, B = pencil.assemble_dense(spec.as_dict(), d)
    lam, X, kap = eig.interior(A, pencil.boundary_rows(d))
    sigma = 0.2 + 0.1j
    idx = eig.nearest(lam, sigma, 8)
    P = klst.Pencil(spec)
    F = P.factor(sigma, precision=klst.FP64)
    om, _, res, info = F.jd_eigs(8, ncv=24, kmin=4, tol=1e-12, v0=to_dev(wl.start_vector(P.n, 3)))
    _check_against(om, lam[idx], kap[idx], np.linalg.norm(A, "fro"))
    assert np.max(res) <= 1e-10


def test_jd_block_preconditioner(klst):
    """The block-inverse preconditioner (K_k^{-1} alone, without the moment coupling) on a tiny pencil,
    where GMRES can resolve the coupling's low rank (4 Nx = 36): the same eigenvalues as the exact
    Woodbury preconditioner, with more inner iterations.  (At C1 the dropped coupling is as large as
    the diagonal and GMRES(30) within 200 iterations no longer yields useful corrections.)"""
    spec = wl.tiny(nx=9, qx=4, qy=3, beta=1.0, mach=3.0)
    d = gas.pencil_data(spec.as_dict())
    A, B = pencil.assemble_dense(spec.as_dict(), d)
    lam, X, kap = eig.interior(A, pencil.boundary_rows(d))
    sigma = 0.2 + 0.1j
    idx = eig.nearest(lam, sigma, 6)
    P = klst.Pencil(spec)
    F = P.factor(sigma, precision=klst.FP64)
    v0 = to_dev(wl.start_vector(P.n, 5))
    out = {}
    for pc in (klst.JD_PREC_FULL, klst.JD_PREC_BLOCK):
        om, _, res, info = F.jd_eigs(6, ncv=24, kmin=4, tol=1e-12, precond=pc, v0=v0, gmres_m=64, gmres_max=1000,
                                     gmres_rtol=1e-12, gmres_atol=0.0)
        assert info["nconv"] == 6 and np.max(res) <= 1e-10
        _check_against(om, lam[idx], kap[idx], np.linalg.norm(A, "fro"))
        out[pc] = info
    assert out[klst.JD_PREC_BLOCK]["inner"] >= out[klst.JD_PREC_FULL]["inner"]


def test_jd_c3_residual(klst):
    """The full-size C3 pencil (n = 281,088): 10 eigenpairs nearest sigma, every residual checked with
    the oracle's matrix-free float64 operator, eigenvalues equal to the Krylov-Schur ones to 1e-9."""
    spec, es = wl.c3()
    P = klst.Pencil(spec)
    F = P.factor(es.sigma, precision=klst.FP64)
    v0 = to_dev(wl.start_vector(P.n, es.seed))
    om, vec, res, info = F.jd_eigs(10, ncv=30, kmin=6, tol=1e-11, v0=v0, vectors=True)
    assert info["nconv"] == 10 and np.max(res) <= 1e-10
    d = gas.pencil_data(spec.as_dict())
    r = eig.residuals(spec.as_dict(), d, om, to_host(vec).T)
    assert np.max(r) <= 1e-10, np.max(r)
    omk, _, resk, _ = F.eigs(10, 40, tol=1e-12, v0=v0)
    perm = eig.match(omk, om)
    assert np.max(np.abs(om[perm] - omk) / np.abs(omk)) <= 1e-9


def test_jd_invalid_options(klst):
    spec = wl.tiny(nx=9, qx=4, qy=2)
    P = klst.Pencil(spec)
    F = P.factor(0.1j, precision=klst.FP64)
    for kw in ({"ncv": 3}, {"ncv": 65}, {"kmin": 40, "ncv": 40}, {"gmres_m": 0}, {"gmres_m": 65}, {"tol": 0.0},
               {"precond": 7}):
        with pytest.raises(klst.KlstError) as ei:
            F.jd_eigs(4, **kw)
        assert ei.value.code == klst.KLST_EINVAL
    Fm = P.factor(0.1j, precision=klst.MIXED)
    with pytest.raises(klst.KlstError) as ei:
        Fm.jd_eigs(4)
    assert ei.value.code == klst.KLST_EINVAL
