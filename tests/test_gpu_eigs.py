"""GPU Krylov-Schur shift-invert eigensolve vs the oracle (QZ / interior problem / dense LU + ARPACK)."""
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
    return err


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_tiny_all_nearest(klst, prec):
    spec = wl.tiny(nx=9, qx=4, qy=3, beta=1.0, mach=3.0)
    d = gas.pencil_data(spec.as_dict())
    A, B = pencil.assemble_dense(spec.as_dict(), d)
    lam, X, kap = eig.interior(A, pencil.boundary_rows(d))
    sigma = 0.2 + 0.1j
    idx = eig.nearest(lam, sigma, 10)
    P = klst.Pencil(spec)
    F = P.factor(sigma, precision=prec)
    om, vec, res, info = F.eigs(10, 30, tol=1e-13, v0=to_dev(wl.start_vector(P.n, 1)), vectors=True)
    _check_against(om, lam[idx], kap[idx], np.linalg.norm(A, "fro"))
    assert np.max(res) <= 1e-10
    V = to_host(vec)
    r = eig.residuals(spec.as_dict(), d, om, V.T)
    assert np.max(r) <= 1e-10
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0)


@pytest.mark.parametrize("prec,arith", [(0, 0), (1, 0), (0, 1), (1, 1), (2, 1)],
                         ids=["fp64", "mixed", "fp64-df64basis", "mixed-df64", "df64"])
def test_c1_against_golden(klst, prec, arith):
    spec, es = wl.c1()
    ref, kap, _ = read_golden("c1_eigs.txt")
    d = gas.pencil_data(spec.as_dict())
    A, B = pencil.assemble_dense(spec.as_dict(), d)
    P = klst.Pencil(spec)
    F = P.factor(es.sigma, precision=prec)
    om, vec, res, info = F.eigs(es.nev, es.ncv, tol=1e-13, v0=to_dev(wl.start_vector(P.n, es.seed)), vectors=True,
                                arith=arith)
    _check_against(om, ref, kap, pencil_norm2_est(d, spec.beta))
    assert np.max(res) <= 1e-10
    r = eig.residuals(spec.as_dict(), d, om, to_host(vec).T)
    assert np.max(r) <= 1e-10
    # nearest-first ordering
    assert np.all(np.diff(np.abs(om - es.sigma)) >= -1e-12)


@pytest.mark.parametrize("prec,arith", [(0, 0), (1, 0), (1, 1), (2, 1)], ids=["fp64", "mixed", "mixed-df64", "df64"])
def test_c2_against_golden(klst, prec, arith):
    spec, es = wl.c2()
    ref, kap, _ = read_golden("c2_eigs.txt")
    d = gas.pencil_data(spec.as_dict())
    normA = pencil_norm2_est(d, spec.beta)
    P = klst.Pencil(spec)
    F = P.factor(es.sigma, precision=prec)
    om, vec, res, info = F.eigs(es.nev, es.ncv, tol=1e-13, v0=to_dev(wl.start_vector(P.n, es.seed)), vectors=True,
                                arith=arith)
    _check_against(om, ref, kap, normA)
    assert np.max(res) <= 1e-10
    r = eig.residuals(spec.as_dict(), d, om, to_host(vec).T)
    assert np.max(r) <= 1e-10


def test_no_restarts_reports_noconv(klst):
    """max_restarts = 0 with a tight tolerance and a basis barely larger than nev -> KLST_ENOCONV."""
    spec, es = wl.c1()
    P = klst.Pencil(spec)
    F = P.factor(es.sigma)
    om, vec, res, info = F.eigs(20, 22, tol=1e-14, max_restarts=0, check=False)
    assert info["status"] == klst.KLST_ENOCONV
    assert info["nconv"] < 20


def test_invalid_options_rejected(klst):
    spec, es = wl.c1()
    P = klst.Pencil(spec)
    F = P.factor(es.sigma)
    with pytest.raises(klst.KlstError) as ei:
        F.eigs(20, 21)
    assert ei.value.code == klst.KLST_EINVAL
