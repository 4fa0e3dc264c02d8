"""Block inverses K_k^{-1} of the shifted factorisation (Eq. parLUfactor for the blocks K_k) formed by a
complex float32 Gauss-Jordan inverse and float64-accurate Newton-Schulz steps on the tensor cores."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import eig, gas, pencil
from paper_2607_27440_b300 import workloads as wl
from tests.helpers import cond1, to_dev, to_host

pytestmark = pytest.mark.gpu

CASES = [
    (wl.tiny(nx=9, qx=4, qy=2, mach=3.0), 0.1j),
    (wl.tiny(nx=33, qx=9, qy=6, mach=3.5), 0.05 + 0.2j),
    (wl.tiny(nx=61, qx=5, qy=4, mach=4.0), 0.05 + 0.2j),
    (wl.tiny(nx=128, qx=6, qy=4, mach=4.0, beta=0.6), 0.1j),
]


@pytest.fixture(scope="module")
def klst():
    from paper_2607_27440_b300 import klst as k
    k.load()
    return k


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp64", "mixed", "df64"])
@pytest.mark.parametrize("spec,sigma", CASES, ids=["9x4x2", "33x9x6", "61x5x4", "128x6x4"])
def test_newton_schulz_inverse_is_used_and_converges(klst, spec, sigma, prec):
    """Every precision forms K_k^{-1} on the tensor cores for Nx <= 128: two steps, no fallback, and the
    residual before the last step small enough that the one after it is at the float64 level."""
    P = klst.Pencil(spec)
    klst.prof_reset()
    klst.prof_enable(True)
    F = P.factor(sigma, precision=prec)
    klst.prof_enable(False)
    groups = klst.prof_read()
    info = F.inverse_info()
    assert info["method"] == 1 and info["fallback"] == 0, info
    assert info["steps"] == 2, info
    assert info["resid"] * spec.nx <= 1e-6, info
    for g in ("factor_gj32", "factor_ns_resid", "factor_ns_update"):
        assert g in groups, sorted(groups)
    assert "factor_gj64" not in groups


@pytest.mark.parametrize("spec,sigma", CASES, ids=["9x4x2", "33x9x6", "61x5x4", "128x6x4"])
def test_newton_schulz_apply_matches_gauss_jordan(klst, spec, sigma, monkeypatch):
    """T x from the tensor-core inverses against the float64 Gauss-Jordan inverses (KLST_NO_TC=1),
    element by element at float64 level, and both against the oracle's dense LU solve."""
    X = wl.random_vectors(spec.n, 2, 53)
    d = gas.pencil_data(spec.as_dict())
    A, B = pencil.assemble_dense(spec.as_dict(), d)
    si = eig.ShiftInvert(A, B, sigma)
    ref = np.stack([si.apply(x) for x in X])
    tol = max(1e-12, 64 * cond1(A - sigma * B, si.lu) * 2.220446049250313e-16)
    P = klst.Pencil(spec)
    out = []
    for env in ("0", "1"):
        monkeypatch.setenv("KLST_NO_TC", env)
        F = P.factor(sigma, precision=klst.FP64)
        assert F.inverse_info()["method"] == (1 if env == "0" else 0)
        out.append(to_host(F.apply(to_dev(X))))
    scale = np.abs(ref).max(axis=1)
    assert np.all(np.abs(out[0] - out[1]).max(axis=1) / scale <= tol)
    assert np.all(np.abs(out[0] - ref).max(axis=1) / scale <= tol)


def test_block_ranges_do_not_change_the_result(klst, monkeypatch):
    """Blocks are independent: processing 54 blocks in ranges of 7 (a ragged last range of 5) gives
    bit-identical inverses, hence bit-identical T x."""
    spec, sigma = CASES[1]
    X = to_dev(wl.random_vectors(spec.n, 2, 59))
    P = klst.Pencil(spec)
    out = []
    for rng in ("", "7"):
        if rng:
            monkeypatch.setenv("KLST_NS_RANGE", rng)
        else:
            monkeypatch.delenv("KLST_NS_RANGE", raising=False)
        F = P.factor(sigma, precision=klst.FP64)
        assert F.inverse_info()["method"] == 1
        out.append(to_host(F.apply(X)))
    assert np.array_equal(out[0], out[1])


def _near_singular_block_shift(spec):
    """A shift 1e-6 (relative) from a finite eigenvalue of the block pencil (K_0(0), E_0), E_0 = I with
    the inflow rows zeroed: K_0(sigma) then has condition number ~1e8, beyond the float32 start."""
    d = gas.pencil_data(spec.as_dict())
    beta = gas._p(spec.as_dict(), "beta")
    nx, k = spec.nx, 0
    K = d["xi_x"][k] * d["Dx"] + np.diag(d["nu"] + 1j * beta * d["xi_y"][k])
    E = np.eye(nx)
    for j in range(nx):
        if d["bc"][j, k]:
            K[j, :] = 0.0
            K[j, j] = 1.0
            E[j, j] = 0.0
    w = sla.eig(K, E, right=False)
    w = w[np.isfinite(w)]
    return complex(w[np.argmin(np.abs(w))] * (1 + 1e-6)), d


def test_ill_conditioned_block_falls_back_to_float64_gauss_jordan(klst, monkeypatch):
    """A block whose float32 inverse is too poor for Newton-Schulz (max |I - K X_0| Nx >= 1/2) is
    inverted by float64 Gauss-Jordan instead: T x then has the backward error of the all-float64
    factorisation (KLST_NO_TC=1) on this ill-conditioned shift, within a factor of 10."""
    spec = wl.tiny(nx=16, qx=4, qy=2, mach=3.0, beta=0.5)
    sigma, d = _near_singular_block_shift(spec)
    A, B = pencil.assemble_dense(spec.as_dict(), d)
    M = A - sigma * B
    X = wl.random_vectors(spec.n, 1, 61)
    P = klst.Pencil(spec)
    monkeypatch.setenv("KLST_NS_RANGE", "1")
    back = []
    for env in ("0", "1"):
        monkeypatch.setenv("KLST_NO_TC", env)
        F = P.factor(sigma, precision=klst.FP64)
        info = F.inverse_info()
        if env == "0":
            assert info["method"] == 1 and 1 <= info["fallback"] < spec.nxi, info
        y = to_host(F.apply(to_dev(X)))[0]
        r = M @ y - B @ X[0]
        back.append(np.linalg.norm(r) / (np.linalg.norm(M, 1) * np.linalg.norm(y) + np.linalg.norm(B @ X[0])))
    assert back[0] <= 10 * back[1] + 1e-14, back
