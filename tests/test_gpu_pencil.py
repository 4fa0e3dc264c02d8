"""GPU pencil assembly vs the oracle, entry by entry (Sec. 2.2, 3.1, 3.2; Eqs. comp_ghat1Dshock/comp_hhat1Dshock)."""
import numpy as np
import pytest

from oracle import gas, pencil
from paper_2607_27440_b300 import workloads as wl
from tests.helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

SPECS = [
    wl.tiny(nx=9, qx=4, qy=2, mach=3.0),
    wl.tiny(nx=7, qx=5, qy=3, mach=4.0, beta=0.7),
    wl.tiny(nx=12, qx=6, qy=4, mach=1.2, base="tanh", noneq=0, width=0.4),
    wl.tiny(nx=10, qx=7, qy=5, mach=2.2, conservative=0, beta=1.9),
    wl.tiny(nx=33, qx=9, qy=6, mach=3.5, noneq=0),
    wl.c1()[0],
]


@pytest.fixture(scope="module")
def klst():
    from paper_2607_27440_b300 import klst as k
    k.load()
    return k


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: f"nx{s.nx}q{s.qx}x{s.qy}M{s.mach}")
def test_tables_match_oracle(klst, spec):
    d = gas.pencil_data(spec.as_dict())
    P = klst.Pencil(spec)
    t = P.tables()
    assert np.max(np.abs(t["x"] - d["x"])) <= 1e-13 * np.max(np.abs(d["x"]))
    assert np.max(np.abs(t["Dx"] - d["Dx"])) <= 1e-13 * np.max(np.abs(d["Dx"]))
    assert np.max(np.abs(t["xi_x"] - d["xi_x"])) <= 1e-13 * max(1, np.max(np.abs(d["xi_x"])))
    assert np.max(np.abs(t["xi_y"] - d["xi_y"])) <= 1e-13 * max(1, np.max(np.abs(d["xi_y"])))
    assert np.allclose(t["W"], d["W"], rtol=1e-12, atol=0)
    assert np.allclose(t["nu"], d["nu"], rtol=1e-12, atol=0)
    G = np.transpose(t["G"], (1, 2, 3, 0))  # (c, a, j, k)
    w = np.transpose(t["w"], (1, 2, 3, 0))
    assert np.max(np.abs(G - d["G"])) <= 1e-10 * np.max(np.abs(d["G"]))
    assert np.max(np.abs(w - d["w"])) <= 1e-12 * np.max(np.abs(d["w"]))
    assert np.array_equal(t["bc"].astype(bool), d["bc"])


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: f"nx{s.nx}q{s.qx}x{s.qy}M{s.mach}")
def test_dense_export_is_oracle_pencil(klst, spec):
    """K - U V^H exported from the device equals the oracle's A - sigma B entry by entry."""
    sigma = 0.05 + 0.2j
    d = gas.pencil_data(spec.as_dict())
    A, B = pencil.assemble_dense(spec.as_dict(), d)
    P = klst.Pencil(spec)
    Ag, Bg = P.export_dense(sigma)
    ref = A - sigma * B
    assert np.array_equal(Bg, np.diag(B).real)
    assert np.max(np.abs(Ag - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert np.array_equal(Ag != 0, ref != 0)


@pytest.mark.parametrize("spec", SPECS[:4] + [wl.c2()[0]], ids=lambda s: f"nx{s.nx}q{s.qx}x{s.qy}")
def test_apply_pencil_matches_oracle(klst, spec):
    """Matrix-free float64 (A - omega B) x on the device vs the oracle's matrix-free rows."""
    d = gas.pencil_data(spec.as_dict())
    P = klst.Pencil(spec)
    X = wl.random_vectors(P.n, 3, 5)
    om = np.array([0.0, 0.3 - 0.1j, -1.0 + 2.0j])
    Y = to_host(P.apply(to_dev(X), omega=om))
    ref = (pencil.apply_A(spec.as_dict(), d, X.T) - pencil.apply_B(d, X.T) * om[None, :]).T
    err = np.max(np.abs(Y - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert np.all(err < 1e-12), err
