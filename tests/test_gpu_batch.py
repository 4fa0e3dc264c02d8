"""Batched sweeps (klst_batch_eigs) and the serving loop (klst_server_*): every pencil's result in the
batch or in the request mix equals its result alone, bit for bit, and matches the oracle."""
import numpy as np
import pytest

from oracle import eig, gas, pencil
from paper_2607_27440_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def klst():
    from paper_2607_27440_b300 import klst as k
    k.load()
    return k


SMALL = [
    (wl.tiny(nx=16, qx=6, qy=4, mach=1.5, beta=0.3), 0.10j),
    (wl.tiny(nx=24, qx=8, qy=6, mach=2.7, beta=1.1), 0.15j),
    (wl.tiny(nx=16, qx=8, qy=6, mach=3.9, beta=1.8), 0.12j),
    (wl.tiny(nx=20, qx=6, qy=4, mach=2.0, beta=0.0), 0.20j),
    (wl.tiny(nx=24, qx=6, qy=4, mach=1.2, base="tanh", noneq=0, width=0.4), 0.10j),
    (wl.tiny(nx=32, qx=6, qy=4, mach=3.0, beta=0.7), 0.18j),
]
NEV, NCV = 6, 20


def _alone(klst, spec, sigma, prec, seed, arith=0):
    P = klst.Pencil(spec)
    F = P.factor(sigma, precision=prec)
    om, _, res, info = F.eigs(NEV, NCV, tol=1e-11, conv=klst.CONV_RESID, seed=seed, arith=arith)
    return om, res


@pytest.mark.parametrize("prec,arith", [(0, 0), (1, 0), (2, 1)], ids=["fp64", "mixed", "df64"])
def test_batch_equals_alone_and_oracle(klst, prec, arith):
    specs = [s for s, _ in SMALL]
    sig = [z for _, z in SMALL]
    om, res, st, infos = klst.batch_eigs(specs, sig, NEV, NCV, precision=prec, nworkers=4, tol=1e-11,
                                         conv=klst.CONV_RESID, seed=100, arith=arith)
    assert np.all(st == 0), st
    for i, (spec, z) in enumerate(SMALL):
        o1, r1 = _alone(klst, spec, z, prec, 100 + i, arith)
        assert np.array_equal(o1, om[i]) and np.array_equal(r1, res[i]), i
        assert np.max(res[i]) <= 1e-10
    for i in (0, 3, 5):
        spec, z = SMALL[i]
        d = gas.pencil_data(spec.as_dict())
        A, B = pencil.assemble_dense(spec.as_dict(), d)
        lam, _, kap = eig.interior(A, pencil.boundary_rows(d))
        ref = lam[eig.nearest(lam, z, NEV)]
        perm = eig.match(ref, om[i])
        assert np.max(np.abs(om[i][perm] - ref) / np.abs(ref)) <= 1e-8


def test_server_results_equal_alone(klst):
    S = klst.Server(hbm_budget_bytes=8 << 30, max_slots=3)
    tickets = []
    for i, (spec, z) in enumerate(SMALL):
        tickets.append(S.submit(spec, z, NEV, NCV, precision=klst.MIXED if i % 2 else klst.FP64, tol=1e-11,
                                conv=klst.CONV_RESID, seed=7 + i))
    out = [S.poll(t, wait=True) for t in tickets]
    for i, (spec, z) in enumerate(SMALL):
        om, res, info, lat, code = out[i]
        assert code == 0 and lat > 0
        o1, r1 = _alone(klst, spec, z, klst.MIXED if i % 2 else klst.FP64, 7 + i)
        assert np.array_equal(o1, om) and np.array_equal(r1, res), i
    assert S.stats() == (0, 0, 0)
    S.close()


def test_server_rejects_request_beyond_budget(klst):
    S = klst.Server(hbm_budget_bytes=32 << 20, max_slots=1)
    with pytest.raises(klst.KlstError) as ei:
        S.submit(wl.c2()[0], 0.1j, 40, 80)
    assert ei.value.code == klst.KLST_ENOMEM
    S.close()


def test_sweep_shapes_in_one_batch(klst):
    """A slice of the Mach/beta/Nx/Nxi sweep: all pencils converge with residual <= 1e-10."""
    sweep = wl.sweep(npencils=8, seed=4)
    specs = [s for s, _ in sweep]
    sig = [z for _, z in sweep]
    om, res, st, infos = klst.batch_eigs(specs, sig, 20, 40, precision=klst.MIXED, tol=2e-11, conv=klst.CONV_RESID,
                                         seed=4)
    assert np.all(st == 0), st
    assert np.max(res) <= 1e-10
