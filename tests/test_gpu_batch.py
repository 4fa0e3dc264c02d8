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


def _pool():
    """Reset/read helpers for the default stream-ordered pool's used-memory high-water mark (bytes
    the library had allocated at once, over what was in use when the mark was reset)."""
    import torch
    from cuda.bindings import runtime as rt
    from cuda.bindings.driver import cuuint64_t as _cuuint64
    err, pool = rt.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())
    assert err == rt.cudaError_t.cudaSuccess
    hi, cur = rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent

    def get(a):
        e, v = rt.cudaMemPoolGetAttribute(pool, a)
        assert e == rt.cudaError_t.cudaSuccess
        return int(v)

    def reset():
        torch.cuda.synchronize()
        (e,) = rt.cudaMemPoolSetAttribute(pool, hi, _cuuint64(0))
        assert e == rt.cudaError_t.cudaSuccess
        return get(cur)

    return reset, lambda: get(hi)


@pytest.mark.parametrize("prec,arith", [(0, 0), (1, 0), (2, 1), (0, 1)], ids=["fp64", "mixed", "df64", "fp64-df64basis"])
def test_admission_footprint_covers_measured_peak(klst, prec, arith):
    """klst_solve_footprint (the server's admission size) is at least the device memory one solve
    actually holds at its peak, measured as the stream-ordered pool's high-water mark."""
    spec, es = wl.c2()
    fp = klst.solve_footprint(spec, es.nev, es.ncv, precision=prec, arith=arith)
    reset, high = _pool()
    base = reset()
    om, res, st, infos = klst.batch_eigs([spec], [es.sigma], es.nev, es.ncv, precision=prec, nworkers=1, tol=1e-11,
                                         conv=klst.CONV_RESID, seed=2, arith=arith)
    assert st[0] == 0
    peak = high() - base
    assert 0 < peak <= fp, (peak, fp)


def test_server_admission_under_memory_pressure(klst):
    """A budget that holds one large request or a few small ones: requests queue, are admitted as
    memory frees up, a later small request may backfill past a waiting large one, and every result
    equals the solve alone."""
    import time
    small = [(wl.tiny(nx=16, qx=6, qy=4, mach=1.5 + 0.1 * i, beta=0.3), 0.1j) for i in range(6)]
    large = (wl.tiny(nx=48, qx=12, qy=8, mach=3.0, beta=0.5), 0.1j)
    f_small = klst.solve_footprint(small[0][0], NEV, NCV)
    f_large = klst.solve_footprint(large[0], NEV, NCV)
    budget = f_large + f_small - 1  # two small requests fit together, the large one only alone
    assert f_large > f_small and 2 * f_small <= budget
    S = klst.Server(hbm_budget_bytes=budget, max_slots=3)
    reqs = small[:2] + [large] + small[2:]
    t0 = time.perf_counter()
    tickets = [S.submit(sp, z, NEV, NCV, tol=1e-11, conv=klst.CONV_RESID, seed=30 + i) for i, (sp, z) in enumerate(reqs)]
    peak_running, peak_bytes = 0, 0
    while True:
        q, r, b = S.stats()
        peak_running, peak_bytes = max(peak_running, r), max(peak_bytes, b)
        assert b <= budget
        if q == 0 and r == 0:
            break
        time.sleep(0.002)
        assert time.perf_counter() - t0 < 300
    out = [S.poll(t, wait=True) for t in tickets]
    for i, (sp, z) in enumerate(reqs):
        om, res, info, lat, code = out[i]
        assert code == 0
        o1, r1 = _alone(klst, sp, z, 0, 30 + i)
        assert np.array_equal(o1, om) and np.array_equal(r1, res), i
    assert peak_bytes <= budget
    S.close()


def test_server_large_request_is_not_starved(klst):
    """Backfill is bounded: one large request submitted among many small ones completes before the
    small requests that arrived after it have all run (it is not passed over indefinitely)."""
    import time
    large = (wl.tiny(nx=48, qx=12, qy=8, mach=3.0, beta=0.5), 0.1j)
    small = wl.tiny(nx=16, qx=6, qy=4, mach=2.0, beta=0.3)
    f_small = klst.solve_footprint(small, NEV, NCV)
    f_large = klst.solve_footprint(large[0], NEV, NCV)
    budget = f_large + f_small - 1  # two small requests fit together, the large one only alone
    assert f_large > f_small and 2 * f_small <= budget
    S = klst.Server(hbm_budget_bytes=budget, max_slots=2)
    sub = {}
    tickets = []
    for i in range(3):
        tickets.append(S.submit(small, 0.1j, NEV, NCV, tol=1e-11, conv=klst.CONV_RESID, seed=i))
        sub[tickets[-1]] = time.perf_counter()
    tl = S.submit(large[0], large[1], NEV, NCV, tol=1e-11, conv=klst.CONV_RESID, seed=99)
    sub[tl] = time.perf_counter()
    for i in range(3, 30):
        tickets.append(S.submit(small, 0.1j, NEV, NCV, tol=1e-11, conv=klst.CONV_RESID, seed=i))
        sub[tickets[-1]] = time.perf_counter()
    done = {}
    for t in tickets + [tl]:
        om, res, info, lat, code = S.poll(t, wait=True)
        assert code == 0
        done[t] = sub[t] + lat / 1e3
    later = [done[t] for t in tickets[3:]]
    assert done[tl] < max(later), "the large request ran after every small request behind it"
    S.close()


def test_server_and_batch_reject_bad_options(klst):
    """Options klst_eigs would reject are rejected at submission, before any worker sizes a buffer."""
    S = klst.Server(hbm_budget_bytes=1 << 30, max_slots=1)
    for kw in (dict(nev=-3, ncv=20), dict(nev=6, ncv=7), dict(nev=6, ncv=400)):
        with pytest.raises(klst.KlstError) as ei:
            S.submit(SMALL[0][0], 0.1j, kw["nev"], kw["ncv"])
        assert ei.value.code == klst.KLST_EINVAL
    with pytest.raises(klst.KlstError):
        S.submit(SMALL[0][0], 0.1j, NEV, NCV, precision=7)
    S.close()
    with pytest.raises(klst.KlstError) as ei:
        klst.batch_eigs([SMALL[0][0]], [0.1j], 6, 6, precision=0)
    assert ei.value.code == klst.KLST_EINVAL and "invalid eigs options" in str(ei.value)


_FRESH_BATCH = r"""
import sys
sys.path.insert(0, sys.argv[1])
from paper_2607_27440_b300 import klst, workloads as wl
klst.load()
specs = [wl.tiny(nx=128, qx=4 + (i % 3), qy=2, mach=1.2 + 0.3 * i) for i in range(8)]
sig = [0.05 + 0.2j + 0.01j * i for i in range(8)]
om, res, st, infos = klst.batch_eigs(specs, sig, 4, 12, precision=klst.FP64, nworkers=8, tol=1e-10)
print(list(st))
sys.exit(0 if all(s == 0 for s in st) else 1)
"""


def test_first_use_in_concurrent_workers_is_safe():
    """A fresh process whose first GPU work is eight Nx = 128 pencils on eight worker threads: the
    kernels that need more than 48 KB of shared memory get their attribute set before any thread
    launches them (a set-once flag that a second thread could pass before the first thread had set
    the attribute made such launches fail with KLST_ECUDA)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", _FRESH_BATCH, root], capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, (r.stdout, r.stderr[-2000:])
