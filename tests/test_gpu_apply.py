"""GPU shift-and-invert apply (Eq. parShiftInvert, Woodbury form) vs the oracle's dense LU solve."""
import numpy as np
import pytest

from oracle import eig, gas, pencil
from paper_2607_27440_b300 import workloads as wl
from tests.helpers import cond1, to_dev, to_host

pytestmark = pytest.mark.gpu

SMALL = [
    (wl.tiny(nx=9, qx=4, qy=2, mach=3.0), 0.1j),
    (wl.tiny(nx=7, qx=5, qy=3, mach=4.0, beta=0.7), 0.3 + 0.05j),
    (wl.tiny(nx=33, qx=9, qy=6, mach=3.5), 0.05 + 0.2j),
    (wl.c1()[0], 0.1j),
    (wl.tiny(nx=48, qx=10, qy=6, mach=2.5, beta=1.4), 0.1j),
]


@pytest.fixture(scope="module")
def klst():
    from paper_2607_27440_b300 import klst as k
    k.load()
    return k


def _oracle(spec, sigma):
    d = gas.pencil_data(spec.as_dict())
    A, B = pencil.assemble_dense(spec.as_dict(), d)
    return d, A, B, eig.ShiftInvert(A, B, sigma)


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp64", "mixed", "df64"])
@pytest.mark.parametrize("spec,sigma", SMALL, ids=lambda v: str(v)[:40])
def test_apply_matches_dense_lu(klst, spec, sigma, prec):
    """||y_gpu - y_oracle|| / ||y_oracle|| <= max(1e-12, 64 cond(A - sigma B) eps) on three seeded vectors."""
    d, A, B, si = _oracle(spec, sigma)
    X = wl.random_vectors(A.shape[0], 3, 17)
    ref = np.stack([si.apply(x) for x in X])
    cond = cond1(A - sigma * B, si.lu)
    tol = max(1e-12, 64 * cond * 2.220446049250313e-16)
    P = klst.Pencil(spec)
    F = P.factor(sigma, precision=prec)
    if prec == 1:
        F.set_refine(6, 1e-15)
    Y = to_host(F.apply(to_dev(X)))
    err = np.linalg.norm(Y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= tol), (err, tol, cond)
    # inflow rows of T x vanish (range of T excludes the B-null space)
    br = pencil.boundary_rows(d)
    assert np.max(np.abs(Y[:, br])) <= tol * np.max(np.abs(Y))


def test_multi_rhs_equals_single(klst):
    spec, sigma = SMALL[2]
    P = klst.Pencil(spec)
    F = P.factor(sigma)
    X = to_dev(wl.random_vectors(P.n, 4, 3))
    Y = to_host(F.apply(X))
    for i in range(4):
        yi = to_host(F.apply(X[i]))
        assert np.array_equal(yi, Y[i])


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp64", "mixed", "df64"])
@pytest.mark.parametrize("which", ["c2", "c3"])
def test_apply_full_size_residual(klst, which, prec):
    """Full workload sizes: the oracle's matrix-free rows give ||(A - sigma B) y - B x|| / ||B x||."""
    spec, es = getattr(wl, which)()
    d = gas.pencil_data(spec.as_dict())
    P = klst.Pencil(spec)
    F = P.factor(es.sigma, precision=prec)
    x = wl.start_vector(P.n, 21)
    y = to_host(F.apply(to_dev(x)))
    r = pencil.apply_A(spec.as_dict(), d, y) - es.sigma * pencil.apply_B(d, y) - pencil.apply_B(d, x)
    rel = np.linalg.norm(r) / np.linalg.norm(pencil.apply_B(d, x))
    # backward error of a float64 solve: O(eps * ||A - sigma B|| * ||y|| / ||B x||)
    normA = np.abs(d["Dx"]).sum(axis=1).max() * np.abs(d["xi_x"]).max() + np.abs(d["nu"]).max() + abs(es.sigma)
    bound = 1e3 * 2.220446049250313e-16 * normA * np.linalg.norm(y) / np.linalg.norm(pencil.apply_B(d, x))
    assert rel <= max(bound, 1e-12), (rel, bound)


def test_exactly_singular_block_is_reported(klst):
    """beta = 0 and odd qx: the xi_x = 0 block is diag(nu - sigma); sigma = nu_j makes it exactly singular."""
    spec = wl.tiny(nx=8, qx=5, qy=2, beta=0.0)
    P = klst.Pencil(spec)
    nu = P.tables()["nu"]
    with pytest.raises(klst.KlstError) as ei:
        P.factor(complex(nu[3], 0.0))
    assert ei.value.code == klst.KLST_ESINGULAR


@pytest.mark.parametrize("nx", [32, 64, 96, 128], ids=["r128", "r256", "r384", "r512"])
def test_capacitance_inverse_cluster_coop_and_per_pivot_agree(klst, nx, monkeypatch):
    """C^{-1} by one thread-block-cluster launch (8 CTAs up to r = 256, 16 at r = 384; r = 512 does
    not fit), by one cooperative launch with grid barriers between the pivots (KLST_NO_CLUSTER_GJ=1)
    and by one launch per pivot (also KLST_NO_COOP_GJ=1) follow the same operations: the applies
    agree bit for bit, and the per-pivot factorisation launches about r more kernels."""
    spec = wl.tiny(nx=nx, qx=6, qy=4, mach=3.0, beta=0.5) if nx < 128 else wl.tiny(nx=nx, qx=4, qy=2, mach=3.0, beta=0.5)
    x = to_dev(wl.start_vector(spec.n, 7))
    P = klst.Pencil(spec)
    lib = klst.load()
    ys, counts = [], []
    for env in ({}, {"KLST_NO_CLUSTER_GJ": "1"}, {"KLST_NO_CLUSTER_GJ": "1", "KLST_NO_COOP_GJ": "1"}):
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        c0 = lib.klst_launch_count()
        ys.append(to_host(P.factor(0.1j, precision=0).apply(x)))
        counts.append(lib.klst_launch_count() - c0)
    r = 4 * nx
    assert counts[2] - counts[1] >= r - 2 and counts[2] - counts[0] >= r - 2, counts
    assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])


def test_refinement_shortfall_reports_erefine(klst):
    """MIXED factors: an apply whose refinement cannot reach refine_tol within max_refine sweeps raises
    the factor's flag; klst_factor_check reports KLST_EREFINE once and clears it, and klst_eigs returns
    KLST_EREFINE with every output filled.  A reachable tolerance reports KLST_OK."""
    spec, sigma = SMALL[2]
    P = klst.Pencil(spec)
    F = P.factor(sigma, precision=klst.MIXED)
    X = to_dev(wl.random_vectors(P.n, 2, 5))
    F.set_refine(6, 1e-11)
    F.apply(X)
    assert F.check() == klst.KLST_OK
    F.set_refine(1, 1e-30)  # unreachable: one sweep cannot bring ||r|| / ||B x|| to 1e-30
    Y = to_host(F.apply(X))
    assert np.all(np.isfinite(Y))
    assert F.check() == klst.KLST_EREFINE
    assert F.check() == klst.KLST_OK  # the flag was cleared
    om, vec, res, info = F.eigs(6, 20, tol=1e-8, max_refine=2, refine_tol=1e-30, seed=3, check=False)
    assert info["status"] == klst.KLST_EREFINE
    assert info["nconv"] == 6 and np.all(np.isfinite(om)) and np.all(np.isfinite(res))
    assert info["max_refine_resid"] > 1e-30


def _pool_used():
    import torch
    from cuda.bindings import runtime as rt
    torch.cuda.synchronize()
    err, pool = rt.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())
    e, v = rt.cudaMemPoolGetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent)
    return int(v)


def test_injected_allocation_failure_returns_enomem(klst):
    """Host-injected device allocation failure at every allocation of build + factor + eigs in turn:
    each failing call returns KLST_ENOMEM with no handle, frees what it had taken (the pool's in-use
    bytes return to the baseline), and the next full solve gives the same eigenvalues as before."""
    spec, sigma = wl.tiny(nx=12, qx=6, qy=4, mach=3.0, beta=0.5), 0.1j
    for prec in (klst.FP64, klst.MIXED):
        ref = klst.Pencil(spec).factor(sigma, precision=prec).eigs(6, 20, tol=1e-11, seed=9)[0]
        base = _pool_used()
        ok_at = None
        for n in range(200):
            klst.fail_alloc_after(n)
            try:
                P = klst.Pencil(spec)
                F = P.factor(sigma, precision=prec)
                om = F.eigs(6, 20, tol=1e-11, seed=9)[0]
            except klst.KlstError as e:
                assert e.code == klst.KLST_ENOMEM, (n, e)
                assert "out of memory" in str(e) or "cudaMalloc" in str(e), str(e)
                continue
            finally:
                klst.fail_alloc_after(-1)
                import gc
                gc.collect()
            ok_at = n
            assert np.array_equal(om, ref)
            del F, P
            break
        assert ok_at is not None and ok_at >= 10, ok_at  # the solve makes at least ten allocations
        import gc
        gc.collect()
        assert _pool_used() == base


# Nx = 128 with a small velocity grid: the full-size tile path (the block Gauss-Jordan of a 128 x 128
# block leaves shared memory and works in global memory, and r = 4 Nx = 512 takes the per-pivot
# capacitance inverse) at sizes the dense oracle still factors in seconds.
NX128 = [
    (wl.tiny(nx=128, qx=4, qy=2, mach=3.0, beta=1.0), 0.05 + 0.2j),
    (wl.tiny(nx=128, qx=6, qy=4, mach=4.0, beta=0.6), 0.1j),
]


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp64", "mixed", "df64"])
@pytest.mark.parametrize("spec,sigma", NX128, ids=["128x4x2", "128x6x4"])
def test_apply_nx128_matches_dense_lu(klst, spec, sigma, prec):
    """Element by element against the oracle's dense LU solve of A - sigma B at Nx = 128."""
    d, A, B, si = _oracle(spec, sigma)
    X = wl.random_vectors(A.shape[0], 2, 23)
    ref = np.stack([si.apply(x) for x in X])
    cond = cond1(A - sigma * B, si.lu)
    tol = max(1e-12, 64 * cond * 2.220446049250313e-16)
    P = klst.Pencil(spec)
    F = P.factor(sigma, precision=prec)
    if prec == 1:
        F.set_refine(6, 1e-15)
    Y = to_host(F.apply(to_dev(X)))
    err = np.abs(Y - ref).max(axis=1) / np.abs(ref).max(axis=1)
    assert np.all(err <= tol), (err, tol, cond)


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp64", "mixed", "df64"])
def test_apply_c3_paper_shape_residual(klst, prec):
    """The paper's own 281,088-unknown shape (Nx = 61, 48 x 48): the oracle's matrix-free rows give
    ||(A - sigma B) y - B x|| / ||B x|| at the float64 level."""
    spec, es = wl.c3_paper_shape()
    d = gas.pencil_data(spec.as_dict())
    P = klst.Pencil(spec)
    F = P.factor(es.sigma, precision=prec)
    x = wl.start_vector(P.n, 22)
    y = to_host(F.apply(to_dev(x)))
    r = pencil.apply_A(spec.as_dict(), d, y) - es.sigma * pencil.apply_B(d, y) - pencil.apply_B(d, x)
    rel = np.linalg.norm(r) / np.linalg.norm(pencil.apply_B(d, x))
    normA = np.abs(d["Dx"]).sum(axis=1).max() * np.abs(d["xi_x"]).max() + np.abs(d["nu"]).max() + abs(es.sigma)
    bound = 1e3 * 2.220446049250313e-16 * normA * np.linalg.norm(y) / np.linalg.norm(pencil.apply_B(d, x))
    assert rel <= max(bound, 1e-12), (rel, bound)


@pytest.mark.parametrize("spec,sigma", [SMALL[2], NX128[1]], ids=["33x9x6", "128x6x4"])
def test_mixed_residual_tensor_core_matches_cuda_core(klst, spec, sigma, monkeypatch):
    """The MIXED refinement residual with its D_x products on the tensor cores (default) and on the
    float64 CUDA cores (KLST_NO_TC=1) refine to the same solution at float64 level."""
    X = to_dev(wl.random_vectors(spec.n, 2, 31))
    P = klst.Pencil(spec)
    out = []
    for env in ("0", "1"):
        monkeypatch.setenv("KLST_NO_TC", env)
        F = P.factor(sigma, precision=klst.MIXED)
        F.set_refine(6, 1e-15)
        out.append(to_host(F.apply(X)))
    err = np.abs(out[0] - out[1]).max(axis=1) / np.abs(out[1]).max(axis=1)
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("spec,sigma", [SMALL[0], SMALL[2], SMALL[4], NX128[1]], ids=["9x4x2", "33x9x6", "48x10x6", "128x6x4"])
def test_fp64_tensor_core_solve_matches_cuda_core(klst, spec, sigma, monkeypatch):
    """The float64 block solves on the tensor cores (integer slices of K_k^{-1}, the default) and as
    complex128 products on the float64 pipe (KLST_NO_TC=1) give the same T x at float64 level, on
    ragged Nx (9, 33) and full 128-row tiles, with 1, 2 and 3 right-hand sides (odd counts leave
    a CTA's second slot empty)."""
    P = klst.Pencil(spec)
    for nrhs in (1, 2, 3):
        X = to_dev(wl.random_vectors(spec.n, nrhs, 41 + nrhs))
        out = []
        for env in ("0", "1"):
            monkeypatch.setenv("KLST_NO_TC", env)
            F = P.factor(sigma, precision=klst.FP64)
            klst.prof_reset()
            klst.prof_enable(True)
            out.append(to_host(F.apply(X)))
            klst.prof_enable(False)
            groups = klst.prof_read()
            assert ("solve_pass1_tc" in groups) == (env == "0"), sorted(groups)
        err = np.abs(out[0] - out[1]).max(axis=-1) / np.abs(out[1]).max(axis=-1)
        assert np.all(err <= 1e-12), (nrhs, err)
