"""klst_apply_pencil_noalloc (fixed device scratch, no allocation) against klst_apply_pencil.

Callers that cannot allocate device memory when they apply the operator (a host framework with
its own memory pool that forbids library allocations in its steady-state loop, a latency-critical
serving loop, code that must not hit out-of-memory mid-solve) use the no-allocation variant; it must
give the same result as the allocating entry point.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2607_27440_b300 import workloads as wl
from tests.helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def klst():
    from paper_2607_27440_b300 import klst as k
    k.load()
    return k


def _close(a, b):
    err = np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)
    assert np.all(err < 1e-12), err


def test_noalloc_matches_allocating_operator_twice(klst):
    spec = wl.c2()[0]
    P = klst.Pencil(spec)
    X = to_dev(wl.random_vectors(P.n, 3, 41))
    om = np.array([0.1j, 0.3 - 0.2j, -1.0 + 0.5j])
    ref1 = to_host(P.apply(X, omega=om))
    out = X.new_empty(X.shape)
    got1 = to_host(P.apply_noalloc(X, omega=om, out=out))
    _close(got1, ref1)
    # second call in a row: different right-hand sides, no shifts
    X2 = to_dev(wl.random_vectors(P.n, 2, 42))
    ref2 = to_host(P.apply(X2))
    got2 = to_host(P.apply_noalloc(X2))
    _close(got2, ref2)


def _pool_high_minus_current():
    """(high-water mark - current use) of the device's default stream-ordered pool, after resetting
    the mark: a call that allocated (and freed) pool memory in between leaves a positive value."""
    import torch
    from cuda.bindings import runtime as rt
    from cuda.bindings.driver import cuuint64_t as _cuuint64
    dev = torch.cuda.current_device()
    err, pool = rt.cudaDeviceGetDefaultMemPool(dev)
    assert err == rt.cudaError_t.cudaSuccess
    attr_hi = rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh
    attr_cur = rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent

    def reset():
        torch.cuda.synchronize()
        (e,) = rt.cudaMemPoolSetAttribute(pool, attr_hi, _cuuint64(0))
        assert e == rt.cudaError_t.cudaSuccess

    def read():
        torch.cuda.synchronize()
        e1, hi = rt.cudaMemPoolGetAttribute(pool, attr_hi)
        e2, cur = rt.cudaMemPoolGetAttribute(pool, attr_cur)
        assert e1 == rt.cudaError_t.cudaSuccess and e2 == rt.cudaError_t.cudaSuccess
        return int(hi) - int(cur)

    return reset, read


def test_noalloc_allocates_nothing(klst):
    """The defining property: after a warm-up call, a call with a caller-owned output raises neither
    the stream-ordered pool's high-water mark nor PyTorch's allocation count.  The allocating
    operator, run the same way, does raise the mark (the check can see an allocation)."""
    import torch
    spec = wl.c2()[0]
    P = klst.Pencil(spec)
    X = to_dev(wl.random_vectors(P.n, 2, 44))
    out = X.new_empty(X.shape)
    om = np.array([0.2j, -0.1 + 0.3j])
    P.apply_noalloc(X, omega=om, out=out)  # warm-up: resolves the scratch address once per device
    reset, read = _pool_high_minus_current()
    reset()
    P.apply(X, omega=om)
    assert read() > 0
    reset()
    n_alloc = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    P.apply_noalloc(X, omega=om, out=out)
    P.apply_noalloc(X, out=out)
    assert read() == 0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == n_alloc


def test_noalloc_checks_the_output_buffer(klst):
    import torch
    spec = wl.c1()[0]
    P = klst.Pencil(spec)
    X = to_dev(wl.random_vectors(P.n, 2, 45))
    for bad in (X.new_empty((1, P.n)), torch.empty(X.shape, dtype=torch.complex64, device="cuda"),
                X.new_empty((P.n, 2)).t(), X):
        with pytest.raises(ValueError):
            P.apply_noalloc(X, out=bad)


def test_noalloc_rejects_work_beyond_the_fixed_array(klst):
    lib = klst.load()
    cap = lib.klst_apply_pencil_noalloc_capacity()
    assert cap == 4 << 20
    spec = wl.c3()[0]  # nx = 128: at most 15 right-hand sides fit
    P = klst.Pencil(spec)
    X = to_dev(wl.random_vectors(P.n, 16, 43))
    Y = X.new_empty(X.shape)
    code = lib.klst_apply_pencil_noalloc(P.handle, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), 16,
                                         None, klst._stream(None))
    assert code == klst.KLST_EINVAL
    assert b"fixed array holds" in lib.klst_last_error()
