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
