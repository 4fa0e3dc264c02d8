"""Post-processing on the GPU (Sec. 5: Eq. L2norm, Eq. Unormpert and the perturbation moments) against
the oracle's point-by-point definitions, on the same vectors."""
import numpy as np
import pytest

from oracle import gas, post
from paper_2607_27440_b300 import workloads as wl
from tests.helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def klst():
    from paper_2607_27440_b300 import klst as k
    k.load()
    return k


@pytest.mark.parametrize("which", ["c1", "c2"])
def test_eneq_matches_oracle(klst, which):
    spec, es = getattr(wl, which)()
    d = gas.pencil_data(spec.as_dict())
    ref = post.eneq(d)
    got = klst.Pencil(spec).base_noneq()
    if spec.noneq == 0:
        assert np.all(got == 0.0)
    else:
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(ref)


def test_eigenvector_macro_matches_oracle(klst):
    """The C1 eigenvectors from klst_eigs: GPU (rho^, u^, v^, E^) and max |U^| against the oracle's
    definitions evaluated on the same vectors (1e-12 relative to the largest moment)."""
    spec, es = wl.c1()
    d = gas.pencil_data(spec.as_dict())
    P = klst.Pencil(spec)
    F = P.factor(es.sigma)
    om, vec, res, info = F.eigs(8, 30, tol=1e-12, seed=1, vectors=True)
    m, um = P.eigvec_macro(vec)
    V = to_host(vec)
    for i in range(V.shape[0]):
        ref = post.macro(d, V[i])
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(m[i] - ref)) <= 1e-12 * scale, i
        _, umax = post.unorm(ref)
        assert um[i] == pytest.approx(umax, rel=1e-12)


def test_macro_of_random_vectors_multi_rhs(klst):
    spec = wl.tiny(nx=20, qx=8, qy=6, mach=3.0)
    d = gas.pencil_data(spec.as_dict())
    X = wl.random_vectors(spec.n, 3, 9)
    m, um = klst.Pencil(spec).eigvec_macro(to_dev(X))
    for i in range(3):
        ref = post.macro(d, X[i])
        assert np.max(np.abs(m[i] - ref)) <= 1e-12 * np.max(np.abs(ref))
