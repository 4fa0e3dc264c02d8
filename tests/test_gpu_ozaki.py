"""klst_gemm_f64_tc: float64-accurate GEMM on the tensor cores (the basis rotation's building block)
against the product in extended precision (numpy longdouble, 64-bit significand)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def klst():
    from paper_2607_27440_b300 import klst as k
    k.load()
    return k


def _ref(A, B):
    return (A.astype(np.longdouble) @ B.astype(np.longdouble))


@pytest.mark.parametrize("M,N,K", [(128, 32, 16), (300, 70, 240), (1000, 140, 240), (257, 33, 9), (64, 200, 128),
                                   (5000, 96, 256)])
def test_gemm_matches_extended_precision(klst, M, N, K):
    """Error per entry within a few float64 ulps of the row and column maxima times K, and no worse than
    numpy's own float64 product against the same extended-precision reference (up to a factor 4)."""
    import torch
    rng = np.random.default_rng(M * 131 + N * 7 + K)
    # entries spread over several orders of magnitude within rows and columns
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-3, 1, size=(M, K))
    B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-2, 2, size=(K, N))
    C = klst.gemm_f64_tc(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    R = _ref(A, B)
    err = np.abs(C - R).astype(np.float64)
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :] * K
    assert np.all(err <= 8 * 2.0 ** -53 * scale), (err / scale).max()
    err64 = np.abs((A @ B) - R).astype(np.float64)
    assert np.linalg.norm(err) <= 4 * np.linalg.norm(err64) + 1e-300


def test_gemm_exact_on_small_integers(klst):
    """Integer matrices whose products fit in float64 exactly come out exact."""
    import torch
    rng = np.random.default_rng(5)
    A = rng.integers(-1000, 1000, size=(256, 64)).astype(np.float64)
    B = rng.integers(-1000, 1000, size=(64, 48)).astype(np.float64)
    C = klst.gemm_f64_tc(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    assert np.array_equal(C, A @ B)


def test_gemm_zero_rows_and_columns(klst):
    import torch
    A = np.zeros((130, 32))
    A[3, 5] = 2.5
    B = np.zeros((32, 40))
    B[5, 7] = -4.0
    C = klst.gemm_f64_tc(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    E = np.zeros((130, 40))
    E[3, 7] = -10.0
    assert np.array_equal(C, E)


def test_gemm_rejects_k_beyond_exactness_bound(klst):
    import torch
    with pytest.raises(klst.KlstError) as ei:
        klst.gemm_f64_tc(torch.zeros((8, 300), dtype=torch.float64, device="cuda"),
                         torch.zeros((300, 8), dtype=torch.float64, device="cuda"))
    assert ei.value.code == klst.KLST_EINVAL
