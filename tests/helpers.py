"""Shared helpers for the GPU parity tests (inputs from the seeded workloads, references from the oracle)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def torch_cuda():
    import torch
    return torch


def to_dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.complex128, device="cuda")


def to_host(t):
    return t.detach().cpu().numpy()


def read_golden(name):
    """Rows (omega, kappa, residual) of a stored eigenvalue file written by tests/golden/make_golden.py."""
    rows = np.loadtxt(os.path.join(GOLDEN, name), comments="#")
    return rows[:, 0] + 1j * rows[:, 1], rows[:, 2], rows[:, 3]


def eig_gate(omega_ref, kappa, normA):
    """Eigenvalues whose oracle value is itself accurate to well below 1e-8 relative.

    First-order perturbation theory bounds the oracle's own error by kappa * eps * ||A||;
    an eigenvalue is gated when that bound is below 1e-10 |omega| (two orders of margin
    under the 1e-8 parity tolerance), otherwise it is reported only.
    """
    return kappa * 2.220446049250313e-16 * normA < 1e-10 * np.abs(omega_ref)


def cond1(A, lu=None):
    """1-norm condition estimate ||A||_1 ||A^{-1}||_1 (Higham-Tisseur estimator on the LU solve)."""
    import scipy.linalg as sla
    import scipy.sparse.linalg as spla
    lu = sla.lu_factor(A) if lu is None else lu
    n = A.shape[0]
    op = spla.LinearOperator((n, n), matvec=lambda x: sla.lu_solve(lu, x),
                             rmatvec=lambda x: sla.lu_solve(lu, x, trans=2), dtype=np.complex128)
    return np.abs(A).sum(axis=0).max() * spla.onenormest(op)


def pencil_norm2_est(data, beta):
    """sqrt(||A||_1 ||A||_inf) >= ||A||_2, from the oracle's per-point tables (triangle-inequality sums)."""
    d = data
    nx, nxi = d["Dx"].shape[0], d["W"].size
    axx = np.abs(d["xi_x"])
    rows = axx[None, :] * np.abs(d["Dx"]).sum(axis=1)[:, None]          # (j, k) streaming row sums
    cols = axx[None, :] * np.abs(d["Dx"]).sum(axis=0)[:, None]          # (m, p) streaming column sums
    diag = np.abs(d["nu"][:, None] + 1j * beta * d["xi_y"][None, :])
    cr = np.zeros((2, nx, nxi))
    cc = np.zeros((2, nx, nxi))
    for j in range(nx):
        blk = np.abs(np.einsum("cak,dap->ckdp", d["G"][:, :, j, :], d["w"][:, :, j, :]))
        cr[:, j, :] = blk.sum(axis=(2, 3))
        cc[:, j, :] = blk.sum(axis=(0, 1))
    ninf = np.max(rows[None] + diag[None] + cr)
    n1 = np.max(cols[None] + diag[None] + cc)
    return float(np.sqrt(ninf * n1))
