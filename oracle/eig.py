"""Reference eigen-solutions of the pencil (oracle; test infrastructure only).

* ``qz``            -- all finite eigenpairs of (A, B) by dense QZ (Sec. 4: the
                       QZ algorithm computes every eigenvalue; tiny pencils only).
* ``interior``      -- the same finite spectrum from the standard problem on the
                       interior unknowns: a boundary row reads q_b = omega * 0, so
                       every finite eigenvector vanishes there and A_II q_I = omega q_I.
* ``shift_invert``  -- T = (A - sigma B)^{-1} B by dense LU (Eq. parShiftInvert),
                       eigenvalues mu of T by ARPACK, omega = sigma + 1/mu.
* ``residuals``     -- ||A q - omega B q||_2 / ||q||_2 (the eigenpair residual).
* ``match``         -- one-to-one minimum-cost assignment of two eigenvalue sets.
"""
import numpy as np
import scipy.linalg as sla
import scipy.optimize as sopt
import scipy.sparse.linalg as spla

from . import pencil


def qz(A, B, inf_tol=1e-12):
    """Finite eigenvalues of (A, B) with right/left eigenvectors and condition numbers.

    Infinite eigenvalues (|beta| < inf_tol ||B||) are dropped.  kappa_i =
    ||x|| ||y|| / |y^H B x| is the eigenvalue condition number.
    """
    ab, vl, vr = sla.eig(A, B, left=True, right=True, homogeneous_eigvals=True)
    alpha, beta = ab
    nb = np.linalg.norm(B, 2) if B.shape[0] <= 512 else np.abs(B).max()
    fin = np.abs(beta) > inf_tol * max(nb, 1.0)
    lam = alpha[fin] / beta[fin]
    X, Y = vr[:, fin], vl[:, fin]
    kappa = np.linalg.norm(X, axis=0) * np.linalg.norm(Y, axis=0) / np.abs(np.sum(Y.conj() * (B @ X), axis=0))
    return lam, X, kappa


def interior(A, bc_rows):
    """Finite spectrum via the interior standard problem A_II q_I = omega q_I.

    Returns (omega, X, kappa) with X embedded back into full length (zeros on
    boundary rows) and kappa the standard eigenvalue condition number of A_II.
    """
    n = A.shape[0]
    I = np.setdiff1d(np.arange(n), bc_rows)
    lam, vl, vr = sla.eig(A[np.ix_(I, I)], left=True, right=True)
    X = np.zeros((n, lam.size), dtype=np.complex128)
    X[I, :] = vr
    kappa = np.linalg.norm(vr, axis=0) * np.linalg.norm(vl, axis=0) / np.abs(np.sum(vl.conj() * vr, axis=0))
    return lam, X, kappa


def nearest(omega, sigma, k):
    """Indices of the k eigenvalues closest to the shift sigma."""
    return np.argsort(np.abs(omega - sigma), kind="stable")[:k]


class ShiftInvert:
    """Dense LU of (A - sigma B); ``apply(x)`` returns (A - sigma B)^{-1} B x (Eq. parShiftInvert)."""

    def __init__(self, A, B, sigma):
        self.B = B
        self.sigma = sigma
        self.lu = sla.lu_factor(A - sigma * B, check_finite=False)

    def apply(self, x):
        return sla.lu_solve(self.lu, self.B @ x, check_finite=False)

    def eigs(self, k, ncv, v0=None, tol=1e-13, maxiter=10000):
        """k largest-|mu| eigenpairs of T by ARPACK; returns (omega sorted by |omega - sigma|, X)."""
        n = self.B.shape[0]
        op = spla.LinearOperator((n, n), matvec=self.apply, dtype=np.complex128)
        mu, X = spla.eigs(op, k=k, which="LM", v0=v0, ncv=ncv, tol=tol, maxiter=maxiter)
        omega = self.sigma + 1.0 / mu
        o = np.argsort(np.abs(omega - self.sigma), kind="stable")
        return omega[o], X[:, o]


    def left_eigs(self, k, ncv, v0=None, tol=1e-13, maxiter=10000):
        """Left eigenvectors from ARPACK on the adjoint T^H = B^H (A - sigma B)^{-H}.

        If T^H z = conj(mu) z then y = (A - sigma B)^{-H} z satisfies
        y^H (A - omega B) = 0 with omega = sigma + 1/mu.  Returns (omega, Y)
        sorted by |omega - sigma|.
        """
        n = self.B.shape[0]
        mv = lambda z: self.B.conj().T @ sla.lu_solve(self.lu, z, trans=2, check_finite=False)
        op = spla.LinearOperator((n, n), matvec=mv, dtype=np.complex128)
        nu_, Z = spla.eigs(op, k=k, which="LM", v0=v0, ncv=ncv, tol=tol, maxiter=maxiter)
        Y = np.stack([sla.lu_solve(self.lu, Z[:, i], trans=2, check_finite=False) for i in range(k)], axis=1)
        omega = self.sigma + 1.0 / nu_.conj()
        o = np.argsort(np.abs(omega - self.sigma), kind="stable")
        return omega[o], Y[:, o]


def condition_numbers(B, X, Y):
    """kappa_i = ||x_i|| ||y_i|| / |y_i^H B x_i| for paired right/left eigenvectors."""
    return np.linalg.norm(X, axis=0) * np.linalg.norm(Y, axis=0) / np.abs(np.sum(Y.conj() * (B @ X), axis=0))


def residuals(spec, data, omega, X):
    """||A x - omega B x||_2 / ||x||_2 per column, with the matrix-free A and B."""
    X = np.asarray(X).reshape(X.shape[0], -1)
    R = pencil.apply_A(spec, data, X) - pencil.apply_B(data, X) * np.asarray(omega)[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(X, axis=0)


def match(a, b):
    """Pair a[i] with b[perm[i]] minimising sum |a - b| (one-to-one); returns perm."""
    cost = np.abs(np.asarray(a)[:, None] - np.asarray(b)[None, :])
    r, c = sopt.linear_sum_assignment(cost)
    perm = np.empty(len(a), dtype=int)
    perm[r] = c
    return perm
