"""Post-processing of the base flow and of eigenvectors (oracle; test infrastructure only).

* ``eneq``   -- the translational non-equilibrium measure of Eq. L2norm (Sec. 5):
                E_neq(x_j) = sqrt( sum_k W_k (f(x_j, xi_k) - f^e(x_j, xi_k))^2 ), with f the base
                flow's reduced distribution g_c and f^e its (discrete) local equilibrium g_c^e,
                summed with the full-line Gauss-Hermite product weights W_k.
* ``macro``  -- the macroscopic perturbations of an eigenvector q = [g^; h^] at every point,
                (rho^, u^, v^, E^)(x_j), from the perturbation-moment definitions of Sec. 2.2
                (the linearised moments that Eqs. comp_ghat1Dshock / comp_hhat1Dshock couple):
                rho^ = sum W g^, u^ = sum W (xi_x - u) g^ / rho, v^ = sum W (xi_y - v) g^ / rho,
                E^ = [sum W (|xi|^2 - 2E) g^ + sum W h^] / (2 rho).
* ``unorm``  -- |U^| = sqrt(|u^|^2 + |v^|^2) (Eq. Unormpert) and its maximum over x, the
                normalisation the paper applies to velocity eigenvectors.
"""
import numpy as np


def eneq(data):
    """E_neq at every collocation point from the oracle's pencil tables (gc, gce, W)."""
    d = data
    return np.sqrt(((d["gc"] - d["gce"]) ** 2) @ d["W"])


def macro(data, q):
    """(4, Nx) complex perturbation moments of one eigenvector q (length 2 Nx Nxi, ordering
    q[(c Nxi + k) Nx + j]), written out point by point from the moment definitions."""
    d = data
    nx, nxi = d["Dx"].shape[0], d["W"].size
    Q = np.asarray(q).reshape(2, nxi, nx)          # [c][k][j]
    g, h = Q[0].T, Q[1].T                            # (Nx, Nxi)
    W, xx, xy = d["W"], d["xi_x"], d["xi_y"]
    rho, u, E = d["rho"], d["u"], d["E"]
    out = np.zeros((4, nx), dtype=np.complex128)
    for j in range(nx):
        out[0, j] = np.sum(W * g[j])
        out[1, j] = np.sum(W * (xx - u[j]) * g[j]) / rho[j]
        out[2, j] = np.sum(W * xy * g[j]) / rho[j]           # v = 0 in the 1-D base flow
        out[3, j] = (np.sum(W * (xx ** 2 + xy ** 2 - 2.0 * E[j]) * g[j]) + np.sum(W * h[j])) / (2.0 * rho[j])
    return out


def unorm(m):
    """|U^|(x_j) = sqrt(|u^|^2 + |v^|^2) (Eq. Unormpert) and its maximum over the points."""
    U = np.sqrt(np.abs(m[1]) ** 2 + np.abs(m[2]) ** 2)
    return U, float(U.max())
