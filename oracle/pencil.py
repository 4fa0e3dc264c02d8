"""Assembly of the kLST pencil A q = omega B q (oracle; test infrastructure only).

Unknown ordering: q[(c * Nxi + k) * Nx + j] with component c in (g^, h^),
micro-velocity node k = kx * qy + ky and collocation point j fastest.

For an interior row (c, j, k), Eqs. comp_ghat1Dshock / comp_hhat1Dshock give
    (i beta xi_y,k + nu_j) q_{c,k}(j) + xi_x,k sum_m (D_x)_{jm} q_{c,k}(m)
        - sum_a G^c_a(j, k) m_a(j) = omega q_{c,k}(j),
    m_a(j) = sum_{c', p} w^{c'}_a(j, p) q_{c',p}(j),
so A holds the left-hand side and B = I (Eq. MatrixSystem with the
eigenvalue variable omega = i varpi of Eq. MatrixProblem).  Inflow boundary
rows (Sec. 2.2: g^ = h^ = 0 for incoming xi at x = -s_inf and x = +s_inf)
become e_row^T in A and 0 in B, so B is singular.
"""
import numpy as np

from . import gas


def index(c, k, j, nxi, nx):
    return (c * nxi + k) * nx + j


def assemble_dense(spec, data=None):
    """Dense complex128 (A, B) of size n = 2 Nx Nxi; ``data`` from gas.pencil_data (computed if None)."""
    d = gas.pencil_data(spec) if data is None else data
    nx, nxi = d["Dx"].shape[0], d["W"].size
    n = 2 * nx * nxi
    beta = gas._p(spec, "beta")
    A = np.zeros((n, n), dtype=np.complex128)
    B = np.eye(n, dtype=np.complex128)
    jj = np.arange(nx)
    for c in range(2):
        for k in range(nxi):
            rows = index(c, k, jj, nxi, nx)
            A[np.ix_(rows, rows)] += d["xi_x"][k] * d["Dx"]
            A[rows, rows] += d["nu"] + 1j * beta * d["xi_y"][k]
    kk = np.arange(nxi)
    for j in range(nx):
        # coupling block at point j: rows (c, k), cols (c', p)
        blocks = [[np.einsum("ak,ap->kp", d["G"][c, :, j, :], d["w"][cp, :, j, :]) for cp in range(2)]
                  for c in range(2)]
        for c in range(2):
            rows = index(c, kk, j, nxi, nx)
            for cp in range(2):
                cols = index(cp, kk, j, nxi, nx)
                A[np.ix_(rows, cols)] -= blocks[c][cp]
    for c in range(2):
        jb, kb = np.nonzero(d["bc"])
        rows = index(c, kb, jb, nxi, nx)
        A[rows, :] = 0.0
        A[rows, rows] = 1.0
        B[rows, rows] = 0.0
    return A, B


def boundary_rows(data):
    """Sorted global indices of the inflow boundary rows (the zero rows of B)."""
    nx, nxi = data["Dx"].shape[0], data["W"].size
    jb, kb = np.nonzero(data["bc"])
    return np.sort(np.concatenate([index(c, kb, jb, nxi, nx) for c in range(2)]))


def nnz_formula(nx, qx, qy):
    """Structural nnz(A) = n (Nx + 2 Nxi - 1) - n_bc (Nx + 2 Nxi - 2), n_bc = 4 floor(qx/2) qy.

    Interior rows hold one dense D_x row (Nx entries, diagonal included) plus the
    moment coupling to every (c', p) at the same point (2 Nxi entries, one of
    them the diagonal); boundary rows hold only the diagonal.  Valid when no
    xi_x node is zero (even qx), the configurations of Table benchmark_cases.
    """
    nxi = qx * qy
    n = 2 * nx * nxi
    nbc = 4 * (qx // 2) * qy
    return n * (nx + 2 * nxi - 1) - nbc * (nx + 2 * nxi - 2)


def nnz_numerical(spec, data=None):
    """Count the nonzero entries of A row block by row block without forming A densely."""
    d = gas.pencil_data(spec) if data is None else data
    nx, nxi = d["Dx"].shape[0], d["W"].size
    beta = gas._p(spec, "beta")
    total = 0
    for j in range(nx):
        blocks = np.concatenate([np.concatenate([np.einsum("ak,ap->kp", d["G"][c, :, j, :], d["w"][cp, :, j, :])
                                                 for cp in range(2)], axis=1) for c in range(2)], axis=0)
        diag_cpl = np.diag(blocks).copy()
        np.fill_diagonal(blocks, 0.0)
        cpl_nnz = np.count_nonzero(blocks, axis=1)  # per row (c, k), excluding the diagonal position
        for c in range(2):
            for k in range(nxi):
                if d["bc"][j, k]:
                    total += 1
                    continue
                row = d["xi_x"][k] * d["Dx"][j, :].astype(np.complex128)
                row[j] += d["nu"][j] + 1j * beta * d["xi_y"][k] - diag_cpl[c * nxi + k]
                total += np.count_nonzero(row) + cpl_nnz[c * nxi + k]
    return total


def apply_A(spec, data, q):
    """Matrix-free A q for q of length n (or shape (n, r)); the same rows as ``assemble_dense``."""
    d = data
    nx, nxi = d["Dx"].shape[0], d["W"].size
    beta = gas._p(spec, "beta")
    shp = q.shape
    Q = q.reshape(2, nxi, nx, -1)
    out = np.einsum("jm,ckmr->ckjr", d["Dx"], Q) * d["xi_x"][None, :, None, None]
    out += (d["nu"][None, None, :, None] + 1j * beta * d["xi_y"][None, :, None, None]) * Q
    m = np.einsum("cajp,cpjr->ajr", d["w"], Q)
    out -= np.einsum("cajk,ajr->ckjr", d["G"], m)
    bcT = d["bc"].T  # (nxi, nx)
    out[:, bcT, :] = Q[:, bcT, :]
    return out.reshape(shp)


def apply_B(data, q):
    """B q: q with the inflow boundary rows zeroed."""
    nx, nxi = data["Dx"].shape[0], data["W"].size
    shp = q.shape
    Q = q.reshape(2, nxi, nx, -1).copy()
    Q[:, data["bc"].T, :] = 0.0
    return Q.reshape(shp)
