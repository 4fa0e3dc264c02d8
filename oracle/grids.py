"""Spatial and velocity grids (oracle; test infrastructure only).

Chebyshev collocation with the algebraic map (Sec. 3.1) and Gauss-Hermite
micro-velocity nodes (Sec. 3.2), written out from their definitions in float64.
"""
import numpy as np


def cheb_points(N):
    """Chebyshev-Gauss-Lobatto points y_j = cos(j pi / N), j = 0..N (Eq. ChebPoints)."""
    j = np.arange(N + 1, dtype=np.float64)
    return np.cos(j * np.pi / N)


def cheb_diff(N):
    """(N+1)x(N+1) Chebyshev differentiation matrix D_y.

    Off-diagonal (c_j/c_m)(-1)^(j+m)/(y_j - y_m) with c_0 = c_N = 2 (Eq. ChebOffDiag);
    interior diagonal -y_j / (2(1 - y_j^2)) (Eq. ChebDiag); corners
    D_00 = (2N^2+1)/6 and D_NN = -(2N^2+1)/6 (Eq. ChebBC).
    """
    y = cheb_points(N)
    c = np.ones(N + 1)
    c[0] = 2.0
    c[N] = 2.0
    D = np.zeros((N + 1, N + 1))
    for j in range(N + 1):
        for m in range(N + 1):
            if j != m:
                D[j, m] = (c[j] / c[m]) * (-1.0) ** (j + m) / (y[j] - y[m])
    for j in range(1, N):
        D[j, j] = -y[j] / (2.0 * (1.0 - y[j] ** 2))
    D[0, 0] = (2.0 * N * N + 1.0) / 6.0
    D[N, N] = -(2.0 * N * N + 1.0) / 6.0
    return D


def algebraic_map(y, L, s_inf):
    """Map y in [-1, 1] to x in [-s_inf, s_inf] (Eq. Chebmapping).

    x = L y / sqrt(1 + s - y^2) with s = (L/s_inf)^2.  Returns x, dy/dx and
    d2y/dx2 evaluated at the mapped points (the closed forms printed beside
    Eq. Chebmapping).
    """
    s = (L / s_inf) ** 2
    x = L * y / np.sqrt(1.0 + s - y * y)
    dydx = np.sqrt(1.0 + s) * L * L / (L * L + x * x) ** 1.5
    d2ydx2 = -3.0 * np.sqrt(1.0 + s) * L * L * x / (L * L + x * x) ** 2.5
    return x, dydx, d2ydx2


def mapped_diff(nx, L, s_inf):
    """Mapped grid and first-derivative matrix D_x = diag(dy/dx) D_y (Sec. 3.1).

    ``nx`` is the number of collocation points (N = nx - 1).  Point j = 0 is
    x = +s_inf (downstream end), j = N is x = -s_inf (upstream end).
    """
    N = nx - 1
    y = cheb_points(N)
    x, dydx, _ = algebraic_map(y, L, s_inf)
    Dx = dydx[:, None] * cheb_diff(N)
    return x, Dx


def hermite_functions(x, n):
    """Orthonormal Hermite functions psi_0..psi_{n-1} at points x, shape (n, len(x)).

    psi_m(x) = H_m(x) exp(-x^2/2) / sqrt(2^m m! sqrt(pi)); computed by the
    three-term recurrence of the orthonormal family, which neither overflows
    nor underflows for |x| up to ~35.
    """
    x = np.asarray(x, dtype=np.float64)
    psi = np.zeros((n, x.size))
    psi[0] = np.pi ** -0.25 * np.exp(-0.5 * x * x)
    if n > 1:
        psi[1] = np.sqrt(2.0) * x * psi[0]
    for m in range(1, n - 1):
        psi[m + 1] = np.sqrt(2.0 / (m + 1)) * x * psi[m] - np.sqrt(m / (m + 1.0)) * psi[m - 1]
    return psi


def gauss_hermite(Q):
    """Gauss-Hermite nodes and weights for weight e^{-x^2} (Sec. 3.2).

    Golub-Welsch: nodes are the eigenvalues of the symmetric tridiagonal Jacobi
    matrix of the monic Hermite recurrence, off-diagonal sqrt(k/2), k = 1..Q-1;
    the weights are sqrt(pi) times the squared first eigenvector components.
    The nodes are symmetrised (x_i = -x_{Q-1-i}, exact zero for odd Q) so that
    the inflow classification sign(xi_x) is exact.

    Returns (nodes ascending, w, W) where w are the weights for integrals of
    F(x) e^{-x^2} and W = w e^{x^2} are the full-line weights used on raw
    distribution values.  W is evaluated in the Christoffel form
    W_i = 1 / sum_{m<Q} psi_m(x_i)^2, which equals w_i e^{x_i^2} without the
    underflow of exponentiating w_i for large Q.
    """
    k = np.arange(1, Q, dtype=np.float64)
    J = np.diag(np.sqrt(k / 2.0), 1) + np.diag(np.sqrt(k / 2.0), -1)
    nodes, vecs = np.linalg.eigh(J)
    order = np.argsort(nodes)
    nodes = nodes[order]
    vecs = vecs[:, order]
    nodes = 0.5 * (nodes - nodes[::-1])
    if Q % 2 == 1:
        nodes[Q // 2] = 0.0
    w = np.sqrt(np.pi) * vecs[0, :] ** 2
    psi = hermite_functions(nodes, Q)
    W = 1.0 / np.sum(psi * psi, axis=0)
    return nodes, w, W


def velocity_grid(qx, qy):
    """Tensor-product micro-velocity grid, node index k = kx*qy + ky.

    Returns xi_x, xi_y, W (full-line product weights W_kx W_ky), each of length
    qx*qy.
    """
    nx_, _, Wx = gauss_hermite(qx)
    ny_, _, Wy = gauss_hermite(qy)
    xi_x = np.repeat(nx_, qy)
    xi_y = np.tile(ny_, qx)
    W = np.repeat(Wx, qy) * np.tile(Wy, qx)
    return xi_x, xi_y, W
