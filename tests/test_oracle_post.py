"""Pins for the oracle's post-processing (Eq. L2norm, Eq. Unormpert, the perturbation moments of Sec. 2.2)."""
import numpy as np
import pytest

from oracle import gas, grids, post
from paper_2607_27440_b300 import workloads as wl


def test_eneq_vanishes_for_an_equilibrium_base():
    """EQ mode sets g_c := g_c^e, so the non-equilibrium measure is exactly zero everywhere."""
    spec = wl.tiny(nx=12, qx=8, qy=6, base="tanh", noneq=0, width=0.5, mach=2.0).as_dict()
    assert np.all(post.eneq(gas.pencil_data(spec)) == 0.0)


def test_eneq_of_mott_smith_peaks_inside_the_shock():
    """The bimodal Mott-Smith base deviates from its local Maxwellian inside the shock and not in the
    free streams (both ends are Rankine-Hugoniot Maxwellians, to quadrature error): E_neq is largest
    near x = 0 and orders of magnitude smaller at x = +-s_inf."""
    spec = wl.tiny(nx=24, qx=30, qy=20, mach=3.0, width=0.5).as_dict()
    d = gas.pencil_data(spec)
    e = post.eneq(d)
    jmax = int(np.argmax(e))
    assert abs(d["x"][jmax]) < 2.0 * spec["width"]
    assert e[0] < 1e-3 * e[jmax] and e[-1] < 1e-3 * e[jmax]


def test_eneq_matches_its_definition_for_a_known_deviation():
    """A distribution that differs from the Maxwellian by eps * phi has E_neq = |eps| sqrt(sum W phi^2)."""
    xi_x, xi_y, W = grids.velocity_grid(10, 8)
    ge = gas.maxwellian(np.array([1.0]), np.array([0.3]), np.array([0.0]), np.array([1.2]), xi_x, xi_y)
    phi = np.exp(-(xi_x ** 2 + xi_y ** 2)) * xi_x
    d = {"gc": ge + 1e-3 * phi, "gce": ge, "W": W}
    assert post.eneq(d)[0] == pytest.approx(1e-3 * np.sqrt(np.sum(W * phi[0] ** 2 if phi.ndim > 1 else W * phi ** 2)),
                                            rel=1e-12)


@pytest.mark.parametrize("a", [0, 1, 2, 3])
def test_macro_of_equilibrium_derivative_is_a_unit_moment(a):
    """With the discrete-conservative coefficients (M C = I_4), the perturbation q whose (g^, h^) is the
    derivative of the equilibrium with respect to moment a at point j carries exactly the unit
    perturbation of moment a at that point and nothing else: macro(q) = e_a delta_j."""
    spec = wl.tiny(nx=8, qx=6, qy=5, mach=2.5, beta=0.4).as_dict()
    d = gas.pencil_data(spec)
    nx, nxi = 8, 30
    j = 3
    q = np.zeros(2 * nx * nxi, dtype=np.complex128)
    for c in range(2):
        for k in range(nxi):
            q[(c * nxi + k) * nx + j] = d["C"][c, a, j, k]
    m = post.macro(d, q)
    ref = np.zeros((4, nx))
    ref[a, j] = 1.0
    assert np.max(np.abs(m - ref)) < 1e-12


def test_unorm_definition():
    m = np.zeros((4, 3), dtype=np.complex128)
    m[1] = [3.0, 1j, 0.0]
    m[2] = [4j, 0.0, -2.0]
    U, Umax = post.unorm(m)
    assert np.allclose(U, [5.0, 1.0, 2.0]) and Umax == 5.0
