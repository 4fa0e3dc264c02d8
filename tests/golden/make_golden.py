"""Write the stored reference eigenvalues for the C1 and C2 workloads.

Calls only the CPU oracle (``oracle/``) and the seeded input recipes; run from
the repository root:  python tests/golden/make_golden.py [c1] [c2]

c1_eigs.txt : the 20 finite eigenvalues nearest sigma = 0.1i of the M = 1.2
              tanh-Maxwellian pencil (n = 1,536), from the dense interior
              standard problem, with their condition numbers and residuals.
c2_eigs.txt : the 40 eigenvalues nearest sigma = 0.1i of the M = 3.0
              Mott-Smith pencil (n = 12,288), from dense LU shift-invert +
              ARPACK (right and adjoint runs), with condition numbers and
              residuals.
Columns: re(omega) im(omega) kappa residual.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import eig, gas, pencil  # noqa: E402
from paper_2607_27440_b300 import workloads as wl  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write(name, header, om, kap, res):
    with open(os.path.join(HERE, name), "w") as f:
        f.write("# " + header.replace("\n", "\n# ") + "\n")
        f.write("# re(omega) im(omega) kappa residual\n")
        for o, k, r in zip(om, kap, res):
            f.write(f"{o.real:.17e} {o.imag:.17e} {k:.6e} {r:.3e}\n")


def c1():
    ps, es = wl.c1()
    spec = ps.as_dict()
    d = gas.pencil_data(spec)
    A, B = pencil.assemble_dense(spec, d)
    lam, X, kap = eig.interior(A, pencil.boundary_rows(d))
    idx = eig.nearest(lam, es.sigma, es.nev)
    res = eig.residuals(spec, d, lam[idx], X[:, idx])
    write("c1_eigs.txt", f"C1 {ps}\nsigma={es.sigma} nev={es.nev}; oracle.eig.interior (dense geev on A_II)",
          lam[idx], kap[idx], res)


def c2():
    ps, es = wl.c2()
    spec = ps.as_dict()
    d = gas.pencil_data(spec)
    A, B = pencil.assemble_dense(spec, d)
    t = time.time()
    si = eig.ShiftInvert(A, B, es.sigma)
    print("lu", time.time() - t, flush=True)
    om, X = si.eigs(es.nev, ncv=2 * es.nev + 1, v0=wl.start_vector(A.shape[0], es.seed))
    print("eigs", time.time() - t, flush=True)
    oml, Y = si.left_eigs(es.nev, ncv=2 * es.nev + 1, v0=wl.start_vector(A.shape[0], es.seed + 100))
    print("left", time.time() - t, flush=True)
    perm = eig.match(om, oml)
    assert np.max(np.abs(om - oml[perm]) / np.abs(om)) < 1e-8
    kap = eig.condition_numbers(B, X, Y[:, perm])
    res = eig.residuals(spec, d, om, X)
    write("c2_eigs.txt", f"C2 {ps}\nsigma={es.sigma} nev={es.nev}; oracle.eig.ShiftInvert (dense LU + ARPACK)",
          om, kap, res)


if __name__ == "__main__":
    which = sys.argv[1:] or ["c1", "c2"]
    for w in which:
        globals()[w]()
