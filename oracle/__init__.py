"""Plain FP64 CPU oracle for the kLST shift-and-invert eigensolve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2607_27440_b300``) never imports it, and it
never imports the product path: the two share no code.

What it computes (paper: Karpuzcu, Levin, Theofilis, "Kinetic Linear Stability
Theory for High-Speed Compressible Flows"):

* ``grids``  -- Chebyshev-Gauss-Lobatto points and differentiation matrix
  (Eqs. ChebPoints, ChebDiag, ChebOffDiag, ChebBC), the algebraic map to the
  unbounded domain (Eq. Chebmapping), Gauss-Hermite nodes/weights (Sec. 3.2).
* ``gas``    -- nondimensional argon gas, Rankine-Hugoniot states, synthetic
  base flows, discrete moments, the discrete Maxwellian equilibrium, the
  linearisation coefficients C and G/H (Sec. 2.2, Eq. CompBGKtilde) and the
  nonlinear discrete BGK collision map used to pin them.
* ``pencil`` -- dense assembly of the pencil (A, B) from Eqs. comp_ghat1Dshock
  and comp_hhat1Dshock with the inflow boundary rows, the structural nnz count
  (Table benchmark_cases), and a matrix-free A q.
* ``eig``    -- reference eigen-solutions: QZ on tiny pencils, the exact
  reduction to the interior standard problem, dense LU shift-invert with ARPACK,
  residuals, condition numbers and eigenvalue matching.

Every floating-point quantity is float64 / complex128.  Where the paper is
silent the oracle follows the readings listed in the repository's design
notes (eigenvalue variable, h moment with K = 0, full-line Gauss-Hermite
weights, derived C/G coefficients, map parameters, discrete conservation).

Parity status: every function is pinned by a ``-m "not gpu"`` test except the
agreement of the derived G/H coefficient formulas with Zou et al. (the paper
defers them to that reference, which is not available): "parity unpinned"
against that source; they are pinned instead against the finite-difference
Jacobian of the nonlinear BGK collision map.
"""
