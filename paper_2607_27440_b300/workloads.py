"""Seeded synthetic workloads for the kLST eigensolve (input recipes only, no method arithmetic).

Shared by the CUDA path's callers and by the tests that run the CPU oracle:
it holds descriptors (numbers) and seeded random draws, nothing else.

The paper's base flows come from its BE-BGK solver, which is not part of the
eigensolve path, so synthetic argon normal-shock base flows stand in for them:
a tanh local Maxwellian (equilibrium) and a Mott-Smith bimodal mix of the
Rankine-Hugoniot Maxwellians (non-equilibrium).  Re_Delta comes from the
paper's Table 1DShockThickness (M = 1.2, 3.0, 4.0); Mach sweeps interpolate
it piecewise-linearly.  Map L = 1, s_inf = 30 (shock-thickness units).
"""
from dataclasses import dataclass, asdict, replace

import numpy as np

RE_TABLE = ((1.2, 24.34), (3.0, 9.68), (4.0, 11.03))
LAMBDA_INF_MM = 0.2071          # upstream mean free path of the argon free stream
DELTA_MM = {1.2: 2.548, 3.0: 0.405, 4.0: 0.346}


def re_delta(mach):
    """Re_Delta at Mach ``mach``: table values, piecewise-linear in between, clamped outside."""
    ms = [m for m, _ in RE_TABLE]
    rs = [r for _, r in RE_TABLE]
    return float(np.interp(mach, ms, rs))


@dataclass(frozen=True)
class PencilSpec:
    nx: int
    qx: int
    qy: int
    mach: float
    beta: float = 1.0
    base: str = "mott_smith"     # "tanh" (local Maxwellian), "mott_smith" (bimodal), "gilbarg_paolucci"
    noneq: int = 1                # 0: EQ (f_c := f_c^e), 1: NONEQ
    conservative: int = 1         # discrete-conservative equilibrium and coefficients
    width: float = 0.5            # tanh width in shock thicknesses
    gamma: float = 5.0 / 3.0
    visc_s: float = 0.5
    re_delta: float = 0.0         # 0 -> from the table
    map_L: float = 1.0
    map_sinf: float = 30.0

    def __post_init__(self):
        if self.re_delta == 0.0:
            object.__setattr__(self, "re_delta", re_delta(self.mach))

    @property
    def nxi(self):
        return self.qx * self.qy

    @property
    def n(self):
        return 2 * self.nx * self.nxi

    def as_dict(self):
        return asdict(self)


@dataclass(frozen=True)
class EigsSpec:
    sigma: complex
    nev: int
    ncv: int
    seed: int
    tol: float = 1e-12
    max_restarts: int = 200
    keep: int = 0  # Schur vectors kept at a restart (0: the library default, nev + (ncv - nev) / 2)


def c1():
    """M = 1.2 tanh local-Maxwellian shock (EQ), Nx = 32, Nxi = 6 x 4 (n = 1,536); 20 eigenvalues near 0.1i."""
    w = 5.0 * LAMBDA_INF_MM / DELTA_MM[1.2]
    return PencilSpec(nx=32, qx=6, qy=4, mach=1.2, base="tanh", noneq=0, width=w), EigsSpec(0.1j, 20, 40, 1)


def c2():
    """M = 3.0 Mott-Smith shock, Nx = 64, Nxi = 12 x 8 (n = 12,288); 40 eigenvalues near 0.1i."""
    return PencilSpec(nx=64, qx=12, qy=8, mach=3.0), EigsSpec(0.1j, 40, 80, 2)


def c3():
    """M = 4.0 Mott-Smith shock, Nx = 128, Nxi = 61 x 18 (n = 281,088); 40 eigenvalues near 0.05+0.2i, ncv 120.

    keep = 70: a restart keeps 70 of the 120 Schur vectors.  Among keep = 50, 60, 70, 80, 90, 100
    this took the least time per solve (34 restarts, 1,861 applies); keep = 50 did not converge
    within 200 restarts."""
    return PencilSpec(nx=128, qx=61, qy=18, mach=4.0), EigsSpec(0.05 + 0.2j, 40, 120, 3, keep=70)


def c3_paper_shape():
    """The paper's own 281,088-unknown shape: Nx = 61, 48 x 48, M = 4.0."""
    return PencilSpec(nx=61, qx=48, qy=48, mach=4.0), EigsSpec(0.05 + 0.2j, 40, 120, 3)


def tiny(nx=9, qx=4, qy=2, mach=3.0, **kw):
    """Small odd-shaped pencils for unit tests (QZ-sized)."""
    return PencilSpec(nx=nx, qx=qx, qy=qy, mach=mach, **kw)


def start_vector(n, seed):
    """Seeded complex start vector: i.i.d. N(0,1) real and imaginary parts (NumPy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def random_vectors(n, r, seed):
    """n x r seeded complex Gaussian block (column-major friendly: returned as (r, n))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n))


NX_SWEEP = (32, 48, 64, 96)
NXI_SWEEP = ((8, 6), (12, 8), (16, 12), (16, 16))


def sweep(npencils=256, seed=4):
    """Batched sweep: Mach ~ U[1.2, 4], beta ~ U[0, 2], Nx and (qx, qy) uniform over the lists,
    Mott-Smith NONEQ base, one shift sigma = 0.1i (1 + U[0, 1]) each, 20 eigenvalues."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(npencils):
        m = rng.uniform(1.2, 4.0)
        b = rng.uniform(0.0, 2.0)
        nx = NX_SWEEP[rng.integers(len(NX_SWEEP))]
        qx, qy = NXI_SWEEP[rng.integers(len(NXI_SWEEP))]
        sig = 0.1j * (1.0 + rng.uniform())
        out.append((PencilSpec(nx=nx, qx=qx, qy=qy, mach=m, beta=b), sig))
    return out


def _factor_q(nxi):
    """Nearest qx x qy >= 2 x 2 factorisation of nxi with qx >= qy and qx/qy <= 4."""
    best = None
    for qy in range(2, int(np.sqrt(nxi)) + 2):
        qx = max(qy, int(round(nxi / qy)))
        if qx > 4 * qy:
            continue
        err = abs(qx * qy - nxi)
        if best is None or err < best[0]:
            best = (err, qx, qy)
    return best[1], best[2]


def serving_requests(rate, duration_s, seed=5, n_min=1536, n_max=281088):
    """Poisson arrivals at ``rate``/s for ``duration_s``: list of (t_arrival, PencilSpec, sigma).

    Mach from {1.2, 3, 4}; n log-uniform in [n_min, n_max]; Nx the largest of
    {32, 64, 128} with n / (2 Nx) >= 24; Nxi = round(n / (2 Nx)) factorised
    as qx x qy; sigma = U[0, 0.2] + i U[0, 0.3]; 20 eigenvalues each.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration_s:
            break
        m = (1.2, 3.0, 4.0)[rng.integers(3)]
        n = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        nx = max(v for v in (32, 64, 128) if n / (2 * v) >= 24 or v == 32)
        qx, qy = _factor_q(max(4, int(round(n / (2 * nx)))))
        sig = rng.uniform(0.0, 0.2) + 1j * rng.uniform(0.0, 0.3)
        out.append((t, PencilSpec(nx=nx, qx=qx, qy=qy, mach=m), sig))
    return out


__all__ = ["PencilSpec", "EigsSpec", "c1", "c2", "c3", "c3_paper_shape", "tiny", "start_vector",
           "random_vectors", "sweep", "serving_requests", "re_delta", "replace"]
