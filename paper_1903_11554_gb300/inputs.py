"""Seeded synthetic inputs for the TT-cross quadrature: 1-D rules, problem
records and workload mixes.

This module is shared by the CUDA path's binding, the tests, the bench and the
CPU oracle.  It holds none of the method's arithmetic (no integrand, no cross
step, no contraction): it only builds the per-mode quadrature nodes and weights
that the method takes as input (Sec. 4.1, Eq. 5), and the problem records
that name an integrand family (Sec. 5.1, Eqs. 9-11) and the stopping
parameters.

Grids:
  * trapezoid rule on the truncated line [-L, L] with N nodes, used by the
    s-in-R^n form of the Ising integrals (the R^n form is the one in which the
    C_n and D_n integrands are written as (sum_j 2 cosh s_j)^-2 times pair
    factors tanh^2((s_i - s_j)/2)); spacing h = 2L/(N-1), end weights h/2.
  * Gauss-Legendre rule mapped to [0, 1] (Sec. 5.2 uses tensor products of
    1-D Gauss-Legendre rules), taken from numpy's leggauss.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

FAMILIES = ("C", "D", "E", "TEST")
FORMS = ("rn", "cube")

# integer codes used across the C ABI (ttq_family / ttq_form in include/ttq.h)
FAMILY_CODE = {"C": 0, "D": 1, "E": 2, "TEST": 3}
FORM_CODE = {"rn": 0, "cube": 1}
PREC_CODE = {"fp64": 0, "dd": 1}


def trapezoid(L: float, N: int):
    """Nodes s_m = -L + m h (m = 0..N-1), h = 2L/(N-1); weights h, h/2 at ends."""
    if N < 2:
        raise ValueError("trapezoid rule needs N >= 2")
    h = 2.0 * L / (N - 1)
    s = np.array([-L + m * h for m in range(N)], dtype=np.float64)
    w = np.full(N, h, dtype=np.float64)
    w[0] = w[-1] = 0.5 * h
    return s, w


def gauss_legendre01(N: int):
    """Gauss-Legendre nodes and weights on [0, 1] (numpy leggauss, mapped)."""
    x, w = np.polynomial.legendre.leggauss(N)
    return 0.5 * (x + 1.0), 0.5 * w


@dataclasses.dataclass
class Problem:
    """One integral request: integrand family and n, per-mode 1-D rules and
    the cross parameters (rank cap, tolerance, sweeps, seed)."""
    family: str                 # "C", "D", "E" (Eqs. 9-11) or "TEST" (separable, exact rank n)
    form: str                   # "rn" (s in R^n, d = n) or "cube" ([0,1]^(n-1), d = n-1)
    n: int                      # Ising index (for TEST: number of separable terms)
    nodes: List[np.ndarray]     # d arrays of node values
    weights: List[np.ndarray]   # d arrays of weights
    rank_cap: int = 16
    tol: float = 1e-12          # relative internal convergence of the integral
    pivot_tol: float = 1e-14    # a pivot is kept when |E*| > pivot_tol * max|core entry|
    conv_window: int = 3        # sweeps in a row whose relative change must be <= tol
    max_sweeps: int = 0         # 0 -> rank_cap + 8
    seed: int = 1
    n_samples: int = 0          # random samples per interface; 0 -> N_k + N_{k+1}
    rook_max: int = 3           # column/row rounds of rook pivoting
    init_samples: int = 64      # random points scanned for the initial multi-indices
    r0: int = 1                 # initial multi-indices (rank of every interface before the first sweep)
    npiv: int = 1               # pivots an interface may add per sweep (1: Alg. 6 as printed)
    precision: str = "fp64"     # "fp64" or "dd" (double-double final contraction)
    name: str = ""

    @property
    def d(self) -> int:
        return len(self.nodes)

    @property
    def N(self) -> List[int]:
        return [len(x) for x in self.nodes]

    def sweeps_limit(self) -> int:
        return self.max_sweeps if self.max_sweeps > 0 else self.rank_cap + 8

    def samples_for(self, k: int) -> int:
        """Random samples for interface k (1-based, between modes k and k+1)."""
        if self.n_samples > 0:
            return self.n_samples
        return self.N[k - 1] + self.N[k]


def modes_for(family: str, form: str, n: int, d: Optional[int] = None) -> int:
    if family == "TEST":
        if d is None:
            raise ValueError("TEST family needs d")
        return d
    if form == "rn":
        if family == "E":
            raise ValueError("E_n is defined on the unit cube only")
        return n
    return n - 1


def make_problem(family: str, form: str, n: int, N: int, *, L: float = 20.0,
                 d: Optional[int] = None, **kw) -> Problem:
    """Same 1-D rule in every mode: trapezoid on [-L, L] for the R^n form,
    Gauss-Legendre on [0, 1] for the unit-cube form and the TEST family."""
    dd = modes_for(family, form, n, d)
    if dd < 1:
        raise ValueError("need at least one mode")
    if form == "rn" and family != "TEST":
        s, w = trapezoid(L, N)
    else:
        s, w = gauss_legendre01(N)
    return Problem(family=family, form=form, n=n, nodes=[s.copy() for _ in range(dd)],
                   weights=[w.copy() for _ in range(dd)], **kw)


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

def config_c4(**kw) -> Problem:
    """C_4 in R^4, trapezoid [-20,20] with 161 nodes/mode (h = 0.25), rank cap 16, tol 1e-12."""
    args = dict(rank_cap=16, tol=1e-12, seed=1, name="C4_rn_N161_r16")
    args.update(kw)
    return make_problem("C", "rn", 4, 161, L=20.0, **args)


def config_d12(**kw) -> Problem:
    """D_12 in R^12, trapezoid [-24,24] with 385 nodes/mode (h = 0.125), rank cap 64, tol 1e-12,
    seeded random initial index set (r0 = 1: the largest |A| of 64 seeded random points)."""
    args = dict(rank_cap=64, tol=1e-12, seed=12, name="D12_rn_N385_r64")
    args.update(kw)
    return make_problem("D", "rn", 12, 385, L=24.0, **args)


def config_d12_r4(**kw) -> Problem:
    """D_12 as config_d12 but from r0 = 4 seeded initial multi-indices, with the
    double-double final contraction: its final cross matrices are conditioned so
    that an FP64 contraction of them (LU or QR) is accurate to ~1e-11 only."""
    args = dict(r0=4, precision="dd", name="D12_rn_N385_r64_r0_4")
    args.update(kw)
    return config_d12(**args)


def config_d12_p4(**kw) -> Problem:
    """D_12 as config_d12 with up to four pivots per interface per sweep (the
    rank-adaptive variant; Alg. 6 adds one)."""
    args = dict(npiv=4, name="D12_rn_N385_r64_p4")
    args.update(kw)
    return config_d12(**args)


def config_e16(**kw) -> Problem:
    """E_16 on [0,1]^15, Gauss-Legendre 128 nodes/mode, rank cap 96, tol 1e-14,
    double-double final contraction."""
    args = dict(rank_cap=96, tol=1e-14, seed=16, precision="dd", name="E16_cube_N128_r96")
    args.update(kw)
    return make_problem("E", "cube", 16, 128, **args)


def config_d_cube(n: int, **kw) -> Problem:
    """D_n in the paper's unit-cube form (Eq. 10) with Gauss-Legendre 129 nodes per
    mode, the rule of the printed D_8, D_16 and D_32 values (Sec. 5.5, Fig. 7):
    D_8 at rank cap 64 (seed 8), D_16 at rank cap 80 (seed 16), D_32 at rank cap
    64 (seed 32), tol 1e-12."""
    caps = {8: 64, 16: 80, 32: 64}
    args = dict(rank_cap=caps.get(n, 64), tol=1e-12, seed=n, name="D%d_cube_N129" % n)
    args.update(kw)
    return make_problem("D", "cube", n, 129, **args)


def config_c_cube(n: int, **kw) -> Problem:
    """C_n in the paper's unit-cube form (Eq. 9) with Gauss-Legendre 33 nodes per
    mode (the rule of the paper's double-precision C_d runs, Sec. 5.3), rank cap
    40, tol 1e-13, seed n."""
    args = dict(rank_cap=40, tol=1e-13, seed=n, name="C%d_cube_N33" % n)
    args.update(kw)
    return make_problem("C", "cube", n, 33, **args)


def config_c_rn_grid(n: int, **kw) -> Problem:
    """C_n in R^n on the trapezoid rule over [-12, 12] with 65 nodes per mode
    (h = 0.375), rank cap 64, tol 1e-13, seed n: a grid whose exact tensor-product
    sum is known in closed form (the separable 1-D integral of the C integrand)."""
    args = dict(rank_cap=64, tol=1e-13, seed=n, name="C%d_rn_N65_L12" % n)
    args.update(kw)
    return make_problem("C", "rn", n, 65, L=12.0, **args)


def batched_mix(count: int = 256, seed: int = 256, *, n_lo: int = 4, n_hi: int = 24,
                node_choices=(65, 129, 257, 513), cap_choices=(8, 16, 32, 64, 128),
                tol: float = 1e-12) -> List[Problem]:
    """Mixed instances: family cyclic C/D/E, n ~ U{n_lo..n_hi}, N ~ U(node_choices),
    rank cap ~ U(cap_choices), per-instance seed seed + i.  C and D use the R^n
    trapezoid form for n <= 8 and the unit-cube Gauss-Legendre form above
    (the truncated-line trapezoid loses accuracy as n grows); E is unit-cube."""
    rng = np.random.default_rng(seed)
    out = []
    fams = ("C", "D", "E")
    for i in range(count):
        fam = fams[i % 3]
        n = int(rng.integers(n_lo, n_hi + 1))
        N = int(rng.choice(node_choices))
        cap = int(rng.choice(cap_choices))
        if fam in ("C", "D") and n <= 8:
            form, L = "rn", (20.0 if fam == "C" else 24.0)
        else:
            form, L = "cube", 0.0
        out.append(make_problem(fam, form, n, N, L=L, rank_cap=cap, tol=tol, seed=seed + i,
                                name="batch%d_%s%d_%s_N%d_r%d" % (i, fam, n, form, N, cap)))
    return out


def serving_stream(count: int = 10000, rate: float = 2000.0, seed: int = 2000, *,
                   n_lo: int = 4, n_hi: int = 32, node_choices=(129, 257, 513),
                   tol_lo: float = 1e-14, tol_hi: float = 1e-8, rank_cap: int = 64):
    """Poisson arrivals (mean `rate` per second) of mixed requests: family
    uniform over C/D/E, n ~ U{n_lo..n_hi}, tol log-uniform in [tol_lo, tol_hi],
    N ~ U(node_choices).  Returns (arrival_times_s, problems)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    probs = []
    for i in range(count):
        fam = ("C", "D", "E")[int(rng.integers(0, 3))]
        n = int(rng.integers(n_lo, n_hi + 1))
        N = int(rng.choice(node_choices))
        tol = float(10.0 ** rng.uniform(math.log10(tol_lo), math.log10(tol_hi)))
        if fam in ("C", "D") and n <= 8:
            form, L = "rn", (20.0 if fam == "C" else 24.0)
        else:
            form, L = "cube", 0.0
        probs.append(make_problem(fam, form, n, N, L=L, rank_cap=rank_cap, tol=tol,
                                  seed=seed + 1 + i, name="req%d" % i))
    return t, probs
