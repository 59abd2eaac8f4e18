"""Closed forms and exact grid values used to pin the oracle.

Closed forms of the Ising-class integrals (values from the literature the
paper builds on, Sec. 5.1; the paper quotes C_inf = 2 exp(-2 gamma)):
    C_1 = 2, C_2 = 1, C_4 = 7 zeta(3) / 12,
    D_2 = 1/3, D_4 = 4 pi^2 / 9 - 1/6 - 7 zeta(3) / 2,
    E_2 = 6 - 8 ln 2.

Exact grid value of C_n in the R^n form (not in the paper; follows from
1/S^2 = int_0^inf t exp(-t S) dt with S = sum_k 2 cosh s_k > 0, which makes
the tensor-product sum separable):
    sum_{i_1..i_n} prod_k w_{k,i_k} (sum_k 2 cosh s_{k,i_k})^-2
        = int_0^inf t prod_k phi_k(t) dt,   phi_k(t) = sum_i w_{k,i} exp(-2 t cosh s_{k,i}).
The 1-D integral is evaluated with mpmath at 40 digits.
"""
from __future__ import annotations

import math


def closed_forms():
    z3 = 1.2020569031595942853997381615114499907649862923405  # zeta(3)
    return {
        ("C", 1): 2.0,
        ("C", 2): 1.0,
        ("C", 4): 7.0 * z3 / 12.0,
        ("D", 2): 1.0 / 3.0,
        ("D", 4): 4.0 * math.pi ** 2 / 9.0 - 1.0 / 6.0 - 7.0 * z3 / 2.0,
        ("E", 2): 6.0 - 8.0 * math.log(2.0),
    }


def c_inf() -> float:
    """Limit of C_n as n -> infinity, 2 exp(-2 gamma) (Sec. 5.3)."""
    gamma = 0.57721566490153286060651209008240243104215933593992
    return 2.0 * math.exp(-2.0 * gamma)


def c_grid_exact(nodes, weights, dps: int = 40) -> float:
    """Exact tensor-product sum of prod w (sum 2cosh s)^-2 over the given
    per-mode rules (no family constant), via the separable 1-D integral."""
    import mpmath as mp
    mp.mp.dps = dps
    tabs = []
    for s, w in zip(nodes, weights):
        tabs.append([(mp.mpf(float(wi)), 2 * mp.cosh(mp.mpf(float(si)))) for si, wi in zip(s, w)])
    cmin = min(min(c for _, c in t) for t in tabs)

    def F(t):
        val = t
        for tab in tabs:
            val *= mp.fsum(wi * mp.exp(-t * c) for wi, c in tab)
        return val

    # integrand decays like exp(-t * n * cmin); split the range for the quadrature
    scale = 1 / (len(tabs) * cmin)
    pts = [0, scale / 8, scale / 2, scale, 4 * scale, 16 * scale, 64 * scale, mp.inf]
    return float(mp.quad(F, pts))
