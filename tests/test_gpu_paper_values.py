"""The paper's own values and the double-double bar, on the GPU (needs a GB300).

  * D_8, D_16 and D_32 in the paper's unit-cube form (Eq. 10) with
    Gauss-Legendre 129 nodes per mode: the printed values of Sec. 5.5 (Fig. 7)
    to 5e-12, and for D_8 and D_16 the stored oracle runs of the same problems
    (tests/golden/oracle_full.json, written by
    tests/golden/make_oracle_values.py) to 1e-12.
  * E_16 at full size (d = 15, Gauss-Legendre 128, rank cap 96, tol 1e-14)
    with the double-double final contraction: value + value_lo against a
    60-digit decimal contraction of the GPU's own final cores (the product of
    2d-1 matrices of Sec. 4.1, read back through the C ABI) to 1e-15, and the
    FP64 oracle's value to 1e-12.
  * C_8 in R^n on a trapezoid grid against the exact tensor-product sum of
    that grid (tests/golden/c_grid_exact.json, from the separable 1-D integral
    of the C integrand evaluated at 40 digits by
    tests/golden/make_c_grid_values.py), within ten times the oracle's own
    error on the same problem.  (From n = 16 on such grids the cross, the
    oracle's as much as the GPU's, reaches the rounding floor: the R^n
    integrand is symmetric in its variables, so a permuted copy of a cross row
    has a zero residual in exact arithmetic and only rounding can select it;
    once selected, the cross matrix has two equal rows and the run stops with
    a singular cross matrix, as the oracle's LU does on C_24.)
  * C_8 .. C_32 in the paper's unit-cube form (Eq. 9, Gauss-Legendre 33): the
    stored oracle runs to 1e-12, and the trend of Sec. 5.3: C_n decreases
    towards C_inf = 2 exp(-2 gamma) from above.
"""
import json
import os
from decimal import Decimal

import numpy as np
import pytest

from oracle import ttcross
from paper_1903_11554_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_11554_gb300 import build
    build.build()


def B():
    from paper_1903_11554_gb300 import binding
    return binding


def golden(name):
    return json.load(open(os.path.join(GOLDEN, "oracle_full.json")))[name]


def printed(name):
    return float(json.load(open(os.path.join(GOLDEN, "paper_values.json")))[name]["value"])


@pytest.mark.parametrize("n", [8, 16])
def test_d_printed_values(n):
    p = inputs.config_d_cube(n)
    got = B().integrate(p)
    assert got["status_name"] == "converged", got
    ref = printed("D_%d" % n)
    assert abs(got["value"] / ref - 1) < 5e-12, (got["value"], ref)
    ora = float(golden("d%d" % n)["value"])
    assert abs(got["value"] / ora - 1) < 1e-12, (got["value"], ora)
    print("D_%d: GPU %.17e, printed rel %.2e, oracle rel %.2e"
          % (n, got["value"], abs(got["value"] / ref - 1), abs(got["value"] / ora - 1)))


def test_d32_printed_value():
    """D_32 (d = 31, the largest printed D_d within the library's d <= 32): the
    cross converges (tol 1e-12, rank 47 of cap 64) and its value meets the
    printed one; there is no stored oracle run of it (hours in the numpy
    oracle), the printed value is the pin."""
    p = inputs.config_d_cube(32)
    got = B().integrate(p)
    assert got["status_name"] == "converged", got
    ref = printed("D_32")
    err = abs(got["value"] / ref - 1)
    print("D_32: GPU %.17e, printed rel %.2e, rank %d, sweeps %d" % (got["value"], err, got["max_rank"], got["sweeps"]))
    assert err < 5e-12, (got["value"], ref)


def test_e16_double_double_at_full_size():
    p = inputs.config_e16()
    plan = B().Plan(p)
    got = plan.run()
    state = plan.get_state()
    ranks = state["ranks"]
    st = ttcross.from_parents(p, state["lpar"], state["lnode"], state["rpar"], state["rnode"])
    assert st.ranks() == ranks
    cores = [plan.get_core(k, (ranks[k - 1], p.N[k - 1], ranks[k])) for k in range(1, p.d + 1)]
    ref = ttcross.contract_decimal(p, st, cores, as_decimal=True)
    dd = Decimal(got["value"]) + Decimal(got["value_lo"])
    err_dd = abs(dd - ref) / abs(ref)
    ora = float(golden("e16")["value"])
    err_oracle = abs(got["value"] - ora) / abs(ora)
    print("E_16: GPU hi %.17e lo %.3e; vs 60-digit contraction of its cores %.2e; vs FP64 oracle %.2e; ranks %s"
          % (got["value"], got["value_lo"], float(err_dd), err_oracle, max(ranks)))
    assert err_dd < Decimal("1e-15"), float(err_dd)
    assert err_oracle < 1e-12


def c_grid_values():
    return json.load(open(os.path.join(GOLDEN, "c_grid_exact.json")))


@pytest.mark.parametrize("n", [8])
def test_c_n_against_exact_grid_value(n):
    entry = c_grid_values()[str(n)]
    p = inputs.config_c_rn_grid(n)
    assert p.name == entry["workload"]
    got = B().integrate(p)
    ref = float(entry["value"])
    err = abs(got["value"] / ref - 1)
    print("C_%d: GPU %.17e, exact grid %.17e, rel %.2e, ranks %d, sweeps %d, status %s"
          % (n, got["value"], ref, err, got["max_rank"], got["sweeps"], got["status_name"]))
    assert err < entry["tolerance"], (err, entry["tolerance"])


def test_c_n_cube_towards_c_infinity():
    from oracle import exact
    c_inf = exact.c_inf()
    prev = None
    for n in (8, 16, 24, 32):
        got = B().integrate(inputs.config_c_cube(n))
        ora = float(golden("c%d_cube" % n)["value"])
        assert abs(got["value"] / ora - 1) < 1e-12, (n, got["value"], ora)
        gap = got["value"] - c_inf
        print("C_%d (unit cube, GL 33): GPU %.17e, oracle rel %.2e, C_n - C_inf %.3e"
              % (n, got["value"], abs(got["value"] / ora - 1), gap))
        assert gap > 0
        if prev is not None:
            assert gap < prev
        prev = gap
