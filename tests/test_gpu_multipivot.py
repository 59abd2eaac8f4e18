"""Several pivots per interface per sweep on the GPU against the oracle's
pivot_search_multi (needs a GB300).

  * sweep by sweep from the oracle's initial set: the integral within 1e-12
    and the nested sets after every sweep identical (the accepted pivots, their
    order and count);
  * whole runs: status, sweeps, evaluations and final ranks equal, value within
    1e-12; the D_12 workload with four pivots per sweep at full size against
    its stored oracle run;
  * D_8 in the unit-cube form with four pivots per sweep against its printed
    value (Sec. 5.5, Fig. 7);
  * the modes that take one pivot per sweep refuse a problem with several.
"""
import json
import os

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


def rel(a, b):
    return abs(a - b) / abs(b)


CASES = {
    "C_rn_3": lambda: inputs.make_problem("C", "rn", 5, 41, L=10.0, rank_cap=14, npiv=3),
    "D_rn_4": lambda: inputs.make_problem("D", "rn", 6, 49, L=12.0, rank_cap=16, npiv=4),
    "D_cube_2": lambda: inputs.make_problem("D", "cube", 7, 33, rank_cap=16, npiv=2),
    "E_cube_4": lambda: inputs.make_problem("E", "cube", 9, 33, rank_cap=16, npiv=4),
    "E_cube_3_r0_2_dd": lambda: inputs.make_problem("E", "cube", 7, 33, rank_cap=14, npiv=3, r0=2, precision="dd"),
}


def same_sets(p, got, st):
    par = ttcross.to_parents(p, st)
    if got["ranks"] != st.ranks():
        return False
    return all(np.array_equal(a, b) for key in ("lpar", "lnode", "rpar", "rnode") for a, b in zip(par[key], got[key]))


@pytest.mark.parametrize("case", sorted(CASES))
def test_sweep_by_sweep_sets(case):
    p = CASES[case]()
    st = ttcross.initial_state(p)
    par = ttcross.to_parents(p, st)
    plan = B().Plan(p)
    plan.set_state(st.ranks(), par["lpar"], par["lnode"], par["rpar"], par["rnode"])
    multi = 0
    for s in range(6):
        value, _, _ = plan.sweep(s, search=True)
        val_o, _, _, piv_o = ttcross.sweep(p, st, s, search=True)
        assert rel(value, val_o) < 1e-12, s
        multi += sum(1 for mp in piv_o if mp is not None and len(mp.pivots) > 1)
        st = ttcross.apply_pivots(p, st, piv_o)
        assert same_sets(p, plan.get_state(), st), s
    assert multi > 0                             # some interface took several pivots


@pytest.mark.parametrize("case", sorted(CASES))
def test_full_run_matches_oracle(case):
    p = CASES[case]()
    ora = ttcross.integrate(p)
    got = B().integrate(p)
    assert (got["status"], got["sweeps"], got["n_eval"], got["ranks"]) == \
        (ora["status"], ora["sweeps"], ora["n_eval"], ora["ranks"]), (got, ora["sweeps"], ora["n_eval"])
    assert rel(got["value"], ora["value"]) < 1e-12


def test_d8_printed_value_with_four_pivots():
    p = inputs.config_d_cube(8, npiv=4)
    got = B().integrate(p)
    ora = ttcross.integrate(p)
    ref = float(json.load(open(os.path.join(GOLDEN, "paper_values.json")))["D_8"]["value"])
    assert got["status_name"] == "converged"
    assert got["sweeps"] == ora["sweeps"]
    assert rel(got["value"], ora["value"]) < 1e-12
    assert rel(got["value"], ref) < 5e-12
    print("D_8, four pivots per sweep: %d sweeps (one pivot: 29), rank %d, printed rel %.2e"
          % (got["sweeps"], got["max_rank"], rel(got["value"], ref)))


def test_d12_four_pivots_full_size():
    """The D_12 workload with up to four pivots per sweep at full size against
    the stored oracle run (tests/golden/oracle_full.json, "d12_p4"): the same
    sweeps, evaluations and final nested sets, the value within 1e-12 of the
    oracle's and of its 60-digit contraction of the oracle's final cores."""
    g = json.load(open(os.path.join(GOLDEN, "oracle_full.json")))["d12_p4"]
    p = inputs.config_d12_p4()
    plan = B().Plan(p)
    got = plan.run()
    assert (got["status"], got["sweeps"], got["n_eval"], got["ranks"]) == (g["status"], g["sweeps"], g["n_eval"], g["ranks"])
    st = plan.get_state()
    for key in ("lpar", "lnode", "rpar", "rnode"):
        for a, b in zip(st[key], g["parents"][key]):
            assert list(map(int, a)) == b, key
    assert rel(got["value"], float(g["value"])) < 1e-12
    assert rel(got["value"], float(g["value_exact_contraction"])) < 1e-12
    print("D_12, four pivots: %d sweeps (one pivot: 64), value rel %.2e to the oracle"
          % (got["sweeps"], rel(got["value"], float(g["value"]))))


def test_one_pivot_modes_refuse_several():
    p = inputs.make_problem("C", "rn", 4, 33, L=8.0, rank_cap=8, npiv=2)
    with pytest.raises(B().TTQError):
        B().Batch([p, p])
    plan = B().Plan(p)
    with pytest.raises(B().TTQError):
        plan.set_sequential(True)
    with pytest.raises(B().TTQError):
        plan.set_search(persistent=True)
    srv = B().Server(1 << 26)
    with pytest.raises(B().TTQError):
        srv.submit(p)
