"""GPU path vs the CPU oracle at the edges of the problem space and at the full
sizes of the bench workloads (needs a GB300).

  * full size: the D_12 and C_4 runs equal the stored oracle runs
    (tests/golden/oracle_full.json, written by make_oracle_values.py from the
    oracle alone): value to 1e-12, and status, sweeps, evaluation count and the
    final nested index sets exactly; E_16 (tolerance 1e-14, so its last sweeps
    sit at the rounding floor where rounding picks the path) to 1e-12 in value;
  * d = 2 (one interface, the sets of both sides are a single mode each) and a
    rank cap of 1 (the run stops at once, no search);
  * the largest shapes the library accepts: d = 32, N = 2048 nodes per mode,
    rank cap 128 — entries at random points, and three sweeps of the cross.
"""
import json
import os

import numpy as np
import pytest

from oracle import integrands, ttcross
from paper_1903_11554_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_full.json")


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


@pytest.mark.parametrize("name", ["c4", "d12", "d12_r4"])
def test_full_size_run_equals_stored_oracle_run(name):
    """Same run as the stored oracle run: status, sweeps, evaluations and the
    final nested sets exactly; the value to 1e-12 of the oracle's 60-digit
    contraction of its own final cores and, in FP64 mode, of its FP64 value.
    (D_12 from r0 = 4 initial multi-indices ends on cross matrices whose FP64
    contraction, the oracle's LU as much as a QR, is good to ~1e-11 only, so
    that workload runs the double-double final contraction.)"""
    ref = json.load(open(GOLDEN))[name]
    p = {"c4": inputs.config_c4, "d12": inputs.config_d12, "d12_r4": inputs.config_d12_r4}[name]()
    plan = B().Plan(p)
    got = plan.run()
    exact = float(ref["value_exact_contraction"])
    value = got["value"] + got["value_lo"]
    print("%s: GPU %.17e (+%.3e), oracle FP64 %s (rel %.2e), oracle cores at 60 digits %.17e (rel %.2e)"
          % (name, got["value"], got["value_lo"], ref["value"], rel(value, float(ref["value"])), exact,
             rel(value, exact)))
    assert rel(value, exact) < 1e-12
    if p.precision == "fp64":
        assert rel(got["value"], float(ref["value"])) < 1e-12
    assert (got["status"], got["sweeps"], got["n_eval"]) == (ref["status"], ref["sweeps"], ref["n_eval"])
    st = plan.get_state()
    assert st["ranks"] == ref["ranks"]
    for key in ("lpar", "lnode", "rpar", "rnode"):
        assert [list(map(int, a)) for a in st[key]] == ref["parents"][key], key


def test_full_size_e16_value_equals_stored_oracle_value():
    ref = json.load(open(GOLDEN))["e16"]
    got = B().integrate(inputs.config_e16())
    assert rel(got["value"], float(ref["value"])) < 1e-12


EDGE = {
    "C2_rn": lambda: inputs.make_problem("C", "rn", 2, 41, L=10.0, rank_cap=8),
    "D2_rn": lambda: inputs.make_problem("D", "rn", 2, 41, L=10.0, rank_cap=8),
    "E3_cube": lambda: inputs.make_problem("E", "cube", 3, 33, rank_cap=8),
    "cap1_C5": lambda: inputs.make_problem("C", "rn", 5, 41, L=10.0, rank_cap=1),
    "cap1_E6": lambda: inputs.make_problem("E", "cube", 6, 17, rank_cap=1),
}


@pytest.mark.parametrize("case", sorted(EDGE))
def test_edge_shapes_match_oracle(case):
    p = EDGE[case]()
    ora = ttcross.integrate(p)
    got = B().integrate(p)
    assert rel(got["value"], ora["value"]) < 1e-12
    assert (got["status"], got["sweeps"], got["n_eval"], got["max_rank"]) == \
        (ora["status"], ora["sweeps"], ora["n_eval"], ora["max_rank"])


MAXIMAL = {
    "D32_rn_N2048": lambda: inputs.make_problem("D", "rn", 32, 2048, L=20.0, rank_cap=128, max_sweeps=3),
    "E33_cube_N2048": lambda: inputs.make_problem("E", "cube", 33, 2048, rank_cap=128, max_sweeps=3),
}


@pytest.mark.parametrize("case", sorted(MAXIMAL))
def test_largest_shapes_entries(case):
    p = MAXIMAL[case]()
    assert p.d == 32 and max(p.N) == 2048
    plan = B().Plan(p)
    g = np.random.default_rng(5)
    idx = np.stack([g.integers(0, N, 2000) for N in p.N], axis=1).astype(np.int32)
    idx[0] = 0                                   # the grid's corners
    idx[1] = np.array(p.N) - 1
    got = plan.eval_points(torch.from_numpy(idx)).cpu().numpy()
    ref = integrands.tensor_entries(p, idx)
    scale = np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(ref) + 1e-15 * scale)


@pytest.mark.parametrize("case", sorted(MAXIMAL))
def test_largest_shapes_three_sweeps(case):
    p = MAXIMAL[case]()
    ora = ttcross.integrate(p)
    got = B().integrate(p)
    assert rel(got["value"], ora["value"]) < 1e-12
    assert (got["status"], got["sweeps"], got["n_eval"], got["max_rank"]) == \
        (ora["status"], ora["sweeps"], ora["n_eval"], ora["max_rank"])
