"""Failure statuses raised on the device and read by the host (needs a GB300).

Both failures are made on the host, through the problem's inputs or the stage
entry points: no kernel is broken and no GPU fault is involved.
  * TTQ_ERR_NONFINITE: a unit-cube E_n problem whose first mode has the node
    x = -1; the pair factor (1 - p) / (1 + p) with p = x_2 divides by zero
    there (Eq. 11), so the first sweep's core entries at that node are inf.
  * TTQ_ERR_SINGULAR: a zero quadrature weight makes every tensor entry that
    uses that node exactly zero; index sets that contain the node in their left
    part make every cross matrix A(I<=k, I>k) the zero matrix, whose QR has
    R_00 = 0 exactly.
In both cases the plan, and the CUDA context, stay usable afterwards.
"""
import numpy as np
import pytest

from oracle import ttcross
from paper_1903_11554_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_11554_gb300 import build
    build.build()


def B():
    from paper_1903_11554_gb300 import binding
    return binding


def test_nonfinite_integrand_is_reported():
    p = inputs.make_problem("E", "cube", 6, 17, rank_cap=8)
    p.nodes[0] = p.nodes[0].copy()
    p.nodes[0][3] = -1.0
    plan = B().Plan(p)
    r = plan.run()
    assert r["status_name"] == "nonfinite", r
    assert plan.run() == r                      # the same plan runs again, same outcome
    # the context is intact: a valid problem still matches the oracle
    q = inputs.make_problem("E", "cube", 6, 17, rank_cap=8)
    got = B().integrate(q)
    ref = ttcross.integrate(q)
    assert abs(got["value"] - ref["value"]) <= 1e-12 * abs(ref["value"])


def _state_through_node(p, node):
    """Rank-1 nested sets built from one multi-index whose first coordinate is `node`."""
    d = p.d
    x = [node] + [p.N[k] // 2 for k in range(1, d)]
    lpar = [[0] for _ in range(d - 1)]
    lnode = [[x[k - 1]] for k in range(1, d)]
    rpar = [[0] for _ in range(d - 1)]
    rnode = [[x[k]] for k in range(1, d)]
    return [1] * (d + 1), lpar, lnode, rpar, rnode


def test_singular_cross_matrix_is_reported():
    p = inputs.make_problem("C", "rn", 4, 41, L=10.0, rank_cap=8)
    p.weights[0] = p.weights[0].copy()
    p.weights[0][5] = 0.0
    plan = B().Plan(p)
    plan.set_state(*_state_through_node(p, 5))
    with pytest.raises(B().TTQError, match="singular"):
        plan.sweep(0, search=False)
    # the same plan with a valid state contracts the oracle's integral
    ranks, lpar, lnode, rpar, rnode = _state_through_node(p, 6)
    plan.set_state(ranks, lpar, lnode, rpar, rnode)
    value, _, _ = plan.sweep(0, search=False)
    st = ttcross.from_parents(p, [np.array(a) for a in lpar], [np.array(a) for a in lnode],
                              [np.array(a) for a in rpar], [np.array(a) for a in rnode])
    cores = [ttcross.core(p, st, k) for k in range(1, p.d + 1)]
    ref = ttcross.integral_plain(p, st, cores)
    assert abs(value - ref) <= 1e-12 * abs(ref)
