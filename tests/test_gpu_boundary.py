"""The boundary's results on the GPU (needs a GB300): the tensor train exported
as device memory (Alg. 6's output: cores, Eq. 3, and nested sets, Eq. 4), the
per-interface ranks of a result, and the r0 seeded initial multi-indices,
each against the oracle."""
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


def test_exported_tensor_train_equals_oracle_cores():
    """After a run, the exported cores, read through their device pointers, are
    the oracle's cores A(I<=k-1, i_k, I>k) on the exported index sets."""
    p = inputs.make_problem("D", "cube", 6, 33, rank_cap=12)
    plan = B().Plan(p)
    res = plan.run()
    tt = plan.export_tt()
    assert tt.ranks == res["ranks"]
    d = p.d
    left = [np.zeros((1, 0), dtype=np.int64)]
    right = [np.zeros((0, d), dtype=np.int64)] * (d + 1)
    right[d] = np.zeros((1, 0), dtype=np.int64)
    cores = []
    for k in range(1, d + 1):
        c, lset, rset = tt.core(k)
        assert tuple(c.shape) == (res["ranks"][k - 1], p.N[k - 1], res["ranks"][k])
        cores.append(c.cpu().numpy())
        if k >= 2:
            assert np.array_equal(lset.cpu().numpy(), left[k - 1]), k
        if k <= d - 1:
            right[k] = rset.cpu().numpy().astype(np.int64)
            _, lnext, _ = tt.core(k + 1)
            left.append(lnext.cpu().numpy().astype(np.int64))
    st = ttcross.CrossState(left, right)
    # nested (Eq. 4): every row of I<=k extends a row of I<=k-1, every row of I>k one of I>k+1
    par = ttcross.to_parents(p, st)
    got = plan.get_state()
    for key in ("lpar", "lnode", "rpar", "rnode"):
        for a, b in zip(par[key], got[key]):
            assert np.array_equal(a, b), key
    scale = max(np.abs(c).max() for c in cores)
    for k in range(1, d + 1):
        ref = ttcross.core(p, st, k)
        assert np.all(np.abs(cores[k - 1] - ref) <= 1e-13 * np.abs(ref) + 1e-15 * scale), k
    # the handle outlives further use of the plan
    plan.run()
    c1, _, _ = tt.core(1)
    assert np.array_equal(c1.cpu().numpy(), cores[0])
    tt.close()


@pytest.mark.parametrize("r0", [1, 3, 6])
def test_initial_sets_match_oracle(r0):
    p = inputs.make_problem("D", "rn", 6, 49, L=12.0, rank_cap=14, r0=r0)
    plan = B().Plan(p)
    plan.init()
    got = plan.get_state()
    st = ttcross.initial_state(p)
    assert got["ranks"] == st.ranks()
    par = ttcross.to_parents(p, st)
    for key in ("lpar", "lnode", "rpar", "rnode"):
        for a, b in zip(par[key], got[key]):
            assert np.array_equal(a, b), (key, a, b)


@pytest.mark.parametrize("r0", [1, 4])
def test_run_with_r0_matches_oracle(r0):
    p = inputs.make_problem("D", "cube", 7, 33, rank_cap=12, r0=r0)
    ora = ttcross.integrate(p)
    got = B().integrate(p)
    assert abs(got["value"] - ora["value"]) <= 1e-12 * abs(ora["value"])
    assert (got["status"], got["sweeps"], got["n_eval"]) == (ora["status"], ora["sweeps"], ora["n_eval"])
    assert got["ranks"] == ora["ranks"]


def test_r0_beyond_the_initial_samples_is_rejected():
    p = inputs.make_problem("C", "rn", 4, 41, L=10.0, rank_cap=8, r0=9, init_samples=8)
    with pytest.raises(B().TTQError):
        B().Plan(p)


def test_plan_runs_after_a_plan_with_smaller_factors_was_made():
    """Kernel shared-memory limits are per function for the whole process: a
    plan made after another with smaller factors (rank cap 8) must not lower
    the limits the first plan's launches need (rank cap 64: the samples'
    factors alone take 64 KB).  Both run, in either order, and give the
    values they give alone."""
    big = inputs.make_problem("D", "rn", 8, 65, L=12.0, rank_cap=64, max_sweeps=6)
    small = inputs.make_problem("C", "rn", 4, 41, L=10.0, rank_cap=8)
    alone_big = B().Plan(big).run()
    alone_small = B().Plan(small).run()
    pb = B().Plan(big)
    ps = B().Plan(small)                         # made after the larger plan
    rb = pb.run()
    rs = ps.run()
    assert (rb["value"], rb["sweeps"], rb["n_eval"]) == (alone_big["value"], alone_big["sweeps"], alone_big["n_eval"])
    assert (rs["value"], rs["sweeps"], rs["n_eval"]) == (alone_small["value"], alone_small["sweeps"], alone_small["n_eval"])
