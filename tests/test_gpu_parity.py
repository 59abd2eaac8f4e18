"""GPU path vs the CPU oracle, through the C ABI (needs a GB300).

Tolerances:
  * integrand entries: |gpu - oracle| <= 1e-13 |oracle| + 1e-15 max|A|
    (both sides round a product of <= n(n-1)/2 + 2n + 3 factors; the unit-cube
    pair factors 1 - x_{i+1}..x_j lose relative accuracy near x = 1, where the
    entries themselves are tiny, hence the absolute term);
  * integrals: 1e-12 relative (FP64), 1e-15 relative for the double-double
    contraction against an exact rational contraction of the same cores.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import integrands, ttcross
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


def rel(a, b):
    return abs(a - b) / abs(b)


CASES = {
    "C_rn": lambda: inputs.make_problem("C", "rn", 5, 41, L=10.0, rank_cap=10),
    "D_rn_uniform": lambda: inputs.make_problem("D", "rn", 6, 49, L=12.0, rank_cap=10),
    "D_rn_generic": lambda: inputs.make_problem("D", "rn", 5, 41, L=10.0 * 0.97, rank_cap=10),
    "C_cube": lambda: inputs.make_problem("C", "cube", 7, 33, rank_cap=12),
    "D_cube": lambda: inputs.make_problem("D", "cube", 7, 33, rank_cap=12),
    "E_cube": lambda: inputs.make_problem("E", "cube", 9, 33, rank_cap=12),
    "TEST": lambda: inputs.make_problem("TEST", "cube", 4, 17, d=6, rank_cap=8),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_eval_points_match_oracle(case):
    p = CASES[case]()
    plan = B().Plan(p)
    g = np.random.default_rng(11)
    idx = np.stack([g.integers(0, N, 4000) for N in p.N], axis=1).astype(np.int32)
    got = plan.eval_points(torch.from_numpy(idx)).cpu().numpy()
    ref = integrands.tensor_entries(p, idx)
    scale = np.abs(ref).max()
    err = np.abs(got - ref)
    assert np.all(err <= 1e-13 * np.abs(ref) + 1e-15 * scale), (case, np.max(err / (np.abs(ref) + scale * 1e-2)))


def oracle_state_after(p, sweeps):
    q = inputs.Problem(**{**p.__dict__, "max_sweeps": sweeps})
    return ttcross.integrate(q)["state"]


@pytest.mark.parametrize("case", ["C_rn", "D_rn_uniform", "D_cube", "E_cube"])
def test_replay_cores_and_integral(case):
    """Fed the oracle's index sets, the GPU evaluates the same cores and
    contracts the same integral."""
    p = CASES[case]()
    st = oracle_state_after(p, 6)
    par = ttcross.to_parents(p, st)
    plan = B().Plan(p)
    plan.set_state(st.ranks(), par["lpar"], par["lnode"], par["rpar"], par["rnode"])
    value, _, _ = plan.sweep(0, search=False)
    cores = [ttcross.core(p, st, k) for k in range(1, p.d + 1)]
    scale = max(np.abs(c).max() for c in cores)
    for k in range(1, p.d + 1):
        got = plan.get_core(k, cores[k - 1].shape)
        assert np.all(np.abs(got - cores[k - 1]) <= 1e-13 * np.abs(cores[k - 1]) + 1e-15 * scale), k
    ref = ttcross.integral_plain(p, st, cores)
    assert rel(value, ref) < 1e-12


@pytest.mark.parametrize("case", ["C_rn", "D_rn_uniform", "D_cube", "E_cube", "TEST"])
def test_one_sweep_pivots_match(case):
    """Same state, same sweep index: Alg. 2 on every interface picks the same
    pivots as the oracle, with the same residual."""
    p = CASES[case]()
    st = oracle_state_after(p, 4)
    par = ttcross.to_parents(p, st)
    plan = B().Plan(p)
    plan.set_state(st.ranks(), par["lpar"], par["lnode"], par["rpar"], par["rnode"])
    s = 3
    value, _, piv = plan.sweep(s, search=True)
    val_o, cores, scale, piv_o = ttcross.sweep(p, st, s, search=True)
    for g, o in zip(piv, piv_o):
        if o is None:
            assert not g["searched"]
            continue
        assert (g["row"], g["col"], g["rounds"], bool(g["accepted"]), g["evals"]) == \
            (o.row, o.col, o.rounds, o.accepted, o.evals), (g, o)
        assert abs(g["err"] - o.err) <= 1e-13 * scale
    # the appended sets equal the oracle's
    new_o = ttcross.apply_pivots(p, st, piv_o)
    got = plan.get_state()
    assert got["ranks"] == new_o.ranks()
    par_o = ttcross.to_parents(p, new_o)
    for key in ("lpar", "lnode", "rpar", "rnode"):
        for a, b in zip(got[key], par_o[key]):
            assert np.array_equal(a, b), key


FULL = {
    "C_rn": lambda: inputs.make_problem("C", "rn", 4, 41, L=10.0, rank_cap=12),
    "D_rn": lambda: inputs.make_problem("D", "rn", 5, 33, L=8.0, rank_cap=12),
    "C_cube": lambda: inputs.make_problem("C", "cube", 6, 33, rank_cap=30),
    "D_cube": lambda: inputs.make_problem("D", "cube", 6, 33, rank_cap=30),
    "E_cube": lambda: inputs.make_problem("E", "cube", 6, 33, rank_cap=30),
    "TEST": lambda: inputs.make_problem("TEST", "cube", 5, 33, d=6, rank_cap=10),
    "C4_config": lambda: inputs.config_c4(),
}


def first_divergence(p, ora):
    """Step the GPU from the oracle's initial set, sweep by sweep on its own
    state (as a run does: bordered QR factors), and compare every search with
    the oracle's record.  Return the first sweep where an interface's pivot,
    round count or evaluation count differ, with that interface's |E*| / scale
    on the oracle's side (None if nothing differs)."""
    st = ttcross.initial_state(p)
    plan = B().Plan(p)
    par = ttcross.to_parents(p, st)
    plan.set_state(st.ranks(), par["lpar"], par["lnode"], par["rpar"], par["rnode"])
    for s, h in enumerate(ora["history"]):
        if not h.pivots:
            break
        _, _, piv = plan.sweep(s, search=True)
        for g, o in zip(piv, h.pivots):
            if o is not None and (g["row"], g["col"], g["rounds"], g["evals"]) != (o.row, o.col, o.rounds, o.evals):
                return s, abs(o.err) / h.scale
    return None


@pytest.mark.parametrize("case", sorted(FULL))
def test_full_run_matches_oracle(case):
    """Whole runs agree to 1e-12.  The searches are identical except where an
    interface has reached the rounding floor (its pivot residual below 1e-12
    of the largest entry): there rounding decides the rook path (several
    pivots, or several paths to one pivot, are equally valid), so the pivot,
    the number of evaluations and the run's length may differ."""
    p = FULL[case]()
    ora = ttcross.integrate(p)
    got = B().integrate(p)
    assert got["status"] == ora["status"]
    assert rel(got["value"], ora["value"]) < 1e-12
    same = (got["sweeps"], got["max_rank"], got["n_eval"]) == (ora["sweeps"], ora["max_rank"], ora["n_eval"])
    if not same:
        div = first_divergence(p, ora)
        assert div is not None
        s, floor = div
        assert floor < 1e-12, (s, floor)


@pytest.mark.parametrize("case", ["C_rn", "D_rn", "E_cube"])
def test_sweep_by_sweep_trajectory(case):
    """Step both sides sweep by sweep from the same initial set: at every sweep
    the integral, the pivots and the evaluation counts agree."""
    p = FULL[case]()
    st = ttcross.initial_state(p)
    par = ttcross.to_parents(p, st)
    plan = B().Plan(p)
    plan.set_state(st.ranks(), par["lpar"], par["lnode"], par["rpar"], par["rnode"])
    for s in range(8):
        value, _, piv = plan.sweep(s, search=True)
        val_o, _, scale, piv_o = ttcross.sweep(p, st, s, search=True)
        assert rel(value, val_o) < 1e-12, s
        for g, o in zip(piv, piv_o):
            if o is None:
                continue
            assert (g["row"], g["col"], g["rounds"], g["evals"]) == (o.row, o.col, o.rounds, o.evals), (s, g, o)
        st = ttcross.apply_pivots(p, st, piv_o)


def test_runs_are_bitwise_reproducible():
    p = FULL["D_cube"]()
    a = B().integrate(p)
    b = B().integrate(p)
    assert a == b


def test_exact_recovery_on_gpu():
    """Thm. 2 on the GPU: the separable rank-n tensor's integral is exact."""
    p = inputs.make_problem("TEST", "cube", 5, 65, d=8, rank_cap=12)
    got = B().integrate(p)
    ex = 0.0
    for t in range(1, 6):
        pr = 1.0
        for k in range(8):
            pr *= float(np.sum(p.weights[k] * np.exp(-t * p.nodes[k] / 8)))
        ex += pr
    assert rel(got["value"], ex) < 1e-13
    assert got["max_rank"] == 5


def exact_contraction(p, st, cores):
    """V_1 G_1^-1 V_2 ... V_d in exact rationals from the given FP64 cores."""
    def inv_apply(G, x):   # x G^-1 by exact Gauss-Jordan on G^T
        n = len(x)
        A = [[Fraction(float(G[j, i])) for j in range(n)] + [x[i]] for i in range(n)]  # rows: G^T | x
        for c in range(n):
            piv = next(r for r in range(c, n) if A[r][c] != 0)
            A[c], A[piv] = A[piv], A[c]
            for r in range(n):
                if r != c and A[r][c] != 0:
                    f = A[r][c] / A[c][c]
                    A[r] = [a - f * b for a, b in zip(A[r], A[c])]
        return [A[i][n] / A[i][i] for i in range(n)]

    def vsum(T):
        r0, N, r1 = T.shape
        return [[sum((Fraction(float(T[a, i, b])) for i in range(N)), Fraction(0)) for b in range(r1)]
                for a in range(r0)]

    x = vsum(cores[0])[0]
    for k in range(1, p.d):
        G = cores[k - 1].reshape(-1, st.rank(k))[ttcross.cross_rows(p, st, k), :]
        x = inv_apply(G, x)
        V = vsum(cores[k])
        x = [sum((x[a] * V[a][b] for a in range(len(x))), Fraction(0)) for b in range(len(V[0]))]
    return x[0] * Fraction(integrands.family_constant(p.family, p.form, p.n))


def test_double_double_contraction_vs_exact():
    p = inputs.make_problem("E", "cube", 6, 17, rank_cap=6, max_sweeps=6, precision="dd")
    st = oracle_state_after(p, 6)
    par = ttcross.to_parents(p, st)
    plan = B().Plan(p)
    plan.set_state(st.ranks(), par["lpar"], par["lnode"], par["rpar"], par["rnode"])
    hi, lo, _ = plan.sweep(0, search=False)
    cores = [plan.get_core(k, (st.rank(k - 1), p.N[k - 1], st.rank(k))) for k in range(1, p.d + 1)]
    ex = exact_contraction(p, st, cores)
    err = abs(Fraction(hi) + Fraction(lo) - ex) / abs(ex)
    assert float(err) < 1e-15
    p64 = inputs.Problem(**{**p.__dict__, "precision": "fp64"})
    plan64 = B().Plan(p64)
    plan64.set_state(st.ranks(), par["lpar"], par["lnode"], par["rpar"], par["rnode"])
    v64, lo64, _ = plan64.sweep(0, search=False)
    assert lo64 == 0.0
    assert float(abs(Fraction(v64) - ex) / abs(ex)) < 1e-13


def test_async_launch_matches_run():
    """ttq_plan_launch / ttq_plan_result (several runs enqueued back to back,
    results read afterwards) give exactly what ttq_plan_run gives."""
    p = FULL["E_cube"]()
    plan = B().Plan(p)
    ref = plan.run()
    for slot in range(3):
        plan.launch(slot)
    for slot in range(3):
        assert plan.result(slot) == ref


def test_plain_launches_match_graph():
    p = FULL["D_rn"]()
    plan = B().Plan(p)
    a = plan.run()
    plan.set_graphs(False)
    b = plan.run()
    assert a == b


@pytest.mark.parametrize("case", ["C_rn", "D_rn", "D_cube", "E_cube", "TEST", "C4_config"])
def test_persistent_search_equals_staged_search(case):
    """The search as one persistent cooperative launch (interface groups handing
    stages on through device flags) and as separate launches per stage give the
    same run bit for bit."""
    p = FULL[case]()
    plan = B().Plan(p)
    plan.set_search(True)
    a = plan.run()
    plan.set_search(False)
    b = plan.run()
    assert a == b


def test_persistent_search_times_out_and_recovers():
    """A wait limit of 1 ns makes the persistent search's first wait between CTAs
    give up: the run ends with TTQ_ERR_TIMEOUT (no GPU fault, no hang), and the
    same plan with the default limit then runs normally."""
    p = FULL["D_cube"]()
    plan = B().Plan(p)
    plan.set_search(True)
    ref = plan.run()
    plan.set_wait_limit(1)
    r = plan.run()
    assert r["status_name"] == "timeout", r
    plan.set_wait_limit(10 ** 9)
    assert plan.run() == ref


SEQ = dict(FULL)
# the unit-cube D_6 and E_6 at rank cap 30 reach the rounding floor (pivot residuals
# ~1e-17 of the largest entry) from its 12th sweep on, where rounding picks
# among equally valid pivots; at cap 8 every pivot stays far above it
SEQ["D_cube"] = lambda: inputs.make_problem("D", "cube", 6, 33, rank_cap=8)
SEQ["E_cube"] = lambda: inputs.make_problem("E", "cube", 6, 33, rank_cap=8)


@pytest.mark.parametrize("case", ["C_rn", "D_rn", "D_cube", "E_cube", "TEST"])
def test_sequential_sweep_matches_oracle(case):
    """Alg. 5 on the GPU (interfaces one after another, each pivot appended at
    once) against the oracle's sequential sweep: the same run, and the same
    final nested sets."""
    p = SEQ[case]()
    ora = ttcross.integrate(p, sequential=True)
    plan = B().Plan(p)
    plan.set_sequential(True)
    got = plan.run()
    assert got["status"] == ora["status"]
    assert rel(got["value"], ora["value"]) < 1e-12
    assert (got["sweeps"], got["n_eval"], got["ranks"]) == (ora["sweeps"], ora["n_eval"], ora["ranks"])
    st = plan.get_state()
    par = ttcross.to_parents(p, ora["state"])
    for key in ("lpar", "lnode", "rpar", "rnode"):
        for a, b in zip(st[key], par[key]):
            assert np.array_equal(a, b), key
