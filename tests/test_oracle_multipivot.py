"""Pins for the oracle's several-pivots-per-sweep variant (pivot_search_multi).

Checked against what the mathematics fixes, not against a restatement:
  * with one pivot per sweep it is the single-pivot search of Alg. 2 (the
    stored full runs of Alg. 6 pin that one);
  * the Schur determinant identity: appending the accepted rows X and columns
    Y to the cross multiplies det A(I<=k, I>k) by det of the old cross's
    residual on X x Y, which greedy elimination in acceptance order factors
    into the accepted pivots; the new cross matrices are built from fresh
    tensor entries, so a wrong residual, Schur update, pivot pairing or append
    order fails it;
  * the rook condition, Eq. (2), of every search against a full superblock
    residual built from Eq. (1);
  * Thm. 2 (exact recovery of a separable tensor of known rank) and the
    printed D_8 (Sec. 5.5, Fig. 7);
  * a planted mistake in the Schur update fails the determinant identity;
  * the meeting rule (a search that meets an earlier running search at the
    same step stops there) changes no accepted pivot: run to their ends, the
    searches it stops end on the pivot of the search they met.
"""
import json
import os

import numpy as np
import pytest

from oracle import integrands, ttcross
from paper_1903_11554_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prepare(p, st):
    cores = [ttcross.core(p, st, k) for k in range(1, p.d + 1)]
    scale = max(float(np.abs(c).max()) for c in cores)
    return cores, scale


def _cross_matrix(p, st, k):
    return ttcross.core(p, st, k).reshape(-1, st.rank(k))[ttcross.cross_rows(p, st, k), :]


def _states(p, sweeps):
    """The run's states after each of its first sweeps (single-pivot run)."""
    st = ttcross.initial_state(p)
    out = [st]
    for s in range(sweeps):
        cores, scale = _prepare(p, st)
        pv = ttcross.search_all(p, st, s, cores, scale)
        st = ttcross.apply_pivots(p, st, pv)
        out.append(st)
    return out


@pytest.mark.parametrize("case", [("C", "rn", 4, 31, 8.0), ("D", "rn", 5, 25, 6.0), ("E", "cube", 6, 17, 0.0)])
def test_one_pivot_is_the_single_search(case):
    fam, form, n, N, L = case
    kw = dict(rank_cap=10, seed=3)
    p = inputs.make_problem(fam, form, n, N, L=L, **kw) if form == "rn" else inputs.make_problem(fam, form, n, N, **kw)
    for s, st in enumerate(_states(p, 4)):
        cores, scale = _prepare(p, st)
        for k in range(1, p.d):
            B = ttcross.maxvol_coefficients(cores[k - 1], ttcross.cross_rows(p, st, k))
            one = ttcross.pivot_search(p, st, k, B, cores[k], s, scale)
            multi = ttcross.pivot_search_multi(p, st, k, B, cores[k], s, scale, 1)
            if one is None:
                assert multi is None
                continue
            srch = multi.searches[0]
            assert (srch.row, srch.col, srch.err, srch.rounds) == (one.row, one.col, one.err, one.rounds)
            assert multi.evals == one.evals
            if one.accepted:
                assert [(q.row, q.col, q.err) for q in multi.pivots] == [(one.row, one.col, one.err)]
            else:
                assert multi.pivots == []


@pytest.mark.parametrize("case", [("C", "rn", 5, 41, 10.0, 3), ("D", "rn", 5, 33, 8.0, 4), ("E", "cube", 7, 21, 0.0, 3)])
def test_schur_determinant_identity(case):
    """det G_k(new) = det G_k(old) * prod(accepted pivots), G from fresh entries."""
    fam, form, n, N, L, npiv = case
    kw = dict(rank_cap=14, seed=11, npiv=npiv)
    p = inputs.make_problem(fam, form, n, N, L=L, **kw) if form == "rn" else inputs.make_problem(fam, form, n, N, **kw)
    st = ttcross.initial_state(p)
    checked = multi_seen = 0
    for s in range(4):
        cores, scale = _prepare(p, st)
        pv = ttcross.search_all(p, st, s, cores, scale)
        new = ttcross.apply_pivots(p, st, pv)
        for k in range(1, p.d):
            mp = pv[k - 1]
            if mp is None or not mp.pivots:
                continue
            g0 = np.linalg.slogdet(_cross_matrix(p, st, k))
            g1 = np.linalg.slogdet(_cross_matrix(p, new, k))
            prod_sign = np.prod(np.sign([q.err for q in mp.pivots]))
            prod_log = np.sum(np.log(np.abs([q.err for q in mp.pivots])))
            assert g1[0] == g0[0] * prod_sign, (s, k)
            assert abs((g1[1] - g0[1]) - prod_log) < 1e-7, (s, k, g1[1] - g0[1], prod_log)
            assert new.rank(k) == st.rank(k) + len(mp.pivots) <= p.rank_cap
            checked += 1
            multi_seen += len(mp.pivots) > 1
        st = new
    assert checked > 0 and multi_seen > 0


def test_greedy_cross_factors_the_taken_block():
    rng = np.random.default_rng(7)
    for m in (2, 3, 4):
        for _ in range(20):
            Mx = rng.standard_normal((m, m))
            ref = Mx.copy()
            out = ttcross.greedy_cross(Mx, 1.0, 1e-14, m)
            assert len(out) == m
            rows = [a for a, _, _ in out]
            cols = [c for _, c, _ in out]
            assert sorted(rows) == list(range(m)) and sorted(cols) == list(range(m))
            det = np.linalg.det(ref[np.ix_(rows, cols)])
            assert abs(np.prod([q for _, _, q in out]) / det - 1) < 1e-10
            # complete pivoting: the first pivot is the largest entry
            assert abs(out[0][2]) == np.abs(ref).max()


def test_rook_condition_of_every_search():
    p = inputs.make_problem("D", "rn", 4, 15, L=6.0, rank_cap=8, rook_max=10, npiv=3)
    st = _states(inputs.make_problem("D", "rn", 4, 15, L=6.0, rank_cap=8), 2)[-1]
    A = np.zeros(p.N)
    grids = np.meshgrid(*[np.arange(N) for N in p.N], indexing="ij")
    idx = np.stack([g.ravel() for g in grids], axis=1)
    A = integrands.tensor_entries(p, idx).reshape(p.N)
    cores, scale = _prepare(p, st)
    seen = 0
    for k in range(1, p.d):
        B = ttcross.maxvol_coefficients(cores[k - 1], ttcross.cross_rows(p, st, k))
        mp = ttcross.pivot_search_multi(p, st, k, B, cores[k], 5, scale, 3)
        left, right = st.left[k - 1], st.right[k + 1]
        Nk, Nk1, rn = p.N[k - 1], p.N[k], len(right)
        S = np.empty((len(left) * Nk, Nk1 * rn))
        for a, pre in enumerate(left):
            for i in range(Nk):
                for j in range(Nk1):
                    for b, suf in enumerate(right):
                        S[a * Nk + i, j * rn + b] = A[tuple(pre) + (i, j) + tuple(suf)]
        I = ttcross.cross_rows(p, st, k)
        J = ttcross.cross_cols(p, st, k)
        E = S - S[:, J] @ np.linalg.solve(S[np.ix_(I, J)], S[I, :])
        for pv in mp.searches:
            if pv.merged:
                continue
            if pv.rounds < p.rook_max:
                assert abs(E[pv.row, pv.col]) >= np.max(np.abs(E[pv.row, :])) * (1 - 1e-9)
                assert abs(E[pv.row, pv.col]) >= np.max(np.abs(E[:, pv.col])) * (1 - 1e-9)
            assert abs(E[pv.row, pv.col] - pv.err) <= 1e-10 * abs(E).max()
            seen += 1
        # the residual matrix of the kept searches is E on their rows and columns
        kept = []
        for pv in mp.searches:
            if not pv.merged and not any(pv.row == q.row or pv.col == q.col for q in kept):
                kept.append(pv)
        sub = E[np.ix_([q.row for q in kept], [q.col for q in kept])]
        assert np.allclose(mp.cross, sub, rtol=0, atol=1e-10 * abs(E).max())
    assert seen >= 2 * (p.d - 1)


@pytest.mark.parametrize("npiv", [2, 3])
def test_exact_recovery_separable_rank(npiv):
    p = inputs.make_problem("TEST", "cube", 5, 33, d=6, rank_cap=10, npiv=npiv)
    r = ttcross.integrate(p)
    assert max(r["ranks"]) <= 5
    d = p.d
    tot = 0.0
    for t in range(1, p.n + 1):
        pr = 1.0
        for k in range(d):
            pr *= float(np.sum(p.weights[k] * np.exp(-t * p.nodes[k] / d)))
        tot += pr
    assert abs(r["value"] / tot - 1) < 1e-13


def test_d8_printed_value_with_four_pivots():
    p = inputs.config_d_cube(8, npiv=4)
    r = ttcross.integrate(p)
    ref = float(json.load(open(os.path.join(GOLDEN, "paper_values.json")))["D_8"]["value"])
    assert r["status"] == ttcross.STATUS_CONVERGED
    assert abs(r["value"] / ref - 1) < 5e-12


def test_planted_schur_sign_fails_the_identity(monkeypatch):
    def wrong(Mx, a, c, rows_left, cols_left):
        piv = Mx[a, c]
        for b in rows_left:
            for e in cols_left:
                Mx[b, e] = Mx[b, e] + (Mx[b, c] * Mx[a, e]) / piv
    monkeypatch.setattr(ttcross, "schur_step", wrong)
    p = inputs.make_problem("D", "rn", 5, 33, L=8.0, rank_cap=14, seed=11, npiv=4)
    st = ttcross.initial_state(p)
    broken = False
    for s in range(4):
        cores, scale = _prepare(p, st)
        pv = ttcross.search_all(p, st, s, cores, scale)
        new = ttcross.apply_pivots(p, st, pv)
        for k in range(1, p.d):
            mp = pv[k - 1]
            if mp is None or len(mp.pivots) < 2:
                continue
            g0 = np.linalg.slogdet(_cross_matrix(p, st, k))
            g1 = np.linalg.slogdet(_cross_matrix(p, new, k))
            prod_log = np.sum(np.log(np.abs([q.err for q in mp.pivots])))
            if abs((g1[1] - g0[1]) - prod_log) > 1e-7:
                broken = True
        st = new
    assert broken


@pytest.mark.parametrize("case", [("C", "rn", 5, 41, 10.0, 4), ("D", "rn", 5, 33, 8.0, 4), ("D", "cube", 7, 25, 0.0, 3),
                                  ("E", "cube", 6, 21, 0.0, 4)])
def test_meeting_rule_keeps_the_pivots(case):
    fam, form, n, N, L, npiv = case
    kw = dict(rank_cap=14, seed=5, npiv=npiv)
    p = inputs.make_problem(fam, form, n, N, L=L, **kw) if form == "rn" else inputs.make_problem(fam, form, n, N, **kw)
    st = ttcross.initial_state(p)
    merged = 0
    for s in range(5):
        cores, scale = _prepare(p, st)
        for k in range(1, p.d):
            B = ttcross.maxvol_coefficients(cores[k - 1], ttcross.cross_rows(p, st, k))
            a = ttcross.pivot_search_multi(p, st, k, B, cores[k], s, scale, npiv)
            b = ttcross.pivot_search_multi(p, st, k, B, cores[k], s, scale, npiv, meet=False)
            if a is None:
                assert b is None
                continue
            assert [(q.row, q.col, q.err) for q in a.pivots] == [(q.row, q.col, q.err) for q in b.pivots]
            assert np.array_equal(a.cross, b.cross)
            assert a.evals <= b.evals
            full = b.searches
            for j, pv in enumerate(a.searches):
                if not pv.merged:
                    assert (pv.row, pv.col, pv.err, pv.evals) == (full[j].row, full[j].col, full[j].err, full[j].evals)
                    continue
                merged += 1
                assert pv.evals < full[j].evals
                # run to its end it stops on the pivot of an earlier search
                assert any((full[q].row, full[q].col) == (full[j].row, full[j].col) for q in range(j))
        pv_all = ttcross.search_all(p, st, s, cores, scale)
        st = ttcross.apply_pivots(p, st, pv_all)
    assert merged > 0
