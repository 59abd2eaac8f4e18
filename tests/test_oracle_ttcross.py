"""Pins for the oracle's TT cross quadrature.

Checked against: the exact recovery theorem (Thm. 2) on a separable tensor of
known rank; the interpolation theorem (Thm. 1) via a full reconstruction; the
rook condition, Eq. (2), against a full superblock residual built from the
matrix cross formula, Eq. (1), directly; brute-force tensor sums; closed
forms; the paper's printed D_8 and D_16 (Sec. 5.5, Fig. 7); the exact grid
value of C_n; mode-reversal symmetry; exact rational contraction.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import brute, exact, integrands, ttcross
from paper_1903_11554_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def separable_exact(p):
    d = p.d
    tot = 0.0
    for t in range(1, p.n + 1):
        pr = 1.0
        for k in range(d):
            pr *= float(np.sum(p.weights[k] * np.exp(-t * p.nodes[k] / d)))
        tot += pr
    return tot


def full_tensor(p):
    grids = np.meshgrid(*[np.arange(N) for N in p.N], indexing="ij")
    idx = np.stack([g.ravel() for g in grids], axis=1)
    return integrands.tensor_entries(p, idx).reshape(p.N)


def tt_full(p, st):
    """Eq. (3) written out on the full grid: A(i1, I>1) G1^-1 A(I<=1, i2, I>2) ... ."""
    cores = [ttcross.core(p, st, k) for k in range(1, p.d + 1)]
    out = cores[0].reshape(p.N[0], -1)                       # N1 x r1
    for k in range(1, p.d):
        G = cores[k - 1].reshape(-1, st.rank(k))[ttcross.cross_rows(p, st, k), :]
        out = np.linalg.solve(G.T, out.T).T
        nxt = cores[k].reshape(st.rank(k), -1)              # r_k x (N_{k+1} r_{k+1})
        out = (out @ nxt).reshape(-1, st.rank(k + 1))
    return out.reshape(p.N)


# --------------------------------------------------------------------------

def test_exact_recovery_separable_rank():
    """Thm. 2: a tensor of exact TT rank n is recovered exactly, so its
    integral equals the closed-form separable sum."""
    p = inputs.make_problem("TEST", "cube", 5, 33, d=6, rank_cap=10)
    r = ttcross.integrate(p)
    assert r["ranks"][1:-1] == [5] * 5
    assert abs(r["value"] / separable_exact(p) - 1) < 1e-13


def test_exact_recovery_full_tensor():
    p = inputs.make_problem("TEST", "cube", 3, 9, d=4, rank_cap=6)
    r = ttcross.integrate(p)
    A = full_tensor(p)
    At = tt_full(p, r["state"])
    assert np.max(np.abs(At - A)) <= 1e-13 * np.max(np.abs(A))


def test_interpolation_on_evaluated_fibers():
    """Thm. 1: with nested sets the TT reproduces every fiber A(I<=k-1, i_k, I>k)."""
    p = inputs.make_problem("D", "cube", 5, 11, rank_cap=6, max_sweeps=5)
    r = ttcross.integrate(p)
    st = r["state"]
    A = full_tensor(p)
    At = tt_full(p, st)
    scale = np.max(np.abs(A))
    for k in range(1, p.d + 1):
        for a in st.left[k - 1]:
            for b in st.right[k]:
                for i in range(p.N[k - 1]):
                    ix = tuple(a) + (i,) + tuple(b)
                    assert abs(At[ix] - A[ix]) <= 1e-12 * scale
    # nestedness, Eq. (4)
    for k in range(1, p.d - 1):
        for row in st.left[k + 1]:
            assert any(np.array_equal(row[:k], x) for x in st.left[k])
        for row in st.right[k]:
            assert any(np.array_equal(row[1:], x) for x in st.right[k + 1])


def test_coefficients_are_identity_on_cross_and_reproduce_fibers():
    p = inputs.make_problem("C", "cube", 5, 13, rank_cap=5, max_sweeps=5)
    st = ttcross.integrate(p)["state"]
    for k in range(1, p.d):
        Y = ttcross.core(p, st, k)
        P = ttcross.cross_rows(p, st, k)
        B = ttcross.maxvol_coefficients(Y, P)
        L = Y.reshape(-1, st.rank(k))
        # B(P,:) = I up to the forward error of a backward-stable solve, cond(G) * eps
        assert np.allclose(B[P, :], np.eye(len(P)), atol=1e-15 * np.linalg.cond(L[P, :]))
        assert np.allclose(B @ L[P, :], L, rtol=0, atol=1e-13 * np.abs(L).max())


def test_rook_condition_against_full_superblock():
    """The pivot Alg. 2 returns is the largest residual in its row and column
    (Eq. 2), with the residual computed from Eq. (1) on the whole superblock."""
    p = inputs.make_problem("D", "rn", 4, 15, L=6.0, rank_cap=8, max_sweeps=3, rook_max=10)
    st = ttcross.integrate(p)["state"]
    A = full_tensor(p)
    cores = [ttcross.core(p, st, k) for k in range(1, p.d + 1)]
    scale = max(np.abs(c).max() for c in cores)
    for k in range(1, p.d):
        B = ttcross.maxvol_coefficients(cores[k - 1], ttcross.cross_rows(p, st, k))
        pv = ttcross.pivot_search(p, st, k, B, cores[k], 7, scale)
        # superblock S(rho, gamma) from the full tensor
        left, right = st.left[k - 1], st.right[k + 1]
        Nk, Nk1 = p.N[k - 1], p.N[k]
        rn = len(right)
        S = np.empty((len(left) * Nk, Nk1 * rn))
        for a, pre in enumerate(left):
            for i in range(Nk):
                for j in range(Nk1):
                    for b, suf in enumerate(right):
                        S[a * Nk + i, j * rn + b] = A[tuple(pre) + (i, j) + tuple(suf)]
        I = ttcross.cross_rows(p, st, k)
        J = ttcross.cross_cols(p, st, k)
        E = S - S[:, J] @ np.linalg.solve(S[np.ix_(I, J)], S[I, :])
        if pv.rounds < p.rook_max:
            assert abs(E[pv.row, pv.col]) >= np.max(np.abs(E[pv.row, :])) * (1 - 1e-9)
            assert abs(E[pv.row, pv.col]) >= np.max(np.abs(E[:, pv.col])) * (1 - 1e-9)
        assert abs(E[pv.row, pv.col] - pv.err) <= 1e-10 * abs(E).max()


def test_parent_pointer_roundtrip():
    p = inputs.make_problem("E", "cube", 6, 17, rank_cap=5, max_sweeps=4)
    st = ttcross.integrate(p)["state"]
    par = ttcross.to_parents(p, st)
    st2 = ttcross.from_parents(p, par["lpar"], par["lnode"], par["rpar"], par["rnode"])
    for k in range(p.d):
        assert np.array_equal(st.left[k], st2.left[k])
    for k in range(1, p.d + 1):
        assert np.array_equal(st.right[k], st2.right[k])


@pytest.mark.parametrize("r0", [1, 4, 9])
def test_initial_sets_by_brute_force(r0):
    """The initial nested sets against a direct restatement of the reading: all
    init_samples points, sorted by |A| (ties by draw order), kept greedily when
    their first and last node indices are new; prefixes and suffixes nested,
    every interface of rank r0, every cross matrix nonsingular."""
    from oracle import rng
    p = inputs.make_problem("D", "rn", 5, 23, L=6.0, rank_cap=12, r0=r0, init_samples=48)
    st = ttcross.initial_state(p)
    d = p.d
    pts = []
    for q in range(p.init_samples):
        x = tuple(rng.draw_index(p.seed, rng.stream_id(0, 0, rng.PURPOSE_INIT), q * d + k, p.N[k])
                  for k in range(d))
        a = abs(float(integrands.tensor_entries(p, np.array([x]))[0]))
        pts.append((-a, q, x))
    kept = []
    for _, q, x in sorted(pts):
        if all(x[0] != y[0] and x[-1] != y[-1] for y in kept):
            kept.append(x)
        if len(kept) == r0:
            break
    assert st.ranks() == [1] + [r0] * (d - 1) + [1]
    for k in range(1, d):
        assert [tuple(r) for r in st.left[k]] == [x[:k] for x in kept]
        assert [tuple(r) for r in st.right[k]] == [x[k:] for x in kept]
    par = ttcross.to_parents(p, st)                     # nested: every row has its parent
    for k in range(1, d):
        assert list(par["lpar"][k - 1]) == (list(range(r0)) if k > 1 else [0] * r0)
        G = ttcross.core(p, st, k).reshape(-1, r0)[ttcross.cross_rows(p, st, k), :]
        assert np.linalg.matrix_rank(G) == r0
    if r0 == 1:                                           # the single largest |A| of the samples
        assert tuple(st.left[d - 1][0]) + (int(st.right[d - 1][0][-1]),) == sorted(pts)[0][2]


def test_decimal_contraction_against_exact_rationals():
    """contract_decimal (60-digit decimals, Gaussian elimination on G^T) against
    the same product of Sec. 4.1 in exact rational arithmetic (Gauss-Jordan on
    G itself, written out here), and against the FP64 integral_plain."""
    p = inputs.make_problem("D", "cube", 5, 9, rank_cap=4, max_sweeps=4)
    st = ttcross.integrate(p)["state"]
    cores = [ttcross.core(p, st, k) for k in range(1, p.d + 1)]

    def vsum(T):
        return [[sum((Fraction(float(v)) for v in T[a, :, b]), Fraction(0)) for b in range(T.shape[2])]
                for a in range(T.shape[0])]

    def times_inverse(x, G):                   # x G^-1: reduce [G | I] to [I | G^-1], then x times it
        n = len(x)
        A = [[Fraction(float(G[i, j])) for j in range(n)] + [Fraction(int(i == j)) for j in range(n)]
             for i in range(n)]
        for c in range(n):
            piv = next(r for r in range(c, n) if A[r][c] != 0)
            A[c], A[piv] = A[piv], A[c]
            A[c] = [v / A[c][c] for v in A[c]]
            for r in range(n):
                if r != c and A[r][c] != 0:
                    A[r] = [a - A[r][c] * b for a, b in zip(A[r], A[c])]
        return [sum((x[i] * A[i][n + j] for i in range(n)), Fraction(0)) for j in range(n)]

    x = vsum(cores[0])[0]
    for k in range(1, p.d):
        G = cores[k - 1].reshape(-1, st.rank(k))[ttcross.cross_rows(p, st, k), :]
        x = times_inverse(x, G)
        V = vsum(cores[k])
        x = [sum((x[a] * V[a][b] for a in range(len(x))), Fraction(0)) for b in range(len(V[0]))]
    exact_value = float(x[0] * Fraction(integrands.family_constant(p.family, p.form, p.n)))
    got = ttcross.contract_decimal(p, st, cores)
    assert abs(got - exact_value) <= 1e-15 * abs(exact_value)
    assert abs(ttcross.integral_plain(p, st, cores) - exact_value) <= 1e-13 * abs(exact_value)


def test_ranks_grow_by_at_most_one_per_sweep():
    p = inputs.make_problem("C", "cube", 6, 33, rank_cap=12)
    r = ttcross.integrate(p)
    prev = None
    for h in r["history"]:
        if prev is not None:
            assert all(0 <= a - b <= 1 for a, b in zip(h.ranks, prev))
        prev = h.ranks


def test_integral_forms_agree():
    p = inputs.make_problem("D", "cube", 6, 33, rank_cap=10, max_sweeps=8)
    st = ttcross.integrate(p)["state"]
    cores = [ttcross.core(p, st, k) for k in range(1, p.d + 1)]
    a = ttcross.integral_plain(p, st, cores)
    Bs = [ttcross.maxvol_coefficients(cores[k - 1], ttcross.cross_rows(p, st, k)) .reshape(cores[k - 1].shape)
          for k in range(1, p.d)]
    b = ttcross.integral_from_coefficients(p, Bs, cores[-1])
    assert abs(a / b - 1) < 1e-13


def test_exact_contraction_matches_float():
    p = inputs.make_problem("E", "cube", 5, 9, rank_cap=4, max_sweeps=4)
    st = ttcross.integrate(p)["state"]
    cores = [ttcross.core(p, st, k) for k in range(1, p.d + 1)]
    Bs = [ttcross.maxvol_coefficients(cores[k - 1], ttcross.cross_rows(p, st, k)).reshape(cores[k - 1].shape)
          for k in range(1, p.d)]
    ex = ttcross.contract_exact(Bs, cores[-1])
    fl = ttcross.integral_from_coefficients(p, Bs, cores[-1]) / integrands.family_constant("E", "cube", 5)
    assert isinstance(ex, Fraction)
    assert abs(float(ex) / fl - 1) < 1e-14


# --------------------------------------------------------------------------
# values against truth

def test_c4_cap40_vs_grid_and_closed_form():
    p = inputs.config_c4(rank_cap=40)
    r = ttcross.integrate(p)
    grid = integrands.family_constant("C", "rn", 4) * brute.brute_sum_symmetric(p)
    assert abs(r["value"] / grid - 1) < 1e-11
    assert abs(r["value"] / exact.closed_forms()[("C", 4)] - 1) < 1e-11


def test_c4_config_rank16_accuracy_limit():
    """The C_4 workload (rank cap 16) stops at the cap with ~2e-7 error:
    rank 16 cannot reach 1e-12 on this grid."""
    p = inputs.config_c4()
    r = ttcross.integrate(p)
    assert r["status"] == ttcross.STATUS_RANK_CAP
    grid = integrands.family_constant("C", "rn", 4) * brute.brute_sum_symmetric(p)
    assert 1e-9 < abs(r["value"] / grid - 1) < 1e-5


@pytest.mark.parametrize("n", [3, 4, 5])
def test_e_vs_brute(n):
    p = inputs.make_problem("E", "cube", n, 48, rank_cap=40)
    r = ttcross.integrate(p)
    ref = 2.0 * brute.brute_sum(p)
    assert abs(r["value"] / ref - 1) < 5e-12


def test_d4_cube_vs_closed_form():
    p = inputs.make_problem("D", "cube", 4, 64, rank_cap=40)
    r = ttcross.integrate(p)
    assert abs(r["value"] / exact.closed_forms()[("D", 4)] - 1) < 1e-13


def test_c6_cube_vs_brute():
    p = inputs.make_problem("C", "cube", 6, 33, rank_cap=30)
    r = ttcross.integrate(p)
    assert abs(r["value"] / (2.0 * brute.brute_sum(p)) - 1) < 5e-12


def test_c8_rn_vs_exact_grid_identity():
    pytest.importorskip("mpmath")
    p = inputs.make_problem("C", "rn", 6, 97, L=18.0, rank_cap=40)
    r = ttcross.integrate(p)
    grid = integrands.family_constant("C", "rn", 6) * exact.c_grid_exact(p.nodes, p.weights)
    assert abs(r["value"] / grid - 1) < 1e-10


def test_d8_printed_value():
    ref = float(json.load(open(os.path.join(GOLDEN, "paper_values.json")))["D_8"]["value"])
    p = inputs.make_problem("D", "cube", 8, 129, rank_cap=64, seed=8)
    r = ttcross.integrate(p)
    assert r["status"] == ttcross.STATUS_CONVERGED
    assert abs(r["value"] / ref - 1) < 5e-12


@pytest.mark.slow
def test_d16_printed_value():
    ref = float(json.load(open(os.path.join(GOLDEN, "paper_values.json")))["D_16"]["value"])
    p = inputs.make_problem("D", "cube", 16, 129, rank_cap=80, seed=16)
    r = ttcross.integrate(p)
    assert abs(r["value"] / ref - 1) < 5e-12


def test_mode_reversal_symmetry():
    """C_n in the R^n form is symmetric in its variables: the cross run on the
    reversed mode order (different pivots) gives the same integral."""
    p = inputs.make_problem("C", "rn", 4, 81, L=16.0, rank_cap=40)
    q = inputs.make_problem("C", "rn", 4, 81, L=16.0, rank_cap=40, seed=99)
    q.nodes, q.weights = q.nodes[::-1], q.weights[::-1]
    a = ttcross.integrate(p)["value"]
    b = ttcross.integrate(q)["value"]
    assert abs(a / b - 1) < 1e-11


# --------------------------------------------------------------------------
# Alg. 5, the sequential sweep (the paper's single-process comparison)

def test_sequential_exact_recovery():
    """Thm. 2 holds for the sequential sweep as well: exact rank, exact integral."""
    p = inputs.make_problem("TEST", "cube", 5, 33, d=6, rank_cap=10)
    r = ttcross.integrate(p, sequential=True)
    assert r["ranks"][1:-1] == [5] * 5
    assert abs(r["value"] / separable_exact(p) - 1) < 1e-13


def test_sequential_superblock_uses_the_updated_left_set():
    """In a sequential sweep the superblock of interface k is built from I<=k-1
    as step k-1 left it (Alg. 5): the pivot is the largest residual of its row
    and column in that superblock, computed from Eq. (1) on the full tensor,
    and its row may lie in the block of the row appended at step k-1."""
    p = inputs.make_problem("D", "rn", 4, 15, L=6.0, rank_cap=8, max_sweeps=3, rook_max=10)
    st = ttcross.integrate(p, sequential=True)["state"]
    A = full_tensor(p)
    cores = [ttcross.core(p, st, k) for k in range(1, p.d + 1)]
    scale = max(np.abs(c).max() for c in cores)
    st2, pivots, _ = ttcross.search_sequential(p, st, 7, cores, scale)
    cur = st
    for k in range(1, p.d):
        pv = pivots[k - 1]
        assert pv is not None
        left, right = cur.left[k - 1], cur.right[k + 1]
        Nk, Nk1 = p.N[k - 1], p.N[k]
        rn = len(right)
        S = np.empty((len(left) * Nk, Nk1 * rn))
        for a, pre in enumerate(left):
            for i in range(Nk):
                for j in range(Nk1):
                    for b, suf in enumerate(right):
                        S[a * Nk + i, j * rn + b] = A[tuple(pre) + (i, j) + tuple(suf)]
        I = ttcross.cross_rows(p, cur, k)
        J = ttcross.cross_cols(p, cur, k)
        E = S - S[:, J] @ np.linalg.solve(S[np.ix_(I, J)], S[I, :])
        if pv.rounds < p.rook_max:
            assert abs(E[pv.row, pv.col]) >= np.max(np.abs(E[pv.row, :])) * (1 - 1e-9)
            assert abs(E[pv.row, pv.col]) >= np.max(np.abs(E[:, pv.col])) * (1 - 1e-9)
        assert abs(E[pv.row, pv.col] - pv.err) <= 1e-10 * abs(E).max()
        if k > 1:
            assert len(left) == st.rank(k - 1) + (1 if pivots[k - 2].accepted else 0)
        if pv.accepted:
            cur = ttcross.apply_pivots(p, cur, [pv])
    assert cur.ranks() == st2.ranks()


def test_sequential_d8_printed_value():
    ref = float(json.load(open(os.path.join(GOLDEN, "paper_values.json")))["D_8"]["value"])
    p = inputs.config_d_cube(8)
    r = ttcross.integrate(p, sequential=True)
    assert r["status"] == ttcross.STATUS_CONVERGED
    assert abs(r["value"] / ref - 1) < 5e-12
