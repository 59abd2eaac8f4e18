"""Pins for the oracle's integrands, brute-force quadrature and exact grid values.

Every check here is against something other than the oracle itself: closed
forms of the Ising-class integrals, an independent restatement of the E_n
integrand in the u_k form, symmetry of C_n / D_n, the two forms of the same
integral, and the separable exact grid value of C_n.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import brute, exact, integrands, rng
from paper_1903_11554_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def const(f, form, n):
    return integrands.family_constant(f, form, n)


def test_splitmix64_published_vector():
    ref = json.load(open(os.path.join(GOLDEN, "splitmix64_seed0.json")))
    got = ["%016x" % rng.splitmix_output(0, m) for m in range(1, 5)]
    assert got == ref["outputs_hex"]


def test_draw_index_range_and_spread():
    M = 385 * 7
    xs = [rng.draw_index(12, rng.stream_id(3, 5, rng.PURPOSE_SAMPLE), t, M) for t in range(4000)]
    assert min(xs) >= 0 and max(xs) < M
    # roughly uniform: every eighth of the range is hit
    hist = np.bincount(np.array(xs) * 8 // M, minlength=8)
    assert hist.min() > 350


def test_gauss_legendre_exactness():
    x, w = inputs.gauss_legendre01(17)
    for p in range(0, 2 * 17):          # exact for degree <= 2N-1
        assert abs(np.sum(w * x ** p) - 1.0 / (p + 1)) < 1e-14


@pytest.mark.parametrize("key", [("C", 1), ("C", 2), ("D", 2)])
def test_closed_forms_rn_brute(key):
    fam, n = key
    p = inputs.make_problem(fam, "rn", n, 321, L=20.0)
    val = const(fam, "rn", n) * brute.brute_sum(p)
    assert abs(val / exact.closed_forms()[key] - 1) < 1e-13


@pytest.mark.parametrize("key", [("C", 2), ("D", 2), ("E", 2)])
def test_closed_forms_cube_brute(key):
    fam, n = key
    p = inputs.make_problem(fam, "cube", n, 40)
    val = const(fam, "cube", n) * brute.brute_sum(p)
    assert abs(val / exact.closed_forms()[key] - 1) < 1e-14


def test_c4_closed_form_rn():
    p = inputs.config_c4()
    val = const("C", "rn", 4) * brute.brute_sum_symmetric(p)
    assert abs(val / exact.closed_forms()[("C", 4)] - 1) < 1e-12


def test_d4_closed_form_both_forms():
    ref = exact.closed_forms()[("D", 4)]
    p = inputs.make_problem("D", "rn", 4, 161, L=20.0)
    assert abs(const("D", "rn", 4) * brute.brute_sum_symmetric(p) / ref - 1) < 5e-11
    p = inputs.make_problem("D", "cube", 4, 64)
    assert abs(const("D", "cube", 4) * brute.brute_sum(p) / ref - 1) < 1e-13


@pytest.mark.parametrize("fam", ["C", "D"])
def test_rn_and_cube_forms_agree_n3(fam):
    rn = inputs.make_problem(fam, "rn", 3, 241, L=20.0)
    cube = inputs.make_problem(fam, "cube", 3, 64)
    a = const(fam, "rn", 3) * brute.brute_sum_symmetric(rn)
    b = const(fam, "cube", 3) * brute.brute_sum(cube)
    assert abs(a / b - 1) < 1e-11


@pytest.mark.parametrize("fam", ["C", "D"])
def test_symmetric_reduction_matches_full_sum(fam):
    p = inputs.make_problem(fam, "rn", 3, 23, L=12.0)
    a = brute.brute_sum(p)
    b = brute.brute_sum_symmetric(p)
    assert abs(a / b - 1) < 1e-14


@pytest.mark.parametrize("fam,form,n", [("C", "rn", 5), ("D", "rn", 6), ("C", "cube", 7),
                                       ("D", "cube", 6), ("E", "cube", 9), ("TEST", "cube", 3)])
def test_numpy_and_c_integrands_agree(fam, form, n):
    d = inputs.modes_for(fam, form, n, 5)
    g = np.random.default_rng(7)
    X = g.uniform(-6, 6, (500, d)) if form == "rn" and fam != "TEST" else g.uniform(0, 1, (500, d))
    a = integrands.g_values(fam, form, n, X)
    b = brute.g_c(fam, form, n, X)
    assert np.max(np.abs(a - b) / np.abs(b)) < 1e-13


def test_e_matches_u_form():
    """E_n restated with u_k = prod_{i<=k} t_i, t_1 = 1:
    prod_{j<k} ((u_k - u_j)/(u_k + u_j))^2."""
    n = 7
    g = np.random.default_rng(3)
    X = g.uniform(0.05, 1, (200, n - 1))
    ours = integrands.g_values("E", "cube", n, X)
    ref = []
    for row in X:
        t = np.concatenate([[1.0], row])
        u = np.cumprod(t)
        v = 1.0
        for k in range(n):
            for j in range(k):
                v *= ((u[k] - u[j]) / (u[k] + u[j])) ** 2
        ref.append(v)
    assert np.max(np.abs(ours / np.array(ref) - 1)) < 1e-13


def test_d_rn_is_symmetric_and_even():
    g = np.random.default_rng(5)
    X = g.uniform(-5, 5, (100, 6))
    base = integrands.g_values("D", "rn", 6, X)
    perm = X[:, [3, 0, 5, 1, 4, 2]]
    assert np.max(np.abs(integrands.g_values("D", "rn", 6, perm) / base - 1)) < 1e-13
    assert np.max(np.abs(integrands.g_values("D", "rn", 6, -X) / base - 1)) < 1e-13


def test_d_vanishes_on_equal_coordinates():
    X = np.array([[0.5, -1.0, 0.5, 2.0]])
    assert integrands.g_values("D", "rn", 4, X)[0] == 0.0


@pytest.mark.parametrize("n", [2, 3, 4])
def test_c_grid_identity_matches_brute_force(n):
    pytest.importorskip("mpmath")
    p = inputs.make_problem("C", "rn", n, 81, L=16.0)
    a = brute.brute_sum(p)
    b = exact.c_grid_exact(p.nodes, p.weights)
    assert abs(a / b - 1) < 1e-14


def test_weighted_entries_fold_weights():
    p = inputs.make_problem("E", "cube", 4, 9)
    idx = np.array([[1, 4, 8], [0, 0, 0]])
    X = np.array([[p.nodes[k][i] for k, i in enumerate(r)] for r in idx])
    W = np.array([np.prod([p.weights[k][i] for k, i in enumerate(r)]) for r in idx])
    assert np.allclose(integrands.tensor_entries(p, idx), W * integrands.g_values("E", "cube", 4, X),
                       rtol=1e-15, atol=0)
