"""Plain CPU TT-cross quadrature (oracle, test infrastructure only).

Follows the paper step by step:
  * TT cross interpolation, Eq. (3): A ~ A(i_1, I_>1) [A(I_<=1, I_>1)]^-1
    A(I_<=1, i_2, I_>2) ... A(I_<=d-1, i_d), with nested index sets, Eq. (4).
  * Weights folded into the tensor, Sec. 4.1: A = w_{i_1}...w_{i_d} f(t).
  * One sweep of the dimension-parallel greedy cross, Alg. 6 with one
    superblock per "process": for every interface k at once, Alg. 2 is applied
    to the superblock A(I_<=k-1 i_k, i_{k+1} I_>k+1) built from the index sets
    of the previous sweep, and all new pivots are appended after the sweep.
  * Alg. 2: random samples, then alternating column / row partial pivoting
    until the rook condition, Eq. (2), holds or the round budget is spent.
  * The coefficient matrix of Alg. 1's first step, B_k = L_k A(I_<=k, I_>k)^-1,
    is one solve with the r_k x r_k cross matrix (LAPACK, partial pivoting).
  * The integral is the product of (2d-1) matrices of Sec. 4.1:
    (sum_i A(i, I_>1)) G_1^-1 (sum_i A(I_<=1, i, I_>2)) ... (sum_i A(I_<=d-1, i)).

Readings where the paper is silent:
  * initial index sets (Alg. 6 needs nested sets to start from): r0 seeded
    random multi-indices x^(1..r0), I_<=k = their prefixes of length k and
    I_>k = their suffixes from mode k+1, in the order chosen (nested by
    construction).  They are taken from `init_samples` seeded random points in
    decreasing |A| (ties by draw order), skipping a point whose first or last
    node index equals that of a point already taken (then all its prefixes and
    suffixes are new, so every interface has rank r0) or whose value is not
    finite and nonzero; r0 = 1 is the single largest |A|;
  * random samples: `samples_for(k)` draws per interface from the counter-based
    SplitMix64 of oracle/rng.py, keyed by (seed, sweep, k); samples that land
    in a row or column of the current cross are skipped (the error is zero
    there, Sec. 2.4);
  * ties in the argmax of Alg. 2: candidates whose |E| is within a noise
    window of the maximum, |E| >= max - (TIE_REL * max + TIE_ABS * scale), are
    tied, and the first in scan order wins (samples in draw order, rows by
    rho = alpha * N_k + i, columns by gamma = j * r_{k+1} + beta); residuals that
    are equal in exact arithmetic (e.g. by the permutation symmetry of C_n and
    D_n) then pick the same pivot whatever the rounding;
  * a pivot is accepted when |E*| > tol * scale, scale = largest |entry| of the
    current cores, and r_k < rank cap;
  * several pivots per interface per sweep (npiv > 1, a rank-adaptive variant
    of Alg. 6, which adds one): the npiv best samples with distinct rows and
    columns start rook searches on the old residual (a search that meets an
    earlier one at the same step stops there, its end being the earlier one's),
    and greedy complete pivoting on the residual matrix of their rows and
    columns keeps the pairs whose Schur pivot passes the acceptance threshold
    (pivot_search_multi);
  * stopping: relative internal convergence |I_s - I_{s-1}| <= tol |I_s|, or
    no pivot accepted in a sweep, or every interface at the rank cap, or the
    sweep limit.
"""
from __future__ import annotations

import dataclasses
from fractions import Fraction
from typing import Dict, List, Optional

import numpy as np

from . import rng
from .integrands import family_constant, tensor_entries

TIE_REL = 1e-12
TIE_ABS = 1e-14

STATUS_CONVERGED = 0
STATUS_NO_PIVOT = 1
STATUS_RANK_CAP = 2
STATUS_MAX_SWEEPS = 3


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def neumaier_sum(a: np.ndarray, axis: int) -> np.ndarray:
    """Neumaier-compensated sum along one axis."""
    a = np.moveaxis(np.asarray(a, dtype=np.float64), axis, 0)
    s = np.zeros(a.shape[1:])
    c = np.zeros(a.shape[1:])
    for x in a:
        t = s + x
        c = c + np.where(np.abs(s) >= np.abs(x), (s - t) + x, (x - t) + s)
        s = t
    return s + c


@dataclasses.dataclass
class CrossState:
    """Nested index sets, Eq. (4): left[k] holds I_<=k as an (r_k, k) array of
    node indices of modes 1..k; right[k] holds I_>k as an (r_k, d-k) array of
    node indices of modes k+1..d.  left[0] and right[d] are the empty tuple."""
    left: List[np.ndarray]
    right: List[np.ndarray]

    @property
    def d(self) -> int:
        return len(self.left)

    def rank(self, k: int) -> int:
        if k == 0 or k == self.d:
            return 1
        return self.left[k].shape[0]

    def ranks(self) -> List[int]:
        return [self.rank(k) for k in range(self.d + 1)]

    def copy(self) -> "CrossState":
        return CrossState([x.copy() for x in self.left], [x.copy() for x in self.right])


def _row_of(table: np.ndarray, row: np.ndarray) -> int:
    hits = np.nonzero(np.all(table == row[None, :], axis=1))[0]
    if len(hits) != 1:
        raise AssertionError("index sets are not nested")
    return int(hits[0])


def cross_rows(problem, st: CrossState, k: int) -> np.ndarray:
    """P_k: positions of I_<=k among the rows (alpha, i) of the k-th fiber
    matrix, rho = alpha * N_k + i (nestedness, Eq. (4), makes them exist)."""
    Nk = problem.N[k - 1]
    out = []
    for a in range(st.rank(k)):
        alpha = _row_of(st.left[k - 1], st.left[k][a, :k - 1])
        out.append(alpha * Nk + int(st.left[k][a, k - 1]))
    return np.array(out, dtype=np.int64)


def cross_cols(problem, st: CrossState, k: int) -> np.ndarray:
    """Q_k: positions of I_>k among the columns (j, beta) of superblock k,
    gamma = j * r_{k+1} + beta."""
    r_next = st.rank(k + 1)
    out = []
    for b in range(st.rank(k)):
        beta = _row_of(st.right[k + 1], st.right[k][b, 1:])
        out.append(int(st.right[k][b, 0]) * r_next + beta)
    return np.array(out, dtype=np.int64)


def to_parents(problem, st: CrossState) -> Dict[str, List[np.ndarray]]:
    """Parent-pointer form of the nested sets: I_<=k[a] = (I_<=k-1[lpar], lnode),
    I_>k[b] = (rnode, I_>k+1[rpar]), for k = 1..d-1."""
    lpar, lnode, rpar, rnode = [], [], [], []
    for k in range(1, problem.d):
        P = cross_rows(problem, st, k)
        Nk = problem.N[k - 1]
        lpar.append(P // Nk)
        lnode.append(P % Nk)
        Q = cross_cols(problem, st, k)
        rn = st.rank(k + 1)
        rnode.append(Q // rn)
        rpar.append(Q % rn)
    return {"lpar": lpar, "lnode": lnode, "rpar": rpar, "rnode": rnode}


def from_parents(problem, lpar, lnode, rpar, rnode) -> CrossState:
    """Inverse of to_parents: rebuild the full multi-index sets."""
    d = problem.d
    left = [np.zeros((1, 0), dtype=np.int64)]
    for k in range(1, d):
        rows = [np.concatenate([left[k - 1][int(p)], [int(i)]]) for p, i in zip(lpar[k - 1], lnode[k - 1])]
        left.append(np.array(rows, dtype=np.int64).reshape(len(rows), k))
    right = [np.zeros((0, d), dtype=np.int64)] * (d + 1)
    right[d] = np.zeros((1, 0), dtype=np.int64)
    for k in range(d - 1, 0, -1):
        rows = [np.concatenate([[int(j)], right[k + 1][int(p)]]) for p, j in zip(rpar[k - 1], rnode[k - 1])]
        right[k] = np.array(rows, dtype=np.int64).reshape(len(rows), d - k)
    return CrossState(left, right)


# ---------------------------------------------------------------------------
# evaluations
# ---------------------------------------------------------------------------

def eval_points(problem, idx: np.ndarray, chunk: int = 1 << 20) -> np.ndarray:
    out = np.empty(idx.shape[0])
    for a in range(0, idx.shape[0], chunk):
        out[a:a + chunk] = tensor_entries(problem, idx[a:a + chunk])
    return out


def core(problem, st: CrossState, k: int) -> np.ndarray:
    """Fiber tensor Y_k = A(I_<=k-1, i_k, I_>k), shape (r_{k-1}, N_k, r_k), Eq. (3)."""
    d = problem.d
    Lset = st.left[k - 1]                  # (r_{k-1}, k-1)
    Rset = st.right[k]                     # (r_k, d-k)
    r0, r1, Nk = Lset.shape[0], Rset.shape[0], problem.N[k - 1]
    idx = np.empty((r0, Nk, r1, d), dtype=np.int64)
    idx[..., :k - 1] = Lset[:, None, None, :]
    idx[..., k - 1] = np.arange(Nk)[None, :, None]
    idx[..., k:] = Rset[None, None, :, :]
    return eval_points(problem, idx.reshape(-1, d)).reshape(r0, Nk, r1)


def superblock_entries(problem, st: CrossState, k: int, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Fresh entries A(I_<=k-1[alpha], i, j, I_>k+1[beta]) of superblock k at
    flattened rows rho = alpha*N_k + i and columns gamma = j*r_{k+1} + beta."""
    d = problem.d
    Nk = problem.N[k - 1]
    rn = st.rank(k + 1)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    idx = np.empty((len(rows), d), dtype=np.int64)
    idx[:, :k - 1] = st.left[k - 1][rows // Nk]
    idx[:, k - 1] = rows % Nk
    idx[:, k] = cols // rn
    idx[:, k + 1:] = st.right[k + 1][cols % rn]
    return eval_points(problem, idx)


# ---------------------------------------------------------------------------
# QR + maxvol coefficients, contraction
# ---------------------------------------------------------------------------

def maxvol_coefficients(Yk: np.ndarray, P: np.ndarray) -> np.ndarray:
    """B_k = A(:, I_>k) A(I_<=k, I_>k)^-1 = L_k G_k^-1 with L_k = Y_k as
    (r_{k-1} N_k) x r_k and G_k = L_k(P_k, :): the coefficient matrix of Alg. 1,
    first step (B(P, :) = identity), as one LAPACK solve with the cross matrix."""
    r = Yk.shape[2]
    Lk = Yk.reshape(-1, r)
    return np.linalg.solve(Lk[P, :].T, Lk.T).T


def integral_plain(problem, st: CrossState, cores: List[np.ndarray]) -> float:
    """Sec. 4.1: (sum_i A(i,I_>1)) G_1^-1 (sum_i A(I_<=1,i,I_>2)) ... (sum_i A(I_<=d-1,i)),
    G_k = A(I_<=k, I_>k); weights are already folded into A; node sums compensated."""
    d = problem.d
    x = neumaier_sum(cores[0], axis=1)                    # 1 x r_1
    for k in range(1, d):
        P = cross_rows(problem, st, k)
        G = cores[k - 1].reshape(-1, st.rank(k))[P, :]
        x = np.linalg.solve(G.T, x.T).T                   # x G_k^-1
        x = x @ neumaier_sum(cores[k], axis=1)            # x V_{k+1}
    return family_constant(problem.family, problem.form, problem.n) * float(x[0, 0])


def integral_from_coefficients(problem, Bs: List[np.ndarray], Yd: np.ndarray) -> float:
    """Same product written with the coefficient cores: prod_k (sum_i B_k(:, i, :)) times sum_i Y_d."""
    x = np.ones((1, 1))
    for B in Bs:
        x = x @ neumaier_sum(B, axis=1)
    x = x @ neumaier_sum(Yd, axis=1)
    return family_constant(problem.family, problem.form, problem.n) * float(x[0, 0])


def contract_exact(Bs: List[np.ndarray], Yd: np.ndarray) -> Fraction:
    """The contraction of given FP64 cores in exact rational arithmetic (no
    constant): the reference for the double-double contraction."""
    x = [Fraction(1)]
    for T in list(Bs) + [Yd]:
        r0, Nk, r1 = T.shape
        W = [[sum((Fraction(float(T[a, i, b])) for i in range(Nk)), Fraction(0)) for b in range(r1)]
             for a in range(r0)]
        x = [sum((x[a] * W[a][b] for a in range(r0)), Fraction(0)) for b in range(r1)]
    return x[0]


def contract_decimal(problem, st: CrossState, cores: List[np.ndarray], digits: int = 60, as_decimal: bool = False):
    """Sec. 4.1's product (sum_i Y_1) G_1^-1 (sum_i Y_2) ... G_{d-1}^-1 (sum_i Y_d)
    of the given FP64 cores (G_k = rows P_k of Y_k, as in integral_plain), every
    step in `digits`-digit decimal arithmetic: node sums, the solves x G_k^-1
    by Gaussian elimination with partial pivoting on G_k^T, the products with
    the node sums.  FP64 values convert to decimals exactly, so the result is
    the contraction of these cores up to ~cond * 10^-digits; returned with the
    family constant, rounded to FP64 (as_decimal: the decimal itself)."""
    from decimal import Decimal, localcontext
    with localcontext() as ctx:
        ctx.prec = digits

        def vsum(T):
            r0, N, r1 = T.shape
            return [[sum((Decimal(float(v)) for v in T[a, :, b]), Decimal(0)) for b in range(r1)]
                    for a in range(r0)]

        def solve_left(G, x):                       # t with t G = x, i.e. G^T t = x
            n = len(x)
            M = [[G[j][i] for j in range(n)] + [x[i]] for i in range(n)]
            for c in range(n):
                p = max(range(c, n), key=lambda r: abs(M[r][c]))
                M[c], M[p] = M[p], M[c]
                for r in range(c + 1, n):
                    f = M[r][c] / M[c][c]
                    if f:
                        M[r] = [a - f * b for a, b in zip(M[r], M[c])]
            t = [Decimal(0)] * n
            for i in range(n - 1, -1, -1):
                t[i] = (M[i][n] - sum((M[i][j] * t[j] for j in range(i + 1, n)), Decimal(0))) / M[i][i]
            return t

        x = vsum(cores[0])[0]
        for k in range(1, problem.d):
            rows = cross_rows(problem, st, k)
            Gf = cores[k - 1].reshape(-1, st.rank(k))[rows, :]
            x = solve_left([[Decimal(float(v)) for v in row] for row in Gf], x)
            V = vsum(cores[k])
            x = [sum((x[a] * V[a][b] for a in range(len(x))), Decimal(0)) for b in range(len(V[0]))]
        c = family_constant(problem.family, problem.form, problem.n)
        v = x[0] * Decimal(repr(c))
        return v if as_decimal else float(v)


# ---------------------------------------------------------------------------
# Alg. 2 on one superblock
# ---------------------------------------------------------------------------

def tie_argmax(score: np.ndarray, scale: float) -> int:
    """First index whose score is within the tie window of the maximum;
    scores < 0 mark candidates that are not eligible.  -1 if none is."""
    ok = score >= 0
    if not ok.any():
        return -1
    smax = float(score[ok].max())
    thr = smax - (TIE_REL * smax + TIE_ABS * scale)
    return int(np.nonzero(ok & (score >= thr))[0][0])


@dataclasses.dataclass
class Pivot:
    k: int
    row: int            # rho = alpha * N_k + i
    col: int            # gamma = j * r_{k+1} + beta
    err: float          # residual A - A~ at the pivot
    accepted: bool
    rounds: int
    evals: int
    merged: bool = False   # several pivots per sweep: stopped where it met an earlier search


@dataclasses.dataclass
class _Superblock:
    """Superblock k of Alg. 6 on the sets of the previous sweep: its sizes, the
    cross's rows and columns (not eligible: the residual vanishes there), and
    the residual E(rho, gamma) = A(rho, gamma) - B_k(rho, :) R_{k+1}(:, gamma)."""
    M: int
    Ncol: int
    row_ok: np.ndarray
    col_ok: np.ndarray
    residual: object


def _superblock(problem, st: CrossState, k: int, B: np.ndarray, Ynext: np.ndarray) -> Optional[_Superblock]:
    Nk = problem.N[k - 1]
    rk = st.rank(k)
    M = st.rank(k - 1) * Nk
    R = Ynext.reshape(rk, -1)
    Ncol = R.shape[1]
    if M <= rk or Ncol <= rk:
        return None                                       # superblock already fully crossed
    row_ok = np.ones(M, dtype=bool)
    row_ok[cross_rows(problem, st, k)] = False
    col_ok = np.ones(Ncol, dtype=bool)
    col_ok[cross_cols(problem, st, k)] = False

    def residual(rows, cols):
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        A = superblock_entries(problem, st, k, rows, cols)
        approx = np.einsum("tb,bt->t", B[rows, :], R[:, cols])
        return A - approx

    return _Superblock(M, Ncol, row_ok, col_ok, residual)


def _sample_scores(problem, sb: _Superblock, k: int, sweep: int):
    """Alg. 2, first step: |E| at the interface's seeded random positions
    (-1 where a sample lies on a cross row or column)."""
    S = problem.samples_for(k)
    stream = rng.stream_id(sweep, k, rng.PURPOSE_SAMPLE)
    srows = np.array([rng.draw_index(problem.seed, stream, 2 * t, sb.M) for t in range(S)], dtype=np.int64)
    scols = np.array([rng.draw_index(problem.seed, stream, 2 * t + 1, sb.Ncol) for t in range(S)], dtype=np.int64)
    ok = sb.row_ok[srows] & sb.col_ok[scols]
    score = np.full(S, -1.0)
    if ok.any():
        score[ok] = np.abs(sb.residual(srows[ok], scols[ok]))
    return srows, scols, score, int(ok.sum())


def _rook(problem, sb: _Superblock, row: int, col: int, scale: float, trace: Optional[list] = None):
    """Rook pivoting from the start (row, col): alternate column and row
    searches until the rook condition, Eq. (2), holds or the round budget is
    spent.  The condition is tested after each search: a column search that
    returns the row searched in the previous round ends the search, since that
    row search returned the current column (the pivot already dominates its
    row and its column, and a repeated row search would return the same
    pivot).  Returns (row, col, E at the pivot, rounds, evaluations).
    trace (a list, or None): gets one entry per search run, in order,
    (kind, row, col, evaluations): kind "c" for a column search (along col,
    row the current row), "r" for a row search (along row, col the current
    column)."""
    rows_all = np.arange(sb.M)
    cols_all = np.arange(sb.Ncol)
    err = 0.0
    rounds = 0
    evals = 0
    prev_row = -1
    for _ in range(max(1, problem.rook_max)):
        rounds += 1
        cscore = np.full(sb.M, -1.0)
        cscore[sb.row_ok] = np.abs(sb.residual(rows_all[sb.row_ok], np.full(int(sb.row_ok.sum()), col)))
        evals += int(sb.row_ok.sum())
        if trace is not None:
            trace.append(("c", row, col, int(sb.row_ok.sum())))
        row = tie_argmax(cscore, scale)
        if row == prev_row:
            break
        rres = np.zeros(sb.Ncol)
        rres[sb.col_ok] = sb.residual(np.full(int(sb.col_ok.sum()), row), cols_all[sb.col_ok])
        evals += int(sb.col_ok.sum())
        if trace is not None:
            trace.append(("r", row, col, int(sb.col_ok.sum())))
        rscore = np.where(sb.col_ok, np.abs(rres), -1.0)
        new_col = tie_argmax(rscore, scale)
        err = float(rres[new_col])
        if new_col == col:
            break
        prev_row = row
        col = new_col
    return row, col, err, rounds, evals


def pivot_search(problem, st: CrossState, k: int, B: np.ndarray, Ynext: np.ndarray,
                 sweep: int, scale: float) -> Optional[Pivot]:
    """Alg. 2 on superblock k with the index sets of the previous sweep (Alg. 6).
    Residual E(rho, gamma) = A(rho, gamma) - B_k(rho, :) R_{k+1}(:, gamma),
    R_{k+1} = Y_{k+1} as r_k x (N_{k+1} r_{k+1}): the best random sample starts
    the rook pivoting; its pivot is accepted when |E| > pivot_tol * scale and
    r_k < rank cap."""
    sb = _superblock(problem, st, k, B, Ynext)
    if sb is None:
        return None
    srows, scols, score, evals = _sample_scores(problem, sb, k, sweep)
    t = tie_argmax(score, scale)
    if t < 0:
        return None
    row, col, err, rounds, ev = _rook(problem, sb, int(srows[t]), int(scols[t]), scale)
    accepted = abs(err) > problem.pivot_tol * scale and st.rank(k) < problem.rank_cap
    return Pivot(k=k, row=row, col=col, err=err, accepted=bool(accepted), rounds=rounds, evals=evals + ev)


def schur_step(Mx: np.ndarray, a: int, c: int, rows_left: List[int], cols_left: List[int]) -> None:
    """Replace the rows and columns left of Mx by the Schur complement of the
    pivot Mx[a, c]: M_be <- M_be - M_bc M_ae / M_ac."""
    piv = Mx[a, c]
    for b in rows_left:
        for e in cols_left:
            Mx[b, e] = Mx[b, e] - (Mx[b, c] * Mx[a, e]) / piv


def greedy_cross(Mx: np.ndarray, scale: float, pivot_tol: float, room: int):
    """Greedy complete pivoting on the square residual matrix Mx (modified in
    place): the largest |M_ac| over the rows and columns left (tie window,
    first in row-major order) while it exceeds pivot_tol * scale and fewer than
    `room` pivots were taken; each taken pivot is followed by schur_step.
    Returns [(a, c, pivot)] in order; the product of the pivots is the
    determinant of Mx restricted to the taken rows and columns, in that order."""
    m = Mx.shape[0]
    rows_left = list(range(m))
    cols_left = list(range(m))
    out = []
    while rows_left and len(out) < room:
        score = np.full((m, m), -1.0)
        for a in rows_left:
            for c in cols_left:
                if np.isfinite(Mx[a, c]):
                    score[a, c] = abs(Mx[a, c])
        t = tie_argmax(score.ravel(), scale)
        if t < 0:
            break
        a, c = divmod(t, m)
        piv = float(Mx[a, c])
        if not abs(piv) > pivot_tol * scale:
            break
        out.append((a, c, piv))
        rows_left.remove(a)
        cols_left.remove(c)
        schur_step(Mx, a, c, rows_left, cols_left)
    return out


@dataclasses.dataclass
class MultiPivot:
    """Interface k's outcome with several pivots per sweep: the rook searches
    run (one Pivot each, with its own residual), the residual matrix of their
    rows and columns, and the pivots accepted from it in acceptance order (err:
    the Schur pivot)."""
    k: int
    searches: List[Pivot]
    cross: np.ndarray
    pivots: List[Pivot]
    evals: int

    @property
    def accepted(self) -> bool:
        return len(self.pivots) > 0


def pivot_search_multi(problem, st: CrossState, k: int, B: np.ndarray, Ynext: np.ndarray,
                       sweep: int, scale: float, npiv: int, meet: bool = True) -> Optional[MultiPivot]:
    """Up to npiv pivots on superblock k in one sweep (a rank-adaptive variant;
    Alg. 6 itself adds one).  On the residual of the sweep's old cross:
      1. starts: the npiv best random samples, taken one at a time as the
         tie-window argmax among the samples whose row and column differ from
         those of the starts already taken;
      2. rook pivoting (Alg. 2) from each start;
      3. a search whose row or column equals that of an earlier search is
         dropped; a search that meets an earlier search still running at the
         same stage (the same column to search in a column step, the same row
         in a row step) stops there: from that stage on both searches take the
         same steps and end on the same pivot (only the round that ends them
         may differ by a half, and then the later one ends on the earlier
         one's pivot), which this rule would drop;
      4. the residuals at the remaining searches' rows x_a and columns y_c
         form the matrix M (M_aa: search a's own residual; the others fresh
         evaluations);
      5. greedy complete pivoting on M (cross approximation of the candidates'
         block): the largest |M_ac| over the rows and columns left (tie
         window, first in row-major order) is accepted while it exceeds
         pivot_tol * scale and the rank stays below the cap; x_a and y_c are
         appended, and M is replaced by its Schur complement
         M_bd - M_bc M_ad / M_ac.
    Each accepted pair extends the cross by a row and a column whose Schur
    pivot is nonzero, so the new cross matrix stays nonsingular:
    det G_k' = det G_k times the product of the accepted pivots.  With
    npiv = 1 this is exactly pivot_search.  meet=False runs every search to
    its end (for the tests of the meeting rule)."""
    sb = _superblock(problem, st, k, B, Ynext)
    if sb is None:
        return None
    srows, scols, score, evals = _sample_scores(problem, sb, k, sweep)
    starts: List[int] = []
    sc = score.copy()
    while len(starts) < npiv:
        t = tie_argmax(sc, scale)
        if t < 0:
            break
        starts.append(t)
        sc[(srows == srows[t]) | (scols == scols[t])] = -1.0
    if not starts:
        return None
    searches: List[Pivot] = []
    ran: List[int] = []                  # per search: the stages it ran before it ended or met another
    traces: List[list] = []
    for t in starts:
        tr: list = []
        row, col, err, rounds, ev = _rook(problem, sb, int(srows[t]), int(scols[t]), scale, tr)
        # stage s of every search is the same step of the sweep (column and row
        # searches alternate from the first column search on)
        n = len(tr)
        for s_, (kind, r_, c_, _) in enumerate(tr if meet else []):
            pos = c_ if kind == "c" else r_
            if any(s_ < ran[q] and (traces[q][s_][2] if kind == "c" else traces[q][s_][1]) == pos
                   for q in range(len(searches))):
                n = s_
                break
        if n < len(tr):
            ev = sum(e for *_, e in tr[:n])
            _, row, col, _ = tr[n]
            searches.append(Pivot(k=k, row=row, col=col, err=0.0, accepted=False, rounds=n // 2 + 1, evals=ev,
                                  merged=True))
        else:
            searches.append(Pivot(k=k, row=row, col=col, err=err, accepted=False, rounds=rounds, evals=ev))
        evals += ev
        ran.append(n)
        traces.append(tr)
    kept: List[Pivot] = []
    for pv in searches:
        if not pv.merged and not any(pv.row == q.row or pv.col == q.col for q in kept):
            kept.append(pv)
    m = len(kept)
    Mx = np.empty((m, m))
    for a in range(m):
        for c in range(m):
            Mx[a, c] = kept[a].err if a == c else float(sb.residual([kept[a].row], [kept[c].col])[0])
    evals += m * (m - 1)
    cross = Mx.copy()
    room = problem.rank_cap - st.rank(k)
    pivots = [Pivot(k=k, row=kept[a].row, col=kept[c].col, err=piv, accepted=True, rounds=kept[a].rounds, evals=0)
              for a, c, piv in greedy_cross(Mx, scale, problem.pivot_tol, room)]
    return MultiPivot(k=k, searches=searches, cross=cross, pivots=pivots, evals=evals)


# ---------------------------------------------------------------------------
# initial set, sweeps, driver
# ---------------------------------------------------------------------------

def initial_state(problem) -> CrossState:
    """r0 seeded multi-indices: the init_samples random points in decreasing
    |A| (ties by draw order), each kept when its first and last node indices
    differ from those of the points already kept, until r0 are kept; their
    prefixes and suffixes are the initial nested sets (Eq. 4)."""
    d = problem.d
    r0 = getattr(problem, "r0", 1)
    stream = rng.stream_id(0, 0, rng.PURPOSE_INIT)
    pts = np.array([[rng.draw_index(problem.seed, stream, p * d + k, problem.N[k]) for k in range(d)]
                    for p in range(problem.init_samples)], dtype=np.int64)
    vals = np.abs(eval_points(problem, pts))
    vals = np.where(np.isfinite(vals), vals, -1.0)
    order = sorted(range(len(pts)), key=lambda p: (-vals[p], p))
    chosen: List[int] = []
    for p in order:
        if not vals[p] > 0:
            break
        if any(pts[p][0] == pts[q][0] or pts[p][d - 1] == pts[q][d - 1] for q in chosen):
            continue
        chosen.append(p)
        if len(chosen) == r0:
            break
    if len(chosen) < r0:
        raise ValueError("fewer than r0 usable initial points among the initial samples")
    X = pts[chosen]                                       # (r0, d)
    left = [X[:, :k].copy() for k in range(d)]
    right = [np.zeros((0, d), dtype=np.int64)] + [X[:, k:].copy() for k in range(1, d + 1)]
    left[0] = np.zeros((1, 0), dtype=np.int64)
    right[d] = np.zeros((1, 0), dtype=np.int64)
    return CrossState(left, right)


def apply_pivots(problem, st: CrossState, pivots: List[Pivot]) -> CrossState:
    """Append every accepted pivot after the whole sweep (Alg. 6): the new row
    (alpha*, i*) extends I_<=k, the new column (j*, beta*) extends I_>k; both are
    nested in the previous sweep's neighbours by construction."""
    new = st.copy()
    flat: List[Pivot] = []
    for pv in pivots:
        if isinstance(pv, MultiPivot):
            flat.extend(pv.pivots)                        # in acceptance order
        elif pv is not None:
            flat.append(pv)
    for pv in flat:
        if not pv.accepted:
            continue
        k = pv.k
        Nk = problem.N[k - 1]
        rn = st.rank(k + 1)
        alpha, i = divmod(pv.row, Nk)
        j, beta = divmod(pv.col, rn)
        lrow = np.concatenate([st.left[k - 1][alpha], [i]]).reshape(1, k)
        rrow = np.concatenate([[j], st.right[k + 1][beta]]).reshape(1, problem.d - k)
        new.left[k] = np.vstack([new.left[k], lrow])
        new.right[k] = np.vstack([new.right[k], rrow])
    return new


@dataclasses.dataclass
class SweepRecord:
    value: float
    ranks: List[int]
    pivots: List[Optional[Pivot]]
    scale: float


def search_all(problem, st: CrossState, s: int, cores: List[np.ndarray], scale: float) -> list:
    """Alg. 6 with one superblock per interface: Alg. 2 on every interface k
    (independently, on the sets of this sweep); interfaces at the cap skip.
    With problem.npiv > 1 every interface runs pivot_search_multi (a
    MultiPivot per interface instead of a Pivot)."""
    npiv = getattr(problem, "npiv", 1)
    pivots: list = []
    for k in range(1, problem.d):
        if st.rank(k) >= problem.rank_cap:
            pivots.append(None)
            continue
        B = maxvol_coefficients(cores[k - 1], cross_rows(problem, st, k))
        if npiv > 1:
            pivots.append(pivot_search_multi(problem, st, k, B, cores[k], s, scale, npiv))
        else:
            pivots.append(pivot_search(problem, st, k, B, cores[k], s, scale))
    return pivots


def search_sequential(problem, st: CrossState, s: int, cores: List[np.ndarray], scale: float):
    """Alg. 5, one left-to-right sweep: for k = 1..d-1 in turn, Alg. 2 on the
    superblock A(I_<=k-1^new i_k, i_{k+1} I_>k+1) built from the left set just
    updated at step k-1 and the right set of the previous sweep, and the pivot
    appended at once.  Cores k-1 and k change with step k-1's append and are
    re-evaluated; scale is the largest |entry| evaluated so far.  Returns the
    updated state, the pivots and the scale."""
    d = problem.d
    cores = list(cores)
    pivots: List[Optional[Pivot]] = []
    for k in range(1, d):
        if k > 1 and pivots[-1] is not None and pivots[-1].accepted:
            for q in (k - 1, k):                     # I_>k-1 and I_<=k-1 grew at step k-1
                cores[q - 1] = core(problem, st, q)
                scale = max(scale, float(np.max(np.abs(cores[q - 1]))))
        if st.rank(k) >= problem.rank_cap:
            pivots.append(None)
            continue
        B = maxvol_coefficients(cores[k - 1], cross_rows(problem, st, k))
        pv = pivot_search(problem, st, k, B, cores[k], s, scale)
        pivots.append(pv)
        if pv is not None and pv.accepted:
            st = apply_pivots(problem, st, [pv])
    return st, pivots, scale


def sweep(problem, st: CrossState, s: int, search: bool = True):
    """One sweep: cores, their largest |entry|, the integral, then (optionally)
    the pivot search on every interface."""
    cores = [core(problem, st, k) for k in range(1, problem.d + 1)]
    scale = max(float(np.max(np.abs(c))) for c in cores)
    value = integral_plain(problem, st, cores)
    pivots = search_all(problem, st, s, cores, scale) if search else []
    return value, cores, scale, pivots


def integrate(problem, state: Optional[CrossState] = None, record: bool = True, sequential: bool = False):
    """Run sweeps until a stopping rule fires.  Returns a dict with the value,
    status, sweeps, N_eval (core entries + search evaluations + initial scan),
    final ranks, per-sweep history and the final state.  sequential: each
    sweep is Alg. 5 (search_sequential) instead of Alg. 6 (search_all)."""
    d = problem.d
    if d < 2:
        raise ValueError("the cross needs d >= 2")
    if sequential and getattr(problem, "npiv", 1) > 1:
        raise ValueError("the sequential sweep takes one pivot per step")
    st = state.copy() if state is not None else initial_state(problem)
    history: List[SweepRecord] = []
    search_evals = 0
    prev = None
    changes: List[float] = []
    status = STATUS_MAX_SWEEPS
    value = float("nan")
    conv = float("inf")
    limit = problem.sweeps_limit()
    for s in range(limit):
        at_cap = all(st.rank(k) >= problem.rank_cap for k in range(1, d))
        last = (s == limit - 1)
        value, cores, scale, _ = sweep(problem, st, s, search=False)
        if prev is not None:
            conv = abs(value - prev) / abs(value) if value != 0 else abs(value - prev)
            changes.append(conv)
        if len(changes) >= problem.conv_window and max(changes[-problem.conv_window:]) <= problem.tol:
            status = STATUS_CONVERGED
            history.append(SweepRecord(value, st.ranks(), [], scale))
            break
        if at_cap:
            status = STATUS_RANK_CAP
            history.append(SweepRecord(value, st.ranks(), [], scale))
            break
        if last:
            status = STATUS_MAX_SWEEPS
            history.append(SweepRecord(value, st.ranks(), [], scale))
            break
        ranks_before = st.ranks()
        if sequential:
            new_st, pivots, scale = search_sequential(problem, st, s, cores, scale)
        else:
            pivots = search_all(problem, st, s, cores, scale)
        search_evals += sum(p.evals for p in pivots if p is not None)
        history.append(SweepRecord(value, ranks_before, pivots, scale))
        if not any(p is not None and p.accepted for p in pivots):
            status = STATUS_NO_PIVOT
            break
        st = new_st if sequential else apply_pivots(problem, st, pivots)
        prev = value
    ranks = st.ranks()
    core_entries = sum(ranks[k - 1] * problem.N[k - 1] * ranks[k] for k in range(1, d + 1))
    return {
        "value": value,
        "status": status,
        "sweeps": len(history),
        "internal_conv": conv,
        "n_eval": core_entries + search_evals + problem.init_samples,
        "ranks": ranks,
        "max_rank": max(ranks),
        "history": history if record else None,
        "state": st,
    }
