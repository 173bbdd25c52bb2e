"""Pins of the oracle's Algorithm 2 (HPSCDP, blocks of thr columns updated from
one residual, Sec. 7) and Algorithm 3 (HPSCDF, greedy feature selection,
Sec. 8), each against something other than itself (no GPU)."""
import numpy as np
import pytest

import oracle
from paper_2104_12570_gb300 import synth


def sys64(m, n, seed, noise=0.05):
    return synth.make_system(m, n, seed=seed, noise=noise, dtype="f64", consistent_rhs_dtype="f64")


def blocks(s, thr, sweeps, **kw):
    return oracle.solve_blocks(s.X, s.y, m=s.m, n=s.n, thr=thr, dtype=s.dtype, tol=0,
                               max_sweeps=sweeps, stop="none", **kw)


# ---------------- Algorithm 2 ----------------

def test_thr_one_is_algorithm_1():
    s = sys64(300, 40, 1)
    o1 = oracle.solve_system(s, tol=0, max_sweeps=6, stop="none")
    o2 = blocks(s, 1, 6)
    np.testing.assert_allclose(o2.a, o1.a, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(o2.hist, o1.hist, rtol=1e-12)


@pytest.mark.parametrize("thr", [3, 7, 16, 40, 100])
def test_one_sweep_is_the_block_splitting(thr):
    """One sweep of Algorithm 2 is a <- a + (D + L_B)^{-1} X^T (y - X a), where
    L_B holds the couplings G_jl of columns l in EARLIER blocks than j (within a
    block every column sees the same residual); thr >= n is the Jacobi iteration."""
    s = sys64(120, 40, 2)
    X = s.dense_f64()
    G = X.T @ X
    n = s.n
    blk = np.arange(n) // thr
    M = np.diag(np.diag(G)) + np.where(blk[:, None] > blk[None, :], G, 0.0)
    a = np.zeros(n)
    for k in range(1, 5):
        a = a + np.linalg.solve(M, X.T @ (s.y - X @ a))
        o = blocks(s, thr, k)
        np.testing.assert_allclose(o.a, a, rtol=1e-9, atol=1e-12)


def test_jacobi_limit_thr_ge_n():
    s = sys64(200, 12, 3)
    X = s.dense_f64()
    d = (X * X).sum(axis=0)
    a = np.zeros(s.n)
    for _ in range(3):
        a = a + (X.T @ (s.y - X @ a)) / d
    np.testing.assert_allclose(blocks(s, 12, 3).a, a, rtol=1e-10)
    np.testing.assert_allclose(blocks(s, 1000, 3).a, a, rtol=1e-10)


def test_blocks_bookkeeping_and_orthogonal_columns():
    s = sys64(150, 30, 4)
    o = blocks(s, 7, 5, want_e=True)
    X = s.dense_f64()
    np.testing.assert_allclose(o.e, s.y - X @ o.a, rtol=0, atol=1e-11 * np.linalg.norm(s.y))
    # orthogonal columns: every block step is exact, one sweep reaches X^T y ⊘ d for any thr
    g = np.random.default_rng(5)
    Q, _ = np.linalg.qr(g.standard_normal((80, 10)))
    Q = Q * np.linspace(1, 3, 10)
    y = g.standard_normal(80)
    Xs = np.ascontiguousarray(Q.T)
    for thr in (1, 3, 10):
        r = oracle.solve_blocks(Xs, y, m=80, n=10, thr=thr, dtype="f64", tol=0, max_sweeps=1,
                                stop="none")
        np.testing.assert_allclose(r.a, (Q.T @ y) / (Q * Q).sum(axis=0), rtol=1e-12)


# ---------------- Algorithm 3 ----------------

def test_selection_minimises_E_by_its_closed_form():
    """E_j = ||e - X_j da_j||^2 = ||e||^2 - <X_j,e>^2 / <X_j,X_j>: the oracle's
    literal argmin over E must be the argmax of the closed form at every step,
    the chosen column is orthogonal to the new residual, and ||e|| never grows."""
    s = sys64(90, 25, 6)
    X = s.dense_f64()
    F = 12
    sel, a, hist = oracle.select(s.X, s.y, m=s.m, n=s.n, F=F, dtype="f64")
    e = s.y.copy()
    d = (X * X).sum(axis=0)
    aa = np.zeros(s.n)
    for f in range(F):
        c = X.T @ e
        score = c * c / d
        j = int(np.argmax(score))
        assert sel[f] == j
        aa[j] += c[j] / d[j]
        e = e - X[:, j] * (c[j] / d[j])
        assert abs(X[:, j] @ e) <= 1e-10 * np.linalg.norm(X[:, j]) * np.linalg.norm(e) + 1e-14
        assert hist[f + 1] <= hist[f] + 1e-15
    np.testing.assert_allclose(a, aa, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(s.y - X @ a, e, atol=1e-12)


def test_orthogonal_features_are_selected_by_correlation():
    g = np.random.default_rng(7)
    Q, _ = np.linalg.qr(g.standard_normal((60, 12)))
    Q = Q * g.uniform(0.5, 2.0, 12)
    y = g.standard_normal(60)
    Xs = np.ascontiguousarray(Q.T)
    sel, a, hist = oracle.select(Xs, y, m=60, n=12, F=12, dtype="f64")
    c = Q.T @ y
    d = (Q * Q).sum(axis=0)
    np.testing.assert_array_equal(sel, np.argsort(-(c * c / d), kind="stable"))
    np.testing.assert_allclose(a, c / d, rtol=1e-12)
    # all features selected: the residual is y's component outside the span
    P = Q @ np.linalg.solve(Q.T @ Q, Q.T @ y)
    assert hist[-1] == pytest.approx(np.linalg.norm(y - P) / np.linalg.norm(y), rel=1e-10)


def test_planted_support_is_found_first():
    g = np.random.default_rng(8)
    m, n = 400, 60
    X = g.standard_normal((m, n))
    S = [5, 17, 33, 48]
    y = X[:, S] @ np.array([3.0, -2.5, 2.0, -1.5])
    Xs = np.ascontiguousarray(X.T)
    sel, a, hist = oracle.select(Xs, y, m=m, n=n, F=4, dtype="f64")
    assert sorted(sel.tolist()) == S
    assert hist[-1] < 0.2


def test_reselection_accumulates_and_keeps_the_bookkeeping():
    """Correlated columns make the greedy step come back to a chosen column; the
    update a_j <- a_j + da_j keeps e = y - X·a (the printed assignment agrees with
    it for a column chosen the first time, where a_j = 0)."""
    g = np.random.default_rng(9)
    base = g.standard_normal(50)
    X = np.stack([base + 0.3 * g.standard_normal(50) for _ in range(4)], axis=1)
    y = X @ np.array([1.0, 1.0, -0.5, 0.7])
    Xs = np.ascontiguousarray(X.T)
    sel, a, hist = oracle.select(Xs, y, m=50, n=4, F=20, dtype="f64")
    assert len(set(sel.tolist())) < len(sel)  # some column was chosen more than once
    e = y - X @ a
    assert np.linalg.norm(e) / np.linalg.norm(y) == pytest.approx(hist[-1], rel=1e-9)
    assert np.all(np.diff(hist) <= 1e-15)


# ---------------- Algorithm 1 with a given column order (Sec. 2's random index variant) ----------------

def order_solve(s, order, sweeps, **kw):
    return oracle.solve_order(s.X, s.y, m=s.m, n=s.n, order=order, dtype=s.dtype, tol=0,
                              max_sweeps=sweeps, stop="none", **kw)


def test_natural_order_is_algorithm_1():
    s = sys64(200, 30, 21)
    order = np.tile(np.arange(30), (5, 1))
    o1 = oracle.solve_system(s, tol=0, max_sweeps=5, stop="none")
    o2 = order_solve(s, order, 5)
    np.testing.assert_array_equal(o2.a, o1.a)
    np.testing.assert_array_equal(o2.hist, o1.hist)


def test_fixed_permutation_is_algorithm_1_on_permuted_columns():
    """Taking the columns in the order pi every sweep is Algorithm 1 on the
    system whose k-th column is X_pi(k); its k-th coefficient is a_pi(k)."""
    s = sys64(150, 25, 22)
    pi = np.random.default_rng(3).permutation(25)
    Xp = np.ascontiguousarray(s.X[pi])  # column-major storage: row k of s.X is column k
    op = oracle.solve(Xp, s.y, m=s.m, n=s.n, dtype="f64", tol=0, max_sweeps=4, stop="none")
    oo = order_solve(s, np.tile(pi, (4, 1)), 4)
    a = np.empty(25)
    a[pi] = op.a
    np.testing.assert_allclose(oo.a, a, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(oo.hist, op.hist, rtol=1e-12)


def test_repeated_index_sweep_is_one_projection():
    """A sweep that takes the same column n times moves only that column, once:
    after the first step <X_q, e> = 0, so the repeats add nothing."""
    s = sys64(120, 10, 23)
    X = s.dense_f64()
    for q in (0, 4, 9):
        o = order_solve(s, np.full((1, 10), q), 1, want_e=True)
        a = np.zeros(10)
        a[q] = X[:, q] @ s.y / (X[:, q] @ X[:, q])
        np.testing.assert_allclose(o.a, a, rtol=1e-12, atol=1e-15)
        assert abs(X[:, q] @ o.e) <= 1e-12 * np.linalg.norm(X[:, q]) * np.linalg.norm(s.y)


def test_random_indices_bookkeeping_monotone_and_limit():
    """Indices drawn with replacement: e = y - X·a, ||e|| never grows, the last
    step's column is orthogonal to the residual, and the iterates reach the
    least-squares solution."""
    s = sys64(300, 20, 24)
    X = s.dense_f64()
    order = np.random.default_rng(4).integers(0, 20, size=(400, 20))
    o = order_solve(s, order, 400, want_e=True)
    np.testing.assert_allclose(o.e, s.y - X @ o.a, atol=1e-11 * np.linalg.norm(s.y))
    assert np.all(np.diff(o.hist) <= 1e-15)
    q = order[-1, -1]
    assert abs(X[:, q] @ o.e) <= 1e-12 * np.linalg.norm(X[:, q]) * np.linalg.norm(s.y)
    a_ls = np.linalg.lstsq(X, s.y, rcond=None)[0]
    np.testing.assert_allclose(o.a, a_ls, rtol=1e-8, atol=1e-10)


def test_order_rejects_indices_outside_the_columns():
    s = sys64(50, 6, 25)
    with pytest.raises(ValueError):
        order_solve(s, np.full((2, 6), 6), 2)
    with pytest.raises(ValueError):
        order_solve(s, np.full((2, 6), -1), 2)


# ---------------- the feature-removal loop of Sec. 8 (swap steps after Algorithm 3) ----------------

def test_swap_with_no_rounds_is_algorithm_3():
    s = sys64(120, 30, 31)
    sel, a, hist = oracle.select(s.X, s.y, m=s.m, n=s.n, F=8, dtype="f64")
    sel2, swaps, a2, hist2 = oracle.select_swap(s.X, s.y, m=s.m, n=s.n, F=8, R=0, dtype="f64")
    np.testing.assert_array_equal(sel2, sel)
    np.testing.assert_array_equal(a2, a)
    np.testing.assert_array_equal(hist2, hist)


def test_swaps_recover_the_planted_support_greedy_missed():
    """Correlated columns (three latent factors) and a planted support {1, 5, 9}:
    the greedy steps take {10, 9, 1}; the swap steps exchange 10 -> 5, 9 -> 11,
    11 -> 9 and end on the planted support.  Every swap lowers the error, the
    refitted column is orthogonal to the residual it leaves (Eq. res-x), and
    e = y - X·a holds."""
    g = np.random.default_rng(1)
    m, n = 200, 16
    base = g.standard_normal((m, 3))
    X = base @ g.standard_normal((3, n)) + 0.5 * g.standard_normal((m, n))
    y = X[:, [1, 5, 9]] @ np.array([1.0, -0.8, 0.6]) + 0.05 * g.standard_normal(m)
    Xs = np.ascontiguousarray(X.T)
    sel, swaps, a, hist = oracle.select_swap(Xs, y, m=m, n=n, F=3, R=4, dtype="f64")
    assert sorted(sel.tolist()) == [1, 9, 10]
    assert swaps.tolist() == [[10, 5], [9, 11], [11, 9], [-1, -1]]
    assert sorted(np.flatnonzero(a).tolist()) == [1, 5, 9]
    assert np.all(np.diff(hist) < 0)
    e = y - X @ a
    assert abs(X[:, 9] @ e) <= 1e-10 * np.linalg.norm(X[:, 9]) * np.linalg.norm(e)
    assert hist[-1] == pytest.approx(np.linalg.norm(e) / np.linalg.norm(y), rel=1e-12)


def test_swap_is_the_best_exchange_and_keeps_the_bookkeeping():
    """Each swap is the single exchange (drop k, add j refitted on the residual
    without k) of least error: brute force over every exchange by a least-squares
    fit of the one new coefficient (numpy lstsq) agrees; e = y - X·a throughout."""
    g = np.random.default_rng(13)
    m, n = 150, 12
    base = g.standard_normal(m)
    X = np.stack([base * (0.6 if c % 3 == 0 else 0.1) + g.standard_normal(m) for c in range(n)], axis=1)
    y = X @ g.standard_normal(n) * 0.5 + X[:, 2] * 2.0
    Xs = np.ascontiguousarray(X.T)
    sel, swaps0, a0, hist0 = oracle.select_swap(Xs, y, m=m, n=n, F=4, R=0, dtype="f64")
    sel, swaps, a1, hist1 = oracle.select_swap(Xs, y, m=m, n=n, F=4, R=1, dtype="f64")
    e0 = y - X @ a0
    best, pair = None, None
    for k in np.flatnonzero(a0):
        ep = e0 + X[:, k] * a0[k]
        for j in range(n):
            if a0[j] != 0:
                continue
            coef = np.linalg.lstsq(X[:, [j]], ep, rcond=None)[0][0]
            E = np.sum((ep - X[:, j] * coef) ** 2)
            if best is None or E < best:
                best, pair = E, (k, j)
    if best < e0 @ e0:
        assert tuple(swaps[0]) == pair
        np.testing.assert_allclose(np.sum((y - X @ a1) ** 2), best, rtol=1e-10)
    else:
        assert tuple(swaps[0]) == (-1, -1)
    np.testing.assert_allclose(hist1[-1], np.linalg.norm(y - X @ a1) / np.linalg.norm(y), rtol=1e-12)


def test_no_swap_when_the_selection_is_already_best():
    g = np.random.default_rng(14)
    Q, _ = np.linalg.qr(g.standard_normal((60, 10)))
    y = Q @ np.array([5.0, 4.0, 3.0, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1])
    sel, swaps, a, hist = oracle.select_swap(np.ascontiguousarray(Q.T), y, m=60, n=10, F=3, R=4,
                                             dtype="f64")
    assert sorted(sel.tolist()) == [0, 1, 2]
    assert np.all(swaps == -1) and len(hist) == 4


# ---------------- worked 2 x 2 example, closed forms by hand ----------------
#
# X = [[1, 1], [0, 1]] (rows), so X_1 = (1, 0), X_2 = (1, 1), d = (1, 2); y = (2, 1),
# whose unique solution is a = (1, 1).  Every iterate below is a dyadic rational,
# so float64 reproduces it exactly.

X22 = np.array([[1.0, 1.0], [0.0, 1.0]])
Y22 = np.array([2.0, 1.0])


def _col22():
    return np.ascontiguousarray(X22.T)  # column-major storage


def test_worked_2x2_algorithm_2_is_jacobi_in_closed_form():
    """thr = 2 puts both columns in one block: every step uses the residual at the
    start of the sweep (Jacobi on G = [[1, 1], [1, 2]]).  The error a - (1, 1)
    is multiplied by M = I - D^-1 G = [[0, -1], [-1/2, 0]] each sweep, so from
    a = 0: after 2k sweeps a = (1 - 2^-k)(1, 1), e = (2^(1-k), 2^-k); after 2k + 1
    sweeps a = (1 + 2^-k, 1 + 2^-(k+1)), e = -(3, 1)·2^-(k+1)."""
    for s in range(1, 9):
        k = s // 2
        if s % 2 == 0:
            a = [1 - 2.0 ** -k, 1 - 2.0 ** -k]
            e = [2.0 ** (1 - k), 2.0 ** -k]
        else:
            a = [1 + 2.0 ** -k, 1 + 2.0 ** -(k + 1)]
            e = [-3 * 2.0 ** -(k + 1), -(2.0 ** -(k + 1))]
        r = oracle.solve_blocks(_col22(), Y22, m=2, n=2, thr=2, dtype="f64", tol=0, max_sweeps=s,
                                stop="none", want_e=True)
        np.testing.assert_array_equal(r.a, a)
        np.testing.assert_array_equal(r.e, e)
        assert r.hist[s] == pytest.approx(np.hypot(*e) / np.sqrt(5.0), rel=1e-15)


def test_worked_2x2_algorithm_3_alternates_in_closed_form():
    """Greedy selection from a = 0: step 1 compares E_1 = 1 with E_2 = 1/2 and takes
    column 2; from then on the column orthogonal to the residual gains nothing and
    the steps alternate 2, 1, 2, 1, ...  After 2k steps a = (1 - 2^-k, 1 + 2^-k),
    e = (0, -2^-k); after 2k + 1 steps a = (1 - 2^-k, 1 + 2^-(k+1)),
    e = 2^-(k+1)·(1, -1)."""
    for F in range(1, 9):
        sel, a, hist = oracle.select(_col22(), Y22, m=2, n=2, F=F, dtype="f64")
        assert list(sel) == [1 if i % 2 == 0 else 0 for i in range(F)]  # 0-based
        k = F // 2
        if F % 2 == 0:
            a_cf, e_cf = [1 - 2.0 ** -k, 1 + 2.0 ** -k], [0.0, -(2.0 ** -k)]
        else:
            a_cf, e_cf = [1 - 2.0 ** -k, 1 + 2.0 ** -(k + 1)], [2.0 ** -(k + 1), -(2.0 ** -(k + 1))]
        np.testing.assert_array_equal(a, a_cf)
        assert hist[F] == pytest.approx(np.hypot(*e_cf) / np.sqrt(5.0), rel=1e-15)


def test_worked_2x2_given_order_repeating_one_column():
    """Sweep 1 takes column 2 twice, sweep 2 column 1 twice: the repeat of a column
    right after its own step finds <X_j, e> = 0 and changes nothing, so
    a = (0, 3/2), e = (1/2, -1/2) after sweep 1 and a = (1/2, 3/2), e = (0, -1/2)
    after sweep 2."""
    order = np.array([[1, 1], [0, 0]])
    r1 = oracle.solve_order(_col22(), Y22, m=2, n=2, order=order[:1], dtype="f64", tol=0,
                            max_sweeps=1, stop="none", want_e=True)
    np.testing.assert_array_equal(r1.a, [0.0, 1.5])
    np.testing.assert_array_equal(r1.e, [0.5, -0.5])
    r2 = oracle.solve_order(_col22(), Y22, m=2, n=2, order=order, dtype="f64", tol=0,
                            max_sweeps=2, stop="none", want_e=True)
    np.testing.assert_array_equal(r2.a, [0.5, 1.5])
    np.testing.assert_array_equal(r2.e, [0.0, -0.5])
