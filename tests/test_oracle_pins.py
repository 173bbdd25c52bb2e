"""Pins of the float64 CPU oracle of Algorithm 1 to facts fixed by the paper
and by mathematics, independent of the oracle's own code.

Each test names the passage it follows.  Together they are chosen so that a
plausible slip in the oracle (a sign, a dropped term, a wrong index, a Jacobi
instead of a Gauss-Seidel order, a transposed layout) fails at least one of
them; test_oracle_mutants.py plants such slips and checks exactly that.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2104_12570_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def col_major(Xd):
    """(m, n) float64 array -> oracle column-major storage (n, m)."""
    return np.ascontiguousarray(np.asarray(Xd, dtype=np.float64).T)


def run(Xd, y, **kw):
    m, n = Xd.shape
    return oracle.solve(col_major(Xd), y, m=m, n=n, layout="col", dtype="f64", **kw)


# --- worked example (Algorithm 1 by hand; tests/golden/hand_2x2.json) -------------------

def test_hand_worked_2x2():
    g = json.load(open(os.path.join(GOLDEN, "hand_2x2.json")))
    Xd = np.array(g["X_rows"])
    y = np.array(g["y"])
    for rec in g["sweeps"]:
        r = run(Xd, y, tol=0, max_sweeps=rec["s"], stop="none", want_e=True)
        assert r.sweeps == rec["s"]
        np.testing.assert_array_equal(r.a, rec["a"])      # exact: powers of two
        np.testing.assert_array_equal(r.e, rec["e"])
        assert r.hist[0] == 1.0
        for s in range(1, rec["s"] + 1):
            assert r.hist[s] == pytest.approx(np.sqrt(0.4) * 2.0 ** -s, rel=1e-15)


# --- closed form for a single column (Eq. da, Eq. da2) ----------------------------------

def test_single_column_closed_form():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((37, 1))
    y = rng.standard_normal(37)
    r = run(x, y, tol=0, max_sweeps=3, stop="none", want_e=True)
    a_cf = float(x[:, 0] @ y) / float(x[:, 0] @ x[:, 0])
    assert r.a[0] == pytest.approx(a_cf, rel=1e-14)
    # a second sweep changes nothing: the residual is already orthogonal to x
    assert r.hist[1] == pytest.approx(r.hist[3], rel=1e-13)
    np.testing.assert_allclose(r.e, y - x[:, 0] * a_cf, rtol=0, atol=1e-13)


# --- orthogonality after each column step (Eq. res-x) and monotone decrease (Eq. decr) ---

def test_orthogonality_and_monotone_decrease_per_column_step():
    rng = np.random.default_rng(2)
    m, n = 23, 7
    Xd = rng.standard_normal((m, n))
    y = rng.standard_normal(m)
    prev = np.linalg.norm(y)
    for k in range(1, 3 * n + 1):
        r = run(Xd, y, tol=0, max_sweeps=5, stop="none", max_col_steps=k, want_e=True)
        j = (k - 1) % n
        xj = Xd[:, j]
        # right after the step on column j, the residual is orthogonal to X_j
        assert abs(xj @ r.e) <= 1e-13 * np.linalg.norm(xj) * max(np.linalg.norm(r.e), 1e-300)
        cur = np.linalg.norm(r.e)
        assert cur <= prev * (1 + 1e-15)
        prev = cur


# --- bookkeeping: e always equals y - X·a (Eq. ek1-ek) ---------------------------------

@pytest.mark.parametrize("sweeps", [1, 2, 5])
def test_residual_bookkeeping(sweeps):
    rng = np.random.default_rng(3)
    Xd = rng.standard_normal((31, 11))
    y = rng.standard_normal(31)
    a0 = rng.standard_normal(11)
    r = run(Xd, y, a0=a0, tol=0, max_sweeps=sweeps, stop="none", want_e=True)
    np.testing.assert_allclose(r.e, y - Xd @ r.a, rtol=0, atol=1e-12 * np.linalg.norm(y))
    e2, nrm = oracle.residual(col_major(Xd), y, r.a, m=31, n=11, layout="col", dtype="f64")
    np.testing.assert_allclose(e2, y - Xd @ r.a, rtol=0, atol=1e-12 * np.linalg.norm(y))


# --- square consistent systems: the limit equals Gaussian elimination (Sec. 4, e_min = 0) --

def gaussian_elimination(A, b):
    """Textbook Gaussian elimination with partial pivoting (tiny inputs)."""
    A = np.array(A, dtype=np.float64)
    b = np.array(b, dtype=np.float64)
    n = len(b)
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        A[[k, p]], b[[k, p]] = A[[p, k]], b[[p, k]]
        for i in range(k + 1, n):
            f = A[i, k] / A[k, k]
            A[i, k:] -= f * A[k, k:]
            b[i] -= f * b[k]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (b[i] - A[i, i + 1:] @ x[i + 1:]) / A[i, i]
    return x


@pytest.mark.parametrize("n", [1, 5, 20, 50])
def test_square_consistent_matches_gaussian_elimination(n):
    rng = np.random.default_rng(10 + n)
    Xd = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    a_star = rng.uniform(-1, 1, n)
    y = Xd @ a_star
    r = run(Xd, y, tol=1e-14, max_sweeps=5000, stop="rel_res")
    assert r.status == "ok"
    ge = gaussian_elimination(Xd, y)
    np.testing.assert_allclose(ge, np.linalg.solve(Xd, y), rtol=1e-12, atol=1e-13)
    assert np.linalg.norm(r.a - ge) <= 1e-9 * np.linalg.norm(ge)
    # residual goes to zero on a consistent system (Theorem 1 with e_min = 0)
    assert r.hist[-1] <= 1e-14


# --- tall least squares: the limit is the normal-equations solution (Sec. 4, e_min > 0) --

def test_tall_least_squares_matches_normal_equations():
    s = synth.make_system(200, 50, seed=5, dtype="f64", noise=0.3, consistent_rhs_dtype="f64")
    Xd = s.dense_f64()
    # the change of ||e|| is second order in the coefficient error, so run a
    # fixed number of sweeps rather than a change-based stop
    r = oracle.solve_system(s, tol=0, max_sweeps=300, stop="none")
    G = Xd.T @ Xd
    L = np.linalg.cholesky(G)
    z = scipy.linalg.solve_triangular(L, Xd.T @ s.y, lower=True)
    a_ne = scipy.linalg.solve_triangular(L.T, z, lower=False)
    a_ls = np.linalg.lstsq(Xd, s.y, rcond=None)[0]
    np.testing.assert_allclose(a_ne, a_ls, rtol=1e-10, atol=1e-12)
    assert np.linalg.norm(r.a - a_ls) <= 1e-9 * np.linalg.norm(a_ls)
    # the limit residual is e_min of Sec. 4
    e_min = np.linalg.norm(s.y - Xd @ a_ls) / np.linalg.norm(s.y)
    assert r.rel_res == pytest.approx(e_min, rel=1e-12)


# --- orthogonal columns: one sweep is exact, a = X^T y ⊘ d ------------------------------

def test_orthogonal_columns_one_sweep():
    rng = np.random.default_rng(6)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 9)))
    Xd = Q * rng.uniform(0.5, 3.0, 9)  # orthogonal, not normalised
    y = rng.standard_normal(40)
    r1 = run(Xd, y, tol=0, max_sweeps=1, stop="none")
    d = np.einsum("ij,ij->j", Xd, Xd)
    np.testing.assert_allclose(r1.a, (Xd.T @ y) / d, rtol=1e-13, atol=1e-14)
    r2 = run(Xd, y, tol=0, max_sweeps=2, stop="none")
    np.testing.assert_allclose(r2.a, r1.a, rtol=1e-13, atol=1e-14)


# --- one sweep of Algorithm 1 is one Gauss-Seidel sweep on X^T X a = X^T y -------------
# (a textbook equivalence: coordinate-wise exact line search on ||y - Xa||^2;
#  the iterate is written here in the matrix splitting form, not per column)

@pytest.mark.parametrize("shape", [(30, 8), (8, 30), (12, 12)])
def test_gauss_seidel_equivalence(shape):
    m, n = shape
    rng = np.random.default_rng(7)
    Xd = rng.standard_normal((m, n))
    y = rng.standard_normal(m)
    a0 = rng.standard_normal(n)
    G = Xd.T @ Xd
    DL = np.tril(G)
    a = a0.copy()
    for s in range(1, 5):
        a = a + scipy.linalg.solve_triangular(DL, Xd.T @ y - G @ a, lower=True)
        r = run(Xd, y, a0=a0, tol=0, max_sweeps=s, stop="none")
        np.testing.assert_allclose(r.a, a, rtol=1e-10, atol=1e-10 * np.linalg.norm(a))


# --- wide consistent systems: residual -> 0, a is one of infinitely many solutions ------

def test_wide_consistent_residual_to_zero():
    s = synth.make_system(20, 60, seed=8, layout="row", dtype="f64", consistent_rhs_dtype="f64")
    r = oracle.solve_system(s, tol=1e-12, max_sweeps=10000, stop="rel_res")
    assert r.status == "ok" and r.rel_res <= 1e-12
    Xd = s.dense_f64()
    assert np.linalg.norm(s.y - Xd @ r.a) <= 1e-11 * np.linalg.norm(s.y)
    # the hist is non-increasing (Eq. decr, sweep by sweep)
    assert np.all(np.diff(r.hist) <= 0)


# --- the stored workload: config-1 shape, consistent, converges to a_true ---------------

def test_tall_200x50_converges_to_a_true():
    s = synth.workload("tall_200x50_f64")
    r = oracle.solve_system(s, tol=1e-10, max_sweeps=1000, stop="rel_res")
    assert r.status == "ok" and r.rel_res <= 1e-10
    assert np.all(np.diff(r.hist) <= 0)
    assert np.linalg.norm(r.a - s.a_true) <= 1e-8 * np.linalg.norm(s.a_true)


# --- zero columns are skipped; warm starts; stopping rules ------------------------------

def test_zero_column_is_skipped():
    rng = np.random.default_rng(9)
    Xd = rng.standard_normal((25, 6))
    Xd[:, 2] = 0.0
    a_star = rng.uniform(-1, 1, 6)
    a_star[2] = 0.0
    y = Xd @ a_star
    a0 = np.zeros(6)
    a0[2] = 0.75
    r = run(Xd, y - Xd @ a0, tol=1e-13, max_sweeps=500, stop="rel_res")
    assert np.all(np.isfinite(r.a)) and r.a[2] == 0.0
    r2 = run(Xd, y, a0=a0, tol=1e-13, max_sweeps=500, stop="rel_res")
    assert r2.a[2] == 0.75  # never touched
    keep = [0, 1, 3, 4, 5]
    np.testing.assert_allclose(r2.a[keep], a_star[keep], rtol=1e-10, atol=1e-11)


def test_warm_start_at_solution_stops_at_sweep_zero():
    s = synth.workload("tall_200x50_f64")
    Xd = s.dense_f64()
    r = oracle.solve_system(s, a0=s.a_true, tol=1e-10, max_sweeps=10, stop="rel_res")
    assert r.sweeps == 0 and r.status == "ok"
    assert r.hist[0] == pytest.approx(np.linalg.norm(s.y - Xd @ s.a_true) / np.linalg.norm(s.y),
                                      abs=1e-15)


def test_stopping_rules():
    s = synth.make_system(120, 30, seed=11, dtype="f64", noise=0.1, consistent_rhs_dtype="f64")
    tol = 1e-6
    r = oracle.solve_system(s, tol=tol, max_sweeps=500, stop="rel_change")
    h = r.hist
    assert r.status == "ok"
    assert abs(h[-2] - h[-1]) < tol * h[-2]
    for k in range(1, len(h) - 1):
        assert not abs(h[k - 1] - h[k]) < tol * h[k - 1]
    r2 = oracle.solve_system(s, tol=1e-3, max_sweeps=2, stop="rel_res")
    assert r2.status == "not_converged" and r2.sweeps == 2  # e_min > 1e-3 here


# --- storage formats are exact promotions of the same system ----------------------------

def test_layouts_and_bf16_promote_exactly():
    s = synth.make_system(40, 13, seed=12, layout="col", dtype="bf16")
    vals = synth.bf16_bits_to_f32(s.X)  # (n, m) float32
    r_bf = oracle.solve_system(s, tol=0, max_sweeps=3, stop="none")
    r_f32 = oracle.solve(np.ascontiguousarray(vals), s.y, m=40, n=13, layout="col", dtype="f32",
                         tol=0, max_sweeps=3, stop="none")
    r_row = oracle.solve(np.ascontiguousarray(vals.T.astype(np.float64)), s.y, m=40, n=13,
                         layout="row", dtype="f64", tol=0, max_sweeps=3, stop="none")
    np.testing.assert_array_equal(r_bf.a, r_f32.a)
    np.testing.assert_array_equal(r_bf.a, r_row.a)


def test_binary16_decode_is_exact_for_every_finite_pattern():
    """The oracle widens IEEE binary16 from the format's definition: for all
    63,488 finite bit patterns (normals, subnormals, both zeros) the residual
    y - X·a with y = 0, a = 1 returns -x exactly as numpy's float16 -> float64
    conversion gives it, through the column-major and row-major readers."""
    bits = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    bits = bits[((bits >> 10) & 31) != 31]
    x16 = bits.view(np.float16)
    m = len(x16)
    want = -x16.astype(np.float64)
    for layout in ("col", "row"):
        X = np.ascontiguousarray(x16.reshape((1, m) if layout == "col" else (m, 1)))
        e, _ = oracle.residual(X, np.zeros(m), np.ones(1), m=m, n=1, layout=layout, dtype="f16")
        np.testing.assert_array_equal(e, want)
    assert want[bits == 0x0001][0] == -2.0 ** -24 and want[bits == 0x7bff][0] == -65504.0


def test_binary16_storage_is_the_float32_system():
    """A binary16 system solves exactly like the float32 system of the same
    values (every binary16 value is a float32)."""
    s = synth.make_system(50, 11, seed=13, layout="col", dtype="f16")
    vals = s.X.astype(np.float32)
    r16 = oracle.solve_system(s, tol=0, max_sweeps=4, stop="none")
    r32 = oracle.solve(np.ascontiguousarray(vals), s.y, m=50, n=11, layout="col", dtype="f32",
                       tol=0, max_sweeps=4, stop="none")
    np.testing.assert_array_equal(r16.a, r32.a)
    np.testing.assert_array_equal(r16.hist, r32.hist)


def test_empty_and_degenerate_shapes():
    y = np.array([1.0, 2.0, 3.0])
    r = oracle.solve(np.zeros((0, 3)), y, m=3, n=0, layout="col", dtype="f64", tol=1e-6,
                     max_sweeps=4, stop="rel_res")
    assert r.status == "not_converged" and np.all(r.hist == 1.0)
    r = oracle.solve(np.zeros((2, 0)), np.zeros(0), m=0, n=2, layout="col", dtype="f64",
                     tol=1e-6, max_sweeps=4, stop="rel_res")
    assert r.status == "ok" and r.sweeps == 0 and np.all(r.a == 0)
    # y = 0: relative residual falls back to the absolute norm
    r = run(np.ones((4, 2)), np.zeros(4), tol=1e-12, max_sweeps=3, stop="rel_res")
    assert r.sweeps == 0 and np.all(r.a == 0)


def test_nonfinite_inputs_are_reported():
    """A NaN in y makes ||e_0|| NaN (reported before any sweep); an infinite
    entry of X makes d_j infinite and the first column step NaN (reported after
    sweep 1)."""
    s = synth.make_system(60, 8, seed=12, dtype="f64", consistent_rhs_dtype="f64")
    y = s.y.copy()
    y[4] = np.nan
    o = oracle.solve(s.X, y, m=s.m, n=s.n, dtype="f64", tol=1e-6, max_sweeps=10)
    assert o.status == "nonfinite" and o.sweeps == 0
    X = s.X.copy()
    X[2, 7] = np.inf
    o = oracle.solve(X, s.y, m=s.m, n=s.n, dtype="f64", tol=1e-6, max_sweeps=10)
    assert o.status == "nonfinite" and o.sweeps == 1


@pytest.mark.parametrize("layout,dtype,stop", [("col", "f32", "rel_change"), ("col", "bf16", "rel_res"),
                                               ("col", "f16", "rel_res"), ("row", "f32", "none")])
def test_threaded_oracle_is_algorithm_1(layout, dtype, stop):
    """The CPU baseline's threaded Algorithm 1 (row loops split over threads,
    column order sequential): bitwise the sequential oracle at one thread, and
    the same iterates up to summation order at several."""
    s = synth.make_system(3001, 40, seed=31, noise=0.01, layout=layout, dtype=dtype)
    a0 = np.linspace(-0.5, 0.5, s.n)
    kw = dict(tol=1e-8, max_sweeps=12, stop=stop)
    ref = oracle.solve_system(s, a0=a0, **kw)
    one, used1 = oracle.solve_mt(s.X, s.y, m=s.m, n=s.n, layout=layout, dtype=dtype, a0=a0,
                                 threads=1, **kw)
    assert used1 == 1 and one.sweeps == ref.sweeps and one.status == ref.status
    np.testing.assert_array_equal(one.a, ref.a)
    np.testing.assert_array_equal(one.hist, ref.hist)
    many, _ = oracle.solve_mt(s.X, s.y, m=s.m, n=s.n, layout=layout, dtype=dtype, a0=a0,
                              threads=5, **kw)
    assert many.sweeps == ref.sweeps
    np.testing.assert_allclose(many.a, ref.a, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(many.hist, ref.hist, rtol=1e-12)
