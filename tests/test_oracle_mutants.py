"""Plants plausible slips in a private copy of the CPU oracle and checks that the
pins catch every one of them.  The mutated copies are compiled to a temporary
directory; the real oracle is never modified.
"""
import json
import os
import subprocess

import numpy as np
import pytest
import scipy.linalg

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "hpscd_oracle.c")

MUTANTS = {
    "axpy_sign": ("e[i] -= col[i] * da;", "e[i] += col[i] * da;"),
    "no_coef_update": ("a_out[j] += da;", "a_out[j] += 0.5 * da;"),
    "wrong_denominator_index": ("num / d[j]", "num / d[0]"),
    "dot_against_y": ("num += col[i] * e[i];", "num += col[i] * y[i];"),
    "denominator_not_squared": ("s += col[i] * col[i];", "s += fabs(col[i]);"),
    "init_residual_sign": ("e[i] -= col[i] * a_out[j];", "e[i] += col[i] * a_out[j];"),
    "norm_without_sqrt": ("  return sqrt(s);", "  return s;"),
    "row_major_transposed": ("Xcopy[j * m + i] = x_elem(X, dt, lay, ld, i, j)",
                             "Xcopy[j * m + i] = x_elem(X, dt, lay, ld, i % n, j % m)"),
    # Algorithm 2 (blocks): the correction uses a instead of a - aprev; a block
    # column sees the residual already updated by its block neighbours
    "blocks_correction_not_delta": ("const double delta = a_out[k] - aprev[k];",
                                    "const double delta = a_out[k];"),
    "blocks_gauss_seidel_inside": ("a_out[k] += d[k] > 0.0 ? dot / d[k] : 0.0;",
                                   "a_out[k] += d[k] > 0.0 ? dot / d[k] : 0.0;"
                                   " { const double dd = d[k] > 0.0 ? dot / d[k] : 0.0;"
                                   " for (int64_t i = 0; i < m; ++i) e[i] -= col[i] * dd;"
                                   " aprev[k] += dd; }"),
    # Algorithm 3 (selection): argmax instead of argmin; the printed assignment
    # instead of the accumulated update; an unsquared error sum
    "select_argmax": ("if (j == 0 || E < best)", "if (j == 0 || E > best)"),
    "select_assign": ("a_out[jhat] += da[jhat];", "a_out[jhat] = da[jhat];"),
    "select_unsquared": ("E += r * r;", "E += r;"),
    # given column order: the index ignored (natural order); the step applied
    # to the coefficient of the wrong column
    "order_ignored": ("const int64_t q = order[(s - 1) * n + k];", "const int64_t q = k;"),
    "order_coef_of_step": ("a_out[q] = a_out[q] + step;", "a_out[k] = a_out[k] + step;"),
    # the swap steps: a swap kept although it does not lower the error; the
    # removed column's contribution not put back into the residual
    "swap_accepts_worse": ("if (bk < 0 || !(bestE < ee)) break;",
                           "if (bk < 0 || !(bestE < 1.5 * ee)) break;"),
    "swap_forgets_removed": ("e[i] = (e[i] + xk[i] * a_out[bk]) - xj[i] * bestd;",
                             "e[i] = e[i] - xj[i] * bestd;"),
}


def build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", str(so),
                           str(path), "-lm"])
    return oracle.load_library(str(so))


def battery(lib):
    """A compact set of the pins; returns the names of those that fail."""
    failed = []

    def solve(Xd, y, **kw):
        m, n = Xd.shape
        return oracle.solve(np.ascontiguousarray(Xd.T), y, m=m, n=n, layout="col",
                            dtype="f64", lib=lib, **kw)

    g = json.load(open(os.path.join(HERE, "golden", "hand_2x2.json")))
    rec = g["sweeps"][2]
    r = solve(np.array(g["X_rows"]), np.array(g["y"]), tol=0, max_sweeps=3, stop="none")
    if not (np.array_equal(r.a, rec["a"]) and
            abs(r.hist[3] - np.sqrt(0.4) / 8) <= 1e-15):
        failed.append("hand_2x2")

    rng = np.random.default_rng(0)
    Xd = rng.standard_normal((30, 8))
    y = rng.standard_normal(30)
    a0 = rng.standard_normal(8)
    G = Xd.T @ Xd
    a_gs = a0 + scipy.linalg.solve_triangular(np.tril(G), Xd.T @ y - G @ a0, lower=True)
    r = solve(Xd, y, a0=a0, tol=0, max_sweeps=1, stop="none")
    if not np.allclose(r.a, a_gs, rtol=1e-10, atol=1e-10):
        failed.append("gauss_seidel")
    r = solve(Xd, y, tol=0, max_sweeps=2, stop="none", want_e=True)
    if not np.allclose(r.e, y - Xd @ r.a, rtol=0, atol=1e-10):
        failed.append("bookkeeping")
    if not np.isclose(r.hist[2], np.linalg.norm(y - Xd @ r.a) / np.linalg.norm(y), rtol=1e-12):
        failed.append("hist")

    # layout: row-major storage of the same system gives the same iterate
    r_row = oracle.solve(np.ascontiguousarray(Xd), y, m=30, n=8, layout="row", dtype="f64",
                         tol=0, max_sweeps=2, stop="none", lib=lib)
    if not np.allclose(r_row.a, r.a, rtol=1e-13, atol=1e-13):
        failed.append("layout")

    # Algorithm 2: one sweep is the block splitting (D + L_B)^{-1} X^T (y - X a)
    thr = 3
    blk = np.arange(8) // thr
    M = np.diag(np.diag(G)) + np.where(blk[:, None] > blk[None, :], G, 0.0)
    a_b = np.linalg.solve(M, Xd.T @ y)
    a_b = a_b + np.linalg.solve(M, Xd.T @ (y - Xd @ a_b))  # two sweeps
    rb = _blocks(lib, Xd, y, thr, sweeps=2)
    if not (np.allclose(rb[0], a_b, rtol=1e-10, atol=1e-12) and
            np.allclose(rb[1], y - Xd @ rb[0], atol=1e-10)):
        failed.append("blocks_splitting")

    # Algorithm 3: argmax of <X_j,e>^2/<X_j,X_j> each step, e = y - X·a (correlated columns
    # make the selection return to a chosen column)
    base = rng.standard_normal(30)
    Xc = np.stack([base + 0.3 * rng.standard_normal(30) for _ in range(5)], axis=1)
    yc = Xc @ np.array([1.0, 1.0, -0.5, 0.7, 0.2])
    sel, a_s, hist_s = _select(lib, Xc, yc, 12)
    e = yc.copy()
    d = (Xc * Xc).sum(axis=0)
    ok = True
    for f in range(12):
        c = Xc.T @ e
        j = int(np.argmax(c * c / d))
        ok &= sel[f] == j
        e = e - Xc[:, j] * (c[j] / d[j])
    ok &= np.allclose(yc - Xc @ a_s, e, atol=1e-10)
    if not ok:
        failed.append("selection")

    # given column order: a fixed permutation every sweep is Algorithm 1 on the
    # permuted columns
    pi = np.array([3, 0, 7, 5, 1, 6, 2, 4])
    ap = solve(Xd[:, pi], y, tol=0, max_sweeps=2, stop="none").a
    a_pi = np.empty(8)
    a_pi[pi] = ap
    ro = oracle.solve_order(np.ascontiguousarray(Xd.T), y, m=30, n=8, order=np.tile(pi, (2, 1)),
                            dtype="f64", tol=0, max_sweeps=2, stop="none", lib=lib)
    if not np.allclose(ro.a, a_pi, rtol=1e-10, atol=1e-12):
        failed.append("order_permutation")

    # swap steps after the greedy selection: the planted support is recovered,
    # every swap lowers the error and e = y - X·a at the end
    gs = np.random.default_rng(1)
    Xw = gs.standard_normal((200, 3)) @ gs.standard_normal((3, 16)) + 0.5 * gs.standard_normal((200, 16))
    yw = Xw[:, [1, 5, 9]] @ np.array([1.0, -0.8, 0.6]) + 0.05 * gs.standard_normal(200)
    sel_w, sw_w, a_w, h_w = oracle.select_swap(np.ascontiguousarray(Xw.T), yw, m=200, n=16, F=3, R=4,
                                               dtype="f64", lib=lib)
    if not (sw_w.tolist() == [[10, 5], [9, 11], [11, 9], [-1, -1]] and np.all(np.diff(h_w) < 0) and
            abs(h_w[-1] - np.linalg.norm(yw - Xw @ a_w) / np.linalg.norm(yw)) <= 1e-12):
        failed.append("swap")
    return failed


def _blocks(lib, Xd, y, thr, sweeps):
    import ctypes
    m, n = Xd.shape
    Xs = np.ascontiguousarray(Xd.T)
    a = np.zeros(n)
    e = np.zeros(m)
    hist = np.zeros(sweeps + 1)
    sw = ctypes.c_int64(0)
    p = lambda v: v.ctypes.data_as(ctypes.c_void_p)
    lib.hpscd_oracle_solve_blocks(p(Xs), 2, 0, m, n, m, p(np.ascontiguousarray(y)), None, thr,
                                  0.0, sweeps, 2, p(a), p(e), p(hist), ctypes.byref(sw))
    return a, e


def _select(lib, Xd, y, F):
    import ctypes
    m, n = Xd.shape
    Xs = np.ascontiguousarray(Xd.T)
    sel = np.zeros(F, dtype=np.int64)
    a = np.zeros(n)
    hist = np.zeros(F + 1)
    p = lambda v: v.ctypes.data_as(ctypes.c_void_p)
    lib.hpscd_oracle_select(p(Xs), 2, 0, m, n, m, p(np.ascontiguousarray(y)), F, p(sel), p(a),
                            p(hist))
    return sel, a, hist


def test_real_oracle_passes_battery():
    assert battery(oracle._load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    lib = build_mutant(tmp_path, name)
    failed = battery(lib)
    assert failed, f"mutant {name} passed every pin"
