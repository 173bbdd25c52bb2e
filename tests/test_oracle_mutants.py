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
    return failed


def test_real_oracle_passes_battery():
    assert battery(oracle._load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    lib = build_mutant(tmp_path, name)
    failed = battery(lib)
    assert failed, f"mutant {name} passed every pin"
