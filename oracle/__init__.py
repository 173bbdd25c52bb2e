"""ctypes binding of the CPU oracle (hpscd_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline / reference leg.  The CUDA product path never imports
it, and this module imports nothing from the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hpscd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

DTYPES = {"f32": 0, "bf16": 1, "f64": 2, "f16": 3}
LAYOUTS = {"col": 0, "row": 1}
STOP = {"rel_res": 0, "rel_change": 1, "none": 2}
STATUS = {0: "ok", 1: "invalid", 2: "not_converged", 3: "nonfinite", 4: "nomem"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math) into oracle/_build,
    with OpenMP for the threaded Algorithm 1 of the CPU baseline when the
    compiler has it (without it that function runs on one thread)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """Open an oracle shared library and declare its signatures."""
    lib = ctypes.CDLL(path)
    i64, vp, dp = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
    lib.hpscd_oracle_solve.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64, i64, i64,
                                       dp, dp, ctypes.c_double, i64, ctypes.c_int, i64,
                                       dp, dp, dp, ctypes.POINTER(i64)]
    lib.hpscd_oracle_solve.restype = ctypes.c_int
    lib.hpscd_oracle_residual.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64, i64, i64,
                                          dp, dp, dp, ctypes.POINTER(ctypes.c_double)]
    lib.hpscd_oracle_residual.restype = ctypes.c_int
    lib.hpscd_oracle_solve_blocks.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64, i64, i64,
                                              dp, dp, i64, ctypes.c_double, i64, ctypes.c_int,
                                              dp, dp, dp, ctypes.POINTER(i64)]
    lib.hpscd_oracle_solve_blocks.restype = ctypes.c_int
    lib.hpscd_oracle_select.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64, i64, i64, dp, i64,
                                        vp, dp, dp]
    lib.hpscd_oracle_select.restype = ctypes.c_int
    lib.hpscd_oracle_solve_order.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64, i64, i64, dp, dp,
                                             vp, ctypes.c_double, i64, ctypes.c_int, dp, dp, dp,
                                             ctypes.POINTER(i64)]
    lib.hpscd_oracle_solve_order.restype = ctypes.c_int
    lib.hpscd_oracle_select_swap.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64, i64, i64, dp, i64,
                                             i64, vp, vp, dp, dp, ctypes.POINTER(i64)]
    lib.hpscd_oracle_select_swap.restype = ctypes.c_int
    lib.hpscd_oracle_solve_mt.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64, i64, i64, dp, dp,
                                          ctypes.c_double, i64, ctypes.c_int, ctypes.c_int, dp, dp,
                                          ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int)]
    lib.hpscd_oracle_solve_mt.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load_library(_LIB)
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check_x(X, m, n, layout, dtype):
    exp = {"f32": np.float32, "bf16": np.uint16, "f64": np.float64, "f16": np.float16}[dtype]
    if X.dtype != exp or not X.flags.c_contiguous:
        raise TypeError(f"X must be C-contiguous {exp}")
    shape = (n, m) if layout == "col" else (m, n)
    if X.shape != shape:
        raise ValueError(f"X shape {X.shape} != {shape}")


class OracleResult:
    def __init__(self, a, e, hist, sweeps, status):
        self.a, self.e, self.hist, self.sweeps, self.status = a, e, hist, sweeps, status

    @property
    def rel_res(self) -> float:
        return float(self.hist[self.sweeps])


def solve(X, y, *, m, n, layout="col", dtype="f32", a0=None, tol=1e-6, max_sweeps=1000,
          stop="rel_res", max_col_steps=-1, want_e=False, lib=None) -> OracleResult:
    """Algorithm 1 in float64 on the stored system (X as in synth's conventions)."""
    _check_x(X, m, n, layout, dtype)
    lib = lib or _load()
    y64 = np.ascontiguousarray(y, dtype=np.float64)
    a064 = None if a0 is None else np.ascontiguousarray(a0, dtype=np.float64)
    a = np.zeros(n, dtype=np.float64)
    e = np.zeros(m, dtype=np.float64) if want_e else None
    hist = np.full(max_sweeps + 1, np.nan, dtype=np.float64)
    sw = ctypes.c_int64(0)
    ld = max(1, m if layout == "col" else n)
    st = lib.hpscd_oracle_solve(_ptr(X), DTYPES[dtype], LAYOUTS[layout], m, n, ld, _ptr(y64),
                                _ptr(a064), float(tol), int(max_sweeps), STOP[stop],
                                int(max_col_steps), _ptr(a), _ptr(e), _ptr(hist),
                                ctypes.byref(sw))
    if st in (1, 4):
        raise ValueError(f"oracle: {STATUS[st]}")
    return OracleResult(a, e, hist[: sw.value + 1], sw.value, STATUS[st])


def solve_mt(X, y, *, m, n, layout="col", dtype="f32", a0=None, tol=1e-6, max_sweeps=1000,
             stop="rel_res", threads=1, lib=None):
    """Algorithm 1 with its row loops split over `threads` OpenMP threads (the CPU
    baseline); equal to solve() at threads = 1.  Returns (OracleResult without e,
    threads actually used)."""
    _check_x(X, m, n, layout, dtype)
    lib = lib or _load()
    y64 = np.ascontiguousarray(y, dtype=np.float64)
    a064 = None if a0 is None else np.ascontiguousarray(a0, dtype=np.float64)
    a = np.zeros(n, dtype=np.float64)
    hist = np.full(max_sweeps + 1, np.nan, dtype=np.float64)
    sw = ctypes.c_int64(0)
    used = ctypes.c_int(0)
    ld = max(1, m if layout == "col" else n)
    st = lib.hpscd_oracle_solve_mt(_ptr(X), DTYPES[dtype], LAYOUTS[layout], m, n, ld, _ptr(y64),
                                   _ptr(a064), float(tol), int(max_sweeps), STOP[stop],
                                   int(threads), _ptr(a), _ptr(hist), ctypes.byref(sw),
                                   ctypes.byref(used))
    if st in (1, 4):
        raise ValueError(f"oracle: {STATUS[st]}")
    return OracleResult(a, None, hist[: sw.value + 1], sw.value, STATUS[st]), used.value


def solve_blocks(X, y, *, m, n, thr, layout="col", dtype="f32", a0=None, tol=1e-6,
                 max_sweeps=1000, stop="rel_res", want_e=False) -> OracleResult:
    """Algorithm 2 (blocks of thr columns updated from one residual) in float64."""
    _check_x(X, m, n, layout, dtype)
    lib = _load()
    y64 = np.ascontiguousarray(y, dtype=np.float64)
    a064 = None if a0 is None else np.ascontiguousarray(a0, dtype=np.float64)
    a = np.zeros(n, dtype=np.float64)
    e = np.zeros(m, dtype=np.float64) if want_e else None
    hist = np.full(max_sweeps + 1, np.nan, dtype=np.float64)
    sw = ctypes.c_int64(0)
    ld = max(1, m if layout == "col" else n)
    st = lib.hpscd_oracle_solve_blocks(_ptr(X), DTYPES[dtype], LAYOUTS[layout], m, n, ld, _ptr(y64),
                                       _ptr(a064), int(thr), float(tol), int(max_sweeps),
                                       STOP[stop], _ptr(a), _ptr(e), _ptr(hist), ctypes.byref(sw))
    if st in (1, 4):
        raise ValueError(f"oracle: {STATUS[st]}")
    return OracleResult(a, e, hist[: sw.value + 1], sw.value, STATUS[st])


def solve_order(X, y, *, m, n, order, layout="col", dtype="f32", a0=None, tol=1e-6,
                max_sweeps=1000, stop="rel_res", want_e=False, lib=None) -> OracleResult:
    """Algorithm 1 with the column of every step given: step k of sweep s takes
    column order[s-1][k] (order: integer array (max_sweeps, n), entries in [0, n))."""
    _check_x(X, m, n, layout, dtype)
    lib = lib or _load()
    y64 = np.ascontiguousarray(y, dtype=np.float64)
    a064 = None if a0 is None else np.ascontiguousarray(a0, dtype=np.float64)
    o64 = np.ascontiguousarray(np.asarray(order, dtype=np.int64).reshape(-1))
    if o64.size != max_sweeps * n:
        raise ValueError("order must hold max_sweeps * n indices")
    a = np.zeros(n, dtype=np.float64)
    e = np.zeros(m, dtype=np.float64) if want_e else None
    hist = np.full(max_sweeps + 1, np.nan, dtype=np.float64)
    sw = ctypes.c_int64(0)
    ld = max(1, m if layout == "col" else n)
    st = lib.hpscd_oracle_solve_order(_ptr(X), DTYPES[dtype], LAYOUTS[layout], m, n, ld, _ptr(y64),
                                      _ptr(a064), _ptr(o64), float(tol), int(max_sweeps), STOP[stop],
                                      _ptr(a), _ptr(e), _ptr(hist), ctypes.byref(sw))
    if st in (1, 4):
        raise ValueError(f"oracle: {STATUS[st]}")
    return OracleResult(a, e, hist[: sw.value + 1], sw.value, STATUS[st])


def select(X, y, *, m, n, F, layout="col", dtype="f32"):
    """Algorithm 3: (selected index per step, a, hist) in float64."""
    _check_x(X, m, n, layout, dtype)
    lib = _load()
    y64 = np.ascontiguousarray(y, dtype=np.float64)
    sel = np.zeros(max(F, 1), dtype=np.int64)
    a = np.zeros(n, dtype=np.float64)
    hist = np.zeros(F + 1, dtype=np.float64)
    ld = max(1, m if layout == "col" else n)
    st = lib.hpscd_oracle_select(_ptr(X), DTYPES[dtype], LAYOUTS[layout], m, n, ld, _ptr(y64),
                                 int(F), _ptr(sel), _ptr(a), _ptr(hist))
    if st != 0:
        raise ValueError(f"oracle select: {STATUS[st]}")
    return sel[:F], a, hist


def select_swap(X, y, *, m, n, F, R, layout="col", dtype="f32", lib=None):
    """Algorithm 3 for F steps, then at most R swap steps of the feature-removal
    loop: (sel[F], swaps (R, 2) with -1 rows after the last, a, hist[F + 1 + nswaps])."""
    _check_x(X, m, n, layout, dtype)
    lib = lib or _load()
    y64 = np.ascontiguousarray(y, dtype=np.float64)
    sel = np.zeros(max(F, 1), dtype=np.int64)
    swaps = np.full(2 * max(R, 1), -1, dtype=np.int64)
    a = np.zeros(n, dtype=np.float64)
    hist = np.full(F + 1 + R, np.nan, dtype=np.float64)
    ns = ctypes.c_int64(0)
    ld = max(1, m if layout == "col" else n)
    st = lib.hpscd_oracle_select_swap(_ptr(X), DTYPES[dtype], LAYOUTS[layout], m, n, ld, _ptr(y64),
                                      int(F), int(R), _ptr(sel), _ptr(swaps), _ptr(a), _ptr(hist),
                                      ctypes.byref(ns))
    if st != 0:
        raise ValueError(f"oracle select_swap: {STATUS[st]}")
    k = ns.value
    return sel[:F], swaps[: 2 * R].reshape(R, 2), a, hist[: F + 1 + k]


def residual(X, y, a, *, m, n, layout="col", dtype="f32"):
    """(e, ||e||_2) with e = y - X·a in float64."""
    _check_x(X, m, n, layout, dtype)
    lib = _load()
    y64 = np.ascontiguousarray(y, dtype=np.float64)
    a64 = np.ascontiguousarray(a, dtype=np.float64)
    e = np.zeros(m, dtype=np.float64)
    nrm = ctypes.c_double(0.0)
    ld = max(1, m if layout == "col" else n)
    st = lib.hpscd_oracle_residual(_ptr(X), DTYPES[dtype], LAYOUTS[layout], m, n, ld,
                                   _ptr(y64), _ptr(a64), _ptr(e), ctypes.byref(nrm))
    if st != 0:
        raise ValueError(f"oracle residual: {STATUS[st]}")
    return e, nrm.value


def solve_system(s, **kw) -> OracleResult:
    """solve() on a synth.System."""
    return solve(s.X, s.y, m=s.m, n=s.n, layout=s.layout, dtype=s.dtype, **kw)
