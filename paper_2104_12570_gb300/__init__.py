"""Python binding of libhpscd.so, the GB300 (sm_103a) HPSCD column-sweep
library (Algorithm 1 of arXiv 2104.12570).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  There is no CPU or eager-PyTorch fallback; when the library cannot
be built or loaded, every call raises.

X is a 2-D (m, n) array: a torch tensor on the GPU for solve(), a host array
(numpy or CPU torch tensor) for solve_host().  Its strides pick the layout:
stride (1, ld) is column-major, stride (ld, 1) is row-major.  dtypes: float32,
bfloat16 (torch.bfloat16, or numpy uint16 bit patterns for solve_host) and IEEE
binary16 (torch.float16 / numpy float16).
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

__all__ = ["Context", "Batch", "MLP", "solve", "solve_host", "HpscdError", "load", "STATUS"]

STATUS = {0: "ok", 1: "invalid_arg", 2: "not_converged", 3: "nonfinite", 4: "timeout",
          5: "cuda_error", 6: "unsupported", 7: "no_memory"}
STOP = {"rel_res": 0, "rel_change": 1, "none": 2}
F32, BF16, F16 = 0, 1, 2
DTYPE_CODES = {"f32": F32, "bf16": BF16, "f16": F16}
COL, ROW = 0, 1

_lock = threading.Lock()
_lib = None


class HpscdError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        self.status = STATUS.get(code, str(code))
        super().__init__(f"hpscd: {self.status}{(': ' + what) if what else ''}")


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_sweeps", ctypes.c_int64),
                ("stop_rule", ctypes.c_int32), ("refresh_every", ctypes.c_int32),
                ("debug_flags", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class Timing(ctypes.Structure):
    _fields_ = [("setup_ms", ctypes.c_float), ("sweep_ms", ctypes.c_float),
                ("passes", ctypes.c_int64), ("x_bytes", ctypes.c_int64),
                ("grid", ctypes.c_int32), ("kernel_launches", ctypes.c_int32)]


class Sys(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("y", ctypes.c_void_p), ("a", ctypes.c_void_p),
                ("hist", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("a_is_guess", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class SysResult(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("rel_res", ctypes.c_double),
                ("status", ctypes.c_int32), ("passes", ctypes.c_int32)]


RESULT_BYTES = ctypes.sizeof(SysResult)


def results_buffer(count: int, device=None):
    """A CUDA buffer for `count` hpscd_sys_result records (rows of RESULT_BYTES bytes)."""
    import torch
    return torch.zeros((int(count), RESULT_BYTES), dtype=torch.uint8,
                       device=device if device is not None else "cuda")


def read_results(buf) -> dict:
    """sweeps / rel_res / status / passes of the records in a results_buffer."""
    raw = np.ascontiguousarray(buf.cpu().numpy()).reshape(-1, RESULT_BYTES)
    rec = np.frombuffer(raw.tobytes(), dtype=np.dtype([("sweeps", "<i8"), ("rel_res", "<f8"),
                                                       ("status", "<i4"), ("passes", "<i4")]))
    return {"sweeps": rec["sweeps"].copy(), "rel_res": rec["rel_res"].copy(),
            "status": [STATUS.get(int(c), str(int(c))) for c in rec["status"]],
            "passes": rec["passes"].copy()}


class Tuning(ctypes.Structure):
    _fields_ = [("cluster", ctypes.c_int32), ("panel", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


SIGNATURES = {
    "hpscd_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "hpscd_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "hpscd_set_stream": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "hpscd_set_timeout": ([ctypes.c_void_p, ctypes.c_double], ctypes.c_int),
    "hpscd_workspace_size": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                              ctypes.c_int64, ctypes.POINTER(Opts),
                              ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "hpscd_set_workspace": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "hpscd_solve": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                     ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                     ctypes.POINTER(Opts), ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                     ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "hpscd_solve_host": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                          ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Opts), ctypes.c_void_p,
                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)],
                         ctypes.c_int),
    "hpscd_solve_blocks": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                            ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_int, ctypes.c_int64, ctypes.POINTER(Opts), ctypes.c_void_p,
                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)],
                           ctypes.c_int),
    "hpscd_solve_order": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                           ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(Opts), ctypes.c_void_p,
                           ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)],
                          ctypes.c_int),
    "hpscd_select_swap": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                           ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.POINTER(Opts), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "hpscd_select": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                      ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.POINTER(Opts), ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)],
                     ctypes.c_int),
    "hpscd_last_timing": ([ctypes.c_void_p, ctypes.POINTER(Timing)], ctypes.c_int),
    "hpscd_solve_async": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                           ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_int, ctypes.POINTER(Opts), ctypes.c_void_p, ctypes.c_void_p],
                          ctypes.c_int),
    "hpscd_async_timings": ([ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(Timing)], ctypes.c_int),
    "hpscd_gram": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                    ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int], ctypes.c_int),
    "hpscd_solve_noalloc": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                             ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_int, ctypes.POINTER(Opts), ctypes.c_void_p,
                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)],
                            ctypes.c_int),
    "hpscd_set_trace": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "hpscd_get_trace": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int64,
                         ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "hpscd_batch_create": ([ctypes.c_void_p, ctypes.POINTER(Sys), ctypes.c_int64, ctypes.c_int,
                            ctypes.POINTER(Opts), ctypes.POINTER(Tuning),
                            ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "hpscd_batch_launch": ([ctypes.c_void_p], ctypes.c_int),
    "hpscd_batch_results": ([ctypes.c_void_p, ctypes.POINTER(SysResult)], ctypes.c_int),
    "hpscd_batch_tuning": ([ctypes.c_void_p, ctypes.POINTER(Tuning)], ctypes.c_int),
    "hpscd_batch_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "hpscd_autotune_batch": ([ctypes.c_void_p, ctypes.POINTER(Sys), ctypes.c_int64, ctypes.c_int,
                              ctypes.c_int64, ctypes.POINTER(Tuning),
                              ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "hpscd_mlp_create": ([ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p)],
                         ctypes.c_int),
    "hpscd_mlp_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "hpscd_mlp_param_count": ([], ctypes.c_int64),
    "hpscd_mlp_set_params": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "hpscd_mlp_get_params": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "hpscd_mlp_predict": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "hpscd_mlp_gradients": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                            ctypes.c_void_p], ctypes.c_int),
    "hpscd_mlp_train_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_double)],
                            ctypes.c_int),
    "hpscd_batch_set_warm_start": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "hpscd_status_string": ([ctypes.c_int], ctypes.c_char_p),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libhpscd.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_needed:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libhpscd.so not found at {_build.LIB}; run build()")
            lib = ctypes.CDLL(_build.LIB)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def make_opts(tol=1e-6, max_sweeps=1000, stop="rel_res", refresh_every=0, debug_flags=0) -> Opts:
    o = Opts()
    o.debug_flags = int(debug_flags)
    o.tol = float(tol)
    o.max_sweeps = int(max_sweeps)
    o.stop_rule = STOP[stop] if isinstance(stop, str) else int(stop)
    o.refresh_every = int(refresh_every)
    return o


def _describe(X):
    """(ptr, dtype code, layout, m, n, ld) of a 2-D torch tensor or numpy array."""
    try:
        import torch
        is_torch = isinstance(X, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_torch = False
    if is_torch:
        if X.dim() != 2:
            raise ValueError("X must be 2-D (m, n)")
        import torch
        if X.dtype == torch.float32:
            dt = F32
        elif X.dtype == torch.bfloat16:
            dt = BF16
        elif X.dtype == torch.float16:
            dt = F16
        else:
            raise TypeError("X dtype must be float32, bfloat16 or float16")
        m, n = X.shape
        s0, s1 = X.stride()
        ptr = X.data_ptr()
    else:
        X = np.asarray(X)
        if X.ndim != 2:
            raise ValueError("X must be 2-D (m, n)")
        if X.dtype == np.float32:
            dt = F32
        elif X.dtype == np.uint16:
            dt = BF16
        elif X.dtype == np.float16:
            dt = F16
        else:
            raise TypeError("X dtype must be float32, uint16 (bfloat16 bits) or float16")
        m, n = X.shape
        s0, s1 = (s // X.itemsize for s in X.strides)
        ptr = X.ctypes.data
    if m == 0 or n == 0:
        return ptr, dt, COL, m, n, max(1, m)
    if s0 == 1 and s1 >= max(1, m):
        return ptr, dt, COL, m, n, s1
    if n == 1 and s0 == 1:
        return ptr, dt, COL, m, n, max(1, m)
    if s1 == 1 and s0 >= max(1, n):
        return ptr, dt, ROW, m, n, s0
    raise ValueError("X must be column-major (stride (1, ld)) or row-major (stride (ld, 1))")


def _check_vec(v, length: int, name: str, device=None):
    """v must be a contiguous float32 CUDA vector of `length` entries (on `device`
    when given): the library reads and writes exactly that many entries."""
    import torch
    if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float32
            and v.is_contiguous() and v.numel() == length
            and (device is None or v.device == device)):
        raise TypeError(f"{name} must be a contiguous float32 CUDA vector of length {length}"
                        + (f" on {device}" if device is not None else ""))


def _coef_out(X, n, out, a0):
    """The coefficient vector of a device solve: `out` (checked) or a new one,
    filled from a0 (n entries) when a warm start is given."""
    import torch
    if out is not None:
        _check_vec(out, n, "out", X.device)
        a = out
    else:
        a = torch.empty(n, dtype=torch.float32, device=X.device)
    if a0 is not None:
        if int(getattr(a0, "numel", lambda: np.size(a0))()) != n:
            raise ValueError(f"a0 must have n = {n} entries")
        a.copy_(a0 if isinstance(a0, torch.Tensor) else torch.as_tensor(np.asarray(a0, np.float32)))
    return a


@dataclass
class SolveResult:
    a: object
    hist: np.ndarray
    sweeps: int
    rel_res: float
    status: str
    timing: dict = field(default_factory=dict)


class Context:
    """One library context: a device, a stream and a workspace."""

    def __init__(self, device: int = 0, stream=None, timeout_s: float | None = None):
        self._lib = load()
        self.device = device
        h = ctypes.c_void_p()
        rc = self._lib.hpscd_create(ctypes.byref(h), int(device), self._stream_handle(stream))
        if rc != 0:
            raise HpscdError(rc, "hpscd_create")
        self._h = h
        self._children = weakref.WeakSet()  # batches and networks made on this context
        if timeout_s is not None:
            self.set_timeout(timeout_s)

    def _device_args(self, X, y):
        """X must be a CUDA tensor on this context's device and y a float32 CUDA
        vector of its m rows there (the kernels dereference both)."""
        import torch
        if not (isinstance(X, torch.Tensor) and X.is_cuda):
            raise TypeError("X must be a CUDA tensor (use solve_host for host arrays)")
        if X.device.index != self.device:
            raise ValueError(f"X is on {X.device}, the context on cuda:{self.device}")
        _check_vec(y, X.shape[0], "y", X.device)

    @staticmethod
    def _stream_handle(stream):
        if stream is None:
            return None
        if isinstance(stream, int):
            return ctypes.c_void_p(stream)
        return ctypes.c_void_p(stream.cuda_stream)

    def set_stream(self, stream):
        rc = self._lib.hpscd_set_stream(self._h, self._stream_handle(stream))
        if rc:
            raise HpscdError(rc)

    def set_timeout(self, seconds: float):
        rc = self._lib.hpscd_set_timeout(self._h, float(seconds))
        if rc:
            raise HpscdError(rc)

    def close(self):
        """Destroy the context, after the batches and networks made on it (their
        handles point into it)."""
        if getattr(self, "_h", None):
            kids = list(getattr(self, "_children", ()))
            for k in sorted(kids, key=lambda k: isinstance(k, MLP)):  # batches first
                k.close()
            self._lib.hpscd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_trace(self, max_passes: int):
        rc = self._lib.hpscd_set_trace(self._h, int(max_passes))
        if rc:
            raise HpscdError(rc)
        self._trace_passes = int(max_passes)

    def trace(self) -> dict:
        """Phase durations (us) per pass of the last solve, and the spread of the
        CTAs' end-of-streaming times in pass 1."""
        P = getattr(self, "_trace_passes", 0)
        if not P:
            return {}
        buf = (ctypes.c_ulonglong * (P * 6 + 4096))()
        got = ctypes.c_int64(0)
        rc = self._lib.hpscd_get_trace(self._h, buf, P * 6 + 4096, ctypes.byref(got))
        if rc:
            raise HpscdError(rc)
        a = np.frombuffer(buf, dtype=np.uint64)[: got.value].astype(np.int64)
        phases = a[: P * 6].reshape(P, 6)
        rows = []
        for r in phases:
            if r[0] == 0:
                break
            def dt(a, b):
                return (r[b] - r[a]) / 1e3 if r[a] and r[b] else None
            rows.append({"stream_us": dt(0, 1), "barrier_us": dt(1, 2), "reduce_us": dt(2, 3),
                         "subst_us": dt(3, 5)})
        ends = a[P * 6:]
        ends = ends[ends > 0]
        spread = float((ends.max() - ends.min()) / 1e3) if ends.size else None
        return {"passes": rows, "pass1_stream_end_spread_us": spread}

    def trace_raw(self) -> np.ndarray:
        """The device timestamps (ns, global timer) of the last traced solve, 6
        words per traced pass (tall sweep) or column block (wide sweep), then the
        tall sweep's per-CTA end-of-streaming times; 0 where nothing was stamped."""
        P = getattr(self, "_trace_passes", 0)
        if not P:
            return np.zeros(0, dtype=np.int64)
        buf = (ctypes.c_ulonglong * (P * 6 + 4096))()
        got = ctypes.c_int64(0)
        rc = self._lib.hpscd_get_trace(self._h, buf, P * 6 + 4096, ctypes.byref(got))
        if rc:
            raise HpscdError(rc)
        return np.frombuffer(buf, dtype=np.uint64)[: got.value].astype(np.int64)

    def timing(self) -> dict:
        t = Timing()
        self._lib.hpscd_last_timing(self._h, ctypes.byref(t))
        return {"setup_ms": t.setup_ms, "sweep_ms": t.sweep_ms, "passes": t.passes,
                "x_bytes": t.x_bytes, "grid": t.grid, "kernel_launches": t.kernel_launches}

    def solve_async(self, X, y, res, *, tol=1e-6, max_sweeps=1000, stop="rel_res", a0=None,
                    out=None, hist=None):
        """Enqueue a solve of column-major CUDA X on the current stream and return at
        once (hpscd_solve_async).  res: a CUDA tensor of RESULT_BYTES bytes (e.g. a
        row of results_buffer(k)) that receives sweeps / rel_res / status / passes
        when the solve has finished; hist: optional CUDA float64 (max_sweeps + 1,).
        Returns the coefficient tensor (valid once the stream has passed the solve)."""
        import torch
        ptr, dt, lay, m, n, ld = _describe(X)
        self._device_args(X, y)
        if lay != COL:
            raise ValueError("solve_async needs a column-major CUDA X")
        if not (isinstance(res, torch.Tensor) and res.is_cuda and res.device == X.device and res.is_contiguous() and res.numel() * res.element_size() >= RESULT_BYTES):
            raise TypeError("res must be a contiguous CUDA buffer of at least RESULT_BYTES bytes")
        if hist is not None and not (hist.is_cuda and hist.dtype == torch.float64 and
                                     hist.numel() >= int(max_sweeps) + 1):
            raise TypeError("hist must be a CUDA float64 tensor of max_sweeps + 1 entries")
        a = _coef_out(X, n, out, a0)
        o = make_opts(tol, max_sweeps, stop)
        self.set_stream(torch.cuda.current_stream(X.device))
        rc = self._lib.hpscd_solve_async(self._h, ctypes.c_void_p(ptr), dt, m, n, ld,
                                         ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                         1 if a0 is not None else 0, ctypes.byref(o),
                                         ctypes.c_void_p(hist.data_ptr() if hist is not None else 0),
                                         ctypes.c_void_p(res.data_ptr()))
        if rc:
            raise HpscdError(rc, "hpscd_solve_async")
        return a

    def async_timings(self, count: int) -> list:
        """Timings of the last `count` asynchronous solves (waits for the stream)."""
        ts = (Timing * int(count))()
        rc = self._lib.hpscd_async_timings(self._h, int(count), ts)
        if rc:
            raise HpscdError(rc, "hpscd_async_timings")
        return [{"setup_ms": t.setup_ms, "sweep_ms": t.sweep_ms, "x_bytes": t.x_bytes, "grid": t.grid,
                 "kernel_launches": t.kernel_launches} for t in ts]

    def set_workspace(self, ptr: int, nbytes: int):
        """Install caller-owned device memory (256-byte aligned) as the workspace;
        ptr = 0 returns the context to allocating its own."""
        rc = self._lib.hpscd_set_workspace(self._h, ctypes.c_void_p(int(ptr) or None), int(nbytes))
        if rc:
            raise HpscdError(rc)

    def workspace_size(self, m, n, dtype="f32", layout="col", **opt_kw) -> int:
        o = make_opts(**opt_kw)
        b = ctypes.c_size_t(0)
        rc = self._lib.hpscd_workspace_size(self._h, DTYPE_CODES[dtype],
                                            COL if layout == "col" else ROW, int(m), int(n),
                                            ctypes.byref(o), ctypes.byref(b))
        if rc:
            raise HpscdError(rc)
        return b.value

    def _finish(self, rc, hist, sw, rr, a):
        if rc in (1, 4, 5, 6, 7):
            raise HpscdError(rc)
        s = sw.value
        return SolveResult(a=a, hist=hist[: s + 1].copy(), sweeps=s, rel_res=rr.value,
                           status=STATUS[rc], timing=self.timing())

    def solve(self, X, y, *, tol=1e-6, max_sweeps=1000, stop="rel_res", a0=None,
              refresh_every=0, out=None, debug_flags=0) -> SolveResult:
        """Solve X·a ≈ y on the GPU (X, y, a0, out: CUDA tensors on this device)."""
        import torch
        ptr, dt, lay, m, n, ld = _describe(X)
        self._device_args(X, y)
        a = _coef_out(X, n, out, a0)
        o = make_opts(tol, max_sweeps, stop, refresh_every, debug_flags)
        hist = np.full(int(max_sweeps) + 1, np.nan)
        sw, rr = ctypes.c_int64(0), ctypes.c_double(0.0)
        self.set_stream(torch.cuda.current_stream(X.device))
        rc = self._lib.hpscd_solve(self._h, ctypes.c_void_p(ptr), dt, lay, m, n, ld,
                                   ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                   1 if a0 is not None else 0, ctypes.byref(o),
                                   hist.ctypes.data_as(ctypes.c_void_p), ctypes.byref(sw),
                                   ctypes.byref(rr))
        return self._finish(rc, hist, sw, rr, a)

    def solve_blocks(self, X, y, thr: int, *, tol=1e-6, max_sweeps=1000, stop="rel_res",
                     a0=None, out=None) -> SolveResult:
        """Algorithm 2: blocks of thr columns take their steps from one residual."""
        import torch
        ptr, dt, lay, m, n, ld = _describe(X)
        self._device_args(X, y)
        if lay != COL:
            raise ValueError("solve_blocks needs a column-major CUDA X")
        a = _coef_out(X, n, out, a0)
        o = make_opts(tol, max_sweeps, stop)
        hist = np.full(int(max_sweeps) + 1, np.nan)
        sw, rr = ctypes.c_int64(0), ctypes.c_double(0.0)
        self.set_stream(torch.cuda.current_stream(X.device))
        rc = self._lib.hpscd_solve_blocks(self._h, ctypes.c_void_p(ptr), dt, m, n, ld,
                                          ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                          1 if a0 is not None else 0, int(thr), ctypes.byref(o),
                                          hist.ctypes.data_as(ctypes.c_void_p), ctypes.byref(sw),
                                          ctypes.byref(rr))
        return self._finish(rc, hist, sw, rr, a)

    def select_swap(self, X, y, F: int, R: int, *, tol=0.0, stop="none"):
        """Algorithm 3 for F steps, then at most R swap steps of the feature-removal
        loop (Sec. 8); returns (SolveResult, chosen column per selection step,
        (R, 2) array of the (dropped, added) pair of each swap, -1 after the last)."""
        import torch
        ptr, dt, lay, m, n, ld = _describe(X)
        self._device_args(X, y)
        if lay != COL:
            raise ValueError("select_swap needs a column-major CUDA X")
        a = torch.empty(n, dtype=torch.float32, device=X.device)
        o = make_opts(tol, F, stop)
        hist = np.full(int(F) + int(R) + 1, np.nan)
        sel = np.full(max(int(F), 1), -1, dtype=np.int64)
        swaps = np.full(2 * max(int(R), 1), -1, dtype=np.int64)
        sw, rr = ctypes.c_int64(0), ctypes.c_double(0.0)
        self.set_stream(torch.cuda.current_stream(X.device))
        rc = self._lib.hpscd_select_swap(self._h, ctypes.c_void_p(ptr), dt, m, n, ld,
                                         ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                         ctypes.byref(o), int(R), sel.ctypes.data_as(ctypes.c_void_p),
                                         swaps.ctypes.data_as(ctypes.c_void_p),
                                         hist.ctypes.data_as(ctypes.c_void_p), ctypes.byref(sw),
                                         ctypes.byref(rr))
        return (self._finish(rc, hist, sw, rr, a), sel[: int(F)],
                swaps[: 2 * int(R)].reshape(int(R), 2))

    def solve_order(self, X, y, order, *, tol=1e-6, max_sweeps=None, stop="rel_res", a0=None,
                    out=None) -> SolveResult:
        """Algorithm 1 with the column of every step given: step k of sweep s takes
        column order[s-1][k] (order: integer array (max_sweeps, n) on the host,
        entries in [0, n), e.g. drawn at random with replacement)."""
        import torch
        ptr, dt, lay, m, n, ld = _describe(X)
        self._device_args(X, y)
        if lay != COL:
            raise ValueError("solve_order needs a column-major CUDA X")
        ordr = np.ascontiguousarray(np.asarray(order, dtype=np.int32).reshape(-1, n) if n else
                                    np.zeros((0, 0), np.int32))
        if max_sweeps is None:
            max_sweeps = ordr.shape[0]
        if ordr.size != int(max_sweeps) * n:
            raise ValueError("order must hold max_sweeps rows of n indices")
        a = _coef_out(X, n, out, a0)
        o = make_opts(tol, max_sweeps, stop)
        hist = np.full(int(max_sweeps) + 1, np.nan)
        sw, rr = ctypes.c_int64(0), ctypes.c_double(0.0)
        self.set_stream(torch.cuda.current_stream(X.device))
        rc = self._lib.hpscd_solve_order(self._h, ctypes.c_void_p(ptr), dt, m, n, ld,
                                         ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                         1 if a0 is not None else 0,
                                         ordr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o),
                                         hist.ctypes.data_as(ctypes.c_void_p), ctypes.byref(sw),
                                         ctypes.byref(rr))
        return self._finish(rc, hist, sw, rr, a)

    def select(self, X, y, F: int, *, tol=0.0, stop="none"):
        """Algorithm 3: F greedy selection steps; returns (SolveResult, chosen column per step)."""
        import torch
        ptr, dt, lay, m, n, ld = _describe(X)
        self._device_args(X, y)
        if lay != COL:
            raise ValueError("select needs a column-major CUDA X")
        a = torch.empty(n, dtype=torch.float32, device=X.device)
        o = make_opts(tol, F, stop)
        hist = np.full(int(F) + 1, np.nan)
        sel = np.full(max(int(F), 1), -1, dtype=np.int64)
        sw, rr = ctypes.c_int64(0), ctypes.c_double(0.0)
        self.set_stream(torch.cuda.current_stream(X.device))
        rc = self._lib.hpscd_select(self._h, ctypes.c_void_p(ptr), dt, m, n, ld,
                                    ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                    ctypes.byref(o), sel.ctypes.data_as(ctypes.c_void_p),
                                    hist.ctypes.data_as(ctypes.c_void_p), ctypes.byref(sw),
                                    ctypes.byref(rr))
        res = self._finish(rc, hist, sw, rr, a)
        return res, sel[: res.sweeps]

    def gram(self, X, simt: bool = False):
        """G = X^T X (n×n float32 CUDA tensor) for a column-major CUDA X."""
        import torch
        ptr, dt, lay, m, n, ld = _describe(X)
        if not (isinstance(X, torch.Tensor) and X.is_cuda and X.device.index == self.device):
            raise TypeError(f"X must be a CUDA tensor on cuda:{self.device}")
        if lay != COL:
            raise ValueError("gram needs a column-major X")
        G = torch.empty(n, n, dtype=torch.float32, device=X.device)
        self.set_stream(torch.cuda.current_stream(X.device))
        rc = self._lib.hpscd_gram(self._h, ctypes.c_void_p(ptr), dt, m, n, ld,
                                  ctypes.c_void_p(G.data_ptr()), n, 2 if simt else 0)
        if rc:
            raise HpscdError(rc)
        return G

    def solve_host(self, X, y, *, tol=1e-6, max_sweeps=1000, stop="rel_res", a0=None,
                   refresh_every=0) -> SolveResult:
        """End-to-end solve from host memory (numpy arrays or CPU tensors; pinned
        memory makes the copies asynchronous).  Returns a as a numpy array."""
        ptr, dt, lay, m, n, ld = _describe(X)
        y_np = _host_f32(y, m)
        a = np.zeros(n, dtype=np.float32) if a0 is None else np.array(a0, dtype=np.float32).ravel()
        if a.size != n:
            raise ValueError(f"a0 must have n = {n} entries")
        o = make_opts(tol, max_sweeps, stop, refresh_every)
        hist = np.full(int(max_sweeps) + 1, np.nan)
        sw, rr = ctypes.c_int64(0), ctypes.c_double(0.0)
        rc = self._lib.hpscd_solve_host(self._h, ctypes.c_void_p(ptr), dt, lay, m, n, ld,
                                        ctypes.c_void_p(y_np[0]), a.ctypes.data_as(ctypes.c_void_p),
                                        1 if a0 is not None else 0, ctypes.byref(o),
                                        hist.ctypes.data_as(ctypes.c_void_p), ctypes.byref(sw),
                                        ctypes.byref(rr))
        return self._finish(rc, hist, sw, rr, a)


def _sys_array(systems, hist_len=0):
    """ctypes array of hpscd_sys from (X, y, a, a_is_guess[, hist]) CUDA tensors."""
    import torch
    arr = (Sys * max(1, len(systems)))()
    for i, t in enumerate(systems):
        X, y, a, guess = t[:4]
        hist = t[4] if len(t) > 4 else None
        ptr, dt, lay, m, n, ld = _describe(X)
        if dt != F32 or lay != COL:
            raise TypeError("batched systems need a float32 column-major X")
        for v, ln in ((y, m), (a, n)):
            if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float32
                    and v.is_contiguous() and v.numel() == ln):
                raise TypeError("y and a must be contiguous float32 CUDA vectors of length m, n")
        arr[i].X, arr[i].y, arr[i].a = ptr, y.data_ptr(), a.data_ptr()
        if hist is not None and not (isinstance(hist, torch.Tensor) and hist.is_cuda
                                     and hist.dtype == torch.float64 and hist.is_contiguous()
                                     and hist.numel() >= hist_len):
            raise TypeError(f"hist must be a contiguous float64 CUDA tensor of at least {hist_len} entries")
        arr[i].hist = hist.data_ptr() if hist is not None else None
        arr[i].m, arr[i].n, arr[i].ld = m, n, ld
        arr[i].a_is_guess = 1 if guess else 0
    return arr


class Batch:
    """Many independent column-major float32 systems solved in one persistent,
    graph-captured launch (hpscd_batch_*).  `systems` is a list of tuples
    (X, y, a, a_is_guess) or (X, y, a, a_is_guess, hist) of CUDA tensors: X (m, n)
    column-major, y (m,), a (n,) in/out, hist (max_sweeps + 1,) float64 or None.
    The tensors must stay alive while the batch is used (the batch keeps them)."""

    def __init__(self, ctx: "Context", systems, *, tol=1e-6, max_sweeps=1000, stop="rel_res",
                 cluster: int = 0, panel: int = 0):
        import torch
        self._lib = ctx._lib
        self.ctx = ctx
        self.systems = list(systems)
        self.count = len(self.systems)
        self._sys = _sys_array(self.systems, int(max_sweeps) + 1)
        o = make_opts(tol, max_sweeps, stop)
        t = Tuning()
        t.cluster = int(cluster)
        t.panel = int(panel)
        dev = self.systems[0][0].device if self.systems else torch.device("cuda", ctx.device)
        ctx.set_stream(torch.cuda.current_stream(dev))
        h = ctypes.c_void_p()
        rc = self._lib.hpscd_batch_create(ctx._h, self._sys, self.count, F32, ctypes.byref(o),
                                          ctypes.byref(t), ctypes.byref(h))
        if rc:
            raise HpscdError(rc, "hpscd_batch_create")
        self._h = h
        self._res = (SysResult * max(1, self.count))()
        ctx._children.add(self)

    @property
    def cluster(self) -> int:
        t = Tuning()
        self._lib.hpscd_batch_tuning(self._h, ctypes.byref(t))
        return t.cluster

    @property
    def panel(self) -> int:
        t = Tuning()
        self._lib.hpscd_batch_tuning(self._h, ctypes.byref(t))
        return t.panel

    def launch(self):
        rc = self._lib.hpscd_batch_launch(self._h)
        if rc:
            raise HpscdError(rc, "hpscd_batch_launch")

    def results(self) -> dict:
        """Wait for the last launch; per-system sweeps, rel_res, status, passes."""
        rc = self._lib.hpscd_batch_results(self._h, self._res)
        if rc in (1, 5):
            raise HpscdError(rc, "hpscd_batch_results")
        n = self.count
        return {"sweeps": np.array([self._res[i].sweeps for i in range(n)], dtype=np.int64),
                "rel_res": np.array([self._res[i].rel_res for i in range(n)]),
                "status": [STATUS.get(self._res[i].status, str(self._res[i].status))
                           for i in range(n)],
                "passes": np.array([self._res[i].passes for i in range(n)], dtype=np.int64),
                "timing": self.ctx.timing()}

    def run(self) -> dict:
        self.launch()
        return self.results()

    def set_warm_start(self, mlp: "MLP | None", theta=None):
        """Start every system from mlp's prediction for theta (CUDA float32
        (count, 16), row i = system i); None restores the cold start."""
        if mlp is None:
            rc = self._lib.hpscd_batch_set_warm_start(self._h, None, None)
            self._theta = None
        else:
            import torch
            if not (isinstance(theta, torch.Tensor) and theta.is_cuda and theta.dtype == torch.float32
                    and theta.is_contiguous() and tuple(theta.shape) == (self.count, 16)):
                raise TypeError("theta must be a contiguous float32 CUDA tensor (count, 16)")
            self._theta = theta
            self._mlp = mlp
            mlp._users.add(self)
            rc = self._lib.hpscd_batch_set_warm_start(self._h, mlp._h, ctypes.c_void_p(theta.data_ptr()))
        if rc:
            raise HpscdError(rc, "hpscd_batch_set_warm_start")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hpscd_batch_destroy(self._h)
            self._h = None
            mlp = getattr(self, "_mlp", None)
            if mlp is not None:
                mlp._users.discard(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_IN, MLP_HID, MLP_OUT, MLP_THETA = 18, 256, 256, 16
MLP_SHAPES = [(MLP_HID, MLP_IN), (MLP_HID,), (MLP_HID, MLP_HID), (MLP_HID,), (MLP_OUT, MLP_HID),
              (MLP_OUT,)]


def mlp_init(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases, as one flat float32 parameter vector."""
    g = np.random.default_rng(seed)
    parts = []
    for shp in MLP_SHAPES:
        if len(shp) == 2:
            lim = np.sqrt(6.0 / shp[1])
            parts.append(g.uniform(-lim, lim, shp).ravel())
        else:
            parts.append(np.zeros(shp))
    return np.concatenate(parts).astype(np.float32)


def mlp_split(flat: np.ndarray):
    """Flat parameter vector -> [W1, b1, W2, b2, W3, b3] views."""
    out, off = [], 0
    for shp in MLP_SHAPES:
        k = int(np.prod(shp))
        out.append(flat[off: off + k].reshape(shp))
        off += k
    return out


class MLP:
    """Warm-start network phi(theta, m, n) -> a on the GPU (hpscd_mlp_*)."""

    def __init__(self, ctx: "Context", max_batch: int = 4096, params=None, seed: int = 0):
        import torch
        self._lib = ctx._lib
        self.ctx = ctx
        self.max_batch = int(max_batch)
        ctx.set_stream(torch.cuda.current_stream(torch.device("cuda", ctx.device)))
        h = ctypes.c_void_p()
        rc = self._lib.hpscd_mlp_create(ctx._h, self.max_batch, ctypes.byref(h))
        if rc:
            raise HpscdError(rc, "hpscd_mlp_create")
        self._h = h
        self._users = weakref.WeakSet()  # batches that start from this network
        ctx._children.add(self)
        self.n_params = int(self._lib.hpscd_mlp_param_count())
        self.set_params(mlp_init(seed) if params is None else params)

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        if flat.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        rc = self._lib.hpscd_mlp_set_params(self._h, flat.ctypes.data_as(ctypes.c_void_p))
        if rc:
            raise HpscdError(rc, "hpscd_mlp_set_params")

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        rc = self._lib.hpscd_mlp_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p))
        if rc:
            raise HpscdError(rc, "hpscd_mlp_get_params")
        return out

    def _batch_args(self, theta, m, n, target=None):
        """(m, n) as int64 host arrays after checking theta (B, 16) and target
        (B, 256): contiguous float32 CUDA tensors on the context's device."""
        import torch
        m = np.ascontiguousarray(m, dtype=np.int64).ravel()
        n = np.ascontiguousarray(n, dtype=np.int64).ravel()
        B = len(m)
        if len(n) != B:
            raise ValueError("m and n must have one entry per row of theta")
        dev = torch.device("cuda", self.ctx.device)
        for t, cols, name in ((theta, MLP_THETA, "theta"), (target, MLP_OUT, "target")):
            if t is None and name == "target":
                continue
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device == dev
                    and t.dtype == torch.float32 and t.is_contiguous()
                    and tuple(t.shape) == (B, cols)):
                raise TypeError(f"{name} must be a contiguous float32 CUDA tensor ({B}, {cols}) on {dev}")
        return m, n

    def predict(self, theta, m, n):
        """(B, 256) float32 CUDA predictions for theta (B, 16) CUDA, m, n host ints."""
        import torch
        m, n = self._batch_args(theta, m, n)
        B = len(m)
        out = torch.empty(B, MLP_OUT, dtype=torch.float32, device=theta.device)
        rc = self._lib.hpscd_mlp_predict(self._h, ctypes.c_void_p(theta.data_ptr()),
                                         m.ctypes.data_as(ctypes.c_void_p),
                                         n.ctypes.data_as(ctypes.c_void_p), B,
                                         ctypes.c_void_p(out.data_ptr()))
        if rc:
            raise HpscdError(rc, "hpscd_mlp_predict")
        return out

    def gradients(self, theta, m, n, target):
        """(loss, flat float32 gradient) of the masked mean-squared error."""
        m, n = self._batch_args(theta, m, n, target)
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        rc = self._lib.hpscd_mlp_gradients(self._h, ctypes.c_void_p(theta.data_ptr()),
                                           m.ctypes.data_as(ctypes.c_void_p),
                                           n.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.c_void_p(target.data_ptr()), len(m),
                                           ctypes.byref(loss), g.ctypes.data_as(ctypes.c_void_p))
        if rc:
            raise HpscdError(rc, "hpscd_mlp_gradients")
        return loss.value, g

    def train_step(self, theta, m, n, target, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> float:
        m, n = self._batch_args(theta, m, n, target)
        loss = ctypes.c_double(0.0)
        rc = self._lib.hpscd_mlp_train_step(self._h, ctypes.c_void_p(theta.data_ptr()),
                                            m.ctypes.data_as(ctypes.c_void_p),
                                            n.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.c_void_p(target.data_ptr()), len(m),
                                            float(lr), float(beta1), float(beta2), float(eps),
                                            ctypes.byref(loss))
        if rc:
            raise HpscdError(rc, "hpscd_mlp_train_step")
        return loss.value

    def close(self):
        """Destroy the network; batches that start from it go back to the cold start."""
        if getattr(self, "_h", None):
            for b in list(getattr(self, "_users", ())):
                if getattr(b, "_h", None):
                    b.set_warm_start(None)
            self._lib.hpscd_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune_batch(ctx: "Context", systems, trial_sweeps: int = 4):
    """((cluster, panel) of the fastest candidate, {(cluster, panel): ms of
    trial_sweeps sweeps of every system}) over clusters 1, 2, 4, 8 and panel
    policies 0, 1, 2 (see Batch)."""
    import torch
    arr = _sys_array(systems, int(trial_sweeps) + 1)
    t = Tuning()
    ms = (ctypes.c_double * 12)()
    ctx.set_stream(torch.cuda.current_stream(systems[0][0].device))
    rc = ctx._lib.hpscd_autotune_batch(ctx._h, arr, len(systems), F32, int(trial_sweeps),
                                       ctypes.byref(t), ms)
    if rc:
        raise HpscdError(rc, "hpscd_autotune_batch")
    return (t.cluster, t.panel), {(k, p): ms[3 * i + p] for i, k in enumerate((1, 2, 4, 8))
                                  for p in range(3) if ms[3 * i + p] >= 0}


def _host_f32(y, m):
    """(pointer, keep-alive) of a host float32 vector of length m."""
    try:
        import torch
        if isinstance(y, torch.Tensor):
            if y.is_cuda or y.dtype != torch.float32 or not y.is_contiguous() or y.numel() != m:
                raise TypeError("y must be a contiguous float32 host vector of length m")
            return (y.data_ptr(), y)
    except ImportError:  # pragma: no cover
        pass
    yn = np.ascontiguousarray(y, dtype=np.float32)
    if yn.size != m:
        raise ValueError("y must have length m")
    return (yn.ctypes.data, yn)


_default = {}


def _default_ctx(device):
    with _lock:
        c = _default.get(device)
    if c is None:
        c = Context(device)
        with _lock:
            _default[device] = c
    return c


def solve(X, y, **kw) -> SolveResult:
    """Module-level solve on X's device with a shared default context."""
    return _default_ctx(X.device.index or 0).solve(X, y, **kw)


def solve_host(X, y, device: int = 0, **kw) -> SolveResult:
    return _default_ctx(device).solve_host(X, y, **kw)
