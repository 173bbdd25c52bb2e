"""hpscd_solve_noalloc, the allocation-free entry point, through the C ABI.

It exists for callers that must not allocate device memory when they solve
(cudaMalloc/cudaFree can synchronize the device and stall other streams; some
callers run where another allocator or a fixed budget owns device memory).
It runs the same kernels as hpscd_solve with its scratch in a static device
array shared by every call, so two calls in a row must both agree with
hpscd_solve: the second one starts from whatever the first left behind.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2104_12570_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_12570_gb300 as hp  # noqa: E402

RTOL_F32 = 1e-5  # the float32 coefficient tolerance of the other GPU tests


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def solve_noalloc(X, y, a_out, guess=False, **kw):
    """Call hpscd_solve_noalloc on torch's current stream (argument marshalling only).
    guess: a_out holds the initial guess (a_is_guess = 1)."""
    lib = hp.load()
    _, dt, lay, m, n, ld = hp._describe(X)
    assert lay == hp.COL
    o = hp.make_opts(**kw)
    hist = np.full(int(o.max_sweeps) + 1, np.nan)
    sw, rr = ctypes.c_int64(0), ctypes.c_double(0.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.hpscd_solve_noalloc(stream, ctypes.c_void_p(X.data_ptr()), dt, m, n, ld,
                                 ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(a_out.data_ptr()),
                                 1 if guess else 0, ctypes.byref(o),
                                 hist.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.byref(sw), ctypes.byref(rr))
    return rc, hist[: sw.value + 1], sw.value


def gpu_system(s):
    if s.dtype == "bf16":
        X = torch.from_numpy(s.X.view(np.int16)).view(torch.bfloat16).cuda().T
    else:
        X = torch.from_numpy(s.X).cuda().T
    return X, torch.from_numpy(s.y).cuda()


def test_two_calls_in_a_row_match_hpscd_solve():
    s = synth.make_system(150_000, 200, seed=21, noise=0.01)  # ragged n, many panels
    X, y = gpu_system(s)
    ctx = hp.Context(0)
    kw = dict(tol=0.0, max_sweeps=6, stop="none")
    ref = ctx.solve(X, y, **kw)
    ctx.close()
    outs = [torch.full((s.n,), float("nan"), device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    free = []
    for a in outs:
        rc, hist, sweeps = solve_noalloc(X, y, a, **kw)
        free.append(torch.cuda.mem_get_info()[0])
        assert rc == 0 and sweeps == ref.sweeps == 6
        assert rel(a.cpu().numpy(), ref.a.cpu().numpy()) <= RTOL_F32
        np.testing.assert_allclose(hist, ref.hist, rtol=1e-5, atol=1e-7)
    # the defining property: once the first call has run (it may load the
    # library's kernels), further calls take no device memory at all
    assert free[1] == free[0] and free[2] == free[0]


def test_warm_start_matches_hpscd_solve():
    s = synth.make_system(60_000, 128, seed=23, noise=0.01)
    X, y = gpu_system(s)
    guess = torch.from_numpy((s.a_true + 0.05 * np.random.default_rng(1).standard_normal(s.n))
                             .astype(np.float32)).cuda()
    ctx = hp.Context(0)
    kw = dict(tol=0.0, max_sweeps=3, stop="none")
    ref = ctx.solve(X, y, a0=guess, **kw)
    ctx.close()
    for _ in range(2):
        a = guess.clone()
        rc, hist, sweeps = solve_noalloc(X, y, a, guess=True, **kw)
        assert rc == 0 and sweeps == 3
        assert rel(a.cpu().numpy(), ref.a.cpu().numpy()) <= RTOL_F32
        np.testing.assert_allclose(hist, ref.hist, rtol=1e-5, atol=1e-7)


def test_refuses_host_pointers():
    s = synth.make_system(1000, 8, seed=24)
    X, y = gpu_system(s)
    a = torch.empty(s.n, device="cuda")
    y_host = torch.from_numpy(s.y)  # pageable host memory: the kernels cannot read it
    rc, _, _ = solve_noalloc(X, y_host, a, tol=1e-6, max_sweeps=5, stop="rel_res")
    assert rc == 1  # HPSCD_ERR_INVALID_ARG, nothing launched


@pytest.mark.parametrize("dtype", ["f16"])
def test_f16_matches_hpscd_solve(dtype):
    s = synth.make_system(30_001, 64, seed=23, dtype=dtype)
    X, y = gpu_system(s)
    assert X.dtype == torch.float16
    ctx = hp.Context(0)
    ref = ctx.solve(X, y, tol=0, max_sweeps=5, stop="none")
    ctx.close()
    a = torch.empty(s.n, device="cuda")
    rc, hist, sweeps = solve_noalloc(X, y, a, tol=0, max_sweeps=5, stop="none")
    assert rc == 0 and sweeps == 5
    assert rel(a.cpu().numpy(), ref.a.cpu().numpy()) <= RTOL_F32


def test_bf16_and_limits():
    s = synth.make_system(40_000, 96, seed=22, dtype="bf16")
    X, y = gpu_system(s)
    ctx = hp.Context(0)
    ref = ctx.solve(X, y, tol=1e-6, max_sweeps=100, stop="rel_res")
    ctx.close()
    a = torch.empty(s.n, device="cuda")
    rc, hist, sweeps = solve_noalloc(X, y, a, tol=1e-6, max_sweeps=100, stop="rel_res")
    assert rc == 0 and abs(sweeps - ref.sweeps) <= 1
    assert rel(a.cpu().numpy(), ref.a.cpu().numpy()) <= RTOL_F32
    # beyond the stated maximum size: a clear error, nothing launched
    for n_, m_ in ((300, 1000), (1, (1 << 20) + 1)):  # n > 256, m > 2^20
        big = torch.zeros(n_, m_, device="cuda").T
        rc, _, _ = solve_noalloc(big, torch.zeros(m_, device="cuda"),
                                 torch.empty(n_, device="cuda"), tol=1e-6, max_sweeps=10,
                                 stop="rel_res")
        assert rc == 6  # HPSCD_ERR_UNSUPPORTED
