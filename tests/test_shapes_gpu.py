"""Shapes and storage types beyond the tall (column-major, n <= 512) and wide
(row-major, m <= 4096, float32) sweeps, through the C ABI, against the
float64 CPU oracle of Algorithm 1:

  column-major, n > 512      the panel sweep (panels of 512 columns in the
                             paper's column order, each from its diagonal Gram
                             block and the residual left by the panel before)
  row-major, m > 4096        one transpose to column-major in the set-up, then
                             the tall or panel sweep
  row-major 16-bit, m <= 4096  widened once to float32, then the cluster sweep

Every storage type widens exactly to float32, so each case is held to the
float32 bound (relative coefficient error <= 1e-5 at equal sweeps, the oracle
solving the same stored system) and, under REL_RES, to a true residual of the
returned coefficients at the tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_2104_12570_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_12570_gb300 as hp  # noqa: E402

RTOL_F32 = 1e-5


@pytest.fixture(scope="module")
def ctx():
    c = hp.Context(0)
    yield c
    c.close()


def to_gpu(s):
    """synth.System -> (X as a logical (m, n) CUDA tensor in the system's layout, y)."""
    if s.dtype == "bf16":
        Xt = torch.from_numpy(s.X.view(np.int16)).view(torch.bfloat16)
    else:
        Xt = torch.from_numpy(np.ascontiguousarray(s.X))
    Xt = Xt.cuda()
    X = Xt.T if s.layout == "col" else Xt
    return X, torch.from_numpy(np.asarray(s.y, dtype=np.float32)).cuda()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def assert_true_residual(s, r, tol):
    _, nrm = oracle.residual(s.X, s.y, r.a.cpu().numpy(), m=s.m, n=s.n, layout=s.layout, dtype=s.dtype)
    true = nrm / np.linalg.norm(s.y.astype(np.float64))
    assert true <= tol
    assert r.rel_res == pytest.approx(true, rel=1e-6)
    assert r.hist[r.sweeps] == r.rel_res


def equal_sweeps(ctx, s, sweeps_list=(1, 3)):
    X, y = to_gpu(s)
    for sweeps in sweeps_list:
        r = ctx.solve(X, y, tol=0, max_sweeps=sweeps, stop="none")
        o = oracle.solve_system(s, tol=0, max_sweeps=sweeps, stop="none")
        assert r.status == "ok" and r.sweeps == sweeps
        err = rel(r.a.cpu().numpy(), o.a)
        assert err <= RTOL_F32, (s.m, s.n, s.layout, s.dtype, sweeps, err)
        np.testing.assert_allclose(r.hist, o.hist, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("m,n,dtype", [(5000, 600, "f32"), (20_000, 1100, "f32"), (1000, 2049, "f32"),
                                       (300, 777, "f32"), (100_003, 1030, "f32"), (4099, 513, "f32"),
                                       (30_000, 700, "bf16"), (30_001, 1200, "f16")])
def test_panel_sweep_equal_sweeps_matches_oracle(ctx, m, n, dtype):
    """Column-major n > 512: ragged last panels, ragged row tails, m below and
    above one 4096-row segment per CTA, every storage type."""
    s = synth.make_system(m, n, seed=m + n, dtype=dtype, noise=0.05)
    equal_sweeps(ctx, s)


def test_panel_sweep_square_equal_sweeps(ctx):
    n = 1500
    s = synth.make_system(n, n, seed=n, scale=0.5 / np.sqrt(n), diag=1.0)
    equal_sweeps(ctx, s, (1, 4))


def test_panel_sweep_rel_res_stop_on_true_residual(ctx):
    s = synth.make_system(40_000, 800, seed=41)
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=60, stop="rel_res")
    assert r.status == "ok"
    o = oracle.solve_system(s, tol=0, max_sweeps=r.sweeps, stop="none")
    assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32
    assert_true_residual(s, r, 1e-6)
    assert rel(r.a.cpu().numpy(), s.a_true) <= 1e-5


def test_panel_sweep_rel_change_and_warm_start(ctx):
    s = synth.make_system(30_000, 900, seed=42, noise=0.01)
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=1e-7, max_sweeps=100, stop="rel_change")
    o = oracle.solve_system(s, tol=1e-7, max_sweeps=100, stop="rel_change")
    assert r.status == "ok" and o.status == "ok" and abs(r.sweeps - o.sweeps) <= 1
    # the reported residual is that of the returned float32 coefficients
    _, nrm = oracle.residual(s.X, s.y, r.a.cpu().numpy(), m=s.m, n=s.n)
    assert r.rel_res == pytest.approx(nrm / np.linalg.norm(s.y.astype(np.float64)), rel=1e-6)
    a0 = (s.a_true + 0.01 * np.random.default_rng(1).standard_normal(s.n)).astype(np.float32)
    rw = ctx.solve(X, y, tol=0, max_sweeps=2, stop="none", a0=torch.from_numpy(a0).cuda())
    ow = oracle.solve_system(s, tol=0, max_sweeps=2, stop="none", a0=a0.astype(np.float64))
    assert rel(rw.a.cpu().numpy(), ow.a) <= RTOL_F32
    np.testing.assert_allclose(rw.hist, ow.hist, rtol=1e-4, atol=1e-7)


def test_panel_sweep_refresh_bf16(ctx):
    s = synth.make_system(50_000, 640, seed=43, dtype="bf16")
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=60, stop="rel_res", refresh_every=2)
    assert r.status == "ok"
    o = oracle.solve_system(s, tol=0, max_sweeps=r.sweeps, stop="none")
    assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32
    assert_true_residual(s, r, 1e-6)


@pytest.mark.parametrize("m,n,dtype", [(10_000, 300, "f32"), (20_000, 700, "bf16"), (5000, 64, "f16"),
                                       (4097, 1, "f32"), (8193, 513, "f32")])
def test_row_major_tall_is_transposed_then_swept(ctx, m, n, dtype):
    s = synth.make_system(m, n, seed=m + 7 * n, layout="row", dtype=dtype, noise=0.05)
    equal_sweeps(ctx, s)


@pytest.mark.parametrize("m,n,dtype", [(2000, 20_000, "bf16"), (300, 4099, "f16"), (37, 1000, "bf16")])
def test_row_major_16bit_wide_is_widened_then_swept(ctx, m, n, dtype):
    s = synth.make_system(m, n, seed=m + n, layout="row", dtype=dtype)
    equal_sweeps(ctx, s, (1, 2))
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=30, stop="rel_res")
    assert r.status == "ok"
    assert_true_residual(s, r, 1e-6)


def test_panel_and_transposed_paths_through_the_host_entry_point(ctx):
    s = synth.make_system(6000, 700, seed=44, noise=0.05)
    r = ctx.solve_host(s.X.T, s.y, tol=0, max_sweeps=2, stop="none")
    assert rel(r.a, oracle.solve_system(s, tol=0, max_sweeps=2, stop="none").a) <= RTOL_F32
    sr = synth.make_system(9000, 100, seed=45, layout="row", dtype="f16", noise=0.05)
    r = ctx.solve_host(sr.X, sr.y, tol=0, max_sweeps=2, stop="none")
    assert rel(r.a, oracle.solve_system(sr, tol=0, max_sweeps=2, stop="none").a) <= RTOL_F32


def test_panel_sweep_in_caller_workspace(ctx):
    s = synth.make_system(12_000, 1030, seed=46)
    X, y = to_gpu(s)
    need = ctx.workspace_size(s.m, s.n, dtype="f32", layout="col", max_sweeps=3, stop="none")
    buf = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    base = (buf.data_ptr() + 255) // 256 * 256
    c2 = hp.Context(0)
    try:
        c2.set_workspace(base, need)
        r = c2.solve(X, y, tol=0, max_sweeps=3, stop="none")
        assert r.status == "ok"
        assert rel(r.a.cpu().numpy(), oracle.solve_system(s, tol=0, max_sweeps=3, stop="none").a) <= RTOL_F32
    finally:
        c2.close()
    del buf


def test_panel_sweep_barrier_timeout_returns_status(ctx):
    """The panel kernel's first grid barrier made to wait for one CTA too
    many: its bounded wait gives up, the solve returns the timeout status and
    the context still solves."""
    s = synth.make_system(5000, 600, seed=47)
    X, y = to_gpu(s)
    ctx.set_timeout(0.5)
    try:
        with pytest.raises(hp.HpscdError) as ei:
            ctx.solve(X, y, tol=0, max_sweeps=2, stop="none", debug_flags=1)
        assert ei.value.status == "timeout"
    finally:
        ctx.set_timeout(5.0)
    r = ctx.solve(X, y, tol=0, max_sweeps=2, stop="none")
    assert rel(r.a.cpu().numpy(), oracle.solve_system(s, tol=0, max_sweeps=2, stop="none").a) <= RTOL_F32
