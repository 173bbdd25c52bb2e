"""Parity of the CUDA tall sweep (column-major X, n <= 512) with the float64
CPU oracle of Algorithm 1, through the C ABI.

Tolerance: relative coefficient error <= 1e-5 for float32 arithmetic
against the oracle at the same sweep count, and <= 1e-3 for bfloat16 storage
(the oracle solves the same bfloat16-valued system, so storage rounding is not
part of the error; the GPU's float32 accumulation is).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2104_12570_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_12570_gb300 as hp  # noqa: E402

RTOL_F32 = 1e-5
RTOL_BF16 = 1e-3
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    c = hp.Context(0)
    yield c
    c.close()


def to_gpu(s):
    """synth.System -> (X logical (m, n) CUDA tensor with the system's layout, y)."""
    if s.dtype == "bf16":
        Xt = torch.from_numpy(s.X.view(np.int16)).view(torch.bfloat16)
    elif s.dtype == "f16":
        Xt = torch.from_numpy(s.X)
    else:
        Xt = torch.from_numpy(np.ascontiguousarray(s.X, dtype=np.float32))
    Xt = Xt.cuda()
    X = Xt.T if s.layout == "col" else Xt
    y = torch.from_numpy(np.asarray(s.y, dtype=np.float32)).cuda()
    return X, y


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def oracle_same(s, sweeps, a0=None):
    return oracle.solve_system(s, tol=0, max_sweeps=sweeps, stop="none", a0=a0)


def assert_true_residual(s, r, tol):
    """REL_RES stops on y - X·a of the returned float32 coefficients: the
    oracle's float64 residual of the GPU's a meets tol and equals the reported
    residual (the GPU forms it with Dot2)."""
    _, nrm = oracle.residual(s.X, s.y, r.a.cpu().numpy(), m=s.m, n=s.n, dtype=s.dtype)
    true = nrm / np.linalg.norm(s.y.astype(np.float64))
    assert true <= tol
    # Dot2 carries ~48 significant bits: at a residual of 1e-6·||y|| the
    # reported value is within ~1e-7 relative of the float64 one
    assert r.rel_res == pytest.approx(true, rel=1e-6)
    assert r.hist[r.sweeps] == r.rel_res


def test_hand_worked_example_exact(ctx):
    g = json.load(open(os.path.join(GOLDEN, "hand_2x2.json")))
    Xd = np.array(g["X_rows"], dtype=np.float32)
    X = torch.from_numpy(np.ascontiguousarray(Xd.T)).cuda().T
    y = torch.tensor(g["y"], dtype=torch.float32).cuda()
    for rec in g["sweeps"]:
        r = ctx.solve(X, y, tol=0, max_sweeps=rec["s"], stop="none")
        assert r.status == "ok" and r.sweeps == rec["s"]
        np.testing.assert_array_equal(r.a.cpu().numpy(), np.array(rec["a"], dtype=np.float32))
        for s in range(rec["s"] + 1):
            expect = 1.0 if s == 0 else np.sqrt(0.4) * 2.0 ** -s
            assert r.hist[s] == pytest.approx(expect, rel=1e-14)


@pytest.mark.parametrize("m,n", [(200, 50), (1000, 37), (777, 5), (64, 1), (3, 3), (5000, 300),
                                 (4099, 512), (100_000, 64), (33, 129)])
def test_equal_sweeps_matches_oracle(ctx, m, n):
    s = synth.make_system(m, n, seed=m + n, noise=0.05)
    X, y = to_gpu(s)
    for sweeps in (1, 3, 8):
        r = ctx.solve(X, y, tol=0, max_sweeps=sweeps, stop="none")
        o = oracle_same(s, sweeps)
        assert r.sweeps == sweeps
        assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32, (sweeps, rel(r.a.cpu().numpy(), o.a))
        # ||e||/||y|| from a float32 residual carries ~1e-7 absolute error: wide
        # (consistent) systems decay to that floor, where only an absolute bound holds
        np.testing.assert_allclose(r.hist, o.hist, rtol=1e-5, atol=1e-7)


def test_converges_on_consistent_tall(ctx):
    s = synth.make_system(200, 50, seed=0)
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=200, stop="rel_res")
    assert r.status == "ok" and r.rel_res <= 1e-6
    o = oracle_same(s, r.sweeps)
    assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32
    # the stop is taken on the true residual of the returned a: the oracle's
    # float64 residual of the GPU's a meets the tolerance and is the one reported
    assert_true_residual(s, r, 1e-6)
    assert rel(r.a.cpu().numpy(), s.a_true) <= 1e-5


def test_bf16_storage_matches_oracle(ctx):
    s = synth.make_system(20_000, 100, seed=3, dtype="bf16")
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=100, stop="rel_res")
    assert r.status == "ok"
    o = oracle_same(s, r.sweeps)
    assert rel(r.a.cpu().numpy(), o.a) <= RTOL_BF16
    assert rel(r.a.cpu().numpy(), o.a) <= 1e-5  # the storage is exact: f32 arithmetic only


@pytest.mark.parametrize("m,n", [(20_000, 100), (4099, 512), (777, 5), (100_003, 256), (33, 129)])
def test_f16_storage_matches_oracle_at_equal_sweeps(ctx, m, n):
    """IEEE binary16 storage: every value widens exactly to float32, so the
    GPU's error against the oracle (which solves the same binary16-valued
    system) is that of float32 arithmetic: the float32 bound at equal sweeps,
    through the tensor-core set-up (kind::f16) and the 16-bit sweep loads."""
    s = synth.make_system(m, n, seed=m + 3 * n, dtype="f16", noise=0.05)
    X, y = to_gpu(s)
    assert X.dtype == torch.float16
    for sweeps in (1, 4):
        r = ctx.solve(X, y, tol=0, max_sweeps=sweeps, stop="none")
        o = oracle_same(s, sweeps)
        assert r.status == "ok" and r.sweeps == sweeps
        assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32, (sweeps, rel(r.a.cpu().numpy(), o.a))
        np.testing.assert_allclose(r.hist, o.hist, rtol=1e-5, atol=1e-7)


def test_f16_refresh_and_true_residual_stop(ctx):
    """Binary16 storage with true-residual refresh passes every 2 sweeps,
    solved to relative residual 1e-6 on the returned coefficients."""
    s = synth.make_system(60_001, 200, seed=21, dtype="f16")
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=60, stop="rel_res", refresh_every=2)
    assert r.status == "ok"
    o = oracle_same(s, r.sweeps)
    assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32
    assert_true_residual(s, r, 1e-6)


@pytest.mark.parametrize("m,n,dtype", [(200_003, 256, "f32"), (1_000_000, 64, "f32"), (300_001, 512, "bf16")])
def test_residual_on_chip_matches_residual_in_hbm(ctx, m, n, dtype):
    """Where it fits, each CTA keeps the residual of its rows in shared memory;
    the debug bit HPSCD_DEBUG_E_IN_HBM keeps it in HBM.  Both give the oracle's
    iterate at equal sweeps, and the same stop and residual under REL_RES."""
    s = synth.make_system(m, n, seed=m % 97 + n, dtype=dtype, noise=0.01)
    X, y = to_gpu(s)
    o = oracle_same(s, 3)
    for flags in (0, 4):
        r = ctx.solve(X, y, tol=0, max_sweeps=3, stop="none", debug_flags=flags)
        assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32, (flags, rel(r.a.cpu().numpy(), o.a))
        np.testing.assert_allclose(r.hist, o.hist, rtol=1e-5, atol=1e-7)
    on = ctx.solve(X, y, tol=1e-7, max_sweeps=50, stop="rel_change")
    off = ctx.solve(X, y, tol=1e-7, max_sweeps=50, stop="rel_change", debug_flags=4)
    assert on.sweeps == off.sweeps and on.rel_res == pytest.approx(off.rel_res, rel=1e-9)


def test_unaligned_leading_dimension_uses_plain_loads(ctx):
    m, n = 1001, 17
    s = synth.make_system(m, n, seed=4)
    buf = np.zeros((n, m + 1), dtype=np.float32)
    buf[:, :m] = s.X
    Xt = torch.from_numpy(buf).cuda()
    X = Xt[:, :m].T  # stride (1, m + 1): ld*4 not a multiple of 16
    assert X.stride() == (1, m + 1)
    y = torch.from_numpy(s.y).cuda()
    r = ctx.solve(X, y, tol=0, max_sweeps=4, stop="none")
    o = oracle_same(s, 4)
    assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32


def test_warm_start_matches_oracle(ctx):
    s = synth.make_system(3000, 40, seed=5)
    a0 = (s.a_true + 0.01 * np.random.default_rng(0).standard_normal(40)).astype(np.float32)
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=0, max_sweeps=2, stop="none", a0=torch.from_numpy(a0).cuda())
    o = oracle_same(s, 2, a0=a0.astype(np.float64))
    assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32
    # float32 residual arithmetic: hist carries ~1e-8·||y|| absolute error
    np.testing.assert_allclose(r.hist, o.hist, rtol=1e-4, atol=1e-7)
    cold = ctx.solve(X, y, tol=1e-6, max_sweeps=100, stop="rel_res")
    warm = ctx.solve(X, y, tol=1e-6, max_sweeps=100, stop="rel_res", a0=torch.from_numpy(a0).cuda())
    assert warm.sweeps < cold.sweeps


def test_refresh_passes_match_oracle(ctx):
    s = synth.make_system(50_000, 128, seed=6, dtype="bf16")
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=50, stop="rel_res", refresh_every=2)
    assert r.status == "ok"
    o = oracle_same(s, r.sweeps)
    assert rel(r.a.cpu().numpy(), o.a) <= 1e-5
    assert_true_residual(s, r, 1e-6)


def test_zero_column_is_skipped(ctx):
    s = synth.make_system(500, 9, seed=7)
    s.X[4, :] = 0.0
    s.y = (s.dense_f64() @ s.a_true).astype(np.float32)
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=0, max_sweeps=6, stop="none")
    a = r.a.cpu().numpy()
    assert a[4] == 0.0 and np.all(np.isfinite(a))
    assert rel(a, oracle_same(s, 6).a) <= RTOL_F32


def test_stopping_rules_follow_oracle(ctx):
    s = synth.make_system(20_000, 64, seed=8, noise=0.01)
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=1e-7, max_sweeps=100, stop="rel_change")
    o = oracle.solve_system(s, tol=1e-7, max_sweeps=100, stop="rel_change")
    assert r.status == "ok" and abs(r.sweeps - o.sweeps) <= 1
    h = r.hist
    assert abs(h[-2] - h[-1]) < 1e-7 * h[-2]
    nc = ctx.solve(X, y, tol=1e-9, max_sweeps=2, stop="rel_res")
    assert nc.status == "not_converged" and nc.sweeps == 2


def test_degenerate_shapes(ctx):
    y = torch.ones(10, device="cuda")
    X = torch.zeros(10, 0, device="cuda")
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=3, stop="rel_res")
    assert r.status == "not_converged" and np.allclose(r.hist, 1.0)
    X = torch.zeros(0, 4, device="cuda")
    r = ctx.solve(X, torch.zeros(0, device="cuda"), tol=1e-6, max_sweeps=3, stop="rel_res")
    assert r.status == "ok" and r.sweeps == 0 and np.all(r.a.cpu().numpy() == 0)
    s = synth.make_system(100, 10, seed=9)
    Xs, ys = to_gpu(s)
    r = ctx.solve(Xs, ys, tol=0, max_sweeps=0, stop="none")
    assert r.sweeps == 0 and r.hist[0] == pytest.approx(1.0)
    # n > 512 (the panel sweep) with every column zero: each step is skipped
    Xz = torch.zeros(600, 10, device="cuda").T
    r = ctx.solve(Xz, y, tol=1e-6, max_sweeps=3, stop="rel_res")
    assert r.status == "not_converged" and r.sweeps == 3
    assert np.all(r.a.cpu().numpy() == 0) and np.allclose(r.hist, 1.0)


def test_binding_rejects_arguments_the_kernels_would_misread(ctx):
    """Vectors of the wrong length, type or device, and host X for a device call,
    are refused before anything is launched; the context stays usable."""
    s = synth.make_system(300, 20, seed=12)
    X, y = to_gpu(s)
    bad = [dict(y=y[:-1]), dict(y=y.double()), dict(y=y.cpu()),
           dict(out=torch.empty(19, device="cuda")), dict(out=torch.empty(20, device="cuda").double()),
           dict(a0=torch.zeros(21, device="cuda"))]
    for kw in bad:
        args = dict(y=y)
        args.update(kw)
        yy = args.pop("y")
        with pytest.raises((TypeError, ValueError)):
            ctx.solve(X, yy, tol=0, max_sweeps=1, stop="none", **args)
    with pytest.raises((TypeError, ValueError)):
        ctx.solve_blocks(X, y[:-1], 5, tol=0, max_sweeps=1, stop="none")
    with pytest.raises((TypeError, ValueError)):
        ctx.select(X, y.double(), 3)
    with pytest.raises((TypeError, ValueError)):
        ctx.solve_order(X, y, np.zeros((1, 20), np.int32), out=torch.empty(3, device="cuda"))
    with pytest.raises((TypeError, ValueError)):
        ctx.gram(X.cpu())
    with pytest.raises((TypeError, ValueError)):
        ctx.solve_host(s.X.T, s.y, a0=np.zeros(7))
    b = hp.Batch(ctx, [(X, y, torch.zeros(20, device="cuda"), False)], tol=0, max_sweeps=1, stop="none")
    net = hp.MLP(ctx, max_batch=8)
    with pytest.raises(TypeError):
        b.set_warm_start(net, torch.zeros(1, 16, device="cuda", dtype=torch.float64))
    with pytest.raises(TypeError):
        net.predict(torch.zeros(2, 16, device="cuda", dtype=torch.float64), [300, 300], [10, 10])
    with pytest.raises((TypeError, ValueError)):
        net.train_step(torch.zeros(2, 16, device="cuda"), [300, 300], [10], torch.zeros(2, 256, device="cuda"))
    with pytest.raises(TypeError):
        net.gradients(torch.zeros(2, 16, device="cuda"), [300, 300], [10, 10], torch.zeros(2, 255, device="cuda"))
    with pytest.raises(TypeError):
        hp.Batch(ctx, [(X, y, torch.zeros(20, device="cuda"), False,
                        torch.zeros(1, device="cuda", dtype=torch.float64))], tol=0, max_sweeps=1,
                 stop="none")
    b.close()
    net.close()
    r = ctx.solve(X, y, tol=0, max_sweeps=2, stop="none")
    assert rel(r.a.cpu().numpy(), oracle_same(s, 2).a) <= RTOL_F32

def test_barrier_timeout_returns_status_and_context_survives(ctx):
    s = synth.make_system(20_000, 32, seed=10)
    X, y = to_gpu(s)
    ctx.set_timeout(0.2)
    with pytest.raises(hp.HpscdError) as ei:
        ctx.solve(X, y, tol=1e-6, max_sweeps=10, stop="rel_res", debug_flags=1)
    assert ei.value.status == "timeout"
    ctx.set_timeout(5.0)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=50, stop="rel_res")
    assert r.status == "ok"


def test_host_entry_point_end_to_end(ctx):
    s = synth.make_system(4000, 48, seed=11)
    r = ctx.solve_host(s.X.T, s.y, tol=0, max_sweeps=3, stop="none")
    assert rel(r.a, oracle_same(s, 3).a) <= RTOL_F32


@pytest.mark.parametrize("m,n,dtype,ld_pad", [(600_001, 200, "f32", 0), (300_007, 130, "bf16", 0),
                                               (200_003, 72, "f16", 0), (50_001, 40, "f16", 1),
                                               (262_145, 64, "f32", 1), (131_071, 96, "f32", 0)])
def test_host_entry_point_large_ragged_bf16_unaligned(ctx, m, n, dtype, ld_pad):
    """hpscd_solve_host on tall systems: ragged row counts, bfloat16 storage, and
    an unaligned leading dimension (the CUDA-core set-up)."""
    s = synth.make_system(m, n, seed=m % 1000, dtype=dtype, noise=0.01)
    Xh = s.X
    if ld_pad:
        buf = np.zeros((n, m + ld_pad), dtype=s.X.dtype)
        buf[:, :m] = s.X
        Xh = buf[:, :m]
    r = ctx.solve_host(Xh.T, s.y, tol=0, max_sweeps=3, stop="none")
    o = oracle_same(s, 3)
    assert r.status == "ok" and r.sweeps == 3
    assert rel(r.a, o.a) <= (RTOL_BF16 if dtype == "bf16" else RTOL_F32)
    np.testing.assert_allclose(r.hist, o.hist, rtol=1e-4)


@pytest.mark.slow
def test_full_size_tall_1Mx256(ctx):
    """The 1,000,000 x 256 float32 noisy least-squares workload, in the launch
    configuration the benchmark times, against the oracle at equal sweeps."""
    s = synth.workload("tall_1Mx256_f32")
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=1e-7, max_sweeps=50, stop="rel_change")
    assert r.status == "ok"
    o = oracle_same(s, r.sweeps)
    assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32
    np.testing.assert_allclose(r.hist, o.hist, rtol=1e-5)
    assert r.timing["grid"] >= 1


@pytest.mark.slow
def test_full_size_precision_mode_4Mx512_bf16(ctx):
    """The 4,000,000 x 512 bfloat16 system in the benchmark's precision-mode
    configuration (refresh every 4 passes, relative residual 1e-6): the oracle's
    float64 residual of the GPU's coefficients meets the tolerance, and one sweep
    equals the oracle's first sweep (bfloat16-storage tolerance)."""
    s = synth.workload("tall_4Mx512_bf16", seed=0)
    X, y = to_gpu(s)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=100, stop="rel_res", refresh_every=4)
    assert r.status == "ok" and r.rel_res <= 1e-6
    assert_true_residual(s, r, 1e-6)  # the last sweep's pass formed y - X·a (predicted last sweep)
    r1 = ctx.solve(X, y, tol=0, max_sweeps=1, stop="none", refresh_every=4)
    o1 = oracle_same(s, 1)
    assert rel(r1.a.cpu().numpy(), o1.a) <= RTOL_BF16
    np.testing.assert_allclose(r1.hist, o1.hist, rtol=1e-4)

def test_async_solves_equal_the_synchronous_ones(ctx):
    """hpscd_solve_async: several solves enqueued back to back (different systems
    and stopping rules) give the synchronous call's coefficients, history, sweep
    count and status; their event timings come back per call."""
    systems = [synth.make_system(m, n, seed=m + n, noise=0.05) for m, n in
               ((20000, 256), (7777, 130), (4099, 97))]
    dev = [(torch.from_numpy(s.X).cuda().T, torch.from_numpy(s.y).cuda()) for s in systems]
    kw = [dict(tol=1e-6, max_sweeps=60, stop="rel_change"), dict(tol=0, max_sweeps=4, stop="none"),
          dict(tol=1e-9, max_sweeps=6, stop="rel_res")]
    res = hp.results_buffer(6)
    outs, hists = [], []
    for k in range(6):
        X, y = dev[k % 3]
        hist = torch.full((61,), float("nan"), dtype=torch.float64, device="cuda")
        outs.append(ctx.solve_async(X, y, res[k], hist=hist, **kw[k % 3]))
        hists.append(hist)
    times = ctx.async_timings(6)
    got = hp.read_results(res)
    for k in range(6):
        X, y = dev[k % 3]
        r = ctx.solve(X, y, **kw[k % 3])
        assert got["status"][k] == r.status == ("not_converged" if k % 3 == 2 else "ok")
        assert got["sweeps"][k] == r.sweeps and got["passes"][k] == r.timing["passes"]
        assert got["rel_res"][k] == r.rel_res
        assert torch.equal(outs[k], r.a)
        np.testing.assert_array_equal(hists[k][: r.sweeps + 1].cpu().numpy(), r.hist)
        assert times[k]["sweep_ms"] > 0 and times[k]["setup_ms"] > 0
    with pytest.raises(hp.HpscdError):
        ctx.async_timings(65)
