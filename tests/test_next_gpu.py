"""Parity of the CUDA forms of Algorithm 2 (HPSCDP: blocks of thr columns take
their steps from the same residual, Sec. 7) and Algorithm 3 (HPSCDF: greedy
feature selection, Sec. 8) with the float64 CPU oracle, through the C ABI.

Tolerances as for Algorithm 1: relative coefficient error <= 1e-5 and hist rtol
1e-5 at equal sweep counts.  The selected columns of Algorithm 3 are index work
and must match exactly; the workloads plant a support with well separated
weights so that no two scores are within float32 rounding of each other."""
import numpy as np
import pytest

import oracle
from paper_2104_12570_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_12570_gb300 as hp  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = hp.Context(0)
    yield c
    c.close()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def to_gpu(s):
    X = torch.from_numpy(np.ascontiguousarray(s.X, dtype=np.float32)).cuda().T
    y = torch.from_numpy(np.asarray(s.y, dtype=np.float32)).cuda()
    return X, y


@pytest.mark.parametrize("m,n,thr", [(2000, 256, 1), (2000, 256, 25), (2000, 256, 32),
                                     (2000, 256, 64), (2000, 256, 256), (777, 130, 3),
                                     (5000, 512, 51), (333, 40, 7), (4099, 97, 40),
                                     (1000, 64, 1000)])
def test_blocks_equal_sweeps_match_oracle(ctx, m, n, thr):
    s = synth.make_system(m, n, seed=m + thr, noise=0.05)
    X, y = to_gpu(s)
    for sweeps in (1, 4):
        r = ctx.solve_blocks(X, y, thr, tol=0, max_sweeps=sweeps, stop="none")
        o = oracle.solve_blocks(s.X, s.y, m=m, n=n, thr=thr, tol=0, max_sweeps=sweeps, stop="none")
        assert r.status == "ok" and r.sweeps == sweeps
        assert rel(r.a.cpu().numpy(), o.a) <= 1e-5, (m, n, thr, sweeps)
        np.testing.assert_allclose(r.hist, o.hist, rtol=1e-5, atol=1e-7)


def test_blocks_thr_one_is_the_plain_sweep(ctx):
    s = synth.make_system(3000, 200, seed=3, noise=0.05)
    X, y = to_gpu(s)
    r1 = ctx.solve(X, y, tol=0, max_sweeps=5, stop="none")
    r2 = ctx.solve_blocks(X, y, 1, tol=0, max_sweeps=5, stop="none")
    assert torch.equal(r1.a, r2.a)


def test_blocks_stopping_rule_and_warm_start(ctx):
    s = synth.make_system(4000, 128, seed=5, noise=0.05)
    X, y = to_gpu(s)
    r = ctx.solve_blocks(X, y, 13, tol=1e-7, max_sweeps=200, stop="rel_change")
    o = oracle.solve_blocks(s.X, s.y, m=s.m, n=s.n, thr=13, tol=1e-7, max_sweeps=200,
                            stop="rel_change")
    assert r.status == "ok" and abs(r.sweeps - o.sweeps) <= 1
    a0 = (s.a_true + 0.1).astype(np.float32)
    r = ctx.solve_blocks(X, y, 13, tol=0, max_sweeps=3, stop="none", a0=torch.from_numpy(a0).cuda())
    o = oracle.solve_blocks(s.X, s.y, m=s.m, n=s.n, thr=13, a0=a0, tol=0, max_sweeps=3, stop="none")
    assert rel(r.a.cpu().numpy(), o.a) <= 1e-5


def planted(m, n, seed, support, noise=0.01):
    g = np.random.default_rng(seed)
    Xd = g.standard_normal((m, n)).astype(np.float32)
    w = np.linspace(3.0, 1.0, len(support)) * np.where(np.arange(len(support)) % 2, -1, 1)
    y = (Xd[:, support].astype(np.float64) @ w + noise * g.standard_normal(m)).astype(np.float32)
    return synth.System(X=np.ascontiguousarray(Xd.T), y=y, a_true=np.zeros(n), m=m, n=n,
                        layout="col", dtype="f32")


@pytest.mark.parametrize("m,n,F", [(2000, 256, 12), (5000, 100, 8), (1500, 512, 10), (300, 33, 6)])
def test_selection_matches_oracle(ctx, m, n, F):
    support = list(np.random.default_rng(m).choice(n, size=min(F, n) - 2, replace=False))
    s = planted(m, n, m + n, support)
    X, y = to_gpu(s)
    r, sel = ctx.select(X, y, F)
    osel, oa, ohist = oracle.select(s.X, s.y, m=m, n=n, F=F)
    np.testing.assert_array_equal(sel, osel)
    assert rel(r.a.cpu().numpy(), oa) <= 1e-5
    np.testing.assert_allclose(r.hist, ohist, rtol=1e-5)
    assert sorted(set(sel[: len(support)].tolist())) == sorted(support)


def test_selection_stops_when_errors_stop_decreasing(ctx):
    s = planted(3000, 64, 11, [4, 9, 30], noise=0.0)
    X, y = to_gpu(s)
    r, sel = ctx.select(X, y, 50, tol=1e-4, stop="rel_change")
    assert r.status == "ok" and r.sweeps < 50
    assert set(sel[:3].tolist()) == {4, 9, 30}


@pytest.mark.slow
def test_full_size_blocks_and_selection(ctx):
    """The 1,000,000 x 256 benchmark system: Algorithm 2 at thr = n/10 and 20
    selection steps, at equal step counts with the oracle."""
    s = synth.workload("tall_1Mx256_f32", seed=0)
    X, y = to_gpu(s)
    r = ctx.solve_blocks(X, y, 25, tol=0, max_sweeps=3, stop="none")
    o = oracle.solve_blocks(s.X, s.y, m=s.m, n=s.n, thr=25, tol=0, max_sweeps=3, stop="none")
    assert rel(r.a.cpu().numpy(), o.a) <= 1e-5
    r, sel = ctx.select(X, y, 20)
    osel, oa, ohist = oracle.select(s.X, s.y, m=s.m, n=s.n, F=20)
    np.testing.assert_array_equal(sel, osel)
    np.testing.assert_allclose(r.hist, ohist, rtol=1e-5)


# ---- Algorithm 1 with the column of every step given (Sec. 2's random-index variant) ----

@pytest.mark.parametrize("m,n,kind", [(2000, 256, "replace"), (2000, 256, "perm"), (777, 130, "replace"),
                                      (333, 40, "perm"), (4099, 97, "replace"), (5000, 512, "replace"),
                                      (300, 33, "same")])
def test_order_equal_sweeps_match_oracle(ctx, m, n, kind):
    s = synth.make_system(m, n, seed=m + n, noise=0.05)
    X, y = to_gpu(s)
    g = np.random.default_rng(m)
    sweeps = 4
    if kind == "replace":
        order = g.integers(0, n, size=(sweeps, n))
    elif kind == "perm":
        order = np.stack([g.permutation(n) for _ in range(sweeps)])
    else:
        order = np.full((sweeps, n), n // 2)
    for k in (1, sweeps):
        r = ctx.solve_order(X, y, order[:k], tol=0, stop="none")
        o = oracle.solve_order(s.X, s.y, m=m, n=n, order=order[:k], tol=0, max_sweeps=k, stop="none")
        assert r.status == "ok" and r.sweeps == k
        assert rel(r.a.cpu().numpy(), o.a) <= 1e-5, (m, n, kind, k)
        np.testing.assert_allclose(r.hist, o.hist, rtol=1e-5, atol=1e-7)


def test_natural_order_is_the_plain_sweep(ctx):
    s = synth.make_system(3000, 200, seed=13, noise=0.05)
    X, y = to_gpu(s)
    r1 = ctx.solve(X, y, tol=0, max_sweeps=5, stop="none")
    r2 = ctx.solve_order(X, y, np.tile(np.arange(200), (5, 1)), tol=0, stop="none")
    assert torch.equal(r1.a, r2.a)
    np.testing.assert_array_equal(r1.hist, r2.hist)


def test_order_stopping_rule_warm_start_and_bad_index(ctx):
    s = synth.make_system(4000, 128, seed=17, noise=0.05)
    X, y = to_gpu(s)
    order = np.random.default_rng(2).integers(0, 128, size=(200, 128))
    r = ctx.solve_order(X, y, order, tol=1e-7, stop="rel_change")
    o = oracle.solve_order(s.X, s.y, m=s.m, n=s.n, order=order, tol=1e-7, max_sweeps=200,
                           stop="rel_change")
    assert r.status == "ok" and abs(r.sweeps - o.sweeps) <= 1
    a0 = (s.a_true + 0.1).astype(np.float32)
    r = ctx.solve_order(X, y, order[:3], tol=0, stop="none", a0=torch.from_numpy(a0).cuda())
    o = oracle.solve_order(s.X, s.y, m=s.m, n=s.n, order=order[:3], a0=a0, tol=0, max_sweeps=3,
                           stop="none")
    assert rel(r.a.cpu().numpy(), o.a) <= 1e-5
    bad = order[:2].copy()
    bad[1, 5] = 128
    with pytest.raises(hp.HpscdError):
        ctx.solve_order(X, y, bad, tol=0, stop="none")


@pytest.mark.slow
def test_full_size_random_order(ctx):
    """The 1,000,000 x 256 benchmark system, 3 sweeps of indices drawn with replacement."""
    s = synth.workload("tall_1Mx256_f32", seed=0)
    X, y = to_gpu(s)
    order = np.random.default_rng(7).integers(0, 256, size=(3, 256))
    r = ctx.solve_order(X, y, order, tol=0, stop="none")
    o = oracle.solve_order(s.X, s.y, m=s.m, n=s.n, order=order, tol=0, max_sweeps=3, stop="none")
    assert rel(r.a.cpu().numpy(), o.a) <= 1e-5
    np.testing.assert_allclose(r.hist, o.hist, rtol=1e-5)


# ---- the feature-removal loop of Sec. 8: swap steps after Algorithm 3 ----

@pytest.mark.parametrize("seed,m,n,k_lat,supp,F,R", [(1, 200, 16, 3, 3, 3, 4), (3, 200, 16, 3, 3, 3, 4),
                                                     (100, 20000, 96, 4, 5, 5, 6),
                                                     (101, 20000, 96, 4, 5, 5, 6)])
def test_swap_steps_match_oracle(ctx, seed, m, n, k_lat, supp, F, R):
    """Correlated columns where the greedy steps miss part of the planted support:
    the swap steps (dropped and added columns) are index work and must match the
    oracle exactly; coefficients and history at 1e-5."""
    if m == 200:
        # the same draws as the oracle pins use
        g = np.random.default_rng(seed)
        base = g.standard_normal((m, 3))
        Xd = base @ g.standard_normal((3, n)) + 0.5 * g.standard_normal((m, n))
        y = Xd[:, [1, 5, 9]] @ np.array([1.0, -0.8, 0.6]) + 0.05 * g.standard_normal(m)
        s = synth.System(X=np.ascontiguousarray(Xd.T).astype(np.float32), y=y.astype(np.float32),
                         a_true=np.zeros(n), m=m, n=n, layout="col", dtype="f32")
    else:
        g = np.random.default_rng(seed)
        base = g.standard_normal((m, k_lat))
        Xd = base @ g.standard_normal((k_lat, n)) + 0.4 * g.standard_normal((m, n))
        sp = g.choice(n, supp, replace=False)
        w = g.uniform(0.5, 1.5, supp) * np.where(g.random(supp) < 0.5, -1, 1)
        y = Xd[:, sp] @ w + 0.05 * g.standard_normal(m)
        s = synth.System(X=np.ascontiguousarray(Xd.T).astype(np.float32), y=y.astype(np.float32),
                         a_true=np.zeros(n), m=m, n=n, layout="col", dtype="f32")
    X, yv = to_gpu(s)
    r, sel, swaps = ctx.select_swap(X, yv, F, R)
    osel, oswaps, oa, ohist = oracle.select_swap(s.X, s.y, m=m, n=n, F=F, R=R)
    np.testing.assert_array_equal(sel, osel)
    np.testing.assert_array_equal(swaps, oswaps)
    assert (oswaps[:, 0] >= 0).sum() >= 2  # the case exercises the loop
    assert r.status == "ok" and r.sweeps == F + (oswaps[:, 0] >= 0).sum()
    assert rel(r.a.cpu().numpy(), oa) <= 1e-5
    np.testing.assert_allclose(r.hist, ohist, rtol=1e-5)


def test_swap_with_no_rounds_is_selection(ctx):
    s = planted(3000, 64, 11, [4, 9, 30], noise=0.01)
    X, y = to_gpu(s)
    r0, sel0 = ctx.select(X, y, 6)
    r1, sel1, swaps = ctx.select_swap(X, y, 6, 0)
    np.testing.assert_array_equal(sel0, sel1)
    assert torch.equal(r0.a, r1.a) and swaps.shape == (0, 2)
