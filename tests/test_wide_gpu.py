"""Parity of the CUDA wide sweep (row-major X, n >> m: one thread-block
cluster walks the column chain) with the float64 CPU oracle of Algorithm 1,
through the C ABI.  Wide consistent systems have infinitely many solutions,
so coefficients are compared at equal sweep counts (not against a_true), and
the true residual of the GPU's a is recomputed by the oracle."""
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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def gpu(s):
    return torch.from_numpy(s.X).cuda(), torch.from_numpy(s.y).cuda()


def assert_true_residual(s, r, tol):
    """The stop under REL_RES is taken on y - X·a of the returned coefficients:
    the oracle's float64 residual of the GPU's a meets tol, and the reported
    residual is that value."""
    _, nrm = oracle.residual(s.X, s.y, r.a.cpu().numpy(), m=s.m, n=s.n, layout="row")
    true = nrm / np.linalg.norm(s.y.astype(np.float64))
    assert true <= tol
    # Dot2 carries ~48 significant bits: at a residual of 1e-6·||y|| the
    # reported value is within ~1e-7 relative of the float64 one
    assert r.rel_res == pytest.approx(true, rel=1e-6)
    assert r.hist[r.sweeps] == r.rel_res


@pytest.mark.parametrize("m,n", [(20, 64), (37, 1000), (100, 5000), (300, 4099), (2000, 20000),
                                 (4096, 3000), (8, 333)])
def test_wide_equal_sweeps_matches_oracle(ctx, m, n):
    s = synth.make_system(m, n, seed=m * 7 + n, layout="row")
    X, y = gpu(s)
    for sweeps in (1, 2):
        r = ctx.solve(X, y, tol=0, max_sweeps=sweeps, stop="none")
        o = oracle.solve_system(s, tol=0, max_sweeps=sweeps, stop="none")
        assert r.status == "ok" and r.sweeps == sweeps
        assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32, (sweeps, rel(r.a.cpu().numpy(), o.a))
        np.testing.assert_allclose(r.hist, o.hist, rtol=1e-4, atol=2e-7)


def test_wide_warm_start_and_stop(ctx):
    s = synth.make_system(500, 8000, seed=5, layout="row")
    X, y = gpu(s)
    a0 = (0.5 * s.a_true).astype(np.float32)
    r = ctx.solve(X, y, tol=0, max_sweeps=1, stop="none", a0=torch.from_numpy(a0).cuda())
    o = oracle.solve_system(s, tol=0, max_sweeps=1, stop="none", a0=a0.astype(np.float64))
    assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=20, stop="rel_res")
    assert r.status == "ok" and r.rel_res <= 1e-6
    assert_true_residual(s, r, 1e-6)


@pytest.mark.slow
def test_full_size_wide_2000x200k(ctx):
    s = synth.workload("wide_2000x200k_f32")
    X, y = gpu(s)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=10, stop="rel_res")
    assert r.status == "ok" and r.rel_res <= 1e-6
    o = oracle.solve_system(s, tol=0, max_sweeps=r.sweeps, stop="none")
    assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32
    assert_true_residual(s, r, 1e-6)


@pytest.mark.parametrize("n,layout", [(777, "row"), (1024, "row"), (300, "col"), (512, "col")])
def test_square_equal_sweeps_matches_oracle(ctx, n, layout):
    """Square systems (the paper's third shape): row-major through the cluster
    sweep, column-major (n <= 512) through the tall sweep, at equal sweeps."""
    s = synth.make_system(n, n, seed=n, layout=layout, scale=0.5 / np.sqrt(n), diag=1.0)
    X = torch.from_numpy(s.X).cuda()
    if layout == "col":
        X = X.T
    y = torch.from_numpy(s.y).cuda()
    for sweeps in (1, 3):
        r = ctx.solve(X, y, tol=0, max_sweeps=sweeps, stop="none")
        o = oracle.solve_system(s, tol=0, max_sweeps=sweeps, stop="none")
        assert r.status == "ok" and r.sweeps == sweeps
        assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32, (n, layout, sweeps)
        np.testing.assert_allclose(r.hist, o.hist, rtol=1e-4, atol=2e-7)


@pytest.mark.slow
def test_full_size_square_4096(ctx):
    """The 4096 x 4096 square benchmark system to relative residual 1e-6: the
    sweep count and iterate of the oracle, and the oracle's own residual of a."""
    s = synth.workload("square_4096_f32")
    X, y = gpu(s)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=200, stop="rel_res")
    o = oracle.solve_system(s, tol=1e-6, max_sweeps=200, stop="rel_res")
    assert r.status == "ok" and o.status == "ok" and abs(r.sweeps - o.sweeps) <= 1
    o = oracle.solve_system(s, tol=0, max_sweeps=r.sweeps, stop="none")
    assert rel(r.a.cpu().numpy(), o.a) <= RTOL_F32
    assert_true_residual(s, r, 1e-6)
