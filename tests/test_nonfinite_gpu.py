"""Non-finite inputs: a NaN in y or an infinite entry of X makes the residual
norm non-finite, and every path reports it (status "nonfinite", the oracle's
OR_NONFINITE) at the sweep where the oracle does, without a fault or a hang.
In a batch only the affected system reports it."""
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


def test_nan_in_y_tall_and_wide(ctx):
    for layout, (m, n) in (("col", (3000, 200)), ("row", (200, 3000))):
        s = synth.make_system(m, n, seed=31, layout=layout, noise=0.01)
        s.y[17] = np.nan
        X = torch.from_numpy(s.X).cuda()
        if layout == "col":
            X = X.T
        r = ctx.solve(X, torch.from_numpy(s.y).cuda(), tol=1e-6, max_sweeps=20)
        o = oracle.solve_system(s, tol=1e-6, max_sweeps=20)
        assert r.status == o.status == "nonfinite" and r.sweeps == o.sweeps == 0, layout


def test_infinite_column_tall(ctx):
    s = synth.make_system(2000, 100, seed=32, noise=0.01)
    s.X[3, 5] = np.inf  # column 3, row 5 (column-major storage)
    X = torch.from_numpy(s.X).cuda().T
    y = torch.from_numpy(s.y).cuda()
    o = oracle.solve_system(s, tol=1e-6, max_sweeps=20)
    assert o.status == "nonfinite"
    for simt in (0, 2):  # tensor-core and CUDA-core set-up
        r = ctx.solve(X, y, tol=1e-6, max_sweeps=20, debug_flags=simt)
        assert r.status == "nonfinite" and r.sweeps == o.sweeps


def test_nan_in_one_system_of_a_batch(ctx):
    systems, keep = [], []
    for k, (m, n) in enumerate(((900, 60), (1500, 100), (700, 33))):
        s = synth.make_system(m, n, seed=40 + k, noise=0.01)
        if k == 1:
            s.y[3] = np.nan
        X = torch.from_numpy(s.X).cuda().T
        y = torch.from_numpy(s.y).cuda()
        a = torch.zeros(n, device="cuda")
        keep.append(s)
        systems.append((X, y, a, False))
    b = hp.Batch(ctx, systems, tol=0, max_sweeps=4, stop="none")
    r = b.run()
    assert r["status"] == ["ok", "nonfinite", "ok"]
    for k in (0, 2):
        o = oracle.solve_system(keep[k], tol=0, max_sweeps=4, stop="none")
        a = systems[k][2].cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - o.a) / np.linalg.norm(o.a) <= 1e-5
    b.close()


def test_nan_in_an_asynchronous_solve(ctx):
    s = synth.make_system(4000, 128, seed=50, noise=0.01)
    X = torch.from_numpy(s.X).cuda().T
    y = torch.from_numpy(s.y).cuda()
    ybad = y.clone()
    ybad[100] = float("nan")
    res = hp.results_buffer(3)
    ctx.solve_async(X, y, res[0], tol=1e-7, max_sweeps=50, stop="rel_change")
    ctx.solve_async(X, ybad, res[1], tol=1e-7, max_sweeps=50, stop="rel_change")
    ctx.solve_async(X, y, res[2], tol=1e-7, max_sweeps=50, stop="rel_change")
    got = hp.read_results(res)
    assert got["status"] == ["ok", "nonfinite", "ok"]
    assert got["sweeps"][0] == got["sweeps"][2] and got["sweeps"][1] == 0
