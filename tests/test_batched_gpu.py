"""Parity of the batched CUDA sweep (many uneven column-major float32 systems,
one persistent graph-captured launch) with the float64 CPU oracle of
Algorithm 1, system by system, through the C ABI.

Tolerances: relative coefficient error <= 1e-5 against the oracle at the same
sweep count for well-conditioned (iid Gaussian) systems, as for the single
solve.  The RBF family is ill-conditioned (cond(X) up to ~3e4): a float32
sweep is the exact sweep of a system perturbed by O(u) relative (u = 2^-24),
and that perturbation moves the iterate by up to cond(X)·O(u) relative, so each
RBF system is held to max(1e-5, 8·cond(X)·u) of its own
(test_rbf_family_equal_sweeps), with the residual history at rtol 1e-4.
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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def residual_floor(s, sweeps):
    """Absolute bound on |hist_gpu[s] - hist_oracle[s]| from float32 residual
    arithmetic.  A pass of the batched kernel applies its whole sweep to each
    row at once, e_i <- e_i - sum_j X_ij·da_j, summed in float32 to a depth of
    at most D = 33 (16 columns per lane, then 16 warps, then e_i), so it rounds
    row i by at most D·u·(|e_i| + sum_j |X_ij|·|da_j|), u = 2^-24; the next
    sweeps take their steps from the perturbed residual and do not lengthen
    that error.  So the bound after sweep s sums, over the sweeps so far,
    D·u·|| |e_{s-1}| + |X|·|da_s| || / ||y||, with Algorithm 1's iterates in
    float64."""
    u, D = 2.0 ** -24, 33
    X = s.dense_f64()
    y = s.y.astype(np.float64)
    e = y.copy()
    a = np.zeros(s.n)
    d = (X * X).sum(axis=0)
    ny = np.linalg.norm(y) or 1.0
    aX = np.abs(X)
    acc, out = 0.0, [0.0]
    for _ in range(sweeps):
        e0, a0 = np.abs(e), a.copy()
        for j in range(s.n):
            if d[j] > 0:
                da = X[:, j] @ e / d[j]
                e -= X[:, j] * da
                a[j] += da
        acc += D * u * np.linalg.norm(e0 + aX @ np.abs(a - a0)) / ny
        out.append(acc)
    return np.array(out)


# (m, n, extra leading dimension, offset in floats of the first element)
SPECS = [(200, 50, 0, 0), (1, 1, 0, 0), (3, 1, 0, 0), (5, 256, 3, 0), (777, 130, 0, 0),
         (2049, 64, 0, 1), (4099, 255, 5, 0), (100, 8, 0, 0), (9000, 256, 0, 0), (300, 33, 1, 3),
         (128, 32, 0, 0), (129, 31, 0, 0), (16384, 97, 0, 0), (40, 200, 0, 0), (1000, 1, 0, 2),
         (640, 128, 4, 0)]


def gaussian_batch(specs, seed=0, noise=0.05):
    """Host systems and their device copies (with the requested ld and offset)."""
    host, dev, keep = [], [], []
    for i, (m, n, extra, off) in enumerate(specs):
        s = synth.make_system(m, n, seed=seed + 17 * i, noise=noise)
        ld = max(1, m + extra)
        buf = torch.zeros(off + n * ld + 4, dtype=torch.float32, device="cuda")
        if n and m:
            blk = buf[off: off + n * ld].view(n, ld)
            blk[:, :m].copy_(torch.from_numpy(s.X))
            X = blk[:, :m].T
        else:
            X = buf[off: off + max(n * ld, 1)].view(max(n, 1), ld)[:n, :m].T
        y = torch.from_numpy(s.y).cuda()
        a = torch.zeros(n, dtype=torch.float32, device="cuda")
        host.append(s)
        dev.append([X, y, a, False])
        keep.append(buf)
    return host, dev, keep


@pytest.mark.parametrize("cluster,panel", [(1, 0), (2, 0), (4, 0), (8, 0), (1, 1), (1, 2), (4, 2)])
def test_equal_sweeps_match_oracle(ctx, cluster, panel):
    host, dev, keep = gaussian_batch(SPECS, seed=cluster + 10 * panel)
    sweeps = 4
    hists = [torch.full((sweeps + 1,), float("nan"), dtype=torch.float64, device="cuda")
             for _ in dev]
    systems = [tuple(d) + (h,) for d, h in zip(dev, hists)]
    b = hp.Batch(ctx, systems, tol=0, max_sweeps=sweeps, stop="none", cluster=cluster, panel=panel)
    assert b.cluster == cluster and b.panel == panel
    r = b.run()
    for i, s in enumerate(host):
        o = oracle.solve_system(s, tol=0, max_sweeps=sweeps, stop="none")
        assert r["status"][i] == "ok" and r["sweeps"][i] == sweeps
        a = dev[i][2].cpu().numpy()
        assert rel(a, o.a) <= RTOL_F32, (SPECS[i], rel(a, o.a))
        # float32 residual arithmetic: the history carries at most the rounding floor
        # above (it matters for consistent systems whose residual cancels to zero)
        h = hists[i].cpu().numpy()
        assert np.all(np.abs(h - o.hist) <= 1e-5 * o.hist + residual_floor(s, sweeps)), SPECS[i]
        assert r["rel_res"][i] == pytest.approx(o.hist[-1], rel=1e-5, abs=1e-6)
    b.close()


def test_graph_replay_is_deterministic(ctx):
    host, dev, keep = gaussian_batch(SPECS[:8], seed=5)
    b = hp.Batch(ctx, [tuple(d) for d in dev], tol=0, max_sweeps=6, stop="none", cluster=2)
    b.run()
    a1 = [d[2].clone() for d in dev]
    for d in dev:
        d[2].fill_(123.0)  # cold start: the guess is ignored
    b.run()
    for x, d in zip(a1, dev):
        assert torch.equal(x, d[2])
    b.close()


@pytest.mark.parametrize("stop,tol", [("rel_res", 1e-4), ("rel_res", 1e-6), ("rel_change", 1e-6)])
def test_stopping_rules(ctx, stop, tol):
    # tall Gaussian systems (well conditioned: Gauss-Seidel converges in tens of sweeps)
    specs = [(500, 20, 0, 0), (3000, 100, 0, 0), (256, 64, 0, 0), (1200, 250, 0, 0)]
    host, dev, keep = gaussian_batch(specs, seed=11, noise=0.0 if stop == "rel_res" else 0.05)
    b = hp.Batch(ctx, [tuple(d) for d in dev], tol=tol, max_sweeps=500, stop=stop)
    r = b.run()
    for i, s in enumerate(host):
        o = oracle.solve_system(s, tol=tol, max_sweeps=500, stop=stop)
        assert o.status == "ok" and r["status"][i] == "ok", (specs[i], o.status, r["status"][i])
        # the GPU stops where the oracle's history meets the rule (or one sweep
        # off where the test is borderline at float32 precision)
        assert abs(int(r["sweeps"][i]) - o.sweeps) <= 1, (specs[i], r["sweeps"][i], o.sweeps)
        oo = oracle.solve_system(s, tol=0, max_sweeps=int(r["sweeps"][i]), stop="none")
        assert rel(dev[i][2].cpu().numpy(), oo.a) <= 1e-4
        if stop == "rel_res":
            # the stop is confirmed on y - X·a of the returned float32 a (Dot2):
            # the oracle's float64 residual of it meets tol and is the one reported
            _, nrm = oracle.residual(s.X, s.y, dev[i][2].cpu().numpy(), m=s.m, n=s.n)
            true = nrm / np.linalg.norm(s.y.astype(np.float64))
            assert true <= tol and r["rel_res"][i] == pytest.approx(true, rel=1e-6)
    b.close()


def test_warm_start_matches_oracle(ctx):
    host, dev, keep = gaussian_batch(SPECS[:10], seed=21)
    a0s = []
    for s, d in zip(host, dev):
        g = np.random.default_rng(s.m + s.n)
        a0 = (s.a_true + 0.1 * g.standard_normal(s.n)).astype(np.float32)
        d[2].copy_(torch.from_numpy(a0))
        d[3] = True
        a0s.append(a0)
    b = hp.Batch(ctx, [tuple(d) for d in dev], tol=0, max_sweeps=3, stop="none")
    r = b.run()
    for i, s in enumerate(host):
        o = oracle.solve_system(s, tol=0, max_sweeps=3, stop="none", a0=a0s[i])
        assert rel(dev[i][2].cpu().numpy(), o.a) <= RTOL_F32
        assert r["rel_res"][i] == pytest.approx(o.hist[-1], rel=1e-5)
    b.close()


def test_zero_column_and_empty_systems(ctx):
    host, dev, keep = gaussian_batch([(300, 40, 0, 0), (50, 3, 0, 0)], seed=3)
    X0 = dev[0][0]
    X0[:, 7] = 0.0
    host[0].X[7, :] = 0.0
    host[0].y = (host[0].dense_f64() @ host[0].a_true).astype(np.float32)
    dev[0][1].copy_(torch.from_numpy(host[0].y))
    e_m0 = (torch.empty(0, 5, device="cuda").T.contiguous().T, torch.empty(0, device="cuda"),
            torch.zeros(5, device="cuda"), False)
    e_n0 = (torch.empty(0, 7, device="cuda").T, torch.ones(7, device="cuda"),
            torch.empty(0, device="cuda"), False)
    b = hp.Batch(ctx, [tuple(dev[0]), e_m0, e_n0, tuple(dev[1])], tol=0, max_sweeps=5, stop="none")
    r = b.run()
    o = oracle.solve_system(host[0], tol=0, max_sweeps=5, stop="none")
    assert rel(dev[0][2].cpu().numpy(), o.a) <= RTOL_F32
    assert dev[0][2][7].item() == 0.0
    assert r["status"] == ["ok"] * 4
    assert r["rel_res"][1] == 0.0 and torch.count_nonzero(e_m0[2]).item() == 0
    assert r["rel_res"][2] == pytest.approx(1.0)  # n = 0: e = y for ever
    o1 = oracle.solve_system(host[1], tol=0, max_sweeps=5, stop="none")
    assert rel(dev[1][2].cpu().numpy(), o1.a) <= RTOL_F32
    b.close()


def test_invalid_batches_are_rejected(ctx):
    X = torch.zeros(10, 257, device="cuda").T.contiguous().T
    y = torch.zeros(10, device="cuda")
    with pytest.raises(hp.HpscdError) as ei:
        hp.Batch(ctx, [(X, y, torch.zeros(257, device="cuda"), False)], max_sweeps=2)
    assert ei.value.status == "unsupported"
    with pytest.raises(hp.HpscdError) as ei:
        hp.Batch(ctx, [(X[:, :10], y, torch.zeros(10, device="cuda"), False)], cluster=3)
    assert ei.value.status == "invalid_arg"
    b = hp.Batch(ctx, [], max_sweeps=2)  # an empty batch is a no-op
    assert b.run()["status"] == []
    b.close()


def test_rbf_family_equal_sweeps(ctx):
    """The batched family's systems (ill-conditioned RBF features) at equal sweeps."""
    fam = synth.rbf_family(0)
    m, n, th = synth.rbf_params(24, seed=7)
    keep, sysd = synth.device_rbf_batch(fam, m, n, th, "cuda")
    sweeps = 12
    a = [torch.zeros(int(k), device="cuda") for k in n]
    hist = [torch.zeros(sweeps + 1, dtype=torch.float64, device="cuda") for _ in n]
    b = hp.Batch(ctx, [(X, y, ai, False, h) for (X, y), ai, h in zip(sysd, a, hist)],
                 tol=0, max_sweeps=sweeps, stop="none")
    b.run()
    u = 2.0 ** -24
    for i in range(len(m)):
        s = synth.rbf_system(fam, int(m[i]), int(n[i]), th[i])
        o = oracle.solve_system(s, tol=0, max_sweeps=sweeps, stop="none")
        np.testing.assert_allclose(hist[i].cpu().numpy(), o.hist, rtol=1e-4)
        sv = np.linalg.svd(s.dense_f64(), compute_uv=False)
        kappa = sv[0] / sv[-1]
        err = rel(a[i].cpu().numpy(), o.a)
        assert err <= max(RTOL_F32, 8 * kappa * u), (m[i], n[i], kappa, err)
    b.close()


def test_autotuner_picks_cluster_and_panel(ctx):
    fam = synth.rbf_family(0)
    m, n, th = synth.rbf_params(300, seed=9)
    keep, sysd = synth.device_rbf_batch(fam, m, n, th, "cuda")
    systems = [(X, y, torch.zeros(int(k), device="cuda"), False) for (X, y), k in zip(sysd, n)]
    best, ms = hp.autotune_batch(ctx, systems, trial_sweeps=3)
    assert best[0] in (1, 2, 4, 8) and best[1] in (0, 1, 2) and best in ms
    assert ms[best] == min(ms.values()) and all(v >= 0 for v in ms.values())
    assert {p for (k, p) in ms if k == 1} == {0, 1, 2}  # every panel policy timed
