"""The warm-start MLP's CUDA kernels (tcgen05 bfloat16 GEMMs, float32
accumulation) against the float64 CPU oracle (oracle/mlp_oracle.py), through
the C ABI.

The oracle evaluates the network at the bfloat16-rounded weights and features
the GPU multiplies with; the remaining difference is the GPU's rounding of
activations and gradients to bfloat16 between layers (2^-9 relative), so
outputs and gradients are compared at 1e-2 relative (Frobenius norm per
tensor)."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from paper_2104_12570_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_12570_gb300 as hp  # noqa: E402

RTOL = 1e-2


@pytest.fixture(scope="module")
def ctx():
    c = hp.Context(0)
    yield c
    c.close()


def bf16(x):
    return synth.bf16_bits_to_f32(synth.f32_to_bf16_bits(np.asarray(x, dtype=np.float32))).astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def problem(B, seed):
    g = np.random.default_rng(seed)
    theta = g.standard_normal((B, 16)).astype(np.float32)
    m = g.integers(256, 16385, B)
    n = g.integers(1, 257, B)
    n[0] = 256
    target = (0.5 * g.standard_normal((B, 256))).astype(np.float32)
    return theta, m, n, target


def oracle_view(params, theta, m, n):
    """(flat parameters with bf16 weights, bf16 features) as the GPU uses them."""
    W1, b1, W2, b2, W3, b3 = mo.unpack(params)
    flat = mo.pack([bf16(W1), b1, bf16(W2), b2, bf16(W3), b3])
    return flat, bf16(mo.features(theta, m, n))


@pytest.mark.parametrize("B", [1, 300, 1024])
def test_forward_matches_oracle(ctx, B):
    mlp = hp.MLP(ctx, max_batch=1024, seed=B)
    theta, m, n, _ = problem(B, B)
    out = mlp.predict(torch.from_numpy(theta).cuda(), m, n).cpu().numpy()
    flat, phi = oracle_view(mlp.params(), theta, m, n)
    ref, _ = mo.forward(flat, phi)
    assert rel(out, ref) <= RTOL
    mlp.close()


def test_gradients_match_oracle(ctx):
    B = 640
    mlp = hp.MLP(ctx, max_batch=1024, seed=3)
    theta, m, n, target = problem(B, 7)
    loss, g = mlp.gradients(torch.from_numpy(theta).cuda(), m, n, torch.from_numpy(target).cuda())
    flat, phi = oracle_view(mlp.params(), theta, m, n)
    L, gref = mo.loss_and_grads(flat, theta, m, n, target, phi=phi)
    assert loss == pytest.approx(L, rel=RTOL)
    for got, ref, name in zip(mo.unpack(g), mo.unpack(gref), ["W1", "b1", "W2", "b2", "W3", "b3"]):
        assert rel(got, ref) <= RTOL, name


def test_adam_step_matches_oracle(ctx):
    B = 256
    mlp = hp.MLP(ctx, max_batch=B, seed=5)
    p0 = mlp.params().astype(np.float64)
    theta, m, n, target = problem(B, 9)
    th, tg = torch.from_numpy(theta).cuda(), torch.from_numpy(target).cuda()
    _, g = mlp.gradients(th, m, n, tg)
    lr = 1e-3
    mlp.train_step(th, m, n, tg, lr=lr)
    p1 = mlp.params().astype(np.float64)
    ref = mo.Adam(p0.size, lr=lr).step(p0, g.astype(np.float64))
    d = np.abs((p1 - p0) - (ref - p0))
    # Adam's first step is lr * g / (|g| + eps) ~ lr * sign(g): equal wherever g is not ~0
    assert d.max() <= 2 * lr + 1e-6
    assert np.mean(d <= 1e-3 * lr + 1e-7) >= 0.999


def test_training_fits_a_fixed_batch(ctx):
    B = 512
    mlp = hp.MLP(ctx, max_batch=B, seed=11)
    theta, m, n, target = problem(B, 13)
    th, tg = torch.from_numpy(theta).cuda(), torch.from_numpy(target).cuda()
    first = mlp.train_step(th, m, n, tg, lr=2e-3)
    for _ in range(300):
        last = mlp.train_step(th, m, n, tg, lr=2e-3)
    assert last < 0.2 * first


def test_batch_warm_start_uses_the_prediction(ctx):
    fam = synth.rbf_family(0)
    m, n, th = synth.rbf_params(40, seed=3)
    keep, sysd = synth.device_rbf_batch(fam, m, n, th, "cuda")
    a = [torch.full((int(k),), 7.0, device="cuda") for k in n]
    theta = torch.from_numpy(th.astype(np.float32)).cuda()
    mlp = hp.MLP(ctx, max_batch=128, seed=1)  # smaller than the batch: chunked forward
    pred = mlp.predict(theta, m, n)
    b0 = hp.Batch(ctx, [(X, y, ai, False) for (X, y), ai in zip(sysd, a)], tol=0, max_sweeps=0,
                  stop="none")
    b0.set_warm_start(mlp, theta)
    b0.run()
    for i in range(len(m)):
        assert torch.equal(a[i], pred[i, : int(n[i])])  # zero sweeps: a = the prediction
    sweeps = 3
    b = hp.Batch(ctx, [(X, y, ai, False) for (X, y), ai in zip(sysd, a)], tol=0, max_sweeps=sweeps,
                 stop="none")
    b.set_warm_start(mlp, theta)
    b.run()
    import oracle
    for i in range(0, len(m), 7):
        s = synth.rbf_system(fam, int(m[i]), int(n[i]), th[i])
        o = oracle.solve_system(s, tol=0, max_sweeps=sweeps, stop="none",
                                a0=pred[i, : int(n[i])].cpu().numpy())
        assert rel(a[i].cpu().numpy(), o.a) <= 2e-3
    b.set_warm_start(None)  # cold again: the descriptors' own flags (False)
    b.run()
    s = synth.rbf_system(fam, int(m[0]), int(n[0]), th[0])
    o = oracle.solve_system(s, tol=0, max_sweeps=sweeps, stop="none")
    assert rel(a[0].cpu().numpy(), o.a) <= 2e-3
