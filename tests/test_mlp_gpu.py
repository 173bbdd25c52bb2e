"""The warm-start MLP's CUDA kernels (tcgen05 bfloat16 GEMMs, float32
accumulation) against the float64 CPU oracle (oracle/mlp_oracle.py), through
the C ABI.

The oracle evaluates the network at the bfloat16-rounded weights and features
the GPU multiplies with, and rounds to bfloat16 (unit roundoff u = 2^-8)
where the GPU stores in bfloat16: H1, H2 (forward) and dOut, dZ2, dZ1
(backward), so the ReLU masks -- decisions taken in floating point -- are
taken in the kernel's precision on both sides.  Every output and gradient
ELEMENT is then held to u·(|ref| + rms(ref)); per tensor, the GPU is also within
1e-2 of the plain float64 network.
"""
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


U_BF16 = 2.0 ** -8   # unit roundoff of bfloat16 (8 significant bits), round to nearest


def store_bf16(x):
    """The GPU's storage rounding of activations and gradients (nearest bfloat16)."""
    return bf16(np.asarray(x, dtype=np.float32))


def assert_within(got, ref, name):
    """Element by element: |got - ref| <= u·(|ref| + rms(ref)), one bfloat16 unit
    of the element plus one of the tensor's scale.  ref takes the ReLU decisions
    and the storage roundings in the kernel's precision, so what is left is the
    order of float32 accumulation (which, carried through a later rounding, can
    move an element by one bfloat16 unit of the scale: < 0.5 u measured in a
    float32-accumulating emulation over eight random networks)."""
    got = np.asarray(got, np.float64)
    rms = float(np.sqrt(np.mean(ref * ref))) if ref.size else 0.0
    lim = U_BF16 * (np.abs(ref) + rms) + 1e-30
    bad = np.abs(got - ref) > lim
    assert not bad.any(), (name, int(bad.sum()), float((np.abs(got - ref) / lim).max()))


def rbf_bound(s):
    """Coefficient tolerance of an ill-conditioned RBF system at equal sweeps: a
    float32 sweep is the exact sweep of a system perturbed by O(u32) relative,
    which moves the iterate by up to cond(X)·O(u32); max(1e-5, 8·cond(X)·2^-24)."""
    sv = np.linalg.svd(s.dense_f64(), compute_uv=False)
    return max(1e-5, 8 * (sv[0] / sv[-1]) * 2.0 ** -24)


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
    ref, _ = mo.forward(flat, phi, store=store_bf16)
    assert_within(out, ref, "out")
    # and against the plain float64 network: the storage roundings cost ~1e-3
    ref64, _ = mo.forward(flat, phi)
    assert rel(out, ref64) <= RTOL
    mlp.close()


def test_gradients_match_oracle(ctx):
    B = 640
    mlp = hp.MLP(ctx, max_batch=1024, seed=3)
    theta, m, n, target = problem(B, 7)
    loss, g = mlp.gradients(torch.from_numpy(theta).cuda(), m, n, torch.from_numpy(target).cuda())
    flat, phi = oracle_view(mlp.params(), theta, m, n)
    L, gref = mo.loss_and_grads(flat, theta, m, n, target, phi=phi, store=store_bf16)
    assert loss == pytest.approx(L, rel=1e-4)
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    for got, ref, name in zip(mo.unpack(g), mo.unpack(gref), names):
        assert_within(got, ref, name)
    # the plain float64 gradients are within the per-tensor 1e-2 of the storage roundings
    _, g64 = mo.loss_and_grads(flat, theta, m, n, target, phi=phi)
    for got, ref, name in zip(mo.unpack(g), mo.unpack(g64), names):
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
    g64 = g.astype(np.float64)
    ref = mo.Adam(p0.size, lr=lr).step(p0, g64)
    step, rstep = p1 - p0, ref - p0
    # element by element: the float32 update of a float32 master moves it by the
    # oracle's step up to the rounding of the step and of the new master
    tol = 1e-4 * lr + 2.0 ** -23 * np.abs(p0)
    bad = np.abs(step - rstep) > tol
    assert not bad.any(), (int(bad.sum()), float(np.abs(step - rstep).max()))
    # Adam's first step is -lr·g/(|g| + eps): its sign is -sign(g) wherever g is not ~0
    live = np.abs(g64) > 10 * 1e-8
    assert np.all(np.sign(step[live]) == -np.sign(g64[live]))


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
        assert rel(a[i].cpu().numpy(), o.a) <= rbf_bound(s)
    b.set_warm_start(None)  # cold again: the descriptors' own flags (False)
    b.run()
    s = synth.rbf_system(fam, int(m[0]), int(n[0]), th[0])
    o = oracle.solve_system(s, tol=0, max_sweeps=sweeps, stop="none")
    assert rel(a[0].cpu().numpy(), o.a) <= rbf_bound(s)
