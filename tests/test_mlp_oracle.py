"""Pins of the CPU oracle of the warm-start MLP (no GPU): gradients against
central finite differences, closed forms of degenerate networks, the output
mask, and Adam's first step."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo


def small_problem(seed=0, B=6):
    g = np.random.default_rng(seed)
    flat = g.normal(0.0, 0.05, mo.n_params())
    theta = g.standard_normal((B, 16))
    m = g.integers(256, 16385, B)
    n = g.integers(1, 257, B)
    target = g.standard_normal((B, 256))
    return flat, theta, m, n, target


def test_features_follow_the_definition():
    phi = mo.features(np.arange(32, dtype=float).reshape(2, 16), [16384, 256], [256, 8])
    assert phi.shape == (2, 18)
    np.testing.assert_array_equal(phi[:, :16], np.arange(32).reshape(2, 16))
    assert phi[0, 16] == 1.0 and phi[1, 16] == 8 / 256
    assert phi[0, 17] == pytest.approx(1.0) and phi[1, 17] == pytest.approx(8 / 14)


def test_gradients_match_central_differences():
    flat, theta, m, n, target = small_problem()
    L, g = mo.loss_and_grads(flat, theta, m, n, target)
    assert L == pytest.approx(mo.loss(flat, theta, m, n, target), rel=1e-14)
    rng = np.random.default_rng(1)
    sizes = np.cumsum([0] + [int(np.prod(s)) for s in mo.SHAPES])
    # every parameter tensor: random coordinates, plus every output bias
    idx = np.concatenate([rng.integers(sizes[i], sizes[i + 1], 40) for i in range(6)])
    idx = np.concatenate([idx, np.arange(sizes[5], sizes[6])])
    h = 1e-5
    for k in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[k] += h
        fm[k] -= h
        fd = (mo.loss(fp, theta, m, n, target) - mo.loss(fm, theta, m, n, target)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-10), k


def test_zero_network_closed_form():
    """With all weights zero the output is b3, so L = mean_valid (b3_j - T_bj)^2 and
    dL/db3_j = 2 sum_b [j < n_b] (b3_j - T_bj) / C; every other gradient is zero."""
    flat, theta, m, n, target = small_problem(2)
    W1, b1, W2, b2, W3, b3 = mo.unpack(np.zeros(mo.n_params()))
    b3 = np.linspace(-1, 1, 256)
    flat = mo.pack([W1, b1, W2, b2, W3, b3])
    L, g = mo.loss_and_grads(flat, theta, m, n, target)
    mask = np.arange(256)[None, :] < n[:, None]
    C = mask.sum()
    assert L == pytest.approx(float((((b3[None, :] - target) ** 2) * mask).sum() / C), rel=1e-14)
    gp = mo.unpack(g)
    np.testing.assert_allclose(gp[5], 2 * ((b3[None, :] - target) * mask).sum(axis=0) / C, rtol=1e-13)
    for t in gp[:5]:
        assert not np.any(t)


def test_linear_regime_matches_matrix_product():
    """Positive weights and inputs keep every ReLU open: the net is the product
    W3 W2 W1 applied to phi plus the propagated biases."""
    g = np.random.default_rng(3)
    W1, W2, W3 = g.uniform(0, 0.1, (256, 18)), g.uniform(0, 0.1, (256, 256)), g.uniform(-1, 1, (256, 256))
    b1, b2, b3 = g.uniform(0, 1, 256), g.uniform(0, 1, 256), g.uniform(-1, 1, 256)
    flat = mo.pack([W1, b1, W2, b2, W3, b3])
    theta = g.uniform(0, 1, (3, 16))
    phi = mo.features(theta, [300, 400, 500], [10, 20, 30])
    out, _ = mo.forward(flat, phi)
    expect = ((phi @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    np.testing.assert_allclose(out, expect, rtol=1e-13)


def test_masked_outputs_do_not_contribute():
    flat, theta, m, n, target = small_problem(4)
    L0, g0 = mo.loss_and_grads(flat, theta, m, n, target)
    t2 = target.copy()
    for b in range(len(n)):
        t2[b, n[b]:] += 100.0
    L1, g1 = mo.loss_and_grads(flat, theta, m, n, t2)
    assert L1 == L0
    np.testing.assert_array_equal(g0, g1)


def test_adam_first_step_is_lr_times_sign():
    """From zero moments m_hat = g and v_hat = g^2, so the step is lr * g / (|g| + eps)."""
    p = np.zeros(5)
    g = np.array([1e-3, -2.0, 5.0, -1e-4, 0.5])
    opt = mo.Adam(5, lr=0.01, eps=1e-8)
    p1 = opt.step(p, g)
    np.testing.assert_allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # second step with the same gradient: the bias-corrected moments are still g and g^2
    p2 = opt.step(p1, g)
    np.testing.assert_allclose(p2 - p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)
