"""CPU oracle of the warm-start MLP (float64 numpy).

TEST INFRASTRUCTURE ONLY: used by tests/ and bench.py's CPU legs, never by
the CUDA product path, and it imports nothing from it.

The network maps the features of a system of a parametric family,
    phi = [theta_1..theta_16, n / 256, log(m) / log(16384)],
to a predicted coefficient vector (256 outputs, the first n used):
    Z1 = phi W1^T + b1,  H1 = relu(Z1)
    Z2 = H1 W2^T + b2,   H2 = relu(Z2)
    Out = H2 W3^T + b3
Loss: L = (1 / C) sum_{b, j < n_b} (Out_bj - T_bj)^2 with C = sum_b n_b.
Gradients by the chain rule written out layer by layer; Adam as published
(Kingma and Ba, "Adam: A Method for Stochastic Optimization", ICLR 2015,
Algorithm 1: biased moments, bias correction, step lr * m_hat / (sqrt(v_hat) + eps)).

Parameter layout (flat): W1 [256][18], b1 [256], W2 [256][256], b2 [256],
W3 [256][256], b3 [256], row-major W[out][in].

store (optional, default none): a rounding applied where an implementation
stores an intermediate in a narrower format -- H1 and H2 in the forward pass,
dOut, dZ2 and dZ1 in the backward pass.  The ReLU masks [Z > 0] are decisions
taken in floating point; a check of such an implementation evaluates them, and
everything after them, in that implementation's precision by passing its
rounding here.  With store = None the arithmetic is plain float64.

Parity status: pinned in tests/test_mlp_oracle.py (central finite
differences, closed forms of degenerate networks, the output mask, Adam's
first step).
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT, N_THETA = 18, 256, 256, 16
SHAPES = [(N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (N_OUT, N_HID), (N_OUT,)]


def n_params() -> int:
    return int(sum(np.prod(s) for s in SHAPES))


def unpack(flat):
    out, off = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(np.asarray(flat[off: off + k], dtype=np.float64).reshape(s))
        off += k
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def features(theta, m, n) -> np.ndarray:
    """phi of each system, shape (B, 18)."""
    theta = np.asarray(theta, dtype=np.float64).reshape(-1, N_THETA)
    m = np.asarray(m, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    return np.concatenate([theta, (n / 256.0)[:, None], (np.log(np.maximum(m, 1.0)) / np.log(16384.0))[:, None]], axis=1)


def _keep(x):
    return x


def forward(flat, phi, store=None):
    st = store or _keep
    W1, b1, W2, b2, W3, b3 = unpack(flat)
    Z1 = phi @ W1.T + b1
    H1 = st(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2.T + b2
    H2 = st(np.maximum(Z2, 0.0))
    out = H2 @ W3.T + b3
    return out, (phi, Z1, H1, Z2, H2)


def output_mask(n, B) -> np.ndarray:
    n = np.asarray(n)
    return (np.arange(N_OUT)[None, :] < n[:, None]).astype(np.float64)


def loss(flat, theta, m, n, target) -> float:
    out, _ = forward(flat, features(theta, m, n))
    mask = output_mask(n, len(n))
    C = mask.sum()
    d = (out - np.asarray(target, dtype=np.float64)) * mask
    return float((d * d).sum() / C) if C > 0 else 0.0


def loss_and_grads(flat, theta, m, n, target, phi=None, store=None):
    """(L, dL/dparams as a flat float64 vector).  phi overrides the features
    (e.g. with the values a lower-precision implementation actually used);
    store: see the module docstring."""
    st = store or _keep
    W1, b1, W2, b2, W3, b3 = unpack(flat)
    if phi is None:
        phi = features(theta, m, n)
    out, (phi, Z1, H1, Z2, H2) = forward(flat, phi, store)
    mask = output_mask(n, len(n))
    C = mask.sum()
    d = (out - np.asarray(target, dtype=np.float64)) * mask
    L = float((d * d).sum() / C) if C > 0 else 0.0
    dOut = st(2.0 * d / C if C > 0 else np.zeros_like(d))
    gW3 = dOut.T @ H2
    gb3 = dOut.sum(axis=0)
    dH2 = dOut @ W3
    dZ2 = st(dH2 * (H2 > 0))
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ W2
    dZ1 = st(dH1 * (H1 > 0))
    gW1 = dZ1.T @ phi
    gb1 = dZ1.sum(axis=0)
    return L, pack([gW1, gb1, gW2, gb2, gW3, gb3])


class Adam:
    """Adam state for a flat parameter vector."""

    def __init__(self, size, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(size)
        self.v = np.zeros(size)
        self.t = 0
        self.lr, self.beta1, self.beta2, self.eps = lr, beta1, beta2, eps

    def step(self, params, grads):
        self.t += 1
        self.m = self.beta1 * self.m + (1.0 - self.beta1) * grads
        self.v = self.beta2 * self.v + (1.0 - self.beta2) * grads * grads
        m_hat = self.m / (1.0 - self.beta1 ** self.t)
        v_hat = self.v / (1.0 - self.beta2 ** self.t)
        return params - self.lr * m_hat / (np.sqrt(v_hat) + self.eps)
