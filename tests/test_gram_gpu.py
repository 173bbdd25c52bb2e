"""The Gram set-up G = X^T X (the denominators <X_j, X_j> of Eq. da2 and the
couplings <X_j, X_l> of Eq. ek1-ek inside a sweep) on the GPU, through the C
ABI, against float64 X^T X computed on the host.

Bound: each entry within 4e-6·sqrt(G_ii G_jj) (float32-grade: float32
accumulation of products that are exact for bfloat16 X and carry ~2^-21
relative error for float32 X split into two tf32 terms; binary16 products are
exact as well)."""
import numpy as np
import pytest

from paper_2104_12570_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_12570_gb300 as hp  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = hp.Context(0)
    yield c
    c.close()


def gpu_X(s):
    if s.dtype == "bf16":
        return torch.from_numpy(s.X.view(np.int16)).view(torch.bfloat16).cuda().T
    return torch.from_numpy(s.X).cuda().T  # float32 or float16


def check(G, s, tol=4e-6):
    Xd = s.dense_f64()
    G64 = Xd.T @ Xd
    d = np.sqrt(np.clip(np.diag(G64), 1e-300, None))
    err = np.abs(G.cpu().numpy().astype(np.float64) - G64) / np.outer(d, d)
    assert err.max() <= tol, err.max()
    np.testing.assert_array_equal(G.cpu().numpy(), G.cpu().numpy().T)  # symmetric


@pytest.mark.parametrize("m,n,dtype", [(64, 1, "f32"), (200, 50, "f32"), (1000, 37, "f32"),
                                       (5000, 256, "f32"), (4099, 129, "f32"),
                                       (777, 300, "bf16"), (3333, 100, "bf16"),
                                       (20000, 512, "bf16"), (130, 256, "bf16"),
                                       (777, 300, "f16"), (20000, 512, "f16"), (4099, 129, "f16")])
def test_gram_matches_float64(ctx, m, n, dtype):
    s = synth.make_system(m, n, seed=m + n, dtype=dtype)
    X = gpu_X(s)
    check(ctx.gram(X), s)
    check(ctx.gram(X, simt=True), s)


def test_gram_tensor_core_vs_cuda_core(ctx):
    s = synth.make_system(100_000, 256, seed=3)
    X = gpu_X(s)
    Gt = ctx.gram(X).cpu().numpy().astype(np.float64)
    Gs = ctx.gram(X, simt=True).cpu().numpy().astype(np.float64)
    d = np.sqrt(np.diag(Gs))
    assert (np.abs(Gt - Gs) / np.outer(d, d)).max() <= 2e-6


def test_solve_same_with_either_gram(ctx):
    s = synth.make_system(30_000, 200, seed=4, noise=0.01)
    X = gpu_X(s)
    y = torch.from_numpy(s.y).cuda()
    a = ctx.solve(X, y, tol=0, max_sweeps=5, stop="none").a.cpu().numpy()
    b = ctx.solve(X, y, tol=0, max_sweeps=5, stop="none", debug_flags=2).a.cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 2e-6


def test_gram_one_signed_columns(ctx):
    """Columns of one sign (uniform on [0, 1)).  The CUDA-core Gram is float32-
    grade here as on any data.  The tensor-core accumulator drops the low bits
    of every partial sum, so over one K slice of L accumulation steps an entry
    can lose up to L ulps of a partial sum bounded by sum_k |x_ki x_kj| <=
    sqrt(G_ii G_jj): error <= L·2^-23·sqrt(G_ii G_jj).  One slice covers
    ceil(m / SMs) rows (n <= 256 float32: one tile group per slice) and takes
    12 steps per 32 rows (4 tf32 K steps × hi·hi, hi·lo, lo·hi).  The diagonal
    is summed on the CUDA cores and stays float32-grade."""
    m, n = 200_000, 256
    g = np.random.default_rng(11)
    Xh = g.uniform(0.0, 1.0, (n, m)).astype(np.float32)
    X = torch.from_numpy(Xh).cuda().T
    Xd = Xh.astype(np.float64)
    G64 = Xd @ Xd.T
    nrm = np.sqrt(np.outer(np.diag(G64), np.diag(G64)))
    Gs = ctx.gram(X, simt=True).cpu().numpy().astype(np.float64)
    assert (np.abs(Gs - G64) / nrm).max() <= 4e-6
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    L = 12 * (-(-(-(-m // sms)) // 32))
    Gt = ctx.gram(X).cpu().numpy().astype(np.float64)
    err = np.abs(Gt - G64) / nrm
    assert err.max() <= L * 2.0 ** -23 + 4e-6, (err.max(), L)
    assert np.abs(np.diag(Gt) - np.diag(G64)).max() / np.diag(G64).min() <= 4e-6


def test_gram_float32_low_bits_reach_the_product(ctx):
    """The float32 split keeps x in place as its high part and relies on a tf32
    operand reading x with its low 13 mantissa bits dropped (hi = x & ~0x1fff);
    lo = x - hi carries those bits.  Elements whose low 13 bits are all ones
    are where dropping and rounding to nearest differ by a full tf32 ulp
    (2^-10 relative): had the operand rounded x instead, every product would
    be off by ~1e-3 and G with it.  Signs and the high bits vary, so the
    entries are sums of products of both signs."""
    m, n = 4096, 160
    g = np.random.default_rng(21)
    hi_bits = (g.integers(0x3f000000, 0x40800000, (n, m), dtype=np.int64) & ~0x1fff).astype(np.uint32)
    Xh = (hi_bits | np.uint32(0x1fff)).view(np.float32) * g.choice([-1.0, 1.0], (n, m)).astype(np.float32)
    Xd = Xh.astype(np.float64)
    G64 = Xd @ Xd.T
    nrm = np.sqrt(np.outer(np.diag(G64), np.diag(G64)))
    Gt = ctx.gram(torch.from_numpy(Xh).cuda().T).cpu().numpy().astype(np.float64)
    assert (np.abs(Gt - G64) / nrm).max() <= 4e-6
