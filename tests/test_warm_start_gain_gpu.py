"""What the trained warm-start network gains over the cold-start sweep.

The shipped weights (paper_2104_12570_gb300/weights/rbf_warm_start.npy) were
trained on 50,000 solutions the batched sweep produced for the RBF family
(seed 1).  On held-out systems of the family (seed 0) the warm start must
reach the stopping rule in fewer sweeps than the cold start, with a final
residual that is no worse, and its first residual must be far below the cold
start's (which is ||y|| / ||y|| = 1)."""
import os

import numpy as np
import pytest

from paper_2104_12570_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_12570_gb300 as hp  # noqa: E402
from paper_2104_12570_gb300 import warm_start as ws  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = hp.Context(0)
    yield c
    c.close()


def test_trained_warm_start_saves_sweeps(ctx):
    assert os.path.exists(ws.WEIGHTS), "trained weights missing"
    fam = synth.rbf_family(0)
    m, n, th = synth.rbf_params(300, seed=0)
    keep, sysd = synth.device_rbf_batch(fam, m, n, th, "cuda")
    cap = 3000
    a = [torch.zeros(int(k), device="cuda") for k in n]
    hist = [torch.zeros(cap + 1, dtype=torch.float64, device="cuda") for _ in n]
    b = hp.Batch(ctx, [(X, y, ai, False, h) for (X, y), ai, h in zip(sysd, a, hist)],
                 tol=ws.TOL, max_sweeps=cap, stop=ws.STOP)
    cold = b.run()
    h0_cold = np.array([h[0].item() for h in hist])
    mlp = ws.load(ctx, max_batch=512)
    b.set_warm_start(mlp, torch.from_numpy(th.astype(np.float32)).cuda())
    warm = b.run()
    h0_warm = np.array([h[0].item() for h in hist])
    b.close()
    assert np.allclose(h0_cold, 1.0)
    # the prediction alone already removes most of the residual a cold start begins with
    assert np.median(h0_warm) < 0.6
    assert warm["sweeps"].sum() < cold["sweeps"].sum()
    # ... and the solve ends no worse (median over systems of warm / cold final residual)
    assert np.median(warm["rel_res"] / cold["rel_res"]) <= 1.0 + 1e-6
    print(f"sweeps cold {cold['sweeps'].mean():.0f} warm {warm['sweeps'].mean():.0f}; "
          f"initial residual warm median {np.median(h0_warm):.3f}")
