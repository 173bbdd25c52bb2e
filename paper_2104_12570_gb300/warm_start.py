"""Train and evaluate the learned warm start for the RBF family of systems.

    python -m paper_2104_12570_gb300.warm_start --train 50000 --out weights.npy

1. Draw (m, n, theta) for the training systems (seed 1; the evaluation batch
   uses seed 0) and solve each with the batched sweep from a cold start under
   the family's stopping rule: the method makes its own labels.
2. Train the MLP phi(theta, m, n) -> a on (theta, m, n, a) with the library's
   GPU kernels (Adam, cosine learning-rate decay, masked mean-squared error).
3. Evaluate on the evaluation batch: sweeps to the stopping rule and the
   final residual, cold start against the MLP's warm start, each as one
   persistent graph-captured launch.

Everything runs through the C ABI (hpscd_batch_*, hpscd_mlp_*); torch only
holds device memory.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import paper_2104_12570_gb300 as hp
    from paper_2104_12570_gb300 import synth
else:
    from . import synth
    import paper_2104_12570_gb300 as hp

# The family's stopping rule: the relative change of ||e|| per sweep falls
# below 1e-6 (the systems are inconsistent, so the residual itself levels off
# well above 1e-6), with at most 10^4 sweeps.
TOL, STOP, MAX_SWEEPS = 1e-6, "rel_change", 10_000
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "rbf_warm_start.npy")


def build_batch(ctx, fam, m, n, th, device="cuda", tol=TOL, stop=STOP, max_sweeps=MAX_SWEEPS,
                cluster=0):
    """(keep, a list, Batch) for the systems (m, n, th) of the family; cluster is
    the CTAs per system or a (cluster, panel) pair from autotune_batch."""
    import torch
    keep, sysd = synth.device_rbf_batch(fam, m, n, th, device)
    a = [torch.zeros(int(k), dtype=torch.float32, device=device) for k in n]
    k, panel = cluster if isinstance(cluster, tuple) else (cluster, 0)
    b = hp.Batch(ctx, [(X, y, ai, False) for (X, y), ai in zip(sysd, a)], tol=tol,
                 max_sweeps=max_sweeps, stop=stop, cluster=k, panel=panel)
    return (keep, sysd), a, b


def solve_family(ctx, fam, m, n, th, chunk=4096, mlp=None, **kw):
    """Solutions as a zero-padded (count, 256) float32 array, plus the sweeps
    and final residuals: from a cold start, or from mlp's prediction when given
    (the solve then continues from where the network puts each system)."""
    import torch
    count = len(m)
    labels = np.zeros((count, 256), dtype=np.float32)
    sweeps = np.zeros(count, dtype=np.int64)
    res = np.zeros(count)
    for c0 in range(0, count, chunk):
        c1 = min(count, c0 + chunk)
        keep, a, b = build_batch(ctx, fam, m[c0:c1], n[c0:c1], th[c0:c1], **kw)
        if mlp is not None:
            theta = torch.from_numpy(np.ascontiguousarray(th[c0:c1], dtype=np.float32)).cuda()
            b.set_warm_start(mlp, theta)
        r = b.run()
        for i, ai in enumerate(a):
            labels[c0 + i, : ai.numel()] = ai.cpu().numpy()
        sweeps[c0:c1] = r["sweeps"]
        res[c0:c1] = r["rel_res"]
        b.close()
        del keep, a
    return labels, sweeps, res


def train(ctx, theta, m, n, labels, *, epochs=400, batch=512, lr=1e-3, lr_min=1e-5, seed=0,
          val_frac=0.1, log=None):
    """Train a fresh MLP; returns (MLP, history)."""
    import torch
    count = len(m)
    g = np.random.default_rng(seed)
    perm = g.permutation(count)
    nval = int(count * val_frac)
    val, tr = perm[:nval], perm[nval:]
    dev = torch.device("cuda", ctx.device)
    th_d = torch.from_numpy(np.ascontiguousarray(theta, dtype=np.float32)).to(dev)
    lab_d = torch.from_numpy(np.ascontiguousarray(labels, dtype=np.float32)).to(dev)
    mlp = hp.MLP(ctx, max_batch=max(batch, 4096), seed=seed)
    steps_per_epoch = max(1, len(tr) // batch)
    total = epochs * steps_per_epoch
    hist = []
    step = 0
    for ep in range(epochs):
        order = tr[g.permutation(len(tr))]
        tl = 0.0
        for k in range(steps_per_epoch):
            idx = np.sort(order[k * batch:(k + 1) * batch])
            it = torch.from_numpy(idx).to(dev)
            cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * step / total))
            tl += mlp.train_step(th_d[it].contiguous(), m[idx], n[idx], lab_d[it].contiguous(), lr=cur)
            step += 1
        if ep == epochs - 1 or ep % 10 == 0:
            vl = val_loss(mlp, th_d, lab_d, m, n, val) if nval else float("nan")
            hist.append({"epoch": ep, "train_loss": tl / steps_per_epoch, "val_loss": vl})
            if log:
                log(hist[-1])
    return mlp, hist


def val_loss(mlp, th_d, lab_d, m, n, idx, chunk=4096):
    import torch
    tot, cnt = 0.0, 0.0
    for c0 in range(0, len(idx), chunk):
        sub = np.sort(idx[c0:c0 + chunk])
        it = torch.from_numpy(sub).to(th_d.device)
        pred = mlp.predict(th_d[it].contiguous(), m[sub], n[sub]).cpu().numpy()
        lab = lab_d[it].cpu().numpy()
        mask = np.arange(256)[None, :] < n[sub][:, None]
        tot += float((((pred - lab) ** 2) * mask).sum())
        cnt += float(mask.sum())
    return tot / max(cnt, 1.0)


def evaluate(ctx, fam, mlp, m, n, th, reps=1, cluster=0, max_sweeps=MAX_SWEEPS):
    """Cold start against warm start on one batch: time (CUDA events around the
    graph launch), sweeps and final residuals.  GBps counts the method's bytes
    (per system: the set-up's read of X and y, then X once per sweep; the
    residual stays in shared memory).  The sweep ratios are also reported on
    the systems that reach the stopping rule in BOTH arms (their counts are not
    clipped by the cap), with their distribution."""
    import torch
    keep, a, b = build_batch(ctx, fam, m, n, th, cluster=cluster, max_sweeps=max_sweeps)
    theta = torch.from_numpy(np.ascontiguousarray(th, dtype=np.float32)).cuda()
    mn = (m * n).astype(np.float64)
    out = {"max_sweeps": int(max_sweeps), "systems": int(len(m))}
    raw = {}
    for name in ("cold", "warm"):
        if name == "warm":
            b.set_warm_start(mlp, theta)
        else:
            b.set_warm_start(None)
        times = []
        for _ in range(reps):
            r = b.run()
            times.append(r["timing"]["sweep_ms"])
        ms = float(np.median(times))
        sw = r["sweeps"]
        nbytes = float((4.0 * mn * (sw + 1) + 4.0 * m).sum())
        out[name] = {"ms": ms, "systems_per_s": len(m) / (ms * 1e-3),
                     "sweeps_mean": float(sw.mean()), "sweeps_median": float(np.median(sw)),
                     "sweeps_p90": float(np.percentile(sw, 90)),
                     "hit_cap": int((sw >= max_sweeps).sum()),
                     "hit_cap_frac": float((sw >= max_sweeps).mean()),
                     "sweeps_per_s": float(sw.sum()) / (ms * 1e-3),
                     "elem_sweeps": float((mn * sw).sum()),
                     "GBps": nbytes / (ms * 1e-3) / 1e9,
                     "rel_res_median": float(np.median(r["rel_res"]))}
        raw[name] = (sw.astype(np.float64), np.asarray(r["rel_res"], np.float64),
                     np.array([st == "ok" for st in r["status"]]))
    ratio = raw["warm"][1] / np.maximum(raw["cold"][1], 1e-300)
    out["warm_over_cold_final_residual_median"] = float(np.median(ratio))
    out["warm_over_cold_final_residual_p90"] = float(np.percentile(ratio, 90))
    out["speedup_time"] = out["cold"]["ms"] / out["warm"]["ms"]
    out["speedup_sweeps"] = out["cold"]["sweeps_mean"] / max(out["warm"]["sweeps_mean"], 1e-9)
    both = raw["cold"][2] & raw["warm"][2] & (raw["cold"][0] < max_sweeps) & (raw["warm"][0] < max_sweeps)
    sc, sw_ = raw["cold"][0][both], raw["warm"][0][both]
    if both.any():
        r_ws = sw_ / np.maximum(sc, 1.0)
        out["converged_in_both"] = {
            "systems": int(both.sum()),
            "sweeps_cold_mean": float(sc.mean()), "sweeps_warm_mean": float(sw_.mean()),
            "speedup_sweeps": float(sc.sum() / max(sw_.sum(), 1.0)),
            "speedup_elem_sweeps": float((mn[both] * sc).sum() / max((mn[both] * sw_).sum(), 1.0)),
            "warm_over_cold_sweeps_p10_p50_p90": [float(np.percentile(r_ws, q)) for q in (10, 50, 90)],
            "warm_fewer_sweeps_frac": float(np.mean(sw_ < sc))}
    b.close()
    return out


def save(mlp, path=WEIGHTS, meta=None):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.save(path, mlp.params())
    if meta is not None:
        with open(os.path.splitext(path)[0] + ".json", "w") as f:
            json.dump(meta, f, indent=1)


def load(ctx, path=WEIGHTS, max_batch=4096):
    return hp.MLP(ctx, max_batch=max_batch, params=np.load(path))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=50_000, help="training systems (seed 1)")
    ap.add_argument("--eval", type=int, default=4096, help="evaluation systems (seed 0)")
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--labels", default="", help="cache file of the training labels (.npz)")
    ap.add_argument("--rounds", type=int, default=1,
                    help="self-training rounds: after each, the training systems are solved again "
                         "from the network's prediction (same rule and cap) and the network is "
                         "retrained on those further-converged solutions")
    ap.add_argument("--init", default="",
                    help="weights (.npy) to continue from: the first labels are solved from this "
                         "network's prediction instead of from a cold start")
    args = ap.parse_args()
    import torch
    ctx = hp.Context(0)
    fam = synth.rbf_family(0)
    m, n, th = synth.rbf_params(args.train, seed=1)
    rounds_log = []
    prev_meta = {}
    if args.init:
        jp = os.path.splitext(args.init)[0] + ".json"
        if os.path.exists(jp):
            with open(jp) as f:
                prev_meta = json.load(f)
        rounds_log = list(prev_meta.get("label_rounds", []))
    t0 = time.time()
    init = load(ctx, args.init) if args.init else None
    if args.labels and os.path.exists(args.labels):
        z = np.load(args.labels)
        labels, sw, res = z["labels"], z["sweeps"], z["res"]
    else:
        labels, sw, res = solve_family(ctx, fam, m, n, th, mlp=init)
        if args.labels:
            np.savez(args.labels, labels=labels, sweeps=sw, res=res)
    if init is not None:
        init.close()
    t1 = time.time()
    rounds_log.append({"round": len(rounds_log), "label_sweeps_mean": float(sw.mean()),
                       "label_hit_cap": int((sw >= MAX_SWEEPS).sum())})
    print(json.dumps({"labels_s": t1 - t0, **rounds_log[-1]}), flush=True)
    mlp, hist = train(ctx, th, m, n, labels, epochs=args.epochs, batch=args.batch, lr=args.lr,
                      log=lambda h: print(json.dumps(h), flush=True))
    for _ in range(1, args.rounds):
        labels, sw, res = solve_family(ctx, fam, m, n, th, mlp=mlp)
        rounds_log.append({"round": len(rounds_log), "label_sweeps_mean": float(sw.mean()),
                           "label_hit_cap": int((sw >= MAX_SWEEPS).sum())})
        print(json.dumps(rounds_log[-1]), flush=True)
        mlp.close()
        mlp, hist = train(ctx, th, m, n, labels, epochs=args.epochs, batch=args.batch, lr=args.lr,
                          log=lambda h: print(json.dumps(h), flush=True))
    t2 = time.time()
    me, ne, te = synth.rbf_params(args.eval, seed=0)
    ev = evaluate(ctx, fam, mlp, me, ne, te)
    made_by = f"python -m paper_2104_12570_gb300.warm_start --rounds {args.rounds}" + \
              (f" --init {os.path.basename(args.init)}" if args.init else "") + " (GB300)"
    meta = {
        "what": "warm-start MLP phi(theta, m, n) -> a for the RBF family (synth.rbf_family(0)); "
                "float32 parameters in the order W1 [256][18], b1, W2 [256][256], b2, W3 [256][256], b3",
        "trained_on": f"{args.train:,} systems synth.rbf_params({args.train}, seed=1); labels = the "
                      f"batched sweep's solutions ({STOP} < {TOL}, at most {MAX_SWEEPS} sweeps): round 0 "
                      "from a cold start, each later round from the previous round's network "
                      "(self-training: the same rule and cap, continued from the prediction)",
        "training": {"rounds_total": len(rounds_log), "epochs": args.epochs, "batch": args.batch,
                     "lr": args.lr, "schedule": "cosine to 1e-5", "optimizer": "Adam(0.9, 0.999, 1e-8)",
                     "final": hist[-1], "labels_s_this_run_first": t1 - t0, "train_s_this_run": t2 - t1},
        "label_rounds": rounds_log,
        "made_by": (prev_meta.get("made_by", "") + ", then " if prev_meta else "") + made_by,
        f"eval_{args.eval}_seed0": ev,
    }
    save(mlp, args.out, meta)
    print(json.dumps(meta), flush=True)
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()
