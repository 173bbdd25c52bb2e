"""Benchmark of the HPSCD column sweep (Algorithm 1) on GB300.

One step = one complete solve of the 1,000,000 x 256 float32 column-major
noisy least-squares system (X iid N(0,1), a_true iid U(-1,1), noise 0.01):
Gram/denominator set-up, then sweeps until the relative change of the
residual norm falls below 1e-7, inputs already resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  value = algorithmic HBM bytes of a solve / time per
solve (GB/s; X is 1.02 GB, larger than L2, so no flush is needed between
steps).  Algorithmic bytes (the method's, not the implementation's): each
sweep reads X once (elem·m·n) and, while the residual e lives in HBM, reads
and writes it (8m); the set-up reads X and y once.  Passes a kernel makes
beyond that (a true-residual confirmation) are not counted.  Under torchrun
every rank solves its own system (independent replicas, weak scaling); rank 0
prints.  The other workloads (wide, square, bfloat16 precision mode, batched
+ learned warm start) follow in the same line, each with its CPU oracle
baseline (all host cores and one core) and the float64 oracle's check of the
GPU result.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "tall_1Mx256_f32"
TOL, STOP, MAX_SWEEPS = 1e-7, "rel_change", 100
METRIC = "time & HBM GB/s to rel. residual 1e-6; learned/BF16 vs plain FP32 on 1 GB300"
FALLBACK_HBM_GBS = 6800.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def sweep_bytes(m, n, esz, sweeps, e_in_hbm=True):
    """Algorithmic bytes of `sweeps` sweeps: X once per sweep, plus the read and
    write of e (8m) when e is not kept on chip."""
    return sweeps * (esz * m * n + (8 * m if e_in_hbm else 0))


def setup_bytes(m, n, esz):
    """The set-up's read of X (Gram matrix, X^T y) and of y."""
    return esz * m * n + 4 * m


def solve_bytes(m, n, esz, sweeps, e_in_hbm=True):
    return setup_bytes(m, n, esz) + sweep_bytes(m, n, esz, sweeps, e_in_hbm)


def cpu_info():
    """(logical cores, CPU model) of this host."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model and os.path.exists("/proc/cpuinfo"):
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    return os.cpu_count() or 1, model


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region.

    The sampler starts before the region and waits for its first reading, so
    that it is running when the region starts; each reading is stamped with the
    host clock, and the summary keeps the readings taken inside the region
    (mark() bounds it), with 30 ms of slack for the sampling period."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0:
                time.sleep(0.005)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, start, end):
        self.window = (start - 0.03, end + 0.03)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if self.window:
            inside = [x for x in lines if self.window[0] <= x[0] <= self.window[1]]
            lines = inside or lines
        for _, ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "in_timed_region": lines is not self.lines}


def traffic_from_profile(src_sha):
    """Per-launch DRAM bytes of the sweep kernel from the committed ncu summary, if the
    kernel source has not changed since it was captured (else None)."""
    p = os.path.join(ROOT, "profiles", "tall_sweep_1Mx256_f32.md")
    if not os.path.exists(p):
        return None
    rec = {}
    for ln in open(p):
        if ln.startswith("<!--") and "bench:" in ln:
            for kv in ln.split("bench:")[1].replace("-->", "").split():
                k, _, v = kv.partition("=")
                rec[k] = v
    if rec.get("kernel_sha") != src_sha or "traffic_bytes_per_launch" not in rec:
        return None
    return float(rec["traffic_bytes_per_launch"])


def kernel_sha():
    h = hashlib.sha256()
    for f in ("tall_sweep.cu", "tall_sweep.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2104_12570_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(
        os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(ms, world, device):
    """The slowest rank's time per step (every rank gets it); ms itself at N = 1."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(bytes_per_rank, world, ms):
    """Whole-job GB/s: every rank solves its own system (replicas, weak scaling), so
    the job moves world × bytes_per_rank in the slowest rank's time."""
    return world * bytes_per_rank / (ms * 1e-3) / 1e9


def oracle_leg(s, stop, tol, max_sweeps, threads, sweeps_cap=None):
    """The CPU oracle's threaded Algorithm 1 (column order sequential, row loops
    over `threads` threads) on system s; sweeps_cap bounds the sweeps timed
    (the time is then extrapolated by the caller).  Returns (result, seconds,
    threads used)."""
    import oracle
    ms = max_sweeps if sweeps_cap is None else min(max_sweeps, sweeps_cap)
    t = time.perf_counter()
    r, used = oracle.solve_mt(s.X, s.y, m=s.m, n=s.n, layout=s.layout, dtype=s.dtype, tol=tol,
                              max_sweeps=ms, stop=stop if sweeps_cap is None else "none",
                              threads=threads)
    return r, time.perf_counter() - t, used


def cpu_baseline(s, esz, stop, tol, max_sweeps, e_in_hbm=True, one_core_sweeps=None, what=""):
    """The oracle timed on this host's cores: on min(nproc, m / 8192) threads to
    the stopping rule (every column step synchronises the threads, so on
    shorter columns more threads only add barrier time), and on one core (to
    the rule, or one_core_sweeps sweeps extrapolated to the threaded run's
    sweep count).  value: GB/s on the same algorithmic bytes as the GPU line."""
    nproc, model = cpu_info()
    threads = max(1, min(nproc, s.m // 8192))
    r_all, t_all, used = oracle_leg(s, stop, tol, max_sweeps, threads)
    nb = solve_bytes(s.m, s.n, esz, r_all.sweeps, e_in_hbm)
    out = {"value": nb / t_all / 1e9, "unit": "GB/s", "cores": used, "kind": "oracle",
           "ms_to_tol": t_all * 1e3, "sweeps": int(r_all.sweeps), "status": r_all.status,
           "nproc": nproc, "cpu_model": model,
           "threads_rule": "min(nproc, m // 8192): one barrier per column step"}
    if used == 1:
        out["one_core"] = {"value": out["value"], "ms_to_tol": out["ms_to_tol"],
                           "sweeps": int(r_all.sweeps), "timed": "the same run (1 thread)"}
        out["sample"] = f"full solve of {what} to {stop}<{tol} on 1 thread"
    elif one_core_sweeps is None:
        r1, t1, _ = oracle_leg(s, stop, tol, max_sweeps, 1)
        out["one_core"] = {"value": nb / t1 / 1e9, "ms_to_tol": t1 * 1e3, "sweeps": int(r1.sweeps),
                           "timed": "full solve"}
        out["sample"] = f"full solve of {what} to {stop}<{tol} on {used} threads and on 1"
    else:
        k = max(1, min(one_core_sweeps, max(1, r_all.sweeps)))
        _, t1, _ = oracle_leg(s, stop, tol, max_sweeps, 1, sweeps_cap=k)
        per_sweep = t1 / k  # the set-up (d, e) is inside; a slight overestimate per sweep
        t1x = per_sweep * max(1, r_all.sweeps)
        out["one_core"] = {"value": nb / t1x / 1e9, "ms_to_tol": t1x * 1e3,
                           "timed": f"{k} sweep(s), extrapolated to {r_all.sweeps}"}
        out["sample"] = (f"{what}: full solve on {used} threads; on 1 thread {k} sweep(s) timed "
                         f"and extrapolated to the threaded run's {r_all.sweeps} sweeps")
    return out, r_all


def oracle_check(s, a_gpu, gpu_sweeps, gpu_rel_res, r_oracle=None):
    """The float64 oracle's view of a GPU result: the residual y - X·a of the
    returned coefficients, and the coefficient error against the oracle's
    iterate when both made the same number of sweeps."""
    import oracle
    a = np.asarray(a_gpu, dtype=np.float64)
    _, nrm = oracle.residual(s.X, s.y, a, m=s.m, n=s.n, layout=s.layout, dtype=s.dtype)
    ny = float(np.linalg.norm(s.y.astype(np.float64)))
    out = {"true_rel_res": nrm / ny if ny > 0 else nrm, "gpu_reported_rel_res": float(gpu_rel_res),
           "gpu_sweeps": int(gpu_sweeps)}
    if r_oracle is not None:
        out["oracle_sweeps"] = int(r_oracle.sweeps)
        out["oracle_rel_res"] = float(r_oracle.rel_res)
        if int(r_oracle.sweeps) == int(gpu_sweeps):
            out["coef_rel_err_equal_sweeps"] = float(np.linalg.norm(a - r_oracle.a) /
                                                     max(np.linalg.norm(r_oracle.a), 1e-300))
    return out


def roofline_block(bytes_, ms, peak, peak_kind, kernel, traffic=None):
    ach = bytes_ / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": peak_kind, "kernel": kernel, "traffic": traffic, "kernel_ms": ms,
            "algorithmic_bytes": bytes_}


def run_reference(args, rank, world):
    """The reference arm: the oracle (float64 CPU Algorithm 1, its row loops on
    every host core) on the benchmark workload, one full solve per step."""
    if rank != 0:
        return
    import oracle  # noqa: F401
    from paper_2104_12570_gb300 import synth
    s = synth.workload(WORKLOAD, seed=0)
    nproc, model = cpu_info()
    times, res, used = [], None, 1
    for i in range(args.warmup + args.steps):
        res, dt, used = oracle_leg(s, STOP, TOL, MAX_SWEEPS, nproc)
        if i >= args.warmup:
            times.append(dt)
    sec = sum(times) / len(times)
    val = solve_bytes(s.m, s.n, 4, res.sweeps) / sec / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "m": s.m, "n": s.n, "stop": f"{STOP}<{TOL}",
                      "sweeps": res.sweeps},
           "cpu_baseline": {"value": val, "unit": "GB/s", "cores": used, "kind": "oracle",
                            "nproc": nproc, "cpu_model": model,
                            "sample": f"full solve of {WORKLOAD} ({res.sweeps} sweeps) per step"},
           "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def precision_comparison(hp, synth, ctx, dev, peak, peak_kind, steps=5, warmup=3, cpu=True):
    """Time to relative residual 1e-6 on the 4,000,000 x 512 consistent system: X
    stored bfloat16 (float32 accumulation, true-residual refresh every 4 sweeps)
    and IEEE binary16 (the same values converted, exact but for the entries below
    2^-17 in magnitude, about 6 per million) against the same values stored
    float32 (plain float32 sweep).  The stop is confirmed on y - X·a of the
    returned float32 coefficients (a Dot2 pass)."""
    import torch
    s = synth.workload("tall_4Mx512_bf16", seed=0)
    Xb = torch.from_numpy(s.X.view(np.int16)).view(torch.bfloat16).to(dev).T
    y = torch.from_numpy(s.y).to(dev)
    out = {"workload": "tall_4Mx512 (X iid N(0,1) rounded to bfloat16, consistent)",
           "stop": "rel_res<=1e-6 (confirmed on the true residual)",
           "bytes": "set-up: elem·m·n + 4m; per sweep: elem·m·n + 8m (e in HBM)"}
    results = {}
    Xh = Xb.T.half().T
    for name, X, kw in (("bf16_refresh4", Xb, dict(refresh_every=4)),
                        ("f16_refresh4", Xh, dict(refresh_every=4)),
                        ("f32_plain", None, {})):
        if X is None:
            del Xh
            X = Xb.T.float().contiguous().T
            del Xb
        for _ in range(warmup):
            r = ctx.solve(X, y, tol=1e-6, max_sweeps=100, stop="rel_res", **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            r = ctx.solve(X, y, tol=1e-6, max_sweeps=100, stop="rel_res", **kw)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        esz = 4 if X.dtype == torch.float32 else 2
        sw = int(r.sweeps)
        out[name] = {"ms_to_tol": ms, "GBps": solve_bytes(s.m, s.n, esz, sw) / (ms * 1e-3) / 1e9,
                     "sweeps": sw, "passes": int(r.timing["passes"]), "rel_res": float(r.rel_res),
                     "setup_ms": float(r.timing["setup_ms"]),
                     "roofline": roofline_block(sweep_bytes(s.m, s.n, esz, sw), float(r.timing["sweep_ms"]),
                                                peak, peak_kind, "tall_sweep_kernel")}
        out[name]["frac_of_peak"] = out[name]["GBps"] / peak
        results[name] = r.a.cpu().numpy()
        del X
    out["bf16_speedup_time_to_tol"] = out["f32_plain"]["ms_to_tol"] / out["bf16_refresh4"]["ms_to_tol"]
    out["f16_speedup_time_to_tol"] = out["f32_plain"]["ms_to_tol"] / out["f16_refresh4"]["ms_to_tol"]
    if cpu:
        cb, ro = cpu_baseline(s, 2, "rel_res", 1e-6, 100, one_core_sweeps=1, what="tall_4Mx512_bf16")
        out["cpu_baseline"] = cb
        for name, a in results.items():
            out[name]["oracle_check"] = oracle_check(s, a, out[name]["sweeps"], out[name]["rel_res"], ro)
    return out


def batched_comparison(hp, synth, ctx, peak, peak_kind, cpu=True):
    """The batched + learned-warm-start workload: 4096 RBF systems (m log-uniform
    in [256, 16384], n uniform in [8, 256]) swept to a relative change of ||e||
    below 1e-6 (at most 10^4 sweeps) in one persistent graph-captured launch,
    cold start against the MLP's warm start (weights trained on 50,000
    method-generated solutions of the family, seed 1)."""
    from paper_2104_12570_gb300 import warm_start as ws
    fam = synth.rbf_family(0)
    m, n, th = synth.rbf_params(4096, seed=0)
    keep, a, b = ws.build_batch(ctx, fam, m, n, th, max_sweeps=4)
    systems = b.systems
    best, tms = hp.autotune_batch(ctx, systems, trial_sweeps=10)
    b.close()
    del keep, a, systems
    out = {"workload": "rbf_batch_4096 (RBF features of U[0,1]^4 inputs, width 0.3; "
                       "y = f_theta(x))",
           "stop": f"{ws.STOP}<{ws.TOL}, max_sweeps {ws.MAX_SWEEPS}",
           "bytes": "per system: set-up 4·m·n + 4m, per sweep 4·m·n (e in shared memory)",
           "x_bytes": int((m * n * 4).sum()),
           "autotune_ms_per_10_sweeps": {f"cluster{k}_panel{p}": v for (k, p), v in tms.items()},
           "cluster": best[0], "panel": best[1]}
    if not os.path.exists(ws.WEIGHTS):
        out["warm"] = "no trained weights"
        return out
    mlp = ws.load(ctx)
    ev = ws.evaluate(ctx, fam, mlp, m, n, th, reps=1, cluster=best)
    # the same comparison on 256 systems of the batch (seed 4) with a 10^5-sweep
    # cap, so that the cap clips (almost) no system in either arm; 8 CTAs per
    # system, since the longest single system bounds the launch
    g = np.random.default_rng(4)
    sub = np.sort(g.choice(len(m), size=256, replace=False))
    ev_unclipped = ws.evaluate(ctx, fam, mlp, m[sub], n[sub], th[sub], reps=1, cluster=(8, 0),
                               max_sweeps=100_000)
    mlp.close()
    for k in ("cold", "warm"):
        if isinstance(ev.get(k), dict):
            ev[k]["frac_of_peak"] = ev[k]["GBps"] / peak
    out.update(ev)
    out["subsample_256_cap_1e5"] = ev_unclipped
    if cpu:
        out["cpu_baseline"], out["oracle_check"] = batched_cpu_and_check(
            hp, synth, ctx, ws, fam, m, n, th, ev["cold"]["elem_sweeps"])
    return out


def batched_cpu_and_check(hp, synth, ctx, ws, fam, m, n, th, gpu_elem_sweeps, count=256, sweeps=20):
    """CPU baseline and parity sample of the batched workload: `count` systems
    drawn from the batch (seed 3), `sweeps` sweeps each (stop rule none), by the
    oracle on every host core (one system per thread) and on one core (a
    quarter of them); the throughput in element-sweeps (m·n per sweep) gives
    the CPU time of the GPU's cold workload.  The same systems swept on the GPU
    give the coefficient error against the oracle at equal sweeps, per system
    against its bound max(1e-5, 8·cond(X)·2^-24)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    nproc, model = cpu_info()
    g = np.random.default_rng(3)
    idx = np.sort(g.choice(len(m), size=count, replace=False))
    syst = [synth.rbf_system(fam, int(m[i]), int(n[i]), th[i]) for i in idx]
    elem = float(sum(s.m * s.n for s in syst)) * sweeps

    def one(s):
        r, _ = oracle.solve_mt(s.X, s.y, m=s.m, n=s.n, tol=0, max_sweeps=sweeps, stop="none", threads=1)
        return r

    t = time.perf_counter()
    with ThreadPoolExecutor(nproc) as ex:
        ores = list(ex.map(one, syst))
    t_all = time.perf_counter() - t
    q = syst[: max(1, count // 4)]
    t = time.perf_counter()
    for s in q:
        one(s)
    t_one = time.perf_counter() - t
    elem_one = float(sum(s.m * s.n for s in q)) * sweeps
    rate_all, rate_one = elem / t_all, elem_one / t_one
    cold_s_all, cold_s_one = gpu_elem_sweeps / rate_all, gpu_elem_sweeps / rate_one
    xbytes_per_elem = 4.0
    cb = {"value": len(m) / cold_s_all, "unit": "systems/s", "cores": nproc, "kind": "oracle",
          "nproc": nproc, "cpu_model": model,
          "GBps": rate_all * xbytes_per_elem / 1e9,
          "s_for_the_cold_batch": cold_s_all,
          "one_core": {"value": len(m) / cold_s_one, "s_for_the_cold_batch": cold_s_one,
                       "GBps": rate_one * xbytes_per_elem / 1e9},
          "sample": (f"{count} systems of the batch x {sweeps} sweeps on {nproc} threads (one "
                     f"system per thread), {len(q)} of them on 1 thread; time of the GPU's cold "
                     "workload (sum of sweeps x m x n) at that element-sweep rate")}
    # the same systems on the GPU, equal sweeps
    keep, sysd = synth.device_rbf_batch(fam, m[idx], n[idx], th[idx], "cuda")
    a = [torch.zeros(int(k), dtype=torch.float32, device="cuda") for k in n[idx]]
    b = hp.Batch(ctx, [(X, y, ai, False) for (X, y), ai in zip(sysd, a)], tol=0, max_sweeps=sweeps,
                 stop="none")
    b.run()
    ratios, errs = [], []
    for s, ai, o in zip(syst, a, ores):
        err = float(np.linalg.norm(ai.cpu().numpy().astype(np.float64) - o.a) /
                    max(np.linalg.norm(o.a), 1e-300))
        Xd = s.dense_f64()
        ev = np.linalg.eigvalsh(Xd.T @ Xd)  # cond(X) = sqrt(cond(X^T X))
        kappa = float(np.sqrt(ev[-1] / max(ev[0], ev[-1] * 1e-300)))
        bound = max(1e-5, 8 * kappa * 2.0 ** -24)
        errs.append(err)
        ratios.append(err / bound)
    b.close()
    chk = {"systems": count, "sweeps": sweeps, "coef_rel_err_median": float(np.median(errs)),
           "coef_rel_err_max": float(np.max(errs)),
           "max_err_over_bound": float(np.max(ratios)),
           "within_1e-5": int(np.sum(np.array(errs) <= 1e-5)),
           "bound": "max(1e-5, 8·cond(X)·2^-24) per system"}
    return cb, chk


def profile_small(hp, synth):
    """A small case for profiler captures (not a bench line): a 512-system batch
    of the RBF family (seed 5), stop rule none, 5 sweeps, cluster 1, launched
    twice; then one training step and one prediction of the warm-start MLP at
    batch 1024."""
    import torch
    from paper_2104_12570_gb300 import warm_start as ws
    ctx = hp.Context(0)
    fam = synth.rbf_family(0)
    m, n, th = synth.rbf_params(512, seed=5)
    keep, a, b = ws.build_batch(ctx, fam, m, n, th, tol=0, stop="none", max_sweeps=5, cluster=1)
    b.run()
    r = b.run()
    mlp = hp.MLP(ctx, max_batch=1024, seed=0)
    g = torch.Generator(device="cuda").manual_seed(0)
    theta = torch.randn(1024, 16, device="cuda", generator=g)
    tgt = torch.randn(1024, 256, device="cuda", generator=g)
    mm, nn = np.full(1024, 4000), np.full(1024, 200)
    mlp.train_step(theta, mm, nn, tgt, lr=1e-4)
    mlp.predict(theta, mm, nn)
    torch.cuda.synchronize()
    print(json.dumps({"profile_small": True, "batch_ms": r["timing"]["sweep_ms"],
                      "x_bytes": int((m * n * 4).sum())}), flush=True)


def next_algorithms(hp, synth, ctx, X, y, s, reps=3):
    """Algorithm 2 (blocks of thr = n/10 columns from one residual, the paper's
    setting) and the random column order variants against Algorithm 1 on the
    benchmark system, all to the relative change of ||e|| < 1e-7; and
    Algorithm 3 (greedy selection) for 32 steps."""
    import torch
    out = {}
    esz = 4
    # the random-index variant of Sec. 2: n indices per sweep drawn uniformly with
    # replacement (seeded), and a fresh random permutation per sweep
    g = np.random.default_rng(11)
    o_rep = g.integers(0, s.n, size=(MAX_SWEEPS, s.n)).astype(np.int32)
    o_perm = np.stack([g.permutation(s.n) for _ in range(MAX_SWEEPS)]).astype(np.int32)
    for name, fn in (("alg1_sweep", lambda: ctx.solve(X, y, tol=TOL, max_sweeps=MAX_SWEEPS, stop=STOP)),
                     ("alg2_blocks_thr25", lambda: ctx.solve_blocks(X, y, max(1, s.n // 10), tol=TOL,
                                                                    max_sweeps=MAX_SWEEPS, stop=STOP)),
                     ("random_indices_with_replacement",
                      lambda: ctx.solve_order(X, y, o_rep, tol=TOL, stop=STOP)),
                     ("random_permutation_per_sweep",
                      lambda: ctx.solve_order(X, y, o_perm, tol=TOL, stop=STOP))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_to_tol": ms, "sweeps": int(r.sweeps), "rel_res": float(r.rel_res),
                     "GBps": solve_bytes(s.m, s.n, esz, int(r.sweeps)) / (ms * 1e-3) / 1e9,
                     "sweep_kernel_GBps": sweep_bytes(s.m, s.n, esz, int(r.sweeps))
                     / (r.timing["sweep_ms"] * 1e-3) / 1e9}
    F = 32
    ctx.select(X, y, F)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        r, sel = ctx.select(X, y, F)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ctx.select_swap(X, y, F, 8)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        rs, sel_s, swaps = ctx.select_swap(X, y, F, 8)
    e1.record()
    torch.cuda.synchronize()
    out["alg3_select_32_then_swaps_8"] = {
        "ms": e0.elapsed_time(e1) / reps, "swaps_made": int((swaps[:, 0] >= 0).sum()),
        "passes": int(rs.timing["passes"]), "rel_res_after": float(rs.rel_res)}
    out["alg3_select_32"] = {"ms": ms, "ms_per_step": r.timing["sweep_ms"] / max(1, r.timing["passes"]),
                             "sweep_kernel_GBps": sweep_bytes(s.m, s.n, esz, r.timing["passes"])
                             / (r.timing["sweep_ms"] * 1e-3) / 1e9,
                             "rel_res_after": float(r.rel_res), "first_selected": sel[:8].tolist()}
    return out


def rowmajor_line(hp, synth, ctx, dev, name, desc, peak, peak_kind, reps=3, flush=False, cpu=True):
    """A row-major workload (the wide cluster kernel) solved to relative residual
    1e-6, the stop confirmed on the true residual of the returned a.  Bytes: the
    set-up reads X (the per-block Gram and the initial residual) and each sweep
    reads X once; e stays in shared memory.  With flush, a buffer larger than L2
    is written before each timed solve (X is smaller than L2)."""
    import torch
    s = synth.workload(name, seed=0)
    X = torch.from_numpy(s.X).to(dev)  # (m, n) row-major
    y = torch.from_numpy(s.y).to(dev)
    buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if flush else None
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=200, stop="rel_res")
    times = []
    for _ in range(reps):
        if buf is not None:
            buf.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = ctx.solve(X, y, tol=1e-6, max_sweeps=200, stop="rel_res")
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = sorted(times)[len(times) // 2]
    sw = int(r.sweeps)
    nb = solve_bytes(s.m, s.n, 4, sw, e_in_hbm=False)
    out = {"workload": desc, "stop": "rel_res<=1e-6 (confirmed on the true residual)",
           "l2": "flushed before each solve (256 MB write)" if flush else "X larger than L2",
           "status": r.status, "sweeps": sw, "rel_res": float(r.rel_res), "ms_to_tol": ms,
           "ms_per_sweep": float(r.timing["sweep_ms"]) / max(1, sw),
           "GBps": nb / (ms * 1e-3) / 1e9, "frac_of_peak": nb / (ms * 1e-3) / 1e9 / peak,
           "bytes": "set-up 4·m·n + 4m, per sweep 4·m·n (e in shared memory)",
           "roofline": roofline_block(sweep_bytes(s.m, s.n, 4, sw, e_in_hbm=False), ms, peak,
                                      peak_kind, "wide_sweep_kernel (set-up and confirmation inside)")}
    a_gpu = r.a.cpu().numpy()
    del X
    if cpu:
        cb, ro = cpu_baseline(s, 4, "rel_res", 1e-6, 200, e_in_hbm=False, what=name)
        out["cpu_baseline"] = cb
        import oracle
        o = oracle.solve_system(s, tol=0, max_sweeps=sw, stop="none") if ro.sweeps != sw else ro
        out["oracle_check"] = oracle_check(s, a_gpu, sw, r.rel_res, o)
        out["oracle_check"]["oracle_sweeps_to_rule"] = int(ro.sweeps)
    return out


def panel_line(hp, synth, ctx, dev, peak, peak_kind, reps=3, cpu=True, rows=0):
    """The column-major 1,000,000 x 1024 consistent float32 system (more than 512
    columns: the panel sweep) solved to relative residual 1e-6, the stop
    confirmed on the true residual of the returned a.  Bytes are the method's:
    set-up 4·m·n + 4m, per sweep 4·m·n + 8m; the panel design reads X twice per
    sweep, so its fraction of the copy peak on those bytes is at most about 1/2."""
    import torch
    name = "tall_1Mx1024_f32"
    s = synth.workload(name, seed=0, **({"m": rows} if rows else {}))
    X = torch.from_numpy(s.X).to(dev).T  # (m, n) column-major
    y = torch.from_numpy(s.y).to(dev)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=100, stop="rel_res")
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = ctx.solve(X, y, tol=1e-6, max_sweeps=100, stop="rel_res")
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = sorted(times)[len(times) // 2]
    sw = int(r.sweeps)
    nb = solve_bytes(s.m, s.n, 4, sw)
    out = {"workload": f"{name} (column-major, consistent, n > 512: the panel sweep)" +
                       (f", m overridden to {s.m}" if rows else ""),
           "stop": "rel_res<=1e-6 (confirmed on the true residual)", "l2": "X larger than L2",
           "status": r.status, "sweeps": sw, "passes": int(r.timing["passes"]),
           "rel_res": float(r.rel_res), "ms_to_tol": ms, "setup_ms": float(r.timing["setup_ms"]),
           "ms_per_sweep": float(r.timing["sweep_ms"]) / max(1, sw),
           "GBps": nb / (ms * 1e-3) / 1e9, "frac_of_peak": nb / (ms * 1e-3) / 1e9 / peak,
           "bytes": "set-up 4·m·n + 4m, per sweep 4·m·n + 8m (X is read twice per sweep)",
           "roofline": roofline_block(sweep_bytes(s.m, s.n, 4, sw), float(r.timing["sweep_ms"]), peak,
                                      peak_kind, "panel_sweep_kernel")}
    a_gpu = r.a.cpu().numpy()
    del X
    if cpu:
        cb, ro = cpu_baseline(s, 4, "rel_res", 1e-6, 100, one_core_sweeps=1, what=name)
        out["cpu_baseline"] = cb
        out["oracle_check"] = oracle_check(s, a_gpu, sw, r.rel_res, ro)
    return out


def profile_wide(hp, synth, cols, blocks=512):
    """The wide cluster kernel alone on a 2,000 x `cols` float32 row-major
    consistent system, solved to relative residual 1e-6 (profiler captures and
    the kernel's own trace; not a bench line).  The trace stamps CTA 0's global
    timer at six points of each of the first `blocks` column blocks: after the
    wait for the block's exchange round and its sum, after the block's steps
    (da = M q - N da_prev), after the next block's M/N copies are issued, after
    the wait for the lookahead slab, after the row pass (update and lookahead
    dots), after the push of the lookahead partials."""
    import torch
    s = synth.workload("wide_2000x200k_f32", seed=0, n=int(cols))
    dev = torch.device("cuda", 0)
    ctx = hp.Context(0)
    X = torch.from_numpy(s.X).to(dev)
    y = torch.from_numpy(s.y).to(dev)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=200, stop="rel_res")  # warm-up, untraced
    ctx.set_trace(blocks)
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=200, stop="rel_res")
    t = ctx.trace_raw()[: 6 * blocks].reshape(blocks, 6)
    t = t[t[:, 5] > 0]
    ctx.set_trace(0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = ctx.solve(X, y, tol=1e-6, max_sweeps=200, stop="rel_res")
    e1.record()
    torch.cuda.synchronize()
    out = {"profile_wide": True, "m": s.m, "n": s.n, "status": r.status, "sweeps": int(r.sweeps),
           "ms_to_tol": e0.elapsed_time(e1), "sweep_kernel_ms": float(r.timing["sweep_ms"]),
           "blocks_per_sweep": -(-s.n // 64)}
    if len(t) > 2:
        prev = t[:-1, 5]
        ph = {"round_wait_and_sum_us": t[1:, 0] - prev, "chain_us": t[1:, 1] - t[1:, 0],
              "next_copies_us": t[1:, 2] - t[1:, 1], "slab_wait_us": t[1:, 3] - t[1:, 2],
              "row_pass_us": t[1:, 4] - t[1:, 3], "push_us": t[1:, 5] - t[1:, 4],
              "block_us": t[1:, 5] - prev}
        out["trace_blocks"] = int(len(t) - 1)
        out["median_per_block"] = {k: float(np.median(v)) / 1e3 for k, v in ph.items()}
    print(json.dumps(out), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the bfloat16-vs-float32 comparison on the 4,000,000 x 512 system")
    ap.add_argument("--no-wide", action="store_true",
                    help="skip the wide 2,000 x 200,000 and square 4096 x 4096 row-major systems")
    ap.add_argument("--no-next", action="store_true",
                    help="skip Algorithm 2 / Algorithm 3 on the benchmark system")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched cold-vs-learned-warm-start comparison (4096 RBF systems)")
    ap.add_argument("--rows", type=int, default=0,
                    help="override m (smaller case for profiler captures; not a bench line)")
    ap.add_argument("--profile-panel", action="store_true",
                    help="the panel sweep alone on the 1,000,000 x 1024 system (not a bench line)")
    ap.add_argument("--profile-small", action="store_true",
                    help="run only the small batched + MLP case used for profiler captures")
    ap.add_argument("--profile-wide", type=int, default=0, metavar="COLS",
                    help="run only the wide kernel on a 2,000 x COLS system (profiler captures)")
    args = ap.parse_args()
    if args.profile_wide:
        import paper_2104_12570_gb300 as hp
        from paper_2104_12570_gb300 import synth
        profile_wide(hp, synth, args.profile_wide)
        return
    if args.profile_small:
        import paper_2104_12570_gb300 as hp
        from paper_2104_12570_gb300 import synth
        profile_small(hp, synth)
        return
    if args.profile_panel:
        import torch
        import paper_2104_12570_gb300 as hp
        from paper_2104_12570_gb300 import synth
        ctx = hp.Context(0)
        peak, peak_kind = peaks()
        out = panel_line(hp, synth, ctx, torch.device("cuda", 0), peak, peak_kind, cpu=False,
                         rows=args.rows)
        print(json.dumps({"profile_panel": True, **out}), flush=True)
        ctx.close()
        return
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    import paper_2104_12570_gb300 as hp
    from paper_2104_12570_gb300 import synth

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s = synth.workload(WORKLOAD, seed=rank, **({"m": args.rows} if args.rows else {}))
    esz = 4
    X = torch.from_numpy(s.X).to(dev).T  # (m, n), column-major
    y = torch.from_numpy(s.y).to(dev)
    ctx = hp.Context(local)
    a = torch.empty(s.n, dtype=torch.float32, device=dev)

    def step():
        return ctx.solve(X, y, tol=TOL, max_sweeps=MAX_SWEEPS, stop=STOP, out=a)

    for _ in range(args.warmup):
        r = step()
    if r.status != "ok":
        raise SystemExit(f"solve did not converge: {r.status}")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # the timed steps are enqueued back to back (hpscd_solve_async): each is the
    # whole solve, set-up included, and writes its status and sweep count to a
    # device record; the records and the per-call kernel timings are read after
    # the timed region
    res = hp.results_buffer(args.steps, dev)
    ctx.solve_async(X, y, res[0], tol=TOL, max_sweeps=MAX_SWEEPS, stop=STOP, out=a)
    with ClockSampler(local) as clk:
        barrier()
        t_start = time.perf_counter()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for k in range(args.steps):
            ctx.solve_async(X, y, res[k], tol=TOL, max_sweeps=MAX_SWEEPS, stop=STOP, out=a)
        ev1.record()
        barrier()
        clk.mark(t_start, time.perf_counter())
    ms = ev0.elapsed_time(ev1) / args.steps
    got = hp.read_results(res)
    if any(st != "ok" for st in got["status"]):
        raise SystemExit(f"a timed solve did not converge: {set(got['status'])}")
    passes = [int(p) for p in got["passes"]]
    times = ctx.async_timings(min(args.steps, 64))
    sweep_ms = [t["sweep_ms"] for t in times]
    launches = int(round(np.mean([t["kernel_launches"] for t in times]) * args.steps))
    sweeps_timed = int(got["sweeps"][-1])
    setup_ms = float(np.mean([t["setup_ms"] for t in times]))
    ms = max_over_ranks(ms, world, dev)
    p_mean = float(np.mean(passes))
    sw_mean = float(np.mean(got["sweeps"]))
    nbytes = solve_bytes(s.m, s.n, esz, sw_mean)
    value = job_value(nbytes, world, ms)

    # end to end through the C ABI from pinned host memory
    e2e = None
    if not args.skip_e2e:
        Xh = torch.from_numpy(s.X).pin_memory().T
        yh = torch.from_numpy(s.y).pin_memory()
        for _ in range(args.warmup):
            ctx.solve_host(Xh, yh, tol=TOL, max_sweeps=MAX_SWEEPS, stop=STOP)
        torch.cuda.synchronize()
        e2e_steps = max(5, args.steps // 2)
        call_ms = []
        t = time.perf_counter()
        for _ in range(e2e_steps):
            t1 = time.perf_counter()
            rh = ctx.solve_host(Xh, yh, tol=TOL, max_sweeps=MAX_SWEEPS, stop=STOP)
            call_ms.append((time.perf_counter() - t1) * 1e3)
        e2e_s = (time.perf_counter() - t) / e2e_steps
        e2e_val = world * solve_bytes(s.m, s.n, esz, int(rh.sweeps)) / e2e_s / 1e9
        # the host link alone: one copy of the same pinned X to the device
        Xd_probe = torch.empty(s.X.shape, dtype=torch.float32, device=dev)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        Xd_probe.copy_(Xh.T, non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        h2d_ms = c0.elapsed_time(c1)
        del Xd_probe
        e2e = {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": int(s.X.nbytes + s.y.nbytes),
               "d2h_bytes_per_step": int(4 * s.n + 8 * (rh.sweeps + 1) + 48),
               "ms_per_step": e2e_s * 1e3, "steps": e2e_steps,
               "call_ms_min_median_max": [min(call_ms), float(np.median(call_ms)), max(call_ms)],
               "slowest_call": int(np.argmax(call_ms)),
               "h2d_copy_ms": h2d_ms,
               "h2d_GBps": s.X.nbytes / (h2d_ms * 1e-3) / 1e9}

    if rank == 0:
        peak, peak_kind = peaks()
        k_ms = float(np.mean(sweep_ms))
        k_bytes = sweep_bytes(s.m, s.n, esz, sw_mean)
        achieved = k_bytes / (k_ms * 1e-3) / 1e9
        tr = traffic_from_profile(kernel_sha())
        out = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if not args.rows else f"{WORKLOAD} with m overridden to {s.m}",
                       "m": s.m, "n": s.n, "layout": "col-major",
                       "stop": f"{STOP}<{TOL}", "sweeps": sweeps_timed,
                       "passes_per_solve": p_mean,
                       "l2": f"inputs larger than L2 ({s.m * s.n * esz / 1e9:.2f} GB X)" if s.m * s.n * esz > 129e6
                       else f"X of {s.m * s.n * esz / 1e6:.0f} MB, below L2",
                       "bytes": "set-up 4·m·n + 4m, per sweep 4·m·n + 8m (e in HBM)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "kernel": "tall_sweep_kernel", "traffic": tr,
                         "kernel_ms": k_ms, "algorithmic_bytes": k_bytes},
            "setup_ms": setup_ms,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        cpu = not args.no_cpu_baseline
        if cpu:
            out["cpu_baseline"], ro = cpu_baseline(s, esz, STOP, TOL, MAX_SWEEPS, what=WORKLOAD)
            out["oracle_check"] = oracle_check(s, a.cpu().numpy(), sweeps_timed,
                                               float(got["rel_res"][-1]), ro)
        if not args.no_next and not args.rows:
            out["next_algorithms"] = next_algorithms(hp, synth, ctx, X, y, s)
        if not args.no_wide and not args.rows:
            out["wide"] = rowmajor_line(hp, synth, ctx, dev, "wide_2000x200k_f32",
                                        "wide_2000x200k_f32 (row-major, consistent)", peak,
                                        peak_kind, reps=3, cpu=cpu)
            out["square"] = rowmajor_line(hp, synth, ctx, dev, "square_4096_f32",
                                          "square_4096_f32 (row-major, consistent, I + 0.5·Z/64)",
                                          peak, peak_kind, reps=3, flush=True, cpu=cpu)
        if not args.no_wide and not args.rows:
            torch.cuda.empty_cache()
            out["panel"] = panel_line(hp, synth, ctx, dev, peak, peak_kind, cpu=cpu)
        if not args.no_compare and not args.rows:
            del X
            torch.cuda.empty_cache()
            out["precision_mode"] = precision_comparison(hp, synth, ctx, dev, peak, peak_kind, cpu=cpu)
        if not args.no_batched and not args.rows:
            torch.cuda.empty_cache()
            out["batched"] = batched_comparison(hp, synth, ctx, peak, peak_kind, cpu=cpu)
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
