"""Seeded synthetic systems X·a = y shaped like the tall, wide and square
workloads of the HPSCD paper (Sec. 2, the system statement; Sec. 9, the
numerical experiments).

This module is the ONLY code shared by the CPU oracle and the CUDA path.  It
holds none of the method's arithmetic: it draws X, a_true and noise, forms the
right-hand side y = X·a_true (+ noise) in float64, and converts storage
formats.  Everything is reproducible from (shape, seed): the random stream is
split into fixed-size chunks, each with its own child seed, so the values do
not depend on how many threads fill them.

Storage conventions (the C-ABI uses the same ones):
  * column-major X (m×n, leading dimension m) is a numpy array of shape (n, m);
    row j of that array is column X_j;
  * row-major X (m×n, leading dimension n) is a numpy array of shape (m, n);
  * BF16 values are kept as uint16 bit patterns.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

CHUNK = 1 << 22  # elements per independent random stream


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def _fill_chunks(out_flat: np.ndarray, seed: int, tag: int, kind: str,
                 lo: float = -1.0, hi: float = 1.0) -> None:
    """Fill out_flat (float32 or float64) with iid draws, chunk by chunk."""
    total = out_flat.size
    nchunks = (total + CHUNK - 1) // CHUNK
    seqs = np.random.SeedSequence([seed, tag]).spawn(max(nchunks, 1))

    def work(c):
        s, e = c * CHUNK, min(total, (c + 1) * CHUNK)
        g = np.random.Generator(np.random.Philox(seqs[c]))
        if kind == "normal":
            out_flat[s:e] = g.standard_normal(e - s, dtype=out_flat.dtype)
        else:
            out_flat[s:e] = g.uniform(lo, hi, e - s).astype(out_flat.dtype)

    if nchunks <= 1:
        if total:
            work(0)
        return
    with ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(work, range(nchunks)))


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (round to nearest, ties to even); returns uint16 bits.
    Inputs are finite."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = (u + np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))) >> np.uint32(16)
    return r.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.ascontiguousarray(b, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


@dataclass
class System:
    """One synthetic system.  X is stored as described in the module docstring."""
    X: np.ndarray          # float32 / uint16(bf16) / float16 / float64 storage array
    y: np.ndarray          # float32 (or float64 for the float64 tiny case), length m
    a_true: np.ndarray     # float64, length n
    m: int
    n: int
    layout: str            # "col" or "row"
    dtype: str             # "f32", "bf16", "f16", "f64"

    @property
    def ld(self) -> int:
        return self.m if self.layout == "col" else self.n

    def x_values_f64_block(self, j0: int, j1: int) -> np.ndarray:
        """Columns j0..j1-1 of X as float64, shape (m, j1-j0) (for forming y / tests)."""
        if self.layout == "col":
            blk = self.X[j0:j1]
            if self.dtype == "bf16":
                blk = bf16_bits_to_f32(blk)
            return np.asarray(blk, dtype=np.float64).T
        blk = self.X[:, j0:j1]
        if self.dtype == "bf16":
            blk = bf16_bits_to_f32(blk)
        return np.asarray(blk, dtype=np.float64)

    def dense_f64(self) -> np.ndarray:
        """The whole X as a float64 (m, n) array.  Small systems only."""
        return self.x_values_f64_block(0, self.n)


def _matvec_f64(sysm: System, a: np.ndarray) -> np.ndarray:
    """y = X·a in float64, streamed in column blocks so large X never exists in float64."""
    y = np.zeros(sysm.m, dtype=np.float64)
    step = max(1, (1 << 24) // max(sysm.m, 1))
    for j0 in range(0, sysm.n, step):
        j1 = min(sysm.n, j0 + step)
        y += sysm.x_values_f64_block(j0, j1) @ a[j0:j1]
    return y


def make_system(m: int, n: int, seed: int = 0, *, layout: str = "col", dtype: str = "f32",
                noise: float = 0.0, consistent_rhs_dtype: str = "f32", scale: float = 1.0,
                diag: float = 0.0) -> System:
    """X = scale·Z + diag·I with Z iid N(0,1) (I the m x n identity), a_true iid
    U(-1,1), y = X·a_true + noise·N(0,1).

    The system solved is the STORED X (after rounding to the storage dtype);
    y is formed from those stored values in float64 and then rounded to
    float32 (or kept float64 when consistent_rhs_dtype == "f64")."""
    if layout not in ("col", "row") or dtype not in ("f32", "bf16", "f16", "f64"):
        raise ValueError("bad layout/dtype")
    shape = (n, m) if layout == "col" else (m, n)

    def shaped(Z):
        if scale != 1.0:
            Z *= Z.dtype.type(scale)
        if diag:
            k = min(m, n)
            Z.reshape(-1)[: k * (shape[1] + 1): shape[1] + 1] += Z.dtype.type(diag)
        return Z

    if dtype == "f64":
        X = np.empty(shape, dtype=np.float64)
        _fill_chunks(X.reshape(-1), seed, 1, "normal")
        X = shaped(X)
    else:
        Xf = np.empty(shape, dtype=np.float32)
        _fill_chunks(Xf.reshape(-1), seed, 1, "normal")
        Xf = shaped(Xf)
        if dtype == "bf16":
            X = f32_to_bf16_bits(Xf).reshape(shape)
        elif dtype == "f16":
            X = Xf.astype(np.float16)  # IEEE binary16, round to nearest even
        else:
            X = Xf
    a_true = np.empty(n, dtype=np.float64)
    _fill_chunks(a_true, seed, 2, "uniform", -1.0, 1.0)
    s = System(X=X, y=np.empty(0), a_true=a_true, m=m, n=n, layout=layout, dtype=dtype)
    y = _matvec_f64(s, a_true)
    if noise:
        z = np.empty(m, dtype=np.float64)
        _fill_chunks(z, seed, 3, "normal")
        y += noise * z
    s.y = y if consistent_rhs_dtype == "f64" else y.astype(np.float32)
    return s


# The paper's workload shapes (Sec. 2: tall, wide and square systems; Sec. 9:
# Float32 storage).  Names state what each one is.
WORKLOADS = {
    # tall, consistent, float64: the small case the oracle finishes in seconds
    "tall_200x50_f64": dict(m=200, n=50, layout="col", dtype="f64", noise=0.0,
                            consistent_rhs_dtype="f64"),
    # tall, noisy least squares, float32 column-major (1.02 GB of X)
    "tall_1Mx256_f32": dict(m=1_000_000, n=256, layout="col", dtype="f32", noise=0.01),
    # wide, consistent, float32 row-major (1.6 GB of X)
    "wide_2000x200k_f32": dict(m=2000, n=200_000, layout="row", dtype="f32", noise=0.0),
    # tall, consistent, float32 column-major with more than 512 columns (4.1 GB
    # of X): the panel sweep
    "tall_1Mx1024_f32": dict(m=1_000_000, n=1024, layout="col", dtype="f32", noise=0.0),
    # tall, consistent, bfloat16 storage (4.1 GB of X)
    "tall_4Mx512_bf16": dict(m=4_000_000, n=512, layout="col", dtype="bf16", noise=0.0),
    # square, consistent, float32 row-major (67 MB of X): I + 0.5·Z/sqrt(n), whose
    # singular values lie in about [0.5, 1.5], so the sweep converges in tens of
    # sweeps (a square Gaussian X has cond ~ n and the sweep barely moves)
    "square_4096_f32": dict(m=4096, n=4096, layout="row", dtype="f32", noise=0.0,
                            scale=0.5 / 64.0, diag=1.0),
}


def workload(name: str, seed: int = 0, **override) -> System:
    kw = dict(WORKLOADS[name])
    kw.update(override)
    m, n = kw.pop("m"), kw.pop("n")
    return make_system(m, n, seed, **kw)


# ---- the batched family: many similar RBF systems (Sec. 9 notes the method
# pays when similar systems are solved many times) ----
#
# Every system of the family takes the first n of 256 fixed centres c_k and the
# first m of 16384 fixed inputs x_i, all iid U[0,1]^4 (drawn once, seed-fixed),
# so a system is determined by (m, n, theta):
#     X_ik = exp(-||x_i - c_k||^2 / (2 * 0.3^2))            (RBF features)
#     y_i  = f_theta(x_i) = sum_k theta_k cos(omega_k . x_i + b_k) / 4
# with omega_k ~ N(0, I_4) and b_k ~ U[0, 2 pi) drawn once, theta ~ N(0, I_16)
# per system, m log-uniform in [256, 16384] and n uniform in [8, 256].
RBF_MAX_M, RBF_MAX_N, RBF_DIM, RBF_THETA = 16384, 256, 4, 16
RBF_WIDTH = 0.3


@dataclass
class RBFFamily:
    C: np.ndarray      # (256, 4) centres
    P: np.ndarray      # (16384, 4) inputs
    omega: np.ndarray  # (16, 4)
    b: np.ndarray      # (16,)
    M: np.ndarray      # (256, 16384) float32: row k = feature column k over all inputs
    F: np.ndarray      # (16384, 16) float64: cos(omega_k . x_i + b_k) / 4


def rbf_family(seed: int = 0) -> RBFFamily:
    g = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 101])))
    C = g.uniform(0.0, 1.0, (RBF_MAX_N, RBF_DIM))
    P = g.uniform(0.0, 1.0, (RBF_MAX_M, RBF_DIM))
    omega = g.standard_normal((RBF_THETA, RBF_DIM))
    b = g.uniform(0.0, 2.0 * np.pi, RBF_THETA)
    d2 = ((C[:, None, :] - P[None, :, :]) ** 2).sum(axis=-1)
    M = np.exp(-d2 / (2.0 * RBF_WIDTH ** 2)).astype(np.float32)
    F = np.cos(P @ omega.T + b) / 4.0
    return RBFFamily(C=C, P=P, omega=omega, b=b, M=M, F=F)


def rbf_params(count: int, seed: int):
    """(m, n, theta) of `count` systems: m log-uniform [256, 16384], n uniform
    [8, 256], theta ~ N(0, I_16)."""
    g = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 102])))
    m = np.rint(np.exp(g.uniform(np.log(256.0), np.log(float(RBF_MAX_M)), count))).astype(np.int64)
    m = np.clip(m, 256, RBF_MAX_M)
    n = g.integers(8, RBF_MAX_N + 1, count).astype(np.int64)
    theta = g.standard_normal((count, RBF_THETA))
    return m, n, theta


def rbf_rhs(fam: RBFFamily, m: int, theta: np.ndarray) -> np.ndarray:
    """y = f_theta(x_1..x_m), formed in float64 and rounded to float32."""
    return (fam.F[:m] @ np.asarray(theta, dtype=np.float64)).astype(np.float32)


def rbf_system(fam: RBFFamily, m: int, n: int, theta: np.ndarray) -> System:
    """One member of the family as a column-major float32 System (a_true unknown: zeros)."""
    X = np.ascontiguousarray(fam.M[:n, :m])
    return System(X=X, y=rbf_rhs(fam, m, theta), a_true=np.zeros(n), m=int(m), n=int(n),
                  layout="col", dtype="f32")


def device_rbf_batch(fam: RBFFamily, m, n, theta, device, share_master: bool = False):
    """The systems (m[i], n[i], theta[i]) of the family as CUDA tensors.

    Returns (keep, systems): systems[i] = (X, y) with X an (m, n) column-major
    float32 view and y (m,) float32 (the values rbf_system/rbf_rhs give).  By
    default every system owns its copy of X (leading dimension m rounded up to
    a multiple of 4, so columns start on 16-byte boundaries); share_master
    makes every X a view of the one 16384-row master matrix (ld = 16384).
    `keep` holds the backing buffers."""
    import torch
    count = len(m)
    Md = torch.from_numpy(fam.M).to(device)
    ys = [rbf_rhs(fam, int(m[i]), theta[i]) for i in range(count)]
    yoff = np.concatenate([[0], np.cumsum([len(v) for v in ys])]).astype(np.int64)
    yflat = torch.from_numpy(np.concatenate(ys) if count else np.zeros(0, np.float32)).to(device)
    systems = []
    if share_master:
        for i in range(count):
            X = Md[: int(n[i]), : int(m[i])].T
            systems.append((X, yflat[yoff[i]: yoff[i + 1]]))
        return (Md, yflat), systems
    lds = [((int(mi) + 3) // 4) * 4 for mi in m]
    offs = np.concatenate([[0], np.cumsum([int(n[i]) * lds[i] for i in range(count)])]).astype(np.int64)
    flat = torch.empty(int(offs[-1]) + 4, dtype=torch.float32, device=device)
    for i in range(count):
        mi, ni, ld = int(m[i]), int(n[i]), lds[i]
        blk = flat[offs[i]: offs[i] + ni * ld].view(ni, ld)
        blk[:, :mi].copy_(Md[:ni, :mi])
        systems.append((blk[:, :mi].T, yflat[yoff[i]: yoff[i + 1]]))
    del Md
    return (flat, yflat), systems
