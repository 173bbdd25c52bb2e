"""The multi-process path of the benchmark on CPU: two gloo ranks (replicas,
one system per rank, no collective on the data path) agree on the slowest
rank's time and on the whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        ms = bench.max_over_ranks(1.5 + r, w, "cpu")  # rank r took 1.5 + r ms per step
        value = bench.job_value(6.0e9, w, ms)
        dist.barrier()
        q.put((r, w, local, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 and g[2] == g[0] for g in got)
    for g in got:
        assert g[3] == pytest.approx(2.5)                      # max over the ranks
        assert g[4] == pytest.approx(2 * 6.0e9 / 2.5e-3 / 1e9)  # both ranks' bytes in that time


def test_single_rank_is_the_identity():
    assert bench.max_over_ranks(1.25, 1, "cpu") == 1.25
    assert bench.job_value(6.0e9, 1, 1.5) == pytest.approx(4000.0)
