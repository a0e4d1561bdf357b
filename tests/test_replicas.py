"""The multi-GPU host path on CPU: two gloo ranks run the replica logic of bench.py (per-rank
seeds, max over ranks of the step times, whole-job throughput) without a GPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2311_11943_gb300 import replicas  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://")
    w, r, _ = replicas.rank_env()
    seed = replicas.rank_seed(2, r)
    ms = [10.0 + 5.0 * r, 1.0 - 0.5 * r]          # rank 1 is slower on the first number
    mx = replicas.max_over_ranks(ms, dist)
    value = replicas.job_throughput(1e12, w, mx[0])
    dist.barrier()
    out.put((r, w, seed, mx, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_times_and_aggregate_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = {r[2] for r in res}
    assert len(seeds) == world                    # independent inputs per rank
    for (r, w, seed, mx, value) in res:
        assert w == world
        assert mx == [15.0, 1.0]                  # max over ranks, element-wise
        assert value == pytest.approx(world * 1e12 / 15e-3 / 1e12)


def test_single_process_is_the_identity():
    assert replicas.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert replicas.job_throughput(2e12, 1, 1000.0) == pytest.approx(2.0)
