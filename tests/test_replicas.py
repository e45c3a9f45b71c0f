"""Multi-rank host logic on CPU (gloo, world size 2): the channel partition of the batched sweep is
disjoint, complete and balanced on every rank without communication, and the job-level reduction
takes the slowest rank's time and the sum of the counts."""
import os

import pytest
import torch.multiprocessing as mp

from paper_1310_7450_gb300 import inputs, replicas


def _worker(rank, world, port, nys, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.partition_channels(nys, world, rank)
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        red = replicas.reduce_job({"wall": ("max", 10.0 + rank), "converged": ("sum", len(mine))}, world)
        q.put((rank, parts, red))
    finally:
        dist.destroy_process_group()


def test_partition_and_reduction_on_two_gloo_ranks():
    ps = inputs.sweep_channel_params(64, 3)
    nys = [q["ny"] for q in ps]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, nys, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, parts, red in got:
        a, b = parts
        assert set(a).isdisjoint(b) and sorted(a + b) == list(range(len(nys)))
        loads = [sum(nys[c] ** 2 for c in part) for part in parts]
        assert max(loads) <= 1.05 * min(loads)
        assert red["wall"] == 11.0 and red["converged"] == len(nys)
        assert parts[rank] == replicas.partition_channels(nys, 2, rank)


def test_partition_single_rank_and_bad_arguments():
    assert replicas.partition_channels([5, 3, 9], 1, 0) == [0, 1, 2]
    with pytest.raises(ValueError):
        replicas.partition_channels([5], 2, 2)
