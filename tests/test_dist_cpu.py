"""The multi-rank path on CPU: two gloo ranks shard uneven instances, time, reduce.

No GPU is involved: the data path has no collective (independent instances), so what
needs checking is that the ranks agree on a balanced, disjoint, complete partition
without communicating, and that the timing reduction takes the maximum.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1605_01715_gb300.dist import gather_to_rank0, max_over_ranks, shard_instances  # noqa: E402


def test_partition_is_complete_disjoint_and_balanced():
    sizes = [1000 * (1 + (i * 37) % 64) for i in range(256)]       # uneven, 1k..64k
    for ws in (1, 2, 3, 8):
        parts = shard_instances(sizes, ws)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)               # LPT bound
    assert shard_instances([5], 4) == [[0], [], [], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard_instances(sizes, world)[rank]
        step_ms = 10.0 + rank                       # rank 1 is the slowest
        worst = max_over_ranks(step_ms)
        done = sum(sizes[i] for i in mine)
        allp = gather_to_rank0((rank, mine, done))
        dist.barrier()
        if rank == 0:
            q.put((worst, allp))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_and_reduce_max():
    sizes = [3000, 200000, 1500, 77000, 64000, 9000, 12000, 150000]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    worst, allp = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert worst == 11.0
    got = sorted(i for _, ids, _ in allp for i in ids)
    assert got == list(range(len(sizes)))
    assert sum(d for _, _, d in allp) == sum(sizes)                 # every unit counted once
