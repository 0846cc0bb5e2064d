"""Host logic of the multi-GPU benchmark on CPU (gloo, world size 2).

Realizations are independent (Algorithm 1's outer loop), so ranks shard them
with disjoint realization ids and no exchange; the job's time is the max
over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # two groups of 8 realizations each (the mixed-size 3D batch)
        bases = [bench.shard_real_base(rank, 16, gb) for gb in (0, 8)]
        ids = [b + i for b in bases for i in range(8)]
        times = bench.max_over_ranks([10.0 + rank, 3.0 * (1 - rank), 7.0], world, "cpu")
        q.put((rank, ids, times))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_realizations_and_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, ids, times = q.get(timeout=120)
        res[rank] = (ids, times)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids0, ids1 = res[0][0], res[1][0]
    assert len(set(ids0)) == 16 and len(set(ids1)) == 16
    assert not set(ids0) & set(ids1)
    assert sorted(ids0 + ids1) == list(range(32))
    assert res[0][1] == res[1][1] == [11.0, 3.0, 7.0]
