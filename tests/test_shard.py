"""Multi-rank path on CPU (gloo, world size 2): domain shards bounded independently, then the only
exchange -- hull min/max and the summed objective -- reproduces the single-rank result."""
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2605_25346_b300 import shard, workloads as wl


@pytest.mark.parametrize("D", [0, 1, 7, 64, 4096])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_ranges_partition_the_domains(D, world):
    ranges = [shard.shard_range(D, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == D
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == D


def test_shard_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def _problem():
    return wl.random_problem(41, [3, 12, 10, 2], D=9, H=3, eps=0.3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    from oracle import reach as orc
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        res = orc.reach(shard.shard_problem(_problem(), rank, world))
        lo, hi = res["hull_lo"].detach().clone(), res["hull_hi"].detach().clone()
        V = res["V"].detach().sum().reshape(1)
        shard.merge_hull(lo, hi)
        shard.merge_objective(V)
        q.put((rank, lo.numpy(), hi.numpy(), V.numpy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_merge_to_the_single_rank_hull():
    from oracle import reach as orc
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = orc.reach(_problem())
    for _, lo, hi, V in got:  # every rank holds the merged result
        np.testing.assert_allclose(lo, full["hull_lo"].detach().numpy(), rtol=1e-12, atol=0)
        np.testing.assert_allclose(hi, full["hull_hi"].detach().numpy(), rtol=1e-12, atol=0)
        np.testing.assert_allclose(V, full["V"].detach().sum().numpy(), rtol=1e-12)
