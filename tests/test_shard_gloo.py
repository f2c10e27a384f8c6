"""N>1 host logic on CPU: domain sharding and max-over-ranks timing, run as
world_size-2 gloo ranks (no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2407_01651_gb300 import shard
from paper_2407_01651_gb300 import workload as wl


def ensemble_sizes():
    # the 96-domain ensemble: 32 each of 256^2, 512x384, 1024x512
    return [256 * 256] * 32 + [512 * 384] * 32 + [1024 * 512] * 32


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shards_partition_and_balance(world):
    sizes = ensemble_sizes()
    parts = shard.shard_domains(sizes, world)
    assert len(parts) == world
    flat = sorted(d for p in parts for d in p)
    assert flat == list(range(len(sizes)))
    loads = [sum(sizes[d] for d in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)


def test_shard_edge_cases():
    assert shard.shard_domains([], 2) == [[], []]
    assert shard.shard_domains([5], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        shard.shard_domains([1, 2], 0)
    with pytest.raises(ValueError):
        shard.job_rate([1], 1, 0.0)
    assert shard.job_rate([10, 20], 3, 2.0) == 45.0
    assert shard.max_over_ranks(3.5) == 3.5


def test_ensemble_layout_sizes_match():
    lays = wl.ensemble_96()
    assert [l.nx * l.ny for l in lays] == ensemble_sizes()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = ensemble_sizes()
        mine = shard.shard_domains(sizes, world)[rank]
        # every rank must compute the same split: gather and compare
        got = [None] * world
        dist.all_gather_object(got, mine)
        ms = 10.0 + rank  # the slower rank decides the job time
        ms_max = shard.max_over_ranks(ms, dist)
        units = [sum(sizes[d] for d in p) for p in got]
        q.put((rank, got, ms_max, shard.job_rate(units, 5, ms_max / 1e3)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_shards_and_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    sizes = ensemble_sizes()
    expect = shard.shard_domains(sizes, world)
    for rank, got, ms_max, rate in res:
        assert got == expect
        assert ms_max == 11.0
        assert rate == pytest.approx(sum(sizes) * 5 / 0.011)
