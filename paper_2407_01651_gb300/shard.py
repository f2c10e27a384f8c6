"""Host-side sharding of independent domains across ranks (one GPU each).

The coupled step has no exchange between domains of an ensemble, so N ranks
split the domain list and step their shares with no collective on the data
path.  The only collective is a MAX of the per-rank timings (and of the
end-to-end wall time), so that the reported rate is whole-job work divided by
the slowest rank.

The split is deterministic and identical on every rank: longest-processing-
time first over site counts (ties broken by domain index), which keeps the
per-rank site counts within one domain's size of each other.
"""
from __future__ import annotations

from typing import Sequence


def shard_domains(sizes: Sequence[int], world: int) -> list[list[int]]:
    """Assign domain indices (by site count ``sizes[d]``) to ``world`` ranks.

    Returns one ascending index list per rank; together they cover every
    domain exactly once.  Raises ValueError for world < 1 or negative sizes."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if any(s < 0 for s in sizes):
        raise ValueError("domain sizes must be >= 0")
    order = sorted(range(len(sizes)), key=lambda d: (-sizes[d], d))
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for d in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(d)
        load[r] += sizes[d]
    return [sorted(x) for x in out]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """MAX of a per-rank scalar over the default process group (identity when
    ``dist`` is None or not initialised)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: Sequence[int], steps: int, seconds_max: float) -> float:
    """Whole-job rate: units all ranks processed per step, times steps, over
    the slowest rank's time (units per second)."""
    if seconds_max <= 0:
        raise ValueError("seconds_max must be > 0")
    return float(sum(units_per_rank)) * steps / seconds_max
