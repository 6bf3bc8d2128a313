"""Sharding of one guiding-centre run over several GPUs (one process per GPU).

Test particles are independent given the field (Sect. 1 of the paper: the test-particle
approach), so a run shards by particle: rank r owns a disjoint id range and a replica of
the field, and advances without any collective. Philox streams are keyed by particle id,
so the union of the shards evolves exactly as the unsharded run. The method's only
exchange is the sum of the snapshot tallies, which are integer counts: the sum is exact
and independent of the order of the ranks.
"""
from __future__ import annotations

import numpy as np

TALLY_KEYS = ("h_mer", "h_age", "h_pad", "m_cnt", "m_sin2", "n_seen")


def id_base(rank: int, n_per_rank: int) -> int:
    """First particle id of ``rank`` when every rank injects ``n_per_rank`` particles."""
    if rank < 0 or n_per_rank < 0:
        raise ValueError("rank and n_per_rank must be >= 0")
    base = rank * n_per_rank
    if base + n_per_rank > 2**32:
        raise ValueError("particle ids exceed 32 bits")
    return base


def reduce_tallies(tallies: dict, group=None) -> dict:
    """Sum integer tallies over all ranks of ``group`` (torch.distributed, any backend).

    Counts travel as int64 (sums of uint32 counts and of uint64 fixed-point moments stay
    exact while they fit in 63 bits); the result is returned in the input dtypes."""
    import torch
    import torch.distributed as dist

    out = {}
    for k in TALLY_KEYS:
        a = np.asarray(tallies[k])
        if a.dtype == np.uint64 and a.size and int(a.max()) >= 2**63:
            raise OverflowError(f"tally {k} exceeds 63 bits")
        t = torch.from_numpy(a.astype(np.int64))
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        out[k] = t.numpy().astype(a.dtype)
    return out
