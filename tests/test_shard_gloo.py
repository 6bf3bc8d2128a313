"""Sharded runs (one process per rank, gloo on CPU): each rank advances its own id range
and the integer tallies are summed across ranks. The result must equal one unsharded run
of all particles, exactly. The per-rank work here is the FP64 oracle (this container has
no GPU); the sharding and reduction logic is the one bench.py and users run on GPUs."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from oracle import AU
from paper_2403_06706_gb300 import shard, synth

WIND = synth.WindSpec(32, 16, 32)
N_PER_RANK = 96
STEPS = 120


def _run(ids_from, count, nodes):
    f = oracle.grid_field(nodes, WIND.r_min_au * AU, WIND.r_max_au * AU)
    p = oracle.params(seed=5)
    ens = [oracle.ensemble(lam_au=0.05, r_out_au=2.0)]
    st = oracle.inject(f, p, ens, [count], id0=ids_from, dt=0.5, n_threads=1)
    T = oracle.TallyArrays(oracle.TallySpec(cadence=10, n_mu=8, n_E=8, n_r=16, n_age=8,
                                            age_max_s=100.0, rwin_lo_au=0.2, rwin_hi_au=0.6,
                                            age_young_s=30.0), 1)
    oracle.advance(f, p, ens, st, 0.0, 0, 0.5, STEPS, tally=T, n_threads=1)
    return st, {k: getattr(T, k) for k in shard.TALLY_KEYS}


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nodes = synth.wind_grid(WIND, dtype=np.float64)
        st, tl = _run(shard.id_base(rank, N_PER_RANK), N_PER_RANK, nodes)
        summed = shard.reduce_tallies(tl)
        q.put((rank, {k: v for k, v in summed.items()}, st["id"].copy(), st["x"].copy()))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_tallies_equal_unsharded_run():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda r: r[0])
    nodes = synth.wind_grid(WIND, dtype=np.float64)
    full, tl_full = _run(0, world * N_PER_RANK, nodes)
    for _, summed, _, _ in res:
        for k in shard.TALLY_KEYS:
            np.testing.assert_array_equal(summed[k], tl_full[k], err_msg=k)
    ids = np.concatenate([r[2] for r in res])
    xs = np.concatenate([r[3] for r in res])
    np.testing.assert_array_equal(ids, full["id"])
    np.testing.assert_array_equal(xs, full["x"])
    assert tl_full["n_seen"][0] == world * N_PER_RANK * (STEPS // 10)


def test_id_base_bounds():
    assert shard.id_base(3, 1000) == 3000
    with pytest.raises(ValueError):
        shard.id_base(2, 2**31)
