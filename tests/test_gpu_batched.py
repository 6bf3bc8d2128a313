"""Batched ensembles in one launch, graph replay, and the launch autotuner.

* 64 ensembles of uneven size (10^3 - 10^5 electrons, log-uniform energies 10-300 keV and
  mean free paths 0.05-2 AU, sites at r 0.1-0.5 AU and latitudes -60..60 deg) advance
  together on the perturbed 256x128x256 field, replayed from a CUDA graph; the oracle
  recomputes 16 particles of every ensemble (ids keyed streams make subsets exact).
* Graph replay gives the same bits as the direct path over repeated calls, with cell
  sorts (which swap the state buffers) and tallies.
* gc_autotune changes the launch shape only: state, clock, counters and tallies are as
  before, and the chosen shape runs.
"""
import numpy as np
import pytest

import oracle
from _cases import compare_states, momentum_scale, oracle_ensembles
from oracle import AU
from paper_2403_06706_gb300 import synth

pytestmark = pytest.mark.gpu
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")


@pytest.fixture(scope="module")
def c3():
    wl = synth.c3_batched()
    return wl, synth.wind_grid(wl.wind, dtype=np.float32)


def test_batched_64_ensembles_graph_replay_parity(c3):
    wl, nodes = c3
    n_steps, calls = 500, 2
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=wl.seed, dt_init=wl.dt) as c:
        c.field_load(nodes, wl.wind.r_min_au, wl.wind.r_max_au)
        c.inject(list(wl.ensembles))
        c.set_launch(block=128, steps_per_launch=250, sort_every=250)
        c.set_graph(True)
        for _ in range(calls):
            c.advance(wl.dt, n_steps)
        g = c.get_state()
        st_ = c.stats()
    assert st_["push_launches"] == calls * (n_steps // 250)
    n_s = 16
    first = np.cumsum([0] + [e.count for e in wl.ensembles])[:-1]
    pick = np.concatenate([f + np.arange(n_s) for f in first])
    gs = {k: (v[:, pick] if v.ndim == 2 else v[pick]) for k, v in g.items()}
    f = oracle.grid_field(nodes, wl.wind.r_min_au * AU, wl.wind.r_max_au * AU)
    p = oracle.params(seed=wl.seed)
    oe = oracle_ensembles(wl.ensembles)
    parts = []
    for k, f0 in enumerate(first):
        counts = [0] * len(oe)
        counts[k] = n_s
        parts.append(oracle.inject(f, p, oe, counts, id0=int(f0), dt=wl.dt))
    st = oracle.StateArrays({k: np.concatenate([q[k] for q in parts], axis=-1) for k in parts[0].arrays})
    np.testing.assert_array_equal(gs["ens"], st["ens"])
    oracle.advance(f, p, oe, st, 0.0, 0, wl.dt, n_steps * calls)
    div = (gs["ncoll"] != st["ncoll"]) | (gs["event"] != st["event"]) | (gs["t_birth"] != st["t_birth"])
    assert div.mean() <= 0.02, div.sum()
    lam = np.array([e.lam_au for e in wl.ensembles])[st["ens"].astype(int)] * AU
    err = compare_states(gs, st.arrays, 1e-4, momentum_scale(st, nodes, wl.wind, wl.ensembles),
                         skip=div, lam=lam)
    for k, v in err.items():
        assert v < (1e-3 if k.startswith("F") else 1e-4), (k, v, err)


WIND = synth.WindSpec(64, 32, 64)
ENS = (synth.EnsembleSpec(700, lam_au=0.05, r_out_au=2.4),
       synth.EnsembleSpec(333, r0_au=0.6, lat_deg=-20.0, lon_deg=101.0, lam_au=0.3, r_out_au=2.4))
TALLY = dict(cadence=50, n_mu=8, n_E=8, n_r=16, n_age=8, age_max_s=500.0)


def _run(graph, nodes, calls=4, n=120, nodes1=None):
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=21) as c:
        c.field_load(nodes, WIND.r_min_au, WIND.r_max_au)
        if nodes1 is not None:
            c.field_load_next(nodes1, 0.0, 300.0)
        c.inject(list(ENS))
        c.set_launch(block=64, steps_per_launch=60, sort_every=90, grid_waves=2)
        c.tally_arm(**TALLY)
        c.set_graph(graph)
        for _ in range(calls):
            c.advance(0.5, n)
        return c.get_state(), c.tally_read(), c.stats()


@pytest.mark.parametrize("time_dependent", [False, True])
def test_graph_replay_is_bitwise_equal_to_direct_path(time_dependent):
    """Graph replay against direct launches; with a time-dependent field the replayed
    kernels take the call's time from device memory, so the blend must still follow it."""
    nodes = synth.wind_grid(WIND, dtype=np.float32)
    nodes1 = None
    if time_dependent:
        nodes1 = synth.wind_grid(synth.WindSpec(64, 32, 64, B1=4.2e-9, u_sw=5.0e5, eps=0.15, n_modes=4,
                                                seed=3), dtype=np.float32)
    a, ta, sa = _run(False, nodes, nodes1=nodes1)
    b, tb, sb = _run(True, nodes, nodes1=nodes1)
    if time_dependent:
        c, _, _ = _run(False, nodes)
        assert np.abs(a["u"] - c["u"]).max() > 0
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    for k in ta:
        np.testing.assert_array_equal(ta[k], tb[k], err_msg=k)
    for k in ("collisions", "rebirths", "particle_steps", "step", "t", "push_launches", "sorts"):
        assert sa[k] == sb[k], k


def test_autotune_keeps_state_and_chooses_a_working_shape():
    nodes = synth.wind_grid(WIND, dtype=np.float32)
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=3) as c:
        c.field_load(nodes, WIND.r_min_au, WIND.r_max_au)
        c.inject(list(ENS))
        c.tally_arm(**TALLY)
        c.advance(0.5, 100)
        before, tb, sb = c.get_state(), c.tally_read(), c.stats()
        best = c.autotune(0.5, trial_steps=100)
        after, ta, sa = c.get_state(), c.tally_read(), c.stats()
        for k in before:
            np.testing.assert_array_equal(before[k], after[k], err_msg=k)
        for k in tb:
            np.testing.assert_array_equal(tb[k], ta[k], err_msg=k)
        for k in ("collisions", "rebirths", "particle_steps", "step", "t", "flags_or"):
            assert sb[k] == sa[k], k
        assert best["trials"] == 24 and best["particle_steps_per_s"] > 0
        assert best["block"] in (64, 128) and best["grid_waves"] in (0, 1, 2, 4)
        c.advance(0.5, 50)  # the chosen shape runs
        assert c.stats()["step"] == 150
