"""Several contexts on one GPU, each on its own stream and driven by its own host thread (the
way the end-to-end benchmark overlaps one shard's host copies with the others' pushes).

Particles are independent given the field and their Philox streams are keyed by id, so a
population split into shards that keep their ids (the id_base option) must evolve exactly
as it does in one context: the same state bit for bit and the same integer tallies. Each
shard copies its state in and out of host memory every call, as in the benchmark."""
import threading

import numpy as np
import pytest

from paper_2403_06706_gb300 import synth

pytestmark = pytest.mark.gpu
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")
torch = pytest.importorskip("torch")

WIND = synth.WindSpec(64, 32, 64, eps=0.1, n_modes=4)
ENS = (synth.EnsembleSpec(700, lam_au=0.05, r_out_au=2.4),
       synth.EnsembleSpec(333, r0_au=0.6, lat_deg=-20.0, lon_deg=101.0, lam_au=0.3, r_out_au=0.62),
       synth.EnsembleSpec(251, r0_au=1.0, lat_deg=10.0, lon_deg=200.0, lam_au=0.5, energy_law=1,
                          E_lo_keV=20, E_hi_keV=500, E_index=3.0, r_out_au=2.4))
TALLY = dict(cadence=10, n_mu=8, n_E=8, n_r=16, n_age=8, age_max_s=500.0)
CALLS, STEPS = 3, 100


def _context(nodes, ens, id_base, stream):
    c = gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=29, stream=stream, id_base=id_base)
    c.field_load(nodes, WIND.r_min_au, WIND.r_max_au)
    c.set_launch(block=128, steps_per_launch=50, sort_every=50)
    c.inject(list(ens))
    c.tally_arm(**TALLY)
    return c


def _run(c, out):
    host = c.get_state()
    for _ in range(CALLS):
        c.set_state(host)
        c.advance(0.5, STEPS)
        host = c.get_state()
    out["state"], out["tally"] = host, c.tally_read()


def test_threaded_shards_reproduce_one_context():
    nodes = synth.wind_grid(WIND, dtype=np.float32)
    one = {}
    with _context(nodes, ENS, 0, torch.cuda.Stream()) as c:
        _run(c, one)
    shards = [(ENS[:1], 0), (ENS[1:], ENS[0].count)]
    ctxs = [_context(nodes, ens, base, torch.cuda.Stream()) for ens, base in shards]
    outs = [{} for _ in ctxs]
    errors = []

    def work(k):
        try:
            _run(ctxs[k], outs[k])
        except Exception as e:  # re-raised below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(len(ctxs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for c in ctxs:
        c.close()
    if errors:
        raise errors[0]
    a, b = outs[0]["state"], outs[1]["state"]
    for k in one["state"]:
        merged = np.concatenate([a[k], b[k]], axis=-1)
        if k == "ens":
            merged = np.concatenate([a[k], b[k] + 1])
        np.testing.assert_array_equal(merged, one["state"][k], err_msg=k)
    for k in ("h_mer", "h_age", "h_pad", "m_cnt", "m_sin2"):
        merged = np.concatenate([outs[0]["tally"][k], outs[1]["tally"][k]], axis=0)
        np.testing.assert_array_equal(merged, one["tally"][k], err_msg=k)
    assert int(one["tally"]["n_seen"][0]) == int(outs[0]["tally"]["n_seen"][0]) + int(outs[1]["tally"]["n_seen"][0])
    assert one["tally"]["h_mer"].sum() > 0
    assert (one["state"]["ncoll"] > 0).mean() > 0.1
