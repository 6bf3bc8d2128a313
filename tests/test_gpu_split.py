"""The split-step push (the neural field's path) on the GPU.

* With the grid evaluated through the sample buffers (GC_FIELD_GRID_SAMPLED) the split-step
  kernels run the same phases on the same field values as the fused push. The injection
  state agrees bit for bit; after 300 steps the integer state (events, collision counts,
  ids, flags), the tally counts and the counters agree exactly, and the floating-point state
  and the tallied sums of sin^2 alpha to a few FP32 roundings per step (the compiler may
  contract a product and a sum into one FMA differently in the two kernels, and a
  collision's new momentum carries such a difference on): 1e-7 of r for positions, 1e-6 of
  the scale for the rest. With collisions in the fixed frame and in the wind frame, and with
  the two-fluid parallel field.
* With the neural field the push is compared with the FP64 oracle running the same network
  (oracle.siren_field, BF16 reading): one short run, increments of R and gamma v_par
  measured against their own size. The network's BF16 noise (about 4e-4 RMS and 7e-3 at
  worst of the field, tests/test_gpu_siren.py) bounds what can agree.
"""
import numpy as np
import pytest

import oracle
from _cases import oracle_ensembles
from oracle import AU
from paper_2403_06706_gb300 import synth

pytestmark = pytest.mark.gpu
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")
torch = pytest.importorskip("torch")

WIND = synth.WindSpec(64, 32, 64, eps=0.1, n_modes=4)
ENS = (synth.EnsembleSpec(700, lam_au=0.05, r_out_au=2.4),
       synth.EnsembleSpec(333, r0_au=0.6, lat_deg=-20.0, lon_deg=101.0, lam_au=0.3, r_out_au=0.62))
TALLY = dict(cadence=25, n_mu=8, n_E=8, n_r=16, n_age=8, age_max_s=500.0)


def _run(source, nodes, n_steps=150, calls=2, wind_u=0.0, ideal=True):
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=17, wind_u=wind_u) as c:
        c.field_load(nodes, WIND.r_min_au, WIND.r_max_au, ideal=ideal)
        c.set_launch(block=128, steps_per_launch=n_steps, sort_every=0)
        if source != gcpush.FIELD_GRID:
            c.field_select(source)
        c.inject(list(ENS))
        st0 = c.get_state()
        c.tally_arm(**TALLY)
        for _ in range(calls):
            c.advance(0.5, n_steps)
        return st0, c.get_state(), c.tally_read(), c.stats()


@pytest.mark.parametrize("wind_u,ideal", [(0.0, True), (4.0e5, True), (0.0, 2)])
def test_grid_sampled_split_push_reproduces_fused_push(wind_u, ideal):
    spec = WIND if ideal is True else synth.WindSpec(64, 32, 64, eps=0.1, n_modes=4, phi1_v=500.0)
    nodes = synth.wind_grid(spec, dtype=np.float32)
    a0, a, ta, sa = _run(gcpush.FIELD_GRID, nodes, wind_u=wind_u, ideal=ideal)
    b0, b, tb, sb = _run(gcpush.FIELD_GRID_SAMPLED, nodes, wind_u=wind_u, ideal=ideal)
    for k in a0:
        np.testing.assert_array_equal(a0[k], b0[k], err_msg="after injection: " + k)
    r = np.sqrt(a["x"] ** 2 + a["y"] ** 2 + a["z"] ** 2)
    for k in a:
        if a[k].dtype.kind in "ui":
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)
            continue
        if k in ("x", "y", "z"):
            err = np.abs(a[k] - b[k]) / r
            bound = 1e-7
        else:
            scale = np.abs(a[k]).max(axis=-1, keepdims=True) if a[k].ndim == 2 else np.abs(a[k]).max()
            err = np.abs(a[k] - b[k]) / np.maximum(scale, 1e-300)
            bound = 1e-6
        print(k, float(err.max()))
        assert err.max() <= bound, (k, err.max())
    for k in ta:
        if k == "m_sin2":
            # sums of sin^2(alpha) in 2^-32 units: the same last-bit differences
            np.testing.assert_allclose(ta[k], tb[k], rtol=1e-6, err_msg=k)
        else:
            np.testing.assert_array_equal(ta[k], tb[k], err_msg=k)
    assert sa["collisions"] == sb["collisions"] > 0
    assert sa["rebirths"] == sb["rebirths"] > 0
    assert sb["field_evals"] >= 2 * 1033 * 300


RS_AU, B_S, E_S = 2.5, 3.5e-9, 3.5e-9 * 4.0e5


def test_neural_push_matches_oracle_on_the_same_network():
    w = synth.WindSpec(64, 32, 64)
    nodes = synth.wind_grid(w, dtype=np.float32)
    ens = (synth.EnsembleSpec(256, lam_au=0.5, r_out_au=2.4),
           synth.EnsembleSpec(256, r0_au=0.5, lat_deg=10.0, lon_deg=30.0, lam_au=0.2, r_out_au=2.4))
    n_steps = 10
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=5) as c:
        c.field_load(nodes, w.r_min_au, w.r_max_au)
        c.siren_set(synth.siren_init(seed=9), omega0=30.0, r_max_au=RS_AU, B_scale=B_S, E_scale=E_S)
        rng = np.random.default_rng(2)
        r = (rng.uniform(0.1**3, 0.96**3, 1 << 16)) ** (1 / 3)
        v = rng.normal(size=(1 << 16, 3))
        xs = (v / np.linalg.norm(v, axis=1, keepdims=True) * r[:, None]).astype(np.float32)
        loss = c.field_fit(xs, n_epochs=30, batch=4096, lr=2e-4)
        print("fit loss", loss[0], loss[-1])
        P = c.siren_get()
        c.field_select(gcpush.FIELD_SIREN)
        c.inject(list(ens))
        g0 = c.get_state()
        c.advance(0.5, n_steps)
        g1 = c.get_state()
        st = c.stats()
    assert st["field_evals"] >= 2 * 512 * (n_steps + 1)
    f = oracle.siren_field(P, 30.0, RS_AU * AU, B_S, E_S, bf16=True)
    p = oracle.params(seed=5)
    oe = oracle_ensembles(ens)
    o0 = oracle.inject(f, p, oe, [e.count for e in ens], id0=0, dt=0.5)
    # injection: mu_B from |B| at the site, start-up history from the network
    rel_u = np.abs(g0["u"] - o0["u"]) / np.abs(o0["u"]).max()
    rel_mub = np.abs(g0["mub"] - o0["mub"]) / np.abs(o0["mub"]).max()
    print("injection: u", rel_u.max(), "mub", rel_mub.max())
    assert rel_u.max() < 1e-12 and rel_mub.max() < 2e-2
    o1 = o0.copy()
    oracle.advance(f, p, oe, o1, 0.0, 0, 0.5, n_steps)
    same = (g1["ncoll"] == o1["ncoll"]) & (g1["t_birth"] == o1["t_birth"])
    assert same.mean() > 0.97
    R0 = np.stack([o0["x"], o0["y"], o0["z"]])
    dRg = np.stack([g1["x"], g1["y"], g1["z"]]) - R0
    dRo = np.stack([o1["x"], o1["y"], o1["z"]]) - R0
    eR = np.linalg.norm(dRg - dRo, axis=0)[same] / np.linalg.norm(dRo, axis=0)[same]
    du_scale = np.abs(o1["u"] - o0["u"])[same] + 1e-3 * np.abs(o0["u"])[same]
    eu = np.abs((g1["u"] - g0["u"]) - (o1["u"] - o0["u"]))[same] / du_scale
    print("increments: R rms", np.sqrt(np.mean(eR**2)), "max", eR.max(), "| u rms", np.sqrt(np.mean(eu**2)),
          "max", eu.max())
    assert np.sqrt(np.mean(eR**2)) < 2e-3 and eR.max() < 3e-2
    assert np.sqrt(np.mean(eu**2)) < 2e-2 and eu.max() < 0.2
