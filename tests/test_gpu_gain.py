"""What the trained neural field gains over the grid it was trained on.

A SIREN is trained on the GPU (the project's own forward, backward and Adam kernels) on
samples of the 64x32x64 Parker grid. Then the FP64 oracle integrates the same electrons,
with E = 0 and without scattering, through the trilinear grid and through the trained
network, at dt = 2, 1 and 0.5 s for 240 s:

* convergence order of the positions (Richardson differences between successive dt): the
  paper's predictor-corrector is third order on a smooth field (the network is C-infinity),
  while the trilinear interpolant's gradient jumps at every cell face, so the drift and
  mirror terms of Eqs. 1-2 are discontinuous there and the order drops to about one;
* energy conservation: with E = 0 the exact motion keeps gamma constant (Eq. 2 with
  E_par = 0 and v.E = 0); the error of the integration is what remains;
* footprint: the network's BF16 weights against the 256x128x256 FP32 grid.
The field error the network pays for this is measured in the benchmark (field_rel_rms).
"""
import numpy as np
import pytest

import oracle
from _cases import oracle_ensembles
from oracle import AU, C_LIGHT, M_E
from paper_2403_06706_gb300 import synth

pytestmark = pytest.mark.gpu
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")


def _gamma(f, st):
    g = np.empty(st.n)
    for i in range(st.n):
        s, _ = oracle.field_eval(f, np.array([st["x"][i], st["y"][i], st["z"][i]]))
        B = np.linalg.norm(s["B"])
        g[i] = np.sqrt(1.0 + (st["u"][i] ** 2 + 2.0 * st["mub"][i] * B / M_E) / C_LIGHT**2)
    return g


def _study(f, oe, counts, p, T=240.0, dts=(2.0, 1.0, 0.5)):
    """convergence order of the positions at time T and the energy error per dt"""
    pos, egy = {}, {}
    for dt in dts:
        st = oracle.inject(f, p, oe, counts, id0=0, dt=dt)
        g0 = _gamma(f, st)
        oracle.advance(f, p, oe, st, 0.0, 0, dt, int(round(T / dt)))
        pos[dt] = np.stack([st["x"], st["y"], st["z"]])
        egy[dt] = float(np.abs(_gamma(f, st) / g0 - 1.0).max())
    d = [np.linalg.norm(pos[a] - pos[b], axis=0).max() for a, b in zip(dts, dts[1:])]
    return float(np.log2(d[0] / d[1])), egy


def test_trained_network_is_smooth_where_the_grid_is_not():
    w = synth.WindSpec(64, 32, 64)
    nodes = synth.wind_grid(w, dtype=np.float32)
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED) as c:
        c.field_load(nodes, w.r_min_au, w.r_max_au)
        c.siren_set(synth.siren_init(seed=11), omega0=30.0, r_max_au=w.r_max_au, B_scale=w.B1,
                    E_scale=w.B1 * w.u_sw)
        loss = c.field_fit(synth.siren_samples(1 << 18, w), n_epochs=40, batch=8192, lr=2e-4)
        P = c.siren_get()
    print("fit loss", loss[0], "->", loss[-1])
    assert loss[-1] < 0.05 * loss[0]

    ens = (synth.EnsembleSpec(16, lam_au=0.5, r_out_au=2.4),)
    oe = oracle_ensembles(ens)
    counts = [e.count for e in ens]
    p = oracle.params(seed=1, no_scatter=True, no_rebirth=True)
    # E = 0 in both fields: zeroed E channels; the network's E scaled away
    nodes0 = nodes.astype(np.float64)
    nodes0[..., 3:6] = 0.0
    fg = oracle.grid_field(nodes0, w.r_min_au * AU, w.r_max_au * AU)
    fs = oracle.siren_field(P, 30.0, w.r_max_au * AU, w.B1, 1e-300)
    order_g, egy_g = _study(fg, oe, counts, p)
    order_s, egy_s = _study(fs, oe, counts, p)
    print(f"convergence order: grid {order_g:.2f}, network {order_s:.2f}")
    print("energy error |gamma/gamma0 - 1| (dt: grid, network):",
          {dt: (egy_g[dt], egy_s[dt]) for dt in egy_g})
    assert order_s > 2.5
    assert order_g < order_s - 1.0
    assert egy_s[0.5] < 0.01 * egy_g[0.5]
    # footprint against the 256x128x256 FP32 grid of the perturbed workload
    net_bytes = 2 * (3 * 65536 + 2048) + 4 * (768 + 4 * 256 + 8)
    assert net_bytes * 500 < 256 * 128 * 256 * 8 * 4
