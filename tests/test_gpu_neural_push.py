"""The neural-field push through the library (gc_field_select(GC_FIELD_SIREN), the split-step
kernels with the tensor-core network evaluation), with a SIREN trained on the GPU by the
library's own kernels on the 64x32x64 Parker grid.

1. Against the oracle running the same network (oracle.siren_field in the BF16 reading) over
   10^3 steps on 1024 electrons (two ensembles, with collisions and rebirths). The two
   evaluations of the network differ by rounding flips of the BF16 values carried between
   layers (tests/test_gpu_siren.py holds them to 1e-3 RMS / 2e-2 max of the outputs' RMS for
   values and 2e-3 / 3e-2 for the Jacobian). Along a trajectory that noise enters every
   step: a field direction off by e moves the position by e per unit of path travelled and
   the mirror force by e_J of its size. Even if the noise kept one sign over the whole path,
   the position would stay within e L (L: the path travelled since the particle's last
   (re)birth, |v| times the time; for the diffusive particles of the short mean free path
   it is far longer than their net displacement) and gamma v_par within e_J of |p|/m. The
   test holds the particles with the same collision and rebirth history as the oracle
   (>= 95 % of them) to those bounds with e = 1e-3, e_J = 2e-3 (RMS) and the maxima at 2e-2,
   3e-2. (The training accumulates its gradients with floating-point atomics, so each run
   trains a slightly different network; the bounds hold for any of them.)
2. What the trained network gains over the grid it was trained on, on the path users run:
   the same electrons with E = 0 and no scattering, pushed by gc_advance in FP32 through the
   grid and through the network at dt = 2, 1 and 0.5 s for 240 s. With E = 0 gamma is
   constant on the exact motion. The grid's interpolant has a gradient that jumps at cell
   faces, so the predictor-corrector is first order there and gamma drifts by an amount that
   shrinks with dt. In exact arithmetic the network is smooth and keeps the third order and
   1e-9 in gamma (tests/test_gpu_gain.py, through the oracle); through the BF16 tensor-core
   evaluation the network's Jacobian carries ~2e-3 of rounding noise, which the mirror force
   turns into an energy error of a few 1e-5 (median) at every dt: a floor, not an order. The
   test pins both behaviours (the finding is a loss of the smoothness gain on this path).
"""
import numpy as np
import pytest

import oracle
from _cases import oracle_ensembles
from oracle import AU, C_LIGHT, M_E
from paper_2403_06706_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")

W = synth.WindSpec(64, 32, 64)
OMEGA0 = 30.0


@pytest.fixture(scope="module")
def trained():
    nodes = synth.wind_grid(W, dtype=np.float32)
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED) as c:
        c.field_load(nodes, W.r_min_au, W.r_max_au)
        c.siren_set(synth.siren_init(seed=11), omega0=OMEGA0, r_max_au=W.r_max_au, B_scale=W.B1,
                    E_scale=W.B1 * W.u_sw)
        loss = c.field_fit(synth.siren_samples(1 << 18, W), n_epochs=40, batch=8192, lr=2e-4)
        P = c.siren_get()
    assert loss[-1] < 0.05 * loss[0]
    return nodes, P


def _siren_context(nodes, P, E_scale, **opt):
    c = gcpush.Context(precision=gcpush.PREC_FP32_MIXED, **opt)
    c.field_load(nodes, W.r_min_au, W.r_max_au)
    c.siren_set(P, omega0=OMEGA0, r_max_au=W.r_max_au, B_scale=W.B1, E_scale=E_scale)
    c.field_select(gcpush.FIELD_SIREN)
    return c


def _absB(f, st):
    return np.array([np.linalg.norm(oracle.field_eval(f, [st["x"][i], st["y"][i], st["z"][i]])[0]["B"])
                     for i in range(st["x"].shape[0])])


def test_neural_push_matches_oracle_over_1000_steps(trained):
    nodes, P = trained
    ens = (synth.EnsembleSpec(512, lam_au=0.5, r_out_au=2.4),
           synth.EnsembleSpec(512, r0_au=0.6, lat_deg=-20.0, lon_deg=101.0, lam_au=0.05, r_out_au=1.2))
    n_steps = 1000
    with _siren_context(nodes, P, W.B1 * W.u_sw, seed=7, dt_init=0.5) as c:
        c.inject(list(ens))
        g0 = c.get_state()
        for _ in range(2):
            c.advance(0.5, n_steps // 2)
        g1 = c.get_state()
    f = oracle.siren_field(P, OMEGA0, W.r_max_au * AU, W.B1, W.B1 * W.u_sw, bf16=True)
    p = oracle.params(seed=7)
    oe = oracle_ensembles(ens)
    o = oracle.inject(f, p, oe, [e.count for e in ens], dt=0.5)
    np.testing.assert_array_equal(g0["u"], o["u"])
    o0 = o.copy()
    oracle.advance(f, p, oe, o, 0.0, 0, 0.5, n_steps)

    same = (g1["ncoll"] == o["ncoll"]) & (g1["t_birth"] == o["t_birth"]) & (g1["event"] == o["event"])
    print("same history", same.mean(), "collisions", int(o["ncoll"].sum()),
          "rebirths", int((o["t_birth"] > 0).sum()))
    assert same.mean() >= 0.95 and int(o["ncoll"].sum()) > 100
    R = lambda s: np.stack([s["x"], s["y"], s["z"]])  # noqa: E731
    pm = np.sqrt(o0["u"] ** 2 + 2 * o0["mub"] * _absB(f, o0) / M_E)  # |p|/m at injection
    speed = pm / np.sqrt(1.0 + (pm / C_LIGHT) ** 2)  # |v|, kept by the inertial-frame collisions
    path = speed * (n_steps * 0.5 - o["t_birth"])     # travelled since the last (re)birth
    eR = np.linalg.norm(R(g1) - R(o), axis=0) / path
    eu = np.abs(g1["u"] - o["u"]) / pm
    emu = np.abs(g1["mub"] - o["mub"]) / np.maximum(np.abs(o["mub"]), 1e-3 * np.abs(o0["mub"]).max())
    for name, e in (("R", eR), ("u", eu), ("mu_B", emu)):
        e = e[same]
        print(f"{name}: rms {np.sqrt(np.mean(e ** 2)):.2e}  p99 {np.percentile(e, 99):.2e}  max {e.max():.2e}")
    assert np.sqrt(np.mean(eR[same] ** 2)) < 1e-3 and eR[same].max() < 2e-2
    assert np.sqrt(np.mean(eu[same] ** 2)) < 2e-3 and eu[same].max() < 3e-2
    assert np.sqrt(np.mean(emu[same] ** 2)) < 2e-3 and emu[same].max() < 3e-2


def _gamma(st, absB):
    return np.sqrt(1.0 + (st["u"] ** 2 + 2.0 * st["mub"] * absB / M_E) / C_LIGHT ** 2)


def _absB_network(c, st):
    """|B| of the library's own network evaluation at the particles' positions (the values
    the push used, up to the float rounding of the position)."""
    import torch

    R = np.stack([st["x"], st["y"], st["z"]], axis=1) / (W.r_max_au * AU)
    x = torch.from_numpy(R.astype(np.float32)).cuda()
    out = torch.empty((R.shape[0], 24), dtype=torch.float32, device="cuda")
    c.siren_field(x, out)
    torch.cuda.synchronize()
    return np.linalg.norm(out[:, 0:3].double().cpu().numpy(), axis=1)


def test_network_gain_through_the_library(trained):
    nodes, P = trained
    nodes0 = nodes.copy()
    nodes0[..., 3:6] = 0.0  # E = 0 in the grid ...
    E_off = 1e-300          # ... and in the network (E = E_scale y_E rounds to 0 in float)
    ens = (synth.EnsembleSpec(64, lam_au=0.5, r_out_au=2.4),)
    fg = oracle.grid_field(nodes0.astype(np.float64), W.r_min_au * AU, W.r_max_au * AU)
    fx = oracle.siren_field(P, OMEGA0, W.r_max_au * AU, W.B1, E_off, bf16=False)  # the exact network
    T = 240.0
    out = {}
    for name in ("grid", "network", "network_exact_B"):
        pos, egy = {}, {}
        for dt in (2.0, 1.0, 0.5):
            opt = dict(seed=1, dt_init=dt, no_scatter=True, no_rebirth=True)
            if name == "grid":
                c = gcpush.Context(precision=gcpush.PREC_FP32_MIXED, **opt)
                c.field_load(nodes0, W.r_min_au, W.r_max_au)
            else:
                c = _siren_context(nodes, P, E_off, **opt)
            with c:
                c.inject(list(ens))
                s0 = c.get_state()
                c.advance(dt, int(round(T / dt)))
                s1 = c.get_state()
                if name == "grid":
                    b0, b1 = _absB(fg, s0), _absB(fg, s1)
                elif name == "network":
                    b0, b1 = _absB_network(c, s0), _absB_network(c, s1)
                else:
                    b0, b1 = _absB(fx, s0), _absB(fx, s1)
            pos[dt] = np.stack([s1["x"], s1["y"], s1["z"]])
            e = np.abs(_gamma(s1, b1) / _gamma(s0, b0) - 1.0)
            egy[dt] = (float(e.max()), float(np.median(e)))
        d = [np.linalg.norm(pos[a] - pos[b], axis=0).max() for a, b in ((2.0, 1.0), (1.0, 0.5))]
        out[name] = (float(np.log2(d[0] / d[1])), egy)
        print(f"{name}: convergence order {out[name][0]:.2f}, |gamma/gamma0 - 1| (max, median) by dt {egy}")
    (order_g, egy_g), (order_s, egy_s), (order_x, egy_x) = out["grid"], out["network"], out["network_exact_B"]
    # the grid: first order (the interpolant's gradient jumps at cell faces), its energy
    # error shrinking with dt
    assert order_g < 1.5 and egy_g[0.5][1] < 0.6 * egy_g[2.0][1]
    # the network on the BF16 tensor-core path: a floor set by the evaluation noise of its
    # Jacobian (which drives the mirror force), the same at every dt within a factor 2,
    # whether gamma is taken with the library's |B| or with the exact network's; its level
    # (3e-5 to 1e-4 in the median over the networks the non-deterministic training gives)
    # within 5e-4
    for e in (egy_s, egy_x):
        med = [e[dt][1] for dt in (2.0, 1.0, 0.5)]
        assert max(med) < 2.0 * min(med) and max(med) < 5e-4
