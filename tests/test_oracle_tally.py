"""Pin of the oracle's snapshot tallies (Sect. 3: snapshots every K steps of the particles
(re)born after t_start; the quantities of Figs. 3, 5 and 9: pitch cosine, kinetic energy,
heliocentric distance, age at 1 AU and the young pitch-angle distribution).

The oracle is advanced in chunks of exactly one tally cadence, so that its one snapshot per
chunk falls on the chunk's last step. After each chunk this test reads the state and rebuilds
every histogram from the definitions, with numpy and explicit bin edges (searchsorted, not the
oracle's floor of a scaled coordinate):

* pitch cosine mu = (gamma v_par) / |p/m| with |p/m|^2 = (gamma v_par)^2 + 2 mu_B |B| / m,
  |B| from the oracle's field evaluation (pinned on its own in test_oracle_field.py);
* kinetic energy (gamma - 1) m c^2 = m |p/m|^2 / (gamma + 1), on log-spaced edges over
  [E_lo, E_hi);
* r on linear edges over [r_lo, r_hi);
* the age x energy histogram of the samples in the window [rwin_lo, rwin_hi) at 1 AU;
* the young pitch distribution: window samples younger than age_young with >= 1 collision;
* sin^2 alpha = 1 - mu^2 in 32-bit fixed point, rounded to nearest, summed per r bin;
* n_seen: every sample taken, and those with energy or r out of range.

The run has many collisions and rebirths (lambda 0.02-0.1 AU, one ensemble in a thin shell
around 1 AU), particles born before t_start (not counted until reborn), energies and radii
on both sides of the tally ranges, and three ensembles (the ensemble index of every
histogram). Every array must equal the oracle's bit for bit.
"""
import math

import numpy as np

import oracle
from oracle import AU, C_LIGHT, KEV, M_E
from paper_2403_06706_gb300 import synth


def _bin(x, edges, lo, hi):
    """Index of the bin [edges[k], edges[k+1]) holding x, -1 outside [lo, hi)."""
    k = np.searchsorted(edges, x, side="right") - 1
    k = np.clip(k, 0, edges.size - 2)
    return np.where((x >= lo) & (x < hi), k, -1)


def _expected(f, st, spec: oracle.TallySpec, n_ens: int, t_new: float, acc: dict):
    """Add the snapshot of state ``st`` at time t_new to the histograms in ``acc``."""
    c2 = C_LIGHT * C_LIGHT
    n = st.n
    Bm = np.empty(n)
    for i in range(n):
        B = oracle.field_eval(f, [st["x"][i], st["y"][i], st["z"][i]], t_new)[0]["B"]
        Bm[i] = math.sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2])
    u = st["u"]
    pm2 = u * u + 2.0 * st["mub"] * Bm / M_E          # (|p| / m)^2
    gamma = np.sqrt(1.0 + pm2 / c2)
    mu = u / np.sqrt(pm2)                              # cos(alpha)
    Ek = M_E * pm2 / (gamma + 1.0)                     # (gamma - 1) m c^2
    r = np.sqrt(st["x"] ** 2 + st["y"] ** 2 + st["z"] ** 2)
    age = t_new - st["t_birth"]
    counted = st["t_birth"] >= spec.t_start
    e = st["ens"].astype(np.int64)

    mu_edges = np.linspace(-1.0, 1.0, spec.n_mu + 1)
    im = np.clip(np.searchsorted(mu_edges, mu, side="right") - 1, 0, spec.n_mu - 1)  # mu = 1 in the top bin
    E_lo, E_hi = spec.E_lo_keV * KEV, spec.E_hi_keV * KEV
    E_edges = E_lo * (E_hi / E_lo) ** (np.arange(spec.n_E + 1) / spec.n_E)
    iE = _bin(Ek, E_edges, E_lo, E_hi)
    r_lo, r_hi = spec.r_lo_au * AU, spec.r_hi_au * AU
    ir = _bin(r, np.linspace(r_lo, r_hi, spec.n_r + 1), r_lo, r_hi)
    ia = _bin(age, np.linspace(0.0, spec.age_max_s, spec.n_age + 1), 0.0, spec.age_max_s)
    in_win = (r >= spec.rwin_lo_au * AU) & (r < spec.rwin_hi_au * AU)
    s2 = np.rint((1.0 - mu * mu) * 2.0 ** 32).astype(np.uint64)

    acc["n_seen"][0] += int(counted.sum())
    acc["n_seen"][1] += int((counted & ((iE < 0) | (ir < 0))).sum())
    m = counted & (iE >= 0) & (ir >= 0)
    np.add.at(acc["h_mer"], (e[m], im[m], iE[m], ir[m]), 1)
    m = counted & (ir >= 0)
    np.add.at(acc["m_cnt"], (e[m], ir[m]), 1)
    np.add.at(acc["m_sin2"], (e[m], ir[m]), s2[m])
    m = counted & in_win & (ia >= 0) & (iE >= 0)
    np.add.at(acc["h_age"], (e[m], ia[m], iE[m]), 1)
    m = counted & in_win & (age < spec.age_young_s) & (st["ncoll"] >= 1)
    np.add.at(acc["h_pad"], (e[m], im[m]), 1)
    return int(counted.sum()), int(m.sum())


def test_tally_bins_follow_their_definitions():
    spec_w = synth.WindSpec(64, 32, 64)
    nodes = synth.wind_grid(spec_w, dtype=np.float64)
    f = oracle.grid_field(nodes, spec_w.r_min_au * AU, spec_w.r_max_au * AU)
    p = oracle.params(seed=11)
    ens = [
        oracle.ensemble(r0_au=0.28, lat_deg=24.0, lam_au=0.05, scatter_law=0),
        oracle.ensemble(r0_au=0.95, lat_deg=10.0, lon_deg=30.0, lam_au=0.02, r_in_au=0.5,
                        scatter_law=1, energy_law=1, E_lo_keV=20.0, E_hi_keV=500.0, E_index=3.0),
        oracle.ensemble(r0_au=1.0, lat_deg=-20.0, lon_deg=200.0, E0_keV=30.0, lam_au=0.1,
                        r_in_au=0.97, r_out_au=1.06),
    ]
    counts = [200, 200, 200]
    dt, K, n_chunks, t0 = 0.5, 20, 60, 100.0
    st = oracle.inject(f, p, ens, counts, t0=t0, dt=dt)
    st["t_birth"][1::2] = 0.0  # born before t_start: not sampled until reborn
    spec = oracle.TallySpec(cadence=K, n_mu=16, n_E=24, n_r=48, n_age=20, t_start=50.0,
                            E_lo_keV=20.0, E_hi_keV=200.0, r_lo_au=0.2, r_hi_au=1.05,
                            age_max_s=1200.0, rwin_lo_au=0.9, rwin_hi_au=1.1, age_young_s=300.0)
    T = oracle.TallyArrays(spec, len(ens))
    acc = {k: np.zeros_like(getattr(T, k)) for k in ("h_mer", "h_age", "h_pad", "m_cnt", "m_sin2", "n_seen")}
    t, n_counted, n_young, stats = t0, 0, 0, np.zeros(2, dtype=np.uint64)
    for j in range(n_chunks):
        stats += oracle.advance(f, p, ens, st, t, j * K, dt, K, tally=T)
        t_new = t + float(K) * dt  # the time of the chunk's last step, as the oracle forms it
        a, b = _expected(f, st, spec, len(ens), t_new, acc)
        n_counted += a
        n_young += b
        t = t_new

    # the run exercises every branch of the definitions
    assert stats[0] > 1000 and stats[1] > 100, stats
    assert 0 < n_counted < n_chunks * sum(counts)
    assert n_young > 50 and acc["h_age"].sum() > 500
    assert 0 < acc["n_seen"][1] < acc["n_seen"][0]
    assert all(acc["h_mer"][e].sum() > 0 for e in range(len(ens)))

    for k in acc:
        got = getattr(T, k)
        np.testing.assert_array_equal(got, acc[k], err_msg=k)
