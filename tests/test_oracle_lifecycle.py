"""Pins of the oracle's particle lifecycle (Sect. 3) and tallies.

* injection at the stated site, energy and pitch laws; the start-up history of Sect. 2.2
  (F^n = F(X^n), F^{n-1} = F(X^n - dt F^n));
* the same start-up after a collision;
* rebirth on leaving the shell with the initial velocity, and its precedence over a
  collision in the same step;
* T11: the number of snapshot samples (every K steps, particles born after t_start), and
  the paper's own count of 9.4e6 snapshot electrons (Sect. 3).
"""
import json
import os

import numpy as np
from scipy import stats

import oracle
from oracle import AU, C_LIGHT, KEV, M_E
from paper_2403_06706_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")


def _parker_grid_field():
    spec = synth.WindSpec(64, 32, 64)
    nodes = synth.wind_grid(spec, dtype=np.float64)
    return spec, oracle.grid_field(nodes, spec.r_min_au * AU, spec.r_max_au * AU)


def _gamma(f, p, st, i):
    R = np.array([st["x"][i], st["y"][i], st["z"][i]])
    return oracle.rhs(f, p, np.r_[R, st["u"][i]], st["mub"][i])[1][0]


def test_injection_state():
    spec, f = _parker_grid_field()
    p = oracle.params(seed=0)
    ens = [oracle.ensemble(r0_au=0.28, lat_deg=24.0, lon_deg=0.0, E0_keV=81.0, lam_au=0.5),
           oracle.ensemble(r0_au=0.4, lat_deg=-10.0, lon_deg=33.0, E0_keV=30.0, lam_au=0.1,
                           mu_law=1)]
    counts = [3000, 10]
    dt = 0.5
    st = oracle.inject(f, p, ens, counts, id0=100, t0=5.0, dt=dt)
    n0 = counts[0]
    lat = np.deg2rad(24)
    np.testing.assert_allclose(st["x"][:n0], 0.28 * AU * np.cos(lat), rtol=1e-15)
    np.testing.assert_allclose(st["z"][:n0], 0.28 * AU * np.sin(lat), rtol=1e-15)
    np.testing.assert_array_equal(st["y"][:n0], 0.0)
    np.testing.assert_array_equal(st["id"], 100 + np.arange(st.n))
    np.testing.assert_array_equal(st["ens"], [0] * n0 + [1] * 10)
    np.testing.assert_array_equal(st["event"], 2)
    np.testing.assert_array_equal(st["t_birth"], 5.0)
    np.testing.assert_array_equal(st["h_prev"], dt)
    gam0 = 1 + 81 * KEV / (M_E * C_LIGHT**2)
    for i in range(0, n0, 97):
        assert abs(_gamma(f, p, st, i) - gam0) < 1e-14 * gam0
    pm = C_LIGHT * np.sqrt(gam0**2 - 1)
    mu0 = st["u"][:n0] / pm
    assert mu0.min() > 0 and mu0.max() <= 1
    assert stats.kstest(mu0, "uniform").pvalue > 1e-3
    # mu0 = 1: all momentum parallel, mu_B = 0 (alpha = 0, Sect. 3)
    np.testing.assert_array_equal(st["mub"][n0:], 0.0)
    # start-up history
    for i in (0, 1, 5, n0 + 3):
        X = np.array([st["x"][i], st["y"][i], st["z"][i], st["u"][i]])
        F0, aux, _ = oracle.rhs(f, p, X, st["mub"][i])
        np.testing.assert_array_equal(st["F0"][:, i], F0)
        F1, _, _ = oracle.rhs(f, p, X - dt * F0, st["mub"][i])
        np.testing.assert_array_equal(st["F1"][:, i], F1)
        assert st["vpar"][i] == aux[1]
    np.testing.assert_array_equal(st["u_inj"], st["u"])
    np.testing.assert_array_equal(st["mub_inj"], st["mub"])


def test_power_law_energies():
    f = oracle.analytic_field(B_unif=(0, 0, 5e-9))
    p = oracle.params(seed=4)
    ens = [oracle.ensemble(energy_law=1, E_lo_keV=20.0, E_hi_keV=500.0, E_index=3.0)]
    st = oracle.inject(f, p, ens, [5000])
    pm2 = st["u"] ** 2 + 2 * st["mub"] * 5e-9 / M_E
    E = (np.sqrt(1 + pm2 / C_LIGHT**2) - 1) * M_E * C_LIGHT**2 / KEV
    a = -2.0
    cdf = lambda e: (e**a - 20.0**a) / (500.0**a - 20.0**a)
    assert E.min() >= 20.0 * (1 - 1e-12) and E.max() <= 500.0 * (1 + 1e-12)
    assert stats.kstest(E, cdf).pvalue > 1e-3


def test_restart_after_collision():
    spec, f = _parker_grid_field()
    p = oracle.params(seed=2)
    ens = [oracle.ensemble(lam_au=0.002, r_out_au=2.4)]
    st = oracle.inject(f, p, ens, [200], dt=0.5)
    before = st.copy()
    oracle.advance(f, p, ens, st, 0.0, 0, 0.5, 1)
    # the same step with scattering off reaches the same R^{n+1} with the old (u, mu_B)
    free = before.copy()
    p_free = oracle.params(seed=2, no_scatter=True)
    oracle.advance(f, p_free, ens, free, 0.0, 0, 0.5, 1)
    hit = np.nonzero(st["ncoll"] > before["ncoll"])[0]
    assert hit.size > 5
    for i in hit[:10]:
        X = np.array([st["x"][i], st["y"][i], st["z"][i], st["u"][i]])
        F0, aux, _ = oracle.rhs(f, p, X, st["mub"][i])
        np.testing.assert_array_equal(st["F0"][:, i], F0)
        F1, _, _ = oracle.rhs(f, p, X - 0.5 * F0, st["mub"][i])
        np.testing.assert_array_equal(st["F1"][:, i], F1)
        assert st["event"][i] == before["event"][i] + 1
        # |p| unchanged by the collision at R^{n+1}
        assert (st["x"][i], st["y"][i], st["z"][i]) == (free["x"][i], free["y"][i], free["z"][i])
        g_pre = _gamma(f, p, free, i)
        assert abs(_gamma(f, p, st, i) - g_pre) < 1e-13 * (g_pre - 1)


def test_rebirth_resets_state_and_takes_precedence():
    spec, f = _parker_grid_field()
    p = oracle.params(seed=9)
    # tiny shell and tiny lambda: the first step leaves the shell and also collides
    ens = [oracle.ensemble(r0_au=0.28, r_in_au=0.28 - 1e-9, r_out_au=0.28 + 1e-9, lam_au=1e-6)]
    st = oracle.inject(f, p, ens, [64], dt=0.5)
    inj = st.copy()
    stats_ = oracle.advance(f, p, ens, st, 10.0, 20, 0.5, 1)
    assert stats_[1] == 64 and stats_[0] == 0
    for k in ("x", "y", "z", "u", "mub", "F0", "F1", "vpar", "h_prev"):
        np.testing.assert_array_equal(st[k], inj[k])
    np.testing.assert_array_equal(st["ncoll"], 0)
    np.testing.assert_array_equal(st["t_birth"], 10.5)
    np.testing.assert_array_equal(st["event"], inj["event"] + 1)


def test_T11_snapshot_count():
    spec, f = _parker_grid_field()
    p = oracle.params(seed=1)
    ens = [oracle.ensemble(lam_au=0.5, r_out_au=2.4)]
    n, K, steps = 300, 25, 230
    st = oracle.inject(f, p, ens, [n], dt=0.5)
    spec_t = oracle.TallySpec(cadence=K)
    T = oracle.TallyArrays(spec_t, 1)
    oracle.advance(f, p, ens, st, 0.0, 0, 0.5, steps, tally=T)
    assert T.n_seen[0] == n * (steps // K)
    assert int(T.h_mer.sum()) + int(T.n_seen[1]) == n * (steps // K)
    assert int(T.m_cnt.sum()) == n * (steps // K)  # every r is inside [0.1, 2.5] AU
    mean_s2 = T.m_sin2.sum() / 2.0**32 / T.m_cnt.sum()
    assert 0.0 <= mean_s2 <= 1.0
    # only particles (re)born at t >= t_start are counted: early rebirths (sunward
    # particles crossing r_in) count after t_start = 1 s, none after the run's end
    st2 = oracle.inject(f, p, ens, [n], dt=0.5)
    T2 = oracle.TallyArrays(oracle.TallySpec(cadence=K, t_start=1.0), 1)
    reb = oracle.advance(f, p, ens, st2, 0.0, 0, 0.5, steps, tally=T2)[1]
    assert 0 < T2.n_seen[0] < n * (steps // K) and reb > 0
    st3 = oracle.inject(f, p, ens, [n], dt=0.5)
    T3 = oracle.TallyArrays(oracle.TallySpec(cadence=K, t_start=steps * 0.5 + 1), 1)
    oracle.advance(f, p, ens, st3, 0.0, 0, 0.5, steps, tally=T3)
    assert T3.n_seen[0] == 0


def test_T11_paper_snapshot_ensemble_arithmetic():
    g = json.load(open(GOLDEN))["snapshot_ensemble"]
    n = g["n_particles"] * (g["t_total_h"] - g["t_start_h"]) * 3600 / (g["dt_s"] * g["cadence_steps"])
    assert abs(n - g["printed_ensemble"]) / g["printed_ensemble"] < 0.01


def test_paper_printed_rates():
    """Recompute two closed forms the paper prints (Sect. 3.2 and Eq. 16)."""
    G = json.load(open(GOLDEN))
    a = G["adiabatic_cooling"]
    rate = -(4.0 / 3.0) * a["u_sw_km_s"] * 1e3 / (a["r_AU"] * AU) * 3600 * 100  # % per hour
    assert abs(rate - a["printed_percent_per_h"]) < 0.01
    # d(p^2)/p^2 -> dE: p^2 c^2 = E (E + 2 m c^2)
    mc2 = M_E * C_LIGHT**2 / KEV
    E = a["E_keV"]
    dE = rate / 100 * E * (E + 2 * mc2) / (2 * (E + mc2))
    assert abs(dE - a["printed_keV_per_h"]) < 0.15
    w = G["random_walk_displacement"]
    v = w["v_over_c"] * C_LIGHT
    for lam, printed in zip(w["lambda_AU"], w["printed_AU"]):
        assert abs(np.sqrt(v * w["t_a_h"] * 3600 * lam * AU) / AU - printed) < 0.06
