"""The perturbed-Parker workload at its full duration: the FP32-mixed push against the FP64
oracle over 48 h simulated (345 600 steps of 0.5 s) on 1024 electrons per mean free path
(lambda = 0.1, 0.5, 1.0 AU; 81 keV from 0.28 AU, 24 deg) on the full 256x128x256 grid, with the
snapshot tallies of Sect. 3 (every 100 steps, particles (re)born after t_start = 8 h: the
paper starts its snapshots after 8.3 h of a 150 h run).

Over hours the FP32 and FP64 trajectories of one particle part ways (a collision or a rebirth
one step apart, a cell face met on the other side), so the two runs are compared as two
samples of the same law. The snapshot samples of one particle life are correlated (the
energy of a life hardly moves, its position drifts slowly), so the KS p-values take as
sample size the number of particle lives the tally can contain (rebirths after t_start, each
counted once; for a histogram with fewer samples than that, its sample count). Counting every
snapshot as independent would claim up to 10^3 times more samples than there are: two FP64
oracle runs that differ only by a 3e-7 relative move of the start state already fall to
p = 0.025 on one marginal that way.

Checks per ensemble:
* every 1-D marginal of every tally (pitch x energy x r; age x energy at 1 AU; the young
  pitch distribution; samples per r bin) by a two-sample KS test at p > 0.01;
* the mean energy against age at 1 AU (the drift-loss signal of Sect. 3, Eqs. 13-14, Fig. 5)
  per age bin within four standard errors (each side's spread over the square root of its
  sample count, capped as above), and the fitted loss rate (keV/h) within its error;
* sample counts, collisions and rebirths within 5 %.
The agreement figures are printed (-s).
"""
import numpy as np
import pytest
from scipy import special

import oracle
from _cases import oracle_ensembles, tally_spec
from oracle import AU
from paper_2403_06706_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")

HOURS = 48
T_START_H = 8
TALLY = dict(cadence=100, n_mu=32, n_E=60, E_lo_keV=60.0, E_hi_keV=90.0, n_r=64, r_lo_au=0.1, r_hi_au=2.5,
             n_age=24, age_max_s=24 * 3600.0, t_start_s=T_START_H * 3600.0, rwin_lo_au=0.9, rwin_hi_au=1.1,
             age_young_s=1200.0)


def _ks_p(ca, cb, n_eff_a, n_eff_b):
    """Two-sample KS statistic of the binned samples ca, cb (counts per bin) and its p-value
    for sample sizes n_eff_a, n_eff_b (asymptotic Kolmogorov law with Stephens' correction)."""
    Fa = np.cumsum(ca) / ca.sum()
    Fb = np.cumsum(cb) / cb.sum()
    D = float(np.abs(Fa - Fb).max())
    en = np.sqrt(n_eff_a * n_eff_b / (n_eff_a + n_eff_b))
    return D, float(special.kolmogorov((en + 0.12 + 0.11 / en) * D))


def _mean_energy_by_age(h_age, E_mid):
    """per age bin: sample count, mean and standard deviation of the energy (bin midpoints)"""
    n = h_age.sum(axis=1).astype(np.float64)
    w = h_age.astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        m = (w * E_mid).sum(axis=1) / n
        v = (w * E_mid ** 2).sum(axis=1) / n - m ** 2
    return n, m, np.sqrt(np.maximum(v, 0.0))


def test_c2_full_duration_fp32_against_oracle():
    wl = synth.c2_perturbed(n_per_lambda=1024)
    nodes = synth.wind_grid(wl.wind, dtype=np.float32)
    dt = wl.dt
    n0 = int(T_START_H * 3600 / dt)
    n1 = int(HOURS * 3600 / dt) - n0
    f = oracle.grid_field(nodes, wl.wind.r_min_au * AU, wl.wind.r_max_au * AU)
    p = oracle.params(seed=wl.seed)
    spec = tally_spec(TALLY)
    E_edges = spec.E_lo_keV * (spec.E_hi_keV / spec.E_lo_keV) ** (np.arange(spec.n_E + 1) / spec.n_E)
    E_mid = np.sqrt(E_edges[:-1] * E_edges[1:])
    age_h = (np.arange(spec.n_age) + 0.5) * spec.age_max_s / spec.n_age / 3600.0
    first = np.cumsum([0] + [e.count for e in wl.ensembles])[:-1]

    for e, ens in enumerate(wl.ensembles):
        with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=wl.seed, dt_init=dt, id_base=int(first[e])) as c:
            c.field_load(nodes, wl.wind.r_min_au, wl.wind.r_max_au)
            c.inject([ens])
            c.tally_arm(**TALLY)
            c.advance(dt, n0)
            s0 = c.stats()
            c.advance(dt, n1)
            s1 = c.stats()
            g = c.tally_read()
        oe = oracle_ensembles([ens])
        st = oracle.inject(f, p, oe, [ens.count], id0=int(first[e]), dt=dt)
        T = oracle.TallyArrays(spec, 1)
        o0 = oracle.advance(f, p, oe, st, 0.0, 0, dt, n0, tally=T)
        o1 = oracle.advance(f, p, oe, st, n0 * dt, n0, dt, n1, tally=T)

        lives_g = int(s1["rebirths"] - s0["rebirths"])
        lives_o = int(o1[1])
        coll_g, coll_o = int(s1["collisions"]), int(o0[0] + o1[0])
        seen_g, seen_o = int(g["n_seen"][0]), int(T.n_seen[0])
        print(f"lambda {ens.lam_au} AU: lives after t_start {lives_g} / {lives_o}, collisions {coll_g} / {coll_o}, "
              f"samples {seen_g} / {seen_o}, out of range {int(g['n_seen'][1])} / {int(T.n_seen[1])}")
        assert lives_o > 500
        for a, b in ((lives_g, lives_o), (coll_g, coll_o), (seen_g, seen_o)):
            assert abs(a - b) <= 0.05 * b, (a, b)

        for k in ("h_mer", "h_age", "h_pad", "m_cnt"):
            a, b = g[k][0].astype(np.int64), getattr(T, k)[0].astype(np.int64)
            assert b.sum() > 0, k
            for axis in range(a.ndim):
                other = tuple(i for i in range(a.ndim) if i != axis)
                ca, cb = a.sum(axis=other), b.sum(axis=other)
                D, pv = _ks_p(ca, cb, min(ca.sum(), lives_g), min(cb.sum(), lives_o))
                print(f"  {k} axis {axis}: samples {ca.sum()} / {cb.sum()}  D {D:.2e}  p {pv:.3f}")
                assert pv > 0.01, (k, axis, D, pv)

        # the drift-loss signal: mean energy against age at 1 AU
        ng, mg, sg = _mean_energy_by_age(g["h_age"][0], E_mid)
        no, mo, so = _mean_energy_by_age(T.h_age[0], E_mid)
        ok = (ng >= 100) & (no >= 100)
        assert ok.sum() >= 6
        se = np.sqrt(sg[ok] ** 2 / np.minimum(ng[ok], lives_g) + so[ok] ** 2 / np.minimum(no[ok], lives_o))
        z = np.abs(mg[ok] - mo[ok]) / se
        print("  mean energy (keV) by age (h):",
              " ".join(f"{h:.1f}:{x:.3f}/{y:.3f}" for h, x, y in zip(age_h[ok], mg[ok], mo[ok])))
        print(f"  max |difference| / standard error {z.max():.2f}")
        assert z.max() < 4.0
        # the loss rate: weighted straight-line fit of the mean energy against age
        rate = []
        for n, m, s, lv in ((ng, mg, sg, lives_g), (no, mo, so, lives_o)):
            wt = np.minimum(n[ok], lv) / np.maximum(s[ok], 1e-3) ** 2
            A = np.stack([np.ones(ok.sum()), age_h[ok]], axis=1)
            cov = np.linalg.inv(A.T @ (A * wt[:, None]))
            coef = cov @ (A.T @ (wt * m[ok]))
            rate.append((coef[1], np.sqrt(cov[1, 1])))
        (rg, eg), (ro, eo) = rate
        print(f"  drift loss {rg:.4f} +- {eg:.4f} keV/h (FP32) vs {ro:.4f} +- {eo:.4f} keV/h (oracle)")
        assert abs(rg - ro) < 4.0 * np.hypot(eg, eo)
