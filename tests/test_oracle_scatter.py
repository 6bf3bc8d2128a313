"""Pins of the oracle's hard-sphere scattering (Sect. 2.3, Eqs. 9, 10, 12).

* T7: the number of collisions is the sum of independent Bernoulli(p(Delta s)) events
  with p = 1 - exp(-Delta s / lambda) (Eq. 9); the exponential free-path trigger and
  the literal per-step draw of Eq. 9 have the same count law; free paths are Exp(lambda).
* T8: in a uniform field the flux-weighted law mu = +-sqrt(a) (Eq. 12) isotropises the
  time-averaged pitch distribution (uniform mu, <sin^2 alpha> = 2/3), while the
  isotropic law mu = 1 - 2a (Eq. 10) does not: it piles particles up at mu ~ 0 (the
  flux argument of Sect. 2.3).
* collisions in the inertial frame conserve gamma exactly (Sect. 3).
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import AU, C_LIGHT, KEV, M_E

B_UNIF = (2e-9, 1e-9, -3e-9)


def _uniform(lam_m, scatter_law=0, seed=0, form=0, n=1000, dt=0.5, E_keV=81.0):
    f = oracle.analytic_field(B_unif=B_UNIF)
    p = oracle.params(seed=seed, collision_form=form, no_rebirth=True)
    ens = [oracle.ensemble(r0_au=1.0, lat_deg=0.0, E0_keV=E_keV, lam_au=lam_m / AU,
                           r_in_au=0.0, r_out_au=1e9, scatter_law=scatter_law)]
    st = oracle.inject(f, p, ens, [n], dt=dt)
    return f, p, ens, st


def _mu(st):
    Bm = np.linalg.norm(B_UNIF)
    pm = np.sqrt(st["u"] ** 2 + 2 * st["mub"] * Bm / M_E)
    return st["u"] / pm


def test_injected_free_paths_are_exponential():
    lam = 0.3 * AU
    _, _, _, st = _uniform(lam, n=4000)
    assert stats.kstest(st["s_rem"] / lam, "expon").pvalue > 1e-3


def test_T7_collision_count_matches_eq9_probabilities():
    lam = 2.0e9
    dt = 0.5
    f, p, ens, st = _uniform(lam, n=800, dt=dt)
    expected = np.zeros(st.n)
    var = np.zeros(st.n)
    t = 0.0
    for k in range(800):
        ds = dt * np.abs(st["vpar"])  # |v_par| is constant in a free flight in a uniform field
        pk = 1.0 - np.exp(-ds / lam)
        expected += pk
        var += pk * (1 - pk)
        oracle.advance(f, p, ens, st, t, k, dt, 1)
        t += dt
    total = st["ncoll"].astype(float).sum()
    assert abs(total - expected.sum()) < 4 * np.sqrt(var.sum()), (total, expected.sum())
    assert total > 2000


def test_T7_exponential_and_bernoulli_forms_agree():
    lam = 2.0e9
    counts = []
    for form, seed in ((0, 1), (1, 2)):
        f, p, ens, st = _uniform(lam, n=3000, form=form, seed=seed)
        oracle.advance(f, p, ens, st, 0.0, 0, 0.5, 600)
        counts.append(st["ncoll"].astype(int))
    hi = max(c.max() for c in counts) + 1
    h0 = np.bincount(counts[0], minlength=hi)
    h1 = np.bincount(counts[1], minlength=hi)
    keep = (h0 + h1) >= 10
    table = np.stack([h0[keep], h1[keep]])
    assert stats.chi2_contingency(table).pvalue > 1e-3
    assert abs(counts[0].mean() - counts[1].mean()) < 0.1 * counts[0].mean()


def _mu_after(scatter_law, steps, n=10000, dt=0.2, lam=1.5e9):
    """One pitch cosine per particle after each entry of ``steps`` (independent samples).
    Delta s / lambda <= 0.02 per step, so the per-step collision probability of Eq. 9 is
    linear in |mu| to 1 %."""
    f, p, ens, st = _uniform(lam, scatter_law=scatter_law, n=n, dt=dt, seed=5)
    out, t, k = [], 0.0, 0
    for s in steps:
        oracle.advance(f, p, ens, st, t, k, dt, s - k)
        t += (s - k) * dt
        k = s
        out.append(_mu(st).copy())
    return out


def test_T8_flux_weighted_law_isotropises():
    (mu,) = _mu_after(1, [1500])
    # Injection draws mu0 on (0, 1]: |mu0| already has the stationary (uniform) law, and
    # ~15 collisions per particle randomise the sign.
    assert stats.kstest(np.abs(mu), "uniform").pvalue > 1e-3
    assert abs((mu < 0).mean() - 0.5) < 4 * 0.5 / np.sqrt(mu.size)
    s2 = 1 - mu**2
    assert abs(s2.mean() - 2.0 / 3.0) < 4 * s2.std() / np.sqrt(mu.size)


def test_T8_isotropic_law_overpopulates_perpendicular_pitch():
    mu1, mu2 = _mu_after(0, [1500, 6000])
    small1, small2 = (np.abs(mu1) < 0.1).mean(), (np.abs(mu2) < 0.1).mean()
    # a uniform distribution puts 10 % there; the 1/|mu| flux weighting keeps piling up
    assert small1 > 0.2 and small2 > small1 + 0.02, (small1, small2)
    assert np.mean(1 - mu2**2) > 2.0 / 3.0 + 0.05


def test_collisions_conserve_gamma_in_uniform_field():
    f, p, ens, st = _uniform(1.0e9, n=500)
    Bm = np.linalg.norm(B_UNIF)
    g0 = np.sqrt(1 + (st["u"] ** 2 + 2 * st["mub"] * Bm / M_E) / C_LIGHT**2)
    mub0 = st["mub"].copy()
    oracle.advance(f, p, ens, st, 0.0, 0, 0.5, 600)
    g1 = np.sqrt(1 + (st["u"] ** 2 + 2 * st["mub"] * Bm / M_E) / C_LIGHT**2)
    hit = st["ncoll"] >= 1
    assert hit.mean() > 0.9
    assert np.all(st["mub"][hit] != mub0[hit])
    np.testing.assert_allclose(g1 - 1, g0 - 1, rtol=1e-12)
