"""Pins of the oracle's predictor-corrector (Eqs. 5-6) and of its start-up rule (Sect. 2.2).

* T1: the coefficients equal those of the variable-step Adams-Bashforth-2 predictor and
  Adams-Moulton-3 corrector, derived here independently by integrating Lagrange
  interpolants of F with SymPy; tau = 1 gives the textbook AB2 / AM3 weights.
* T2: third-order global convergence on a smooth (analytic) field, at fixed dt and at
  alternating dt (tau = 2, 1/2), scattering and rebirth off.
* T3: exact special cases of Eqs. 1-2 (uniform fields), integrated exactly to rounding.
"""
import numpy as np
import pytest
import sympy as sp

import oracle
from oracle import AU, KEV

RNG = np.random.default_rng(7)


def _ab_am_weights():
    t, h, tau = sp.symbols("t h tau", positive=True)
    Fm, F0, Fs = sp.symbols("Fm F0 Fs")
    tm = -h / tau  # t^{n-1}
    # predictor: linear through (t^{n-1}, F^{n-1}), (0, F^n), integrated over [0, h]
    lin = F0 + (F0 - Fm) * (t - 0) / (0 - tm)
    pred = sp.integrate(lin, (t, 0, h))
    # corrector: quadratic through (t^{n-1}, F^{n-1}), (0, F^n), (h, F*)
    quad = (Fm * (t - 0) * (t - h) / ((tm - 0) * (tm - h))
            + F0 * (t - tm) * (t - h) / ((0 - tm) * (0 - h))
            + Fs * (t - tm) * (t - 0) / ((h - tm) * (h - 0)))
    corr = sp.integrate(quad, (t, 0, h))
    return (t, h, tau, Fm, F0, Fs), sp.simplify(pred), sp.simplify(corr)


def test_T1_coefficients_equal_variable_step_ab2_am3():
    (t, h, tau, Fm, F0, Fs), pred, corr = _ab_am_weights()
    pf = sp.lambdify((h, tau, Fm, F0), pred)
    cf = sp.lambdify((h, tau, Fm, F0, Fs), corr)
    for _ in range(50):
        X = RNG.normal(size=4)
        F0v, F1v, Fsv = RNG.normal(size=(3, 4))
        dt = RNG.uniform(0.1, 3.0)
        tv = RNG.uniform(0.25, 4.0)
        Xs = oracle.predictor(X, F0v, F1v, dt, tv)
        X1 = oracle.corrector(X, F0v, F1v, Fsv, dt, tv)
        np.testing.assert_allclose(Xs, X + pf(dt, tv, F1v, F0v), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(X1, X + cf(dt, tv, F1v, F0v, Fsv), rtol=1e-13, atol=1e-13)
    # tau = 1: textbook AB2 (3/2, -1/2) and AM3 (5/12 F*, 8/12 F^n, -1/12 F^{n-1})
    c1 = sp.expand(corr.subs(tau, 1) / h)
    assert sp.simplify(c1 - (sp.Rational(5, 12) * Fs + sp.Rational(8, 12) * F0
                             - sp.Rational(1, 12) * Fm)) == 0
    p1 = sp.expand(pred.subs(tau, 1) / h)
    assert sp.simplify(p1 - (sp.Rational(3, 2) * F0 - sp.Rational(1, 2) * Fm)) == 0
    # the corrector weights in closed form, (3 + tau)/6 etc.
    cw = sp.Poly(sp.expand(corr / h), Fs, F0, Fm)
    assert sp.simplify(cw.coeff_monomial(Fs) - (3 + 2 * tau) / (6 * (1 + tau))) == 0
    assert sp.simplify(cw.coeff_monomial(F0) - (3 + tau) / 6) == 0
    assert sp.simplify(cw.coeff_monomial(Fm) + tau**2 / (6 * (1 + tau))) == 0


def _parker():
    return oracle.analytic_field(parker_B0=3.5e-9, parker_rref=AU, parker_omega=2.7e-6,
                                 parker_u=4e5, parker_E=True)


def _run(f, p, ens, counts, dts):
    """Inject with dts[0] and advance one call per entry of dts."""
    st = oracle.inject(f, p, ens, counts, dt=dts[0])
    t = 0.0
    for k, dt in enumerate(dts):
        oracle.advance(f, p, ens, st, t, k, dt, 1)
        t += dt
    return st


def _run_uniform(f, p, ens, counts, dt, n):
    st = oracle.inject(f, p, ens, counts, dt=dt)
    oracle.advance(f, p, ens, st, 0.0, 0, dt, n)
    return st


def _err(a, b):
    """Max relative position error and u error relative to |u| (floored at 1e3 m/s)."""
    R = np.stack([a["x"], a["y"], a["z"]])
    Rr = np.stack([b["x"], b["y"], b["z"]])
    eR = np.max(np.linalg.norm(R - Rr, axis=0) / np.linalg.norm(Rr, axis=0))
    eu = np.max(np.abs(a["u"] - b["u"]) / np.maximum(np.abs(b["u"]), 1e3))
    return max(eR, eu)


def _ensembles():
    # three pitch cosines at 0.5 AU, 40 deg latitude; never scattered, never reborn
    e = oracle.ensemble(r0_au=0.5, lat_deg=40.0, lon_deg=10.0, E0_keV=81.0, lam_au=1.0,
                        r_in_au=0.0, r_out_au=1e9)
    return [e]


@pytest.mark.parametrize("alternating", [False, True])
def test_T2_third_order_convergence(alternating):
    f = _parker()
    p = oracle.params(seed=3, no_scatter=True, no_rebirth=True)
    ens = _ensembles()
    counts = [6]
    T = 1200.0
    ref = _run_uniform(f, p, ens, counts, 0.15625, int(round(T / 0.15625)))
    errs = []
    hs = [40.0, 20.0, 10.0, 5.0]
    for h in hs:
        if alternating:
            dts = [h, h / 2] * int(round(T / (1.5 * h)))
            st = _run(f, p, ens, counts, dts)
        else:
            st = _run_uniform(f, p, ens, counts, h, int(round(T / h)))
        errs.append(_err(st, ref))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 2.8), (errs, slopes)
    assert np.all(slopes < 3.2), (errs, slopes)


def _uniform_case(B, E, ideal, n=200, dt=0.5):
    f = oracle.analytic_field(B_unif=B, E_unif=E, ideal=ideal)
    p = oracle.params(seed=1, no_scatter=True, no_rebirth=True)
    ens = [oracle.ensemble(r0_au=0.7, lat_deg=10.0, lon_deg=30.0, E0_keV=50.0,
                           r_in_au=0.0, r_out_au=1e9)]
    st0 = oracle.inject(f, p, ens, [16], dt=dt)
    st = st0.copy()
    oracle.advance(f, p, ens, st, 0.0, 0, dt, n)
    return f, p, st0, st, n * dt


def test_T3_uniform_B_straight_line():
    B = np.array([3e-9, -1e-9, 2e-9])
    _, p, st0, st, T = _uniform_case(tuple(B), (0, 0, 0), True)
    b = B / np.linalg.norm(B)
    np.testing.assert_array_equal(st["u"], st0["u"])
    np.testing.assert_array_equal(st["mub"], st0["mub"])
    R0 = np.stack([st0["x"], st0["y"], st0["z"]])
    R = np.stack([st["x"], st["y"], st["z"]])
    vpar = st0["vpar"]
    np.testing.assert_allclose(R, R0 + np.outer(b, vpar) * T, rtol=1e-13, atol=1e-3)


def test_T3_uniform_E_perp_constant_drift():
    B = np.array([0.0, 0.0, 5e-9])
    E = np.array([2e-3, -1e-3, 0.0])
    _, p, st0, st, T = _uniform_case(tuple(B), tuple(E), True)
    vE = np.cross(E, B) / (B @ B)
    np.testing.assert_array_equal(st["u"], st0["u"])
    R0 = np.stack([st0["x"], st0["y"], st0["z"]])
    R = np.stack([st["x"], st["y"], st["z"]])
    expect = R0 + (np.outer(B / np.linalg.norm(B), st0["vpar"]) + vE[:, None]) * T
    np.testing.assert_allclose(R, expect, rtol=1e-13, atol=1e-3)


def test_T3_uniform_E_parallel_linear_momentum():
    B = np.array([0.0, 4e-9, 0.0])
    E = np.array([0.0, 1e-6, 0.0])
    _, p, st0, st, T = _uniform_case(tuple(B), tuple(E), False)
    expect = st0["u"] + oracle.Q_E * E[1] / oracle.M_E * T
    np.testing.assert_allclose(st["u"], expect, rtol=1e-12)
