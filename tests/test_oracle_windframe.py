"""Scattering in the solar-wind frame (Sect. 3.2, Eqs. 15-16), pinned by the paper's closed
form: in a radial field B ~ 1/r^2 with frequent, isotropising collisions in the frame of a
radial wind u, the wind-frame momentum decays as d ln p~^2 / dt = -(4/3) u / r (Eq. 16),
-1.34 %/h at 1 AU for u = 418 km/s. The run keeps only the v_par b drift (the setting of the
paper's Fig. 7), a mean free path far below the focusing length r/2, 81 keV electrons from
r = 1 AU and the flux-weighted law of Eq. 12: with collisions counted per path length
|v_par| dt, that law keeps the time-averaged pitch distribution isotropic, the assumption
behind Eq. 16. The rate is measured over one hour after a 10-minute relaxation and compared
with Eq. 16 at the particles' mean 1/r. Control: collisions in the fixed frame keep |p|."""
import numpy as np

import oracle
from oracle import AU, C_LIGHT, M_E

U_SW = 4.18e5


def _setup(wind_u):
    f = oracle.analytic_field(parker_B0=3.5e-9, parker_rref=AU, parker_omega=0.0, parker_u=U_SW,
                              parker_E=False)
    p = oracle.params(seed=5, drift_mask=1, no_rebirth=True, wind_u=wind_u)
    e = oracle.ensemble(r0_au=1.0, lat_deg=10.0, lon_deg=30.0, E0_keV=81.0, lam_au=0.005, r_out_au=5.0,
                        scatter_law=1)
    return f, p, e


def _p2(f, s, wind_u):
    """(|p|/m)^2 in the frame of the wind (the fixed frame for wind_u = 0) and r"""
    out, rr = np.empty(s.n), np.empty(s.n)
    for i in range(s.n):
        R = np.array([s["x"][i], s["y"][i], s["z"][i]])
        B = oracle.field_eval(f, R)[0]["B"]
        Bm = np.linalg.norm(B)
        r = np.linalg.norm(R)
        V = wind_u * (R @ B) / (r * Bm)
        gV = 1.0 / np.sqrt(1.0 - V * V / C_LIGHT**2)
        pp2 = 2.0 * s["mub"][i] * Bm / M_E
        g = np.sqrt(1.0 + (s["u"][i] ** 2 + pp2) / C_LIGHT**2)
        ut = gV * (s["u"][i] - V * g)
        out[i], rr[i] = ut * ut + pp2, r
    return out, rr


def test_wind_frame_cooling_matches_eq16():
    f, p, e = _setup(U_SW)
    st = oracle.inject(f, p, [e], [4000], dt=0.5)
    oracle.advance(f, p, [e], st, 0.0, 0, 0.5, 1200)
    a, r0 = _p2(f, st, U_SW)
    oracle.advance(f, p, [e], st, 600.0, 1200, 0.5, 7200)
    b, r1 = _p2(f, st, U_SW)
    assert st["ncoll"].mean() > 300  # frequent scattering: lambda far below r / 2
    rel = b / a - 1.0
    rate, se = rel.mean(), rel.std() / np.sqrt(rel.size)
    inv_r = 0.5 * (np.mean(1.0 / r0) + np.mean(1.0 / r1))
    expect = -(4.0 / 3.0) * U_SW * inv_r * 3600.0
    print(f"d ln p~^2 over 1 h: {rate:.4%} +- {se:.4%}; Eq. 16 at <1/r>: {expect:.4%}")
    assert abs(rate - expect) < 0.05 * abs(expect) + 3 * se
    # at 1 AU the closed form is the paper's -1.34 %/h
    assert abs(-(4.0 / 3.0) * U_SW / AU * 3600.0 + 0.0134) < 0.0001


def test_fixed_frame_collisions_keep_momentum():
    f, p, e = _setup(0.0)
    st = oracle.inject(f, p, [e], [300], dt=0.5)
    a, _ = _p2(f, st, 0.0)
    oracle.advance(f, p, [e], st, 0.0, 0, 0.5, 7200)
    b, _ = _p2(f, st, 0.0)
    assert st["ncoll"].mean() > 300
    assert np.abs(b / a - 1.0).max() < 1e-8  # the integration error of one hour
