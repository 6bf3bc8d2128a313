"""Parity at the full size of the perturbed-Parker workload (256x128x256 FP32 grid with
eps = 0.1 and 8 modes; 3 ensembles of 10^6 electrons at 81 keV with lambda = 0.1, 0.5,
1.0 AU), in the launch configuration the benchmark times. The oracle recomputes sampled
particles one by one: the first 512 ids of every ensemble (Philox streams are keyed by
particle id, so a subset evolves exactly as inside the full ensemble).

Tolerances: the trajectory state (R, gamma v_par, v_par, mu_B, free path) within 1e-4 over
the first 10^3 steps, and its bulk (99th percentile of every state error) within 2e-5.
The carried right-hand sides F^n, F^{n-1} are functions of the state; in a field with
10 % structure on 0.1 AU scales a position offset dR moves b and grad|B| by about
0.1 dR / 0.1 AU, so they are held to 1e-3. The tail of the FP32 errors comes from the rare
steps where FP32 and FP64 positions sit on opposite sides of a cell face, across which the
trilinear gradient (hence the mirror force) jumps."""
import numpy as np
import pytest

import oracle
from _cases import bulk_percentiles, compare_states, momentum_scale, oracle_ensembles
from oracle import AU
from paper_2403_06706_gb300 import synth

pytestmark = pytest.mark.gpu
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")

# The bulk of the kept particles must sit far inside the per-particle maxima (1e-4, 1e-3 for
# the carried right-hand sides), so that an error confined to more than 1 % of the
# trajectories cannot hide below the maxima or behind the particles excused for a differing
# history or an ill-conditioned start: the 99th percentile of every state error within
# 2e-5, ten times the FP32 rounding a state accumulates over 10^3 steps (sqrt(1000) x 6e-8
# ~ 2e-6), and of the carried right-hand sides within 1e-4 (their maxima's tenfold ratio to
# the state's). Measured: p99 of 2e-7 to 5e-6 for the state, up to 1.2e-5 for F^n, F^{n-1};
# medians near 1e-7.
BULK_P99 = {"R": 2e-5, "u": 2e-5, "vpar": 2e-5, "mub": 2e-5, "s_rem": 2e-5, "F0_R": 1e-4, "F0_u": 1e-4,
            "F1_R": 1e-4, "F1_u": 1e-4}


def _check_bulk(name, gs, st, pm, skip, lam):
    p50 = bulk_percentiles(gs, st, pm, skip=skip, lam=lam, q=50)
    p99 = bulk_percentiles(gs, st, pm, skip=skip, lam=lam, q=99)
    print(name, "excused", int(skip.sum()), "of", skip.size)
    for k in p99:
        print(f"  {k:6s} p50 {p50[k]:.2e}  p99 {p99[k]:.2e}")
    for k, v in p99.items():
        assert v < BULK_P99[k], (name, k, v)


def test_full_size_fp32_sampled_parity():
    import bench

    wl = synth.c2_perturbed()
    nodes = synth.wind_grid(wl.wind, dtype=np.float32)
    n_steps = 1000
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=wl.seed, dt_init=wl.dt) as c:
        c.field_load(nodes, wl.wind.r_min_au, wl.wind.r_max_au)
        c.inject(list(wl.ensembles))
        c.set_launch(**bench.LAUNCH)
        c.advance(wl.dt, n_steps)
        g = c.get_state()
    n_s = 512
    first = np.cumsum([0] + [e.count for e in wl.ensembles])[:-1]
    pick = np.concatenate([f + np.arange(n_s) for f in first])
    gs = {k: (v[:, pick] if v.ndim == 2 else v[pick]) for k, v in g.items()}

    f = oracle.grid_field(nodes, wl.wind.r_min_au * AU, wl.wind.r_max_au * AU)
    p = oracle.params(seed=wl.seed)
    oe = oracle_ensembles(wl.ensembles)
    parts = []
    for k, f0 in enumerate(first):
        counts = [0] * len(oe)
        counts[k] = n_s
        parts.append(oracle.inject(f, p, oe, counts, id0=int(f0), dt=wl.dt))
    st = oracle.StateArrays({k: np.concatenate([q[k] for q in parts], axis=-1)
                             for k in parts[0].arrays})
    np.testing.assert_array_equal(gs["id"], st["id"])
    oracle.advance(f, p, oe, st, 0.0, 0, wl.dt, n_steps)
    div = (gs["ncoll"] != st["ncoll"]) | (gs["event"] != st["event"]) | (gs["t_birth"] != st["t_birth"])
    assert div.mean() <= 0.01, div.sum()
    lam = np.array([e.lam_au for e in wl.ensembles])[st["ens"].astype(int)] * AU
    pm = momentum_scale(st, nodes, wl.wind, wl.ensembles)
    err = compare_states(gs, st.arrays, 1e-4, pm, skip=div, lam=lam)
    for k, v in err.items():
        assert v < (1e-3 if k.startswith("F") else 1e-4), (k, v, err)
    _check_bulk("plain", gs, st.arrays, pm, div, lam)
    keep = ~div
    R = np.stack([gs["x"], gs["y"], gs["z"]])[:, keep]
    Ro = np.stack([st["x"], st["y"], st["z"]])[:, keep]
    eR = np.linalg.norm(R - Ro, axis=0) / np.linalg.norm(Ro, axis=0)
    assert np.percentile(eR, 99) < 1e-5, np.percentile(eR, [50, 90, 99])
    np.testing.assert_array_equal(gs["flags"], st["flags"])


def _oracle_subset(f, p, wl, n_s, first):
    oe = oracle_ensembles(wl.ensembles)
    parts = []
    for k, f0 in enumerate(first):
        counts = [0] * len(oe)
        counts[k] = n_s
        parts.append(oracle.inject(f, p, oe, counts, id0=int(f0), dt=wl.dt))
    st = oracle.StateArrays({k: np.concatenate([q[k] for q in parts], axis=-1) for k in parts[0].arrays})
    return oe, st


def test_large_grid_fp32_sampled_parity_and_tally_invariants():
    """The large workload: 512x256x512 FP32 grid (2.15 GB, eps = 0.2, 16 modes), 3x10^7
    electrons with an E^-3 spectrum on [20, 500] keV, lambda = 0.3 AU, tallies of
    pitch x energy x r on 64 x 64 x 128 bins; 1000 steps in the benchmark's launch shape.
    The oracle recomputes the first 256 ids; the full tally is checked by its invariants:
    every particle is sampled at every cadence step, and every in-range sample lands in
    exactly one bin."""
    import bench

    wl = synth.c5_large()
    nodes = synth.wind_grid(wl.wind, dtype=np.float32)
    n_steps, cadence = 1000, 100
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=wl.seed, dt_init=wl.dt) as c:
        c.field_load(nodes, wl.wind.r_min_au, wl.wind.r_max_au)
        c.inject(list(wl.ensembles))
        c.set_launch(**bench.LAUNCH)
        c.tally_arm(cadence=cadence, n_mu=64, n_E=64, n_r=128, E_lo_keV=5.0, E_hi_keV=600.0,
                    r_lo_au=wl.wind.r_min_au, r_hi_au=wl.wind.r_max_au)
        c.advance(wl.dt, n_steps)
        g = c.get_state()
        t = c.tally_read()
    n = wl.n_particles
    assert int(t["n_seen"][0]) == n * (n_steps // cadence)
    assert int(t["h_mer"].sum(dtype=np.int64)) == int(t["n_seen"][0]) - int(t["n_seen"][1])
    assert int(t["n_seen"][1]) < 0.01 * int(t["n_seen"][0])
    n_s = 256
    gs = {k: (v[:, :n_s] if v.ndim == 2 else v[:n_s]) for k, v in g.items()}
    f = oracle.grid_field(nodes, wl.wind.r_min_au * AU, wl.wind.r_max_au * AU)
    p = oracle.params(seed=wl.seed)
    oe, st = _oracle_subset(f, p, wl, n_s, [0])
    oracle.advance(f, p, oe, st, 0.0, 0, wl.dt, n_steps)
    div = (gs["ncoll"] != st["ncoll"]) | (gs["event"] != st["event"]) | (gs["t_birth"] != st["t_birth"])
    assert div.mean() <= 0.02, div.sum()
    lam = np.full(n_s, wl.ensembles[0].lam_au * AU)
    pm = momentum_scale(st, nodes, wl.wind, wl.ensembles)
    err = compare_states(gs, st.arrays, 1e-4, pm, skip=div, lam=lam)
    for k, v in err.items():
        assert v < (1e-3 if k.startswith("F") else 1e-4), (k, v, err)
    _check_bulk("large", gs, st.arrays, pm, div, lam)


def test_neural_workload_sampled_parity():
    """The neural-field workload: a SIREN trained on 10^7 samples of the perturbed
    256x128x256 grid, then 10^7 electrons pushed with it for 20 steps. The oracle runs the
    same network (BF16 reading) for the first 256 ids; increments of R and gamma v_par are
    compared against their own size (the network's BF16 noise bounds the agreement,
    tests/test_gpu_split.py)."""
    wn = synth.c4_neural()
    X = wn.extra
    w = wn.wind
    nodes = synth.wind_grid(w, dtype=np.float32)
    n_steps = 20
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=wn.seed, dt_init=wn.dt) as c:
        c.field_load(nodes, w.r_min_au, w.r_max_au)
        c.siren_set(synth.siren_init(seed=0), omega0=X["omega0"], r_max_au=w.r_max_au, B_scale=w.B1,
                    E_scale=w.B1 * w.u_sw)
        samples = synth.siren_samples(X["n_samples"], w)
        for ep, lr in X["schedule"]:  # the benchmark's training schedule
            c.field_fit(samples, n_epochs=ep, batch=X["batch"], lr=lr)
        P = c.siren_get()
        c.field_select(gcpush.FIELD_SIREN)
        c.inject(list(wn.ensembles))
        g0 = c.get_state()
        c.advance(wn.dt, n_steps)
        g1 = c.get_state()
    n_s = 256
    sl = lambda a: {k: (v[:, :n_s] if v.ndim == 2 else v[:n_s]) for k, v in a.items()}  # noqa: E731
    g0, g1 = sl(g0), sl(g1)
    f = oracle.siren_field(P, X["omega0"], w.r_max_au * AU, w.B1, w.B1 * w.u_sw, bf16=True)
    p = oracle.params(seed=wn.seed)
    oe, o0 = _oracle_subset(f, p, wn, n_s, [0])
    np.testing.assert_array_equal(g0["u"], o0["u"])
    o1 = o0.copy()
    oracle.advance(f, p, oe, o1, 0.0, 0, wn.dt, n_steps)
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


def _ks_marginals(a, b, name):
    """Two-sample KS test on every 1-D marginal of the histogram pair (a, b), each bin's
    count expanded into that many samples at the bin index."""
    from scipy import stats

    for axis in range(a.ndim):
        other = tuple(i for i in range(a.ndim) if i != axis)
        ca = a.sum(axis=other).astype(np.int64)
        cb = b.sum(axis=other).astype(np.int64)
        if ca.sum() < 50 or cb.sum() < 50:
            continue
        xa = np.repeat(np.arange(ca.size), ca)
        xb = np.repeat(np.arange(cb.size), cb)
        p = stats.ks_2samp(xa, xb).pvalue
        print(name, "axis", axis, "samples", ca.sum(), cb.sum(), "KS p", p)
        assert p > 0.01, (name, axis, p)


def test_c2_subset_tallies_match_oracle_by_ks():
    """The FP32 push against the FP64 oracle on a 1026-electron subset of the perturbed-Parker
    workload (342 per mean free path, the full 256x128x256 grid), 10^4 steps with tallies every
    10 steps: every marginal of every tally (pitch, energy, r; age x energy at 1 AU; the young
    pitch distribution; the samples per r bin) agrees by a two-sample KS test at p > 0.01."""
    wl = synth.c2_perturbed(n_per_lambda=342)
    nodes = synth.wind_grid(wl.wind, dtype=np.float32)
    tally = dict(cadence=10, n_mu=32, n_E=32, n_r=64, n_age=32, age_max_s=5000.0, rwin_lo_au=0.9,
                 rwin_hi_au=1.1, age_young_s=1200.0)
    calls = [(wl.dt, 5000, 0.0), (wl.dt, 5000, 0.0)]
    from _cases import run_gpu, run_oracle

    g, gt, gs = run_gpu(nodes, wl.wind, list(wl.ensembles), calls, gcpush.PREC_FP32_MIXED,
                        seed=wl.seed, tally=tally)
    o, ot, os_ = run_oracle(nodes, wl.wind, list(wl.ensembles), calls, seed=wl.seed, tally=tally)
    assert int(gt["n_seen"][0]) == int(ot.n_seen[0]) > 0
    assert abs(int(gs["collisions"]) - int(os_[0])) <= 0.01 * int(os_[0])
    for k in ("h_mer", "h_age", "h_pad", "m_cnt"):
        a, b = gt[k], getattr(ot, k)
        assert a.sum() > 0, k
        for e in range(a.shape[0]):
            _ks_marginals(a[e], b[e], f"{k}[{e}]")


@pytest.mark.parametrize("variant", ["wind_frame_collisions", "two_fluid_field", "time_dependent_field"])
def test_full_size_variants_sampled_parity(variant):
    """The method variants the benchmark times, at full size in its launch configuration
    (the perturbed 256x128x256 grid, 3x10^6 electrons, 1000 steps): wind-frame collisions
    (u = 400 km/s), the two-fluid field (a 500 V potential) and a time-dependent field (the
    wind turning faster, stronger and differently perturbed over the run). The oracle
    recomputes the first 512 ids of every ensemble; tolerances as in the plain full-size test,
    with particles whose discrete history differs (near-tie collisions or rebirths) counted
    and bounded."""
    import dataclasses

    import bench

    wl = synth.c2_perturbed()
    nodes = synth.wind_grid(wl.wind, dtype=np.float32)
    opt, ideal, nodes1, window = {}, True, None, None
    if variant == "wind_frame_collisions":
        opt = {"wind_u": 4.0e5}
    elif variant == "two_fluid_field":
        nodes[..., 7] = synth.potential_of(wl.wind, 500.0)[None, None, :].astype(nodes.dtype)
        ideal = 2
    else:
        nodes1 = synth.wind_grid(dataclasses.replace(wl.wind, B1=4.2e-9, u_sw=5.0e5, seed=wl.wind.seed + 1),
                                 dtype=np.float32)
        window = (0.0, 1000 * wl.dt)
    n_steps = 1000
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=wl.seed, dt_init=wl.dt, **opt) as c:
        c.field_load(nodes, wl.wind.r_min_au, wl.wind.r_max_au, ideal=ideal)
        if nodes1 is not None:
            c.field_load_next(nodes1, *window)
        c.inject(list(wl.ensembles))
        c.set_launch(**bench.LAUNCH)
        c.advance(wl.dt, n_steps)
        g = c.get_state()
    n_s = 512
    first = np.cumsum([0] + [e.count for e in wl.ensembles])[:-1]
    pick = np.concatenate([f + np.arange(n_s) for f in first])
    gs = {k: (v[:, pick] if v.ndim == 2 else v[pick]) for k, v in g.items()}
    if nodes1 is None:
        f = oracle.grid_field(nodes, wl.wind.r_min_au * AU, wl.wind.r_max_au * AU, ideal=ideal)
    else:
        f = oracle.grid_field_pair(nodes, nodes1, window[0], window[1], wl.wind.r_min_au * AU,
                                   wl.wind.r_max_au * AU, ideal=ideal)
    p = oracle.params(seed=wl.seed, **opt)
    oe, st = _oracle_subset(f, p, wl, n_s, first)
    np.testing.assert_array_equal(gs["id"], st["id"])
    oracle.advance(f, p, oe, st, 0.0, 0, wl.dt, n_steps)
    pm = momentum_scale(st, nodes, wl.wind, wl.ensembles)
    div = (gs["ncoll"] != st["ncoll"]) | (gs["event"] != st["event"]) | (gs["t_birth"] != st["t_birth"])
    # particles whose oracle trajectory is itself unstable at FP32 resolution (a cell face
    # met within rounding, a collision step decided within it): the oracle rerun from start
    # states moved by +-3e-7 along two seeded directions ends more than half the tolerance
    # away (5e-5 |p|/m in gamma v_par, 5e-4 in the position rows of F^n)
    ill = np.zeros(st["u"].shape[0], dtype=bool)
    for d in range(2):
        for sgn in (1.0, -1.0):
            _, sp = _oracle_subset(f, p, wl, n_s, first)
            rng = np.random.default_rng(1000 + d)
            for k in ("x", "y", "z", "u"):
                sp.arrays[k] *= 1.0 + sgn * 3e-7 * rng.standard_normal(sp.arrays[k].shape)
            oracle.advance(f, p, oe, sp, 0.0, 0, wl.dt, n_steps)
            ill |= np.abs(sp["u"] - st["u"]) > 5e-5 * pm
            # the carried right-hand side likewise (half its 1e-3 tolerance)
            ill |= (np.linalg.norm(sp["F0"][:3] - st["F0"][:3], axis=0)
                    > 5e-4 * np.linalg.norm(st["F0"][:3], axis=0))
    print(variant, "diverged", int(div.sum()), "ill-conditioned", int(ill.sum()))
    assert div.mean() <= 0.01 and ill.mean() <= 0.01, (div.sum(), ill.sum())
    div |= ill
    lam = np.array([e.lam_au for e in wl.ensembles])[st["ens"].astype(int)] * AU
    err = compare_states(gs, st.arrays, 1e-4, pm, skip=div, lam=lam)
    for k, v in err.items():
        assert v < (1e-3 if k.startswith("F") else 1e-4), (k, v, err)
    _check_bulk(variant, gs, st.arrays, pm, div, lam)
    keep = ~div
    R = np.stack([gs["x"], gs["y"], gs["z"]])[:, keep]
    Ro = np.stack([st["x"], st["y"], st["z"]])[:, keep]
    eR = np.linalg.norm(R - Ro, axis=0) / np.linalg.norm(Ro, axis=0)
    assert np.percentile(eR, 99) < 1e-5, np.percentile(eR, [50, 90, 99])
