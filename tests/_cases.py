"""Shared parity-case helpers: run one workload through the CUDA library (C ABI) and
through the FP64 oracle with identical seeded inputs and call structure."""
from __future__ import annotations

import numpy as np

import oracle
from oracle import AU, C_LIGHT, KEV, M_E

try:
    from paper_2403_06706_gb300 import gcpush
except Exception:  # the CPU suite never calls the library
    gcpush = None
from paper_2403_06706_gb300 import synth


def oracle_ensembles(ens):
    return [oracle.ensemble(r0_au=e.r0_au, lat_deg=e.lat_deg, lon_deg=e.lon_deg, E0_keV=e.E0_keV,
                            lam_au=e.lam_au, r_in_au=e.r_in, r_out_au=e.r_out_au,
                            energy_law=e.energy_law, E_lo_keV=e.E_lo_keV, E_hi_keV=e.E_hi_keV,
                            E_index=e.E_index, mu_law=e.mu_law, scatter_law=e.scatter_law)
            for e in ens]


def run_gpu(nodes, wind, ens, calls, precision, seed=0, tally=None, dt_init=None, launch=None,
            ideal=True, nodes1=None, t_snap=None, **opt):
    """calls: list of (dt, n_steps, lambda_au); nodes1, t_snap: a second snapshot and the
    (t0, t1) window of a time-dependent field. Returns (state, tallies, stats)."""
    dt0 = dt_init if dt_init is not None else calls[0][0]
    with gcpush.Context(precision=precision, device=0, seed=seed, dt_init=dt0, **opt) as ctx:
        ctx.field_load(nodes, wind.r_min_au, wind.r_max_au, ideal=ideal)
        if nodes1 is not None:
            ctx.field_load_next(nodes1, *t_snap)
        ctx.inject(ens)
        if launch:
            ctx.set_launch(**launch)
        if tally:
            ctx.tally_arm(**tally)
        for dt, n, lam in calls:
            ctx.advance(dt, n, lam)
        st = ctx.get_state()
        tl = ctx.tally_read() if tally else None
        stats = ctx.stats()
    return st, tl, stats


def tally_spec(t: dict) -> oracle.TallySpec:
    return oracle.TallySpec(cadence=t.get("cadence", 100), n_mu=t.get("n_mu", 32),
                            n_E=t.get("n_E", 32), n_r=t.get("n_r", 64), n_age=t.get("n_age", 32),
                            t_start=t.get("t_start_s", 0.0), E_lo_keV=t.get("E_lo_keV", 5.0),
                            E_hi_keV=t.get("E_hi_keV", 600.0), r_lo_au=t.get("r_lo_au", 0.1),
                            r_hi_au=t.get("r_hi_au", 2.5), age_max_s=t.get("age_max_s", 86400.0),
                            rwin_lo_au=t.get("rwin_lo_au", 0.9), rwin_hi_au=t.get("rwin_hi_au", 1.1),
                            age_young_s=t.get("age_young_s", 1200.0))


def run_oracle(nodes, wind, ens, calls, seed=0, tally=None, dt_init=None, subset=None,
               n_threads=0, ideal=True, nodes1=None, t_snap=None, perturb=None, **opt):
    """perturb: (direction seed, eps) scales R and gamma v_par after injection by
    1 + eps * (a seeded standard normal per particle and component)."""
    if nodes1 is None:
        f = oracle.grid_field(nodes, wind.r_min_au * AU, wind.r_max_au * AU, ideal=ideal)
    else:
        f = oracle.grid_field_pair(nodes, nodes1, t_snap[0], t_snap[1], wind.r_min_au * AU,
                                   wind.r_max_au * AU, ideal=ideal)
    p = oracle.params(seed=seed, **opt)
    oe = oracle_ensembles(ens)
    dt0 = dt_init if dt_init is not None else calls[0][0]
    st = oracle.inject(f, p, oe, [e.count for e in ens], dt=dt0, n_threads=n_threads)
    if subset is not None:
        st = st.subset(subset)
    if perturb is not None:
        rng = np.random.default_rng(perturb[0])
        for k in ("x", "y", "z", "u"):
            st.arrays[k] *= 1.0 + perturb[1] * rng.standard_normal(st.arrays[k].shape)
    T = oracle.TallyArrays(tally_spec(tally), len(ens)) if tally else None
    t, step = 0.0, 0
    stats = np.zeros(2, dtype=np.uint64)
    for dt, n, lam in calls:
        stats += oracle.advance(f, p, oe, st, t, step, dt, n, lambda_override_m=lam * AU,
                                tally=T, n_threads=n_threads)
        t += n * dt
        step += n
    return st, T, stats


def momentum_scale(st, nodes, wind, ens) -> np.ndarray:
    """|p|/m of each particle at injection (m/s): sqrt(u_inj^2 + 2 mu_B,inj |B(R0)| / m)."""
    f = oracle.grid_field(nodes, wind.r_min_au * AU, wind.r_max_au * AU)
    Bm = np.zeros(len(ens))
    for k, e in enumerate(oracle_ensembles(ens)):
        R0 = np.array([e.r0 * np.cos(e.lat) * np.cos(e.lon), e.r0 * np.cos(e.lat) * np.sin(e.lon),
                       e.r0 * np.sin(e.lat)])
        Bm[k] = np.linalg.norm(oracle.field_eval(f, R0)[0]["B"])
    b = Bm[st["ens"].astype(int)]
    return np.sqrt(st["u_inj"] ** 2 + 2 * st["mub_inj"] * b / M_E)


def state_errors(g, o, pm, keep=None, lam=None):
    """Per-particle relative errors of the continuous state (arrays over the kept particles);
    pm: per-particle |p|/m scale; lam: per-particle mean free path (the scale of the remaining
    free path; 0.01 AU if None)."""
    keep = np.ones(g["x"].shape[0], dtype=bool) if keep is None else keep
    R = np.stack([g["x"], g["y"], g["z"]])[:, keep]
    Ro = np.stack([o["x"], o["y"], o["z"]])[:, keep]
    out = {}
    out["R"] = np.linalg.norm(R - Ro, axis=0) / np.linalg.norm(Ro, axis=0)
    out["u"] = np.abs(g["u"][keep] - o["u"][keep]) / pm[keep]
    out["vpar"] = np.abs(g["vpar"][keep] - o["vpar"][keep]) / pm[keep]
    mscale = np.maximum(np.abs(o["mub"][keep]), 1e-30 + np.abs(o["mub_inj"][keep]).max() * 1e-6)
    out["mub"] = np.abs(g["mub"][keep] - o["mub"][keep]) / mscale
    for F in ("F0", "F1"):
        # dR/dt = v_par b + drifts: near a mirror point v_par -> 0 and |dR/dt| shrinks to the
        # drift speed while its error still follows the v_par error, which scales with |p|/m;
        # so the scale is |dR/dt| but not below a tenth of |p|/m
        v = np.maximum(np.linalg.norm(o[F][:3, keep], axis=0), 0.1 * pm[keep])
        out[F + "_R"] = np.linalg.norm(g[F][:3, keep] - o[F][:3, keep], axis=0) / v
        # d(gamma v_par)/dt: the mirror force is ~ v^2 / L ~ (|p|/m) / 1000 s
        out[F + "_u"] = np.abs(g[F][3, keep] - o[F][3, keep]) / (pm[keep] / 1000.0)
    ls = (0.01 * AU) if lam is None else lam[keep]
    out["s_rem"] = np.abs(g["s_rem"][keep] - o["s_rem"][keep]) / ls
    return out


def compare_states(g, o, tol, pm, skip=None, lam=None):
    """Max relative errors of the continuous state (state_errors) over the particles not in
    skip."""
    keep = np.ones(g["x"].shape[0], dtype=bool) if skip is None else ~skip
    return {k: float(np.max(v)) if v.size else 0.0 for k, v in state_errors(g, o, pm, keep, lam).items()}


def bulk_percentiles(g, o, pm, skip=None, lam=None, q=99):
    """The q-th percentile of every relative state error over the particles not in skip."""
    keep = np.ones(g["x"].shape[0], dtype=bool) if skip is None else ~skip
    return {k: float(np.percentile(v, q)) for k, v in state_errors(g, o, pm, keep, lam).items()}


def ill_conditioned(nodes, wind, ens, calls, final, pm, eps=3e-7, n_dir=2, **kw):
    """Particles whose FP64 oracle result is itself unstable at FP32 resolution: the oracle
    rerun with the start state moved by +-eps (relative) along n_dir seeded directions ends
    more than 1e-5 |p|/m away in gamma v_par from ``final`` (the unperturbed oracle run). A
    trajectory that passes within about eps of a cell face is such a case: the trilinear
    field's gradient jumps across the face, so the side a rounding puts the point on
    changes the mirror force there (a tie between two correct values)."""
    bad = np.zeros(final["u"].shape[0], dtype=bool)
    for d in range(n_dir):
        for sgn in (1.0, -1.0):
            o, _, _ = run_oracle(nodes, wind, ens, calls, perturb=(1000 + d, sgn * eps), **kw)
            bad |= np.abs(o["u"] - final["u"]) > 1e-5 * pm
    return bad
