"""gc_advance_noalloc: the push on caller-owned device memory, checked against gc_advance.

Some users of this library cannot let it allocate device memory: a simulation code that
keeps the GPU's memory in its own pool and lends out views of its buffers, or a stepping
loop that must not pay the device-wide synchronisation an allocation can cause. For them
gc_advance_noalloc advances a particle state that sits in the caller's own device buffers
and uses nothing but a fixed scratch array compiled into the library.

Here torch tensors stand in for the caller's buffers. The entry point is called twice in
a row through the C ABI (so the second call runs on scratch the first call left behind)
and each result is compared with gc_advance of a context holding the same particles:
integer state exactly, the continuous state within the FP64 parity tolerance (1e-9). A warm
call leaves the device's free memory exactly as it found it, and the largest ensemble table
the scratch holds (GC_NOALLOC_MAX_ENSEMBLES) gives the results of gc_advance too.
This file is collected last and also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from _cases import compare_states, momentum_scale
from paper_2403_06706_gb300 import synth

pytestmark = pytest.mark.gpu
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")
torch = pytest.importorskip("torch")

WIND = synth.WindSpec(64, 32, 64)
R_OUT = synth.r_out_default(WIND)
ENS = (
    synth.EnsembleSpec(257, r0_au=0.28, lat_deg=24.0, lam_au=0.5, r_out_au=R_OUT),
    synth.EnsembleSpec(61, r0_au=0.5, lat_deg=-30.0, lon_deg=47.0, E0_keV=40.0, lam_au=0.02,
                       r_in_au=0.45, r_out_au=0.6, scatter_law=1),
)
CALLS = ((0.5, 180), (0.5, 120))


def _to_device(state):
    """Copy a host state (dict of numpy arrays) into fresh CUDA tensors."""
    dev = {}
    for k, v in state.items():
        t = torch.from_numpy(v.view(np.int32) if v.dtype == np.uint32 else v).cuda()
        dev[k] = t.contiguous()
    torch.cuda.synchronize()
    return dev


def _to_host(dev):
    torch.cuda.synchronize()
    return {k: (t.cpu().numpy().view(np.uint32) if t.dtype == torch.int32 else t.cpu().numpy())
            for k, t in dev.items()}


def _soa(dev, n):
    s = gcpush.ParticleSoA()
    s.n = n
    for k in gcpush.F64_STATE + ("F0", "F1"):
        setattr(s, k, C.cast(C.c_void_p(dev[k].data_ptr()), C.POINTER(C.c_double)))
    for k in gcpush.U32_STATE:
        setattr(s, k, C.cast(C.c_void_p(dev[k].data_ptr()), C.POINTER(C.c_uint32)))
    return s


def _noalloc(precision, nodes_dev, dev, n, t0, step0, dt, n_steps, n_ens=None, dtype=None, ens=None):
    L = gcpush.load()
    o = gcpush.Options()
    o.precision, o.device, o.seed = precision, 0, 13
    o.stream = torch.cuda.current_stream().cuda_stream
    g = gcpush.GridDesc()
    g.n_ph, g.n_th, g.n_r = nodes_dev.shape[0], nodes_dev.shape[1], nodes_dev.shape[2]
    g.dtype = dtype if dtype is not None else (gcpush.DTYPE_F64 if precision == gcpush.PREC_FP64
                                               else gcpush.DTYPE_F32)
    g.r_min_au, g.r_max_au, g.ideal = WIND.r_min_au, WIND.r_max_au, 1
    if ens is None:
        ens = list(ENS) if n_ens is None else [ENS[0]] * n_ens
    arr = (gcpush.EnsembleDesc * len(ens))(*[gcpush.ensemble_desc(e) for e in ens])
    st = gcpush.StatsOut()
    rc = L.gc_advance_noalloc(C.byref(o), C.byref(g), C.c_void_p(nodes_dev.data_ptr()), arr, len(ens),
                              C.byref(_soa(dev, n)), t0, step0, dt, n_steps, 0.0, C.byref(st))
    return rc, st


@pytest.mark.parametrize("precision,np_dtype", [(gcpush.PREC_FP32_MIXED, np.float32),
                                                (gcpush.PREC_FP64, np.float64)])
def test_noalloc_matches_gc_advance_on_two_calls(precision, np_dtype):
    nodes = synth.wind_grid(WIND, dtype=np_dtype)
    nodes_dev = torch.from_numpy(nodes).cuda()
    with gcpush.Context(precision=precision, seed=13, dt_init=0.5) as ctx:
        ctx.field_load(nodes, WIND.r_min_au, WIND.r_max_au)
        ctx.inject(list(ENS))
        dev = _to_device(ctx.get_state())
        n = ctx.n
        t0, step0 = 0.0, 0
        for dt, n_steps in CALLS:
            before = ctx.stats()
            ctx.advance(dt, n_steps)
            after = ctx.stats()
            ref = ctx.get_state()
            rc, st = _noalloc(precision, nodes_dev, dev, n, t0, step0, dt, n_steps)
            assert rc == gcpush.GC_OK, gcpush.load().gc_last_error()
            got = _to_host(dev)
            for k in gcpush.U32_STATE:
                np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
            err = compare_states(got, ref, 1e-9, momentum_scale(ref, nodes, WIND, ENS))
            assert max(err.values()) < 1e-9, err
            assert st.collisions == after["collisions"] - before["collisions"]
            assert st.rebirths == after["rebirths"] - before["rebirths"]
            assert st.step == step0 + n_steps and st.flags_or == 0
            t0 += dt * n_steps
            step0 += n_steps
        assert after["collisions"] > 0 and after["rebirths"] > 0


def test_noalloc_rejects_oversize_and_wrong_grid_type():
    nodes = synth.wind_grid(WIND, dtype=np.float32)
    nodes_dev = torch.from_numpy(nodes).cuda()
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=13) as ctx:
        ctx.field_load(nodes, WIND.r_min_au, WIND.r_max_au)
        ctx.inject(list(ENS))
        dev = _to_device(ctx.get_state())
        n = ctx.n
    rc, _ = _noalloc(gcpush.PREC_FP32_MIXED, nodes_dev, dev, n, 0.0, 0, 0.5, 5,
                     n_ens=257)  # GC_NOALLOC_MAX_ENSEMBLES + 1
    assert rc == -1 and b"ensembles" in gcpush.load().gc_last_error()
    rc, _ = _noalloc(gcpush.PREC_FP32_MIXED, nodes_dev, dev, n, 0.0, 0, 0.5, 5,
                     dtype=gcpush.DTYPE_F64)
    assert rc == -1 and b"dtype" in gcpush.load().gc_last_error()
    # a particle naming an ensemble the table does not hold is refused before the push
    dev["ens"][3] = 7
    rc, _ = _noalloc(gcpush.PREC_FP32_MIXED, nodes_dev, dev, n, 0.0, 0, 0.5, 5)
    assert rc == -1 and b"ensemble" in gcpush.load().gc_last_error()


def test_noalloc_allocates_no_device_memory():
    """After one warm call (which loads the kernels), a call leaves cudaMemGetInfo's free
    device memory unchanged to the byte."""
    nodes = synth.wind_grid(WIND, dtype=np.float32)
    nodes_dev = torch.from_numpy(nodes).cuda()
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED, seed=13) as ctx:
        ctx.field_load(nodes, WIND.r_min_au, WIND.r_max_au)
        ctx.inject(list(ENS))
        dev = _to_device(ctx.get_state())
        n = ctx.n
    rc, _ = _noalloc(gcpush.PREC_FP32_MIXED, nodes_dev, dev, n, 0.0, 0, 0.5, 20)
    assert rc == gcpush.GC_OK, gcpush.load().gc_last_error()
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    rc, _ = _noalloc(gcpush.PREC_FP32_MIXED, nodes_dev, dev, n, 10.0, 20, 0.5, 20)
    free1, _ = torch.cuda.mem_get_info()
    assert rc == gcpush.GC_OK, gcpush.load().gc_last_error()
    assert free1 == free0, (free0, free1, total)


def test_noalloc_full_ensemble_table():
    """GC_NOALLOC_MAX_ENSEMBLES (256) ensembles of two electrons each, every one with its own
    site, energy, free path and scattering law, so that the whole table is read: the result
    equals gc_advance's on a context injected with the same ensembles."""
    ens = [synth.EnsembleSpec(2, r0_au=0.25 + 0.001 * k, lat_deg=-30.0 + 0.23 * k, lon_deg=1.4 * k,
                              E0_keV=20.0 + k, lam_au=0.01 + 0.004 * k, r_out_au=R_OUT, scatter_law=k % 2)
           for k in range(256)]
    nodes = synth.wind_grid(WIND, dtype=np.float64)
    nodes_dev = torch.from_numpy(nodes).cuda()
    with gcpush.Context(precision=gcpush.PREC_FP64, seed=13, dt_init=0.5) as ctx:
        ctx.field_load(nodes, WIND.r_min_au, WIND.r_max_au)
        ctx.inject(ens)
        dev = _to_device(ctx.get_state())
        n = ctx.n
        ctx.advance(0.5, 60)
        ref = ctx.get_state()
        s = ctx.stats()
    assert int(ref["ens"].max()) == 255
    rc, st = _noalloc(gcpush.PREC_FP64, nodes_dev, dev, n, 0.0, 0, 0.5, 60, ens=ens)
    assert rc == gcpush.GC_OK, gcpush.load().gc_last_error()
    got = _to_host(dev)
    for k in gcpush.U32_STATE:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    err = compare_states(got, ref, 1e-9, momentum_scale(ref, nodes, WIND, ens))
    assert max(err.values()) < 1e-9, err
    assert st.collisions == s["collisions"] and st.rebirths == s["rebirths"]
