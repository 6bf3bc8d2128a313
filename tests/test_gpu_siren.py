"""The neural field on the tensor cores against the FP64 oracle (oracle/siren.py).

* Fused evaluation (values and the forward-mode Jacobian) against the oracle's BF16 reading
  (the same BF16 roundings of W2..W5 and of the values carried between layers, everything
  else exact). The kernel accumulates in FP32 and uses the hardware sine and cosine, so its
  pre-rounding values differ from the oracle's by ~1e-6 relative; each BF16 rounding turns
  such a difference into a full ulp (2^-8) with probability ~1e-6 / 2^-8, and the flipped
  values feed 256 sums of the next layer, so the two BF16 computations decorrelate partly
  over the four layers (measured: a tenth to a sixth of the full BF16 noise in RMS, half of it in
  the maximum). Bounds, relative to the outputs' RMS: values 1e-3 RMS and 2e-2 for any single
  element, Jacobian 2e-3 and 3e-2 (its rows pass through one more rounding per layer), and
  1e-4 for the mean difference of any output over all points (a missing or misplaced term
  would be systematic; rounding noise averages out). Against the exact FP64 network, where the whole BF16
  rounding noise shows: 1e-2 RMS and 5e-2 elementwise.
* Field mode (physical B, E and their gradients): the kernel's product-rule unscaling
  against the oracle's, applied to the kernel's own raw outputs (FP32 rounding only).
* Training: targets, loss and gradient, and Adam, each against the oracle.
Sizes span several 64-point tiles per CTA with a ragged tail; the empty input is a no-op.
"""
import numpy as np
import pytest

from oracle import siren
from paper_2403_06706_gb300 import synth

pytestmark = pytest.mark.gpu
gcpush = pytest.importorskip("paper_2403_06706_gb300.gcpush")
torch = pytest.importorskip("torch")

W0 = 30.0
RS_AU = 2.5
B_S, E_S = 3.5e-9, 3.5e-9 * 4.0e5


def _points(n, seed):
    rng = np.random.default_rng(seed)
    r = (rng.uniform(0.1**3, 1.0, n)) ** (1 / 3) * 0.999
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return (v * r[:, None]).astype(np.float32)


@pytest.fixture(scope="module")
def ctx():
    with gcpush.Context(precision=gcpush.PREC_FP32_MIXED) as c:
        yield c


@pytest.fixture(scope="module")
def params():
    return synth.siren_init(seed=3)


def _eval(c, x, jac=True):
    xd = torch.from_numpy(x).cuda()
    y = torch.full((x.shape[0], 8), float("nan"), device="cuda")
    J = torch.full((x.shape[0], 8, 3), float("nan"), device="cuda") if jac else None
    c.siren_eval(xd, y, J)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64), (J.cpu().numpy().astype(np.float64) if jac else None)


def _rel(a, b):
    s = np.sqrt(np.mean(b * b))
    return np.abs(a - b).max() / s, np.sqrt(np.mean((a - b) ** 2)) / s


def _bias(a, b):
    """largest mean difference of one output over all points, relative to the RMS"""
    d = (a - b).reshape(a.shape[0], -1).mean(0)
    return np.abs(d).max() / np.sqrt(np.mean(b * b))


def _check_bf16(y, J, yo, Jo, what):
    ey, Ey = _rel(y, yo)
    eJ, EJ = _rel(J, Jo)
    by, bJ = _bias(y, yo), _bias(J, Jo)
    print(f"{what}: y max {ey:.2e} rms {Ey:.2e} bias {by:.2e}; J max {eJ:.2e} rms {EJ:.2e} bias {bJ:.2e}")
    assert np.isfinite(y).all() and np.isfinite(J).all()
    assert ey < 2e-2 and Ey < 1e-3 and eJ < 3e-2 and EJ < 2e-3, (ey, Ey, eJ, EJ)
    return by, bJ


def test_eval_matches_bf16_oracle_many_tiles(ctx, params):
    ctx.siren_set(params, omega0=W0, r_max_au=RS_AU, B_scale=B_S, E_scale=E_S)
    n = 64 * 152 * 2 + 37
    x = _points(n, 1)
    y, J = _eval(ctx, x)
    yo, Jo = siren.forward(params.astype(np.float64), x.astype(np.float64), W0, jac=True, bf16=True)
    by, bJ = _check_bf16(y, J, yo, Jo, "bf16 reading")
    assert by < 1e-4 and bJ < 1e-4, (by, bJ)


@pytest.mark.parametrize("n", [1, 63, 64, 65, 200])
def test_eval_small_and_ragged(ctx, params, n):
    ctx.siren_set(params, omega0=W0, r_max_au=RS_AU, B_scale=B_S, E_scale=E_S)
    x = _points(n, 10 + n)
    y, J = _eval(ctx, x)
    yo, Jo = siren.forward(params.astype(np.float64), x.astype(np.float64), W0, jac=True, bf16=True)
    _check_bf16(y, J, yo, Jo, f"n={n}")


def test_eval_empty_is_a_noop(ctx, params):
    ctx.siren_set(params, omega0=W0, r_max_au=RS_AU, B_scale=B_S, E_scale=E_S)
    x = torch.zeros((0, 3), device="cuda")
    y = torch.zeros((0, 8), device="cuda")
    ctx.siren_eval(x, y, None)


def test_eval_bf16_cost_against_exact_network(ctx, params):
    ctx.siren_set(params, omega0=W0, r_max_au=RS_AU, B_scale=B_S, E_scale=E_S)
    x = _points(4096, 2)
    y, J = _eval(ctx, x)
    yo, Jo = siren.forward(params.astype(np.float64), x.astype(np.float64), W0, jac=True)
    print("BF16 vs exact FP64 network: y", _rel(y, yo), "J", _rel(J, Jo))
    assert _rel(y, yo)[1] < 1e-2 and _rel(J, Jo)[1] < 1e-2
    assert _rel(y, yo)[0] < 5e-2 and _rel(J, Jo)[0] < 5e-2


def test_field_mode_matches_oracle_unscaling(ctx, params):
    ctx.siren_set(params, omega0=W0, r_max_au=RS_AU, B_scale=B_S, E_scale=E_S)
    n = 3001
    x = _points(n, 4)
    xd = torch.from_numpy(x).cuda()
    fd = torch.full((n, 24), float("nan"), device="cuda")
    ctx.siren_field(xd, fd)
    torch.cuda.synchronize()
    f = fd.cpu().numpy().astype(np.float64)
    y, J = _eval(ctx, x)
    B, E, dB, dE = siren.physical_field(x.astype(np.float64), y, J, RS_AU * siren.AU, B_S, E_S)
    for name, g, o in (("B", f[:, 0:3], B), ("E", f[:, 3:6], E), ("dB", f[:, 6:15], dB.reshape(n, 9)),
                       ("dE", f[:, 15:24], dE.reshape(n, 9))):
        # the field spans decades in r: compare relative to each point's own scale
        scale = np.sqrt(np.mean(o * o, axis=1, keepdims=True))
        err = np.abs(g - o) / scale
        print(name, err.max())
        assert err.max() < 1e-4, name


@pytest.fixture(scope="module")
def small_grid():
    w = synth.WindSpec(32, 16, 32, eps=0.1, n_modes=4)
    return w, synth.wind_grid(w, dtype=np.float32)


def test_training_targets_match_oracle_interpolant(ctx, params, small_grid):
    w, nodes = small_grid
    ctx.field_load(nodes, w.r_min_au, w.r_max_au)
    ctx.siren_set(params, omega0=W0, r_max_au=RS_AU, B_scale=B_S, E_scale=E_S)
    x = _points(2000, 5)
    t = torch.zeros((2000, 8), device="cuda")
    ctx.field_targets(torch.from_numpy(x).cuda(), t)
    torch.cuda.synchronize()
    to = siren.grid_targets(nodes.astype(np.float64), w.r_min_au * siren.AU, w.r_max_au * siren.AU,
                            x.astype(np.float64), RS_AU * siren.AU, B_S, E_S)
    np.testing.assert_allclose(t.cpu().numpy(), to, rtol=2e-6, atol=2e-6 * np.abs(to).max())


def test_loss_and_gradient_match_bf16_oracle(ctx, params):
    ctx.siren_set(params, omega0=W0, r_max_au=RS_AU, B_scale=B_S, E_scale=E_S)
    n = 512
    rng = np.random.default_rng(6)
    x = _points(n, 6)
    t = (rng.normal(size=(n, 8)) * 0.3).astype(np.float32)
    g = torch.zeros(gcpush.SIREN_NPARAMS, device="cuda")
    loss = ctx.siren_loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), g)
    Lo, go = siren.loss_and_grad(params.astype(np.float64), x.astype(np.float64), t.astype(np.float64), W0,
                                 bf16=True)
    gg = g.cpu().numpy().astype(np.float64)
    print("loss", loss, Lo, "grad rel", np.linalg.norm(gg - go) / np.linalg.norm(go))
    assert abs(loss - Lo) < 1e-4 * Lo
    assert np.linalg.norm(gg - go) / np.linalg.norm(go) < 2e-3
    # every parameter block carries its own gradient
    d = siren.unpack(go)
    dg = siren.unpack(gg)
    for k in d:
        assert np.linalg.norm(dg[k] - d[k]) <= 1e-2 * np.linalg.norm(d[k]) + 1e-12, k


def test_adam_step_matches_oracle(ctx, params, small_grid):
    w, nodes = small_grid
    ctx.field_load(nodes, w.r_min_au, w.r_max_au)
    ctx.siren_set(params, omega0=W0, r_max_au=RS_AU, B_scale=B_S, E_scale=E_S)
    n = 1024
    x = _points(n, 7)
    xd = torch.from_numpy(x).cuda()
    t = torch.zeros((n, 8), device="cuda")
    ctx.field_targets(xd, t)
    g = torch.zeros(gcpush.SIREN_NPARAMS, device="cuda")
    ctx.siren_loss_grad(xd, t, g)
    lr = 1e-3
    ctx.field_fit(xd, n_epochs=1, batch=n, lr=lr)
    p1 = ctx.siren_get().astype(np.float64)
    ref, _, _ = siren.adam_step(params.astype(np.float64), g.cpu().numpy().astype(np.float64),
                                np.zeros(params.size), np.zeros(params.size), 1, lr)
    err = np.abs(p1 - ref)
    print("adam max err / lr", err.max() / lr)
    assert err.max() < 2e-3 * lr + 1e-6


def test_fit_reduces_the_loss(ctx, small_grid):
    w, nodes = small_grid
    ctx.field_load(nodes, w.r_min_au, w.r_max_au)
    ctx.siren_set(synth.siren_init(seed=4), omega0=W0, r_max_au=RS_AU, B_scale=B_S, E_scale=E_S)
    x = _points(1 << 16, 8)
    loss = ctx.field_fit(x, n_epochs=12, batch=4096, lr=1e-4)
    print("loss per epoch", loss)
    assert np.all(np.isfinite(loss))
    assert loss[-1] < 0.2 * loss[0]
