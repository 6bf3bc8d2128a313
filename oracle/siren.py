"""FP64 reference of the neural field: a SIREN (sine-activated MLP, Sitzmann et al. 2020).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests, the smoke check and the
benchmark's CPU leg use it; the CUDA library neither imports nor calls it.

Network (3 -> 256 x 4 -> 8): z1 = w0 (W1 x + b1), h1 = sin z1; z_k = W_k h_{k-1} + b_k,
h_k = sin z_k (k = 2..4); y = W5 h4 + b5. Input x is the position scaled to the unit cube;
the 8 outputs are the scaled field channels. Derivatives:
* forward-mode Jacobian dy/dx: t1 = w0 cos(z1) * W1[:, j], t_k = cos(z_k) * (W_k t_{k-1}),
  J = W5 t4 (the chain rule, one tangent per input direction);
* reverse mode for the mean-squared error L = mean((y - target)^2): dy = 2 (y - t) / size,
  dz_k = (W_{k+1}^T dz_{k+1}) * cos(z_k), dW_k = dz_k^T h_{k-1}, db_k = sum dz_k;
* Adam (Kingma & Ba 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
  theta <- theta - lr m_hat / (sqrt(v_hat) + eps) with bias-corrected m_hat, v_hat.

Parameter vector (float32 or float64, this order): W1 (256 x 3), b1 (256), then for k = 2..4
W_k (256 x 256, [out][in]), b_k (256), then W5 (8 x 256), b5 (8).

BF16 reading (``bf16=True``): the network as the tensor cores run it, with W2..W5 and the
values carried between layers (h_k and the tangents t_k; in the backward pass the dz_k fed to
the weight products) rounded to bfloat16 (8 significant bits, round to nearest even), every
sum and product otherwise exact. W1, the biases, z_1 and the output stay unrounded.

Targets (``grid_targets``): the eight node channels [B, E, |B|, Phi] of a node-centred
spherical grid interpolated trilinearly in (r, theta, phi) index space (poles included,
phi periodic, clamped to the edge cells), scaled to O(1) as the network's outputs:
B and |B| times (r / 1 AU)^2 / B_scale, E times (r / 1 AU) / E_scale, Phi / (E_scale AU).
``physical_field`` undoes that scaling for B and E with the product rule.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_HID_LAYERS, N_OUT = 3, 256, 4, 8
AU = 1.495978707e11


def round_bf16(a):
    """Round to bfloat16 (8 significant bits, ties to even), returned as float64."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)
    return np.ldexp(np.rint(m * 256.0), e - 8)


def _rb(a, on):
    return round_bf16(a) if on else a


def _weights(p, bf16):
    """Weights as the evaluation uses them (W2..W5 rounded in the BF16 reading)."""
    if not bf16:
        return p
    q = dict(p)
    for k in range(2, N_HID_LAYERS + 2):
        q[f"W{k}"] = round_bf16(p[f"W{k}"])
    return q


def shapes(n_h: int = N_H, n_out: int = N_OUT):
    s = [("W1", (n_h, N_IN)), ("b1", (n_h,))]
    for k in range(2, N_HID_LAYERS + 1):
        s += [(f"W{k}", (n_h, n_h)), (f"b{k}", (n_h,))]
    s += [("W5", (n_out, n_h)), ("b5", (n_out,))]
    return s


def n_params(n_h: int = N_H, n_out: int = N_OUT) -> int:
    return int(sum(np.prod(sh) for _, sh in shapes(n_h, n_out)))


def offset(name: str, n_h: int = N_H, n_out: int = N_OUT) -> int:
    """Index of the first element of parameter block `name` in the flat vector."""
    o = 0
    for nm, sh in shapes(n_h, n_out):
        if nm == name:
            return o
        o += int(np.prod(sh))
    raise KeyError(name)


def unpack(flat, n_h: int = N_H, n_out: int = N_OUT) -> dict:
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, sh in shapes(n_h, n_out):
        n = int(np.prod(sh))
        out[name] = flat[o:o + n].reshape(sh)
        o += n
    assert o == flat.size
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel()
                           for name, _ in shapes(p["W1"].shape[0], p["W5"].shape[0])])


def forward(flat, x, omega0: float, jac: bool = False, bf16: bool = False):
    """y (n, 8) and, with jac, J (n, 8, 3) = dy/dx."""
    p = _weights(unpack(flat), bf16)
    x = np.asarray(x, dtype=np.float64)
    z = omega0 * (x @ p["W1"].T + p["b1"])
    h = _rb(np.sin(z), bf16)
    c = np.cos(z)
    t = None
    if jac:
        # t[:, j, :] = d h1 / d x_j
        t = _rb(omega0 * c[:, None, :] * p["W1"].T[None, :, :], bf16)
    for k in range(2, N_HID_LAYERS + 1):
        W, b = p[f"W{k}"], p[f"b{k}"]
        z = h @ W.T + b
        if jac:
            t = _rb(np.cos(z)[:, None, :] * (t @ W.T), bf16)
        h = _rb(np.sin(z), bf16)
    y = h @ p["W5"].T + p["b5"]
    if not jac:
        return y
    J = np.transpose(t @ p["W5"].T, (0, 2, 1))
    return y, J


def loss_and_grad(flat, x, target, omega0: float, bf16: bool = False):
    """MSE over samples and channels and its gradient (same layout as the parameters)."""
    p = _weights(unpack(flat), bf16)
    x = np.asarray(x, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    hs, cs = [], []
    z = omega0 * (x @ p["W1"].T + p["b1"])
    hs.append(_rb(np.sin(z), bf16))
    cs.append(np.cos(z))
    for k in range(2, N_HID_LAYERS + 1):
        z = hs[-1] @ p[f"W{k}"].T + p[f"b{k}"]
        hs.append(_rb(np.sin(z), bf16))
        cs.append(np.cos(z))
    y = hs[-1] @ p["W5"].T + p["b5"]
    r = y - target
    L = float(np.mean(r * r))
    dy = 2.0 * r / r.size
    g = {"W5": dy.T @ hs[-1], "b5": dy.sum(0)}
    dh = dy @ p["W5"]
    for k in range(N_HID_LAYERS, 1, -1):
        dz = dh * cs[k - 1]
        g[f"b{k}"] = dz.sum(0)
        dz = _rb(dz, bf16)
        g[f"W{k}"] = dz.T @ hs[k - 2]
        dh = dz @ p[f"W{k}"]
    dz1 = dh * cs[0] * omega0
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return L, pack(g)


def adam_step(flat, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update; step counts from 1. Returns (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1**step)
    vh = v / (1.0 - beta2**step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def grid_targets(nodes, r_min: float, r_max: float, x, r_scale: float, B_scale: float, E_scale: float):
    """Scaled eight-channel trilinear interpolant of nodes [n_ph][n_th][n_r][8] (SI, radii in
    m) at scaled points x (n, 3), R = x r_scale."""
    nodes = np.asarray(nodes, dtype=np.float64)
    n_ph, n_th, n_r, _ = nodes.shape
    R = np.asarray(x, dtype=np.float64) * r_scale
    out = np.empty((R.shape[0], 8))
    dr = (r_max - r_min) / (n_r - 1)
    for q, (X, Y, Z) in enumerate(R):
        rho = np.hypot(X, Y)
        r = np.sqrt(X * X + Y * Y + Z * Z)
        th = np.arctan2(rho, Z)
        ph = np.arctan2(Y, X) % (2 * np.pi)
        xr, xt, xp = (r - r_min) / dr, th / (np.pi / (n_th - 1)), ph / (2 * np.pi / n_ph)
        i, j, k = int(np.floor(xr)), int(np.floor(xt)), int(np.floor(xp))
        fr, ft, fp = xr - i, xt - j, xp - k
        if i < 0:
            i, fr = 0, 0.0
        elif i > n_r - 2:
            i, fr = n_r - 2, 1.0
        if j < 0:
            j, ft = 0, 0.0
        elif j > n_th - 2:
            j, ft = n_th - 2, 1.0
        k %= n_ph
        v = np.zeros(8)
        for a in (0, 1):
            for b in (0, 1):
                for c in (0, 1):
                    w = (fr if a else 1 - fr) * (ft if b else 1 - ft) * (fp if c else 1 - fp)
                    v += w * nodes[(k + c) % n_ph, j + b, i + a]
        s2, s1 = (r / AU) ** 2 / B_scale, (r / AU) / E_scale
        out[q, 0:3] = v[0:3] * s2
        out[q, 3:6] = v[3:6] * s1
        out[q, 6] = v[6] * s2
        out[q, 7] = v[7] / (E_scale * AU)
    return out


def physical_field(x, y, J, r_scale: float, B_scale: float, E_scale: float):
    """B, E (n, 3) and dB, dE (n, 3, 3) with [d][c] = dF_c / dR_d at R = x r_scale from the
    scaled outputs y (n, 8) and J = dy/dx (n, 8, 3): B = B_scale y_B (AU / r)^2,
    E = E_scale y_E (AU / r)."""
    R = np.asarray(x, dtype=np.float64) * r_scale
    r2 = (R * R).sum(1)
    a = AU / np.sqrt(r2)
    B = B_scale * y[:, 0:3] * (a * a)[:, None]
    E = E_scale * y[:, 3:6] * a[:, None]
    # d(AU/r)^2/dR_d = -2 (AU/r)^2 R_d / r^2 ; d(AU/r)/dR_d = -(AU/r) R_d / r^2
    u = R / r2[:, None]
    dB = B_scale * (a * a)[:, None, None] * (np.transpose(J[:, 0:3, :], (0, 2, 1)) / r_scale
                                              - 2.0 * u[:, :, None] * y[:, None, 0:3])
    dE = E_scale * a[:, None, None] * (np.transpose(J[:, 3:6, :], (0, 2, 1)) / r_scale
                                       - u[:, :, None] * y[:, None, 3:6])
    return B, E, dB, dE
