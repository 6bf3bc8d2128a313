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
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_HID_LAYERS, N_OUT = 3, 256, 4, 8


def shapes(n_h: int = N_H, n_out: int = N_OUT):
    s = [("W1", (n_h, N_IN)), ("b1", (n_h,))]
    for k in range(2, N_HID_LAYERS + 1):
        s += [(f"W{k}", (n_h, n_h)), (f"b{k}", (n_h,))]
    s += [("W5", (n_out, n_h)), ("b5", (n_out,))]
    return s


def n_params(n_h: int = N_H, n_out: int = N_OUT) -> int:
    return int(sum(np.prod(sh) for _, sh in shapes(n_h, n_out)))


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


def forward(flat, x, omega0: float, jac: bool = False):
    """y (n, 8) and, with jac, J (n, 8, 3) = dy/dx."""
    p = unpack(flat)
    x = np.asarray(x, dtype=np.float64)
    z = omega0 * (x @ p["W1"].T + p["b1"])
    h = np.sin(z)
    c = np.cos(z)
    t = None
    if jac:
        # t[:, j, :] = d h1 / d x_j
        t = omega0 * c[:, None, :] * p["W1"].T[None, :, :]
    for k in range(2, N_HID_LAYERS + 1):
        W, b = p[f"W{k}"], p[f"b{k}"]
        z = h @ W.T + b
        if jac:
            t = np.cos(z)[:, None, :] * (t @ W.T)
        h = np.sin(z)
    y = h @ p["W5"].T + p["b5"]
    if not jac:
        return y
    J = np.transpose(t @ p["W5"].T, (0, 2, 1))
    return y, J


def loss_and_grad(flat, x, target, omega0: float):
    """MSE over samples and channels and its gradient (same layout as the parameters)."""
    p = unpack(flat)
    x = np.asarray(x, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    hs, cs = [], []
    z = omega0 * (x @ p["W1"].T + p["b1"])
    hs.append(np.sin(z))
    cs.append(np.cos(z))
    for k in range(2, N_HID_LAYERS + 1):
        z = hs[-1] @ p[f"W{k}"].T + p[f"b{k}"]
        hs.append(np.sin(z))
        cs.append(np.cos(z))
    y = hs[-1] @ p["W5"].T + p["b5"]
    r = y - target
    L = float(np.mean(r * r))
    dy = 2.0 * r / r.size
    g = {"W5": dy.T @ hs[-1], "b5": dy.sum(0)}
    dh = dy @ p["W5"]
    for k in range(N_HID_LAYERS, 1, -1):
        dz = dh * cs[k - 1]
        g[f"W{k}"] = dz.T @ hs[k - 2]
        g[f"b{k}"] = dz.sum(0)
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
