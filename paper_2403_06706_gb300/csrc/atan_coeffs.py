"""Coefficients of the FP32 path's atan: atan(t) ~ t * p(t^2) on [0, 1], p of degree 7.

Fitted here for minimal maximum absolute error by iteratively reweighted least squares
(Lawson's algorithm) on Chebyshev-spaced points; the octant reduction that maps any
(y, x) to t = min(|x|, |y|) / max(|x|, |y|) in [0, 1] is the textbook one. Running this
script prints the coefficients written into gc_device.cuh (max |error| ~ 4e-8; rounded to
float, as the kernel holds them, 7.0e-8 at t = 1).
"""
import numpy as np


def fit(deg: int = 7, iters: int = 30):
    t = (1 - np.cos(np.linspace(0, np.pi, 4000))) / 2
    s = t * t
    A = np.stack([t * s**k for k in range(deg + 1)], 1)
    c, *_ = np.linalg.lstsq(A, np.arctan(t), rcond=None)
    w = np.ones_like(t)
    for _ in range(iters):
        err = A @ c - np.arctan(t)
        w = w * (1 + 50 * np.abs(err) / np.abs(err).max())
        w /= w.mean()
        c, *_ = np.linalg.lstsq(A * w[:, None], np.arctan(t) * w, rcond=None)
    tt = np.linspace(0, 1, 200001)
    return c, float(np.abs(tt * np.polyval(c[::-1], tt * tt) - np.arctan(tt)).max())


if __name__ == "__main__":
    c, e = fit()
    print("max |error|", e)
    for k, v in enumerate(c):
        print(f"c{k} = {v:.9e}f")
