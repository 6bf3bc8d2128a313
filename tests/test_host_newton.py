"""Error bound of the FP32 path's FP64 reciprocal and square root (the collision bookkeeping
of the FP32-mixed push): Newton's method from a float estimate, two steps.

    1/x:        y <- y + y (1 - x y)               (two FMAs a step)
    1/sqrt(x):  y <- y + (y / 2) (1 - (x y) y)      (one product and two FMAs a step)
    sqrt(x) = x / sqrt(x) = x (1/sqrt(x))

The steps are replayed here with every FMA rounded once from the exact rational value (as the
hardware does), starting from the float estimate moved to the edge of the error a float
estimate may have (2^-21 relative on either side; the GPU's estimates are within 2^-22). The
results must lie within 4 ulp of the exact values over 40 decades of x.
"""
from fractions import Fraction as Fr

import numpy as np


def fma(a, b, c):
    return float(Fr(a) * Fr(b) + Fr(c))


def rcp_newton(x, y0):
    y = y0
    for _ in range(2):
        y = fma(y, fma(-x, y, 1.0), y)
    return y


def rsqrt_newton(x, y0):
    y = y0
    for _ in range(2):
        y = fma(0.5 * y, fma(-x * y, y, 1.0), y)
    return y


def _ulps(got, exact):
    return abs(Fr(got) - exact) / (abs(exact) * Fr(2) ** -52)


def test_newton_reciprocal_and_square_root_within_four_ulp():
    rng = np.random.default_rng(5)
    xs = 10.0 ** rng.uniform(-10, 30, 400)
    worst_r = worst_q = worst_s = 0.0
    for x in xs:
        x = float(x)
        for d in (-2.0 ** -21, 2.0 ** -21, float(rng.uniform(-2.0 ** -21, 2.0 ** -21))):
            # float estimates at the edge of their error
            r0 = float(np.float32((1.0 / x) * (1.0 + d)))
            q0 = float(np.float32((1.0 / np.sqrt(x)) * (1.0 + d)))
            r = rcp_newton(x, r0)
            worst_r = max(worst_r, float(_ulps(r, 1 / Fr(x))))
            q = rsqrt_newton(x, q0)
            # exact 1/sqrt(x) to ~1e-30 relative: refine in rationals
            e = Fr(1.0 / np.sqrt(x))
            for _ in range(3):
                e = e * (3 - Fr(x) * e * e) / 2
            worst_q = max(worst_q, float(_ulps(q, e)))
            s = x * q
            worst_s = max(worst_s, float(_ulps(s, Fr(x) * e)))
    print("worst ulp: rcp", worst_r, "rsqrt", worst_q, "sqrt", worst_s)
    assert worst_r < 4 and worst_q < 4 and worst_s < 4
