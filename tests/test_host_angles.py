"""The FP64 path's polar angles without a double-precision atan2 (gc_device.cuh,
`refine_angle`), checked on the CPU: the committed cos/sin table is what its generator writes
and holds correctly rounded values, and the refinement's arithmetic, replayed in float64 from
the FP32 estimate the kernel forms, agrees with numpy's arctan2 to a few ulp everywhere,
including estimates at the worst error the FP32 polynomial can have and points halfway
between reference angles."""
import math
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2403_06706_gb300", "csrc")


def _table():
    text = open(os.path.join(CSRC, "unit_circle_table.h")).read()
    rows = re.findall(r"\{(\S+), (\S+)\},\s+// m = (\d+)", text)
    step = float.fromhex(re.search(r"kCircleStep = (\S+);", text).group(1))
    inv_step = float.fromhex(re.search(r"kCircleInvStep = (\S+);", text).group(1))
    cs = np.array([[float.fromhex(c), float.fromhex(s)] for c, s, _ in rows])
    assert [int(m) for *_, m in rows] == list(range(len(rows)))
    return cs, step, inv_step


def _atan2_f32_coeffs():
    """The FP32 atan polynomial's coefficients as the kernel spells them (highest first)."""
    text = open(os.path.join(CSRC, "gc_device.cuh")).read()
    body = text[text.index("__device__ __forceinline__ float m_atan2"):]
    body = body[:body.index("return copysignf")]
    first = re.search(r"float p = (\S+)f;", body).group(1)
    rest = re.findall(r"p = fmaf\(p, s, (\S+)f\);", body)
    return [np.float32(v) for v in [first, *rest]]


def _atan2_f32(y, x, coeffs):
    """The kernel's FP32 atan2, step for step in float32 (its fast division is within 2 ulp of
    the correctly rounded one used here)."""
    y = y.astype(np.float32)
    x = x.astype(np.float32)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    with np.errstate(invalid="ignore", divide="ignore"):
        t = np.where(mx > 0, mn / mx, np.float32(0)).astype(np.float32)
    s = t * t
    p = np.full_like(t, coeffs[0])
    for c in coeffs[1:]:
        p = (p * s + c).astype(np.float32)
    r = t * p
    r = np.where(ay > ax, np.float32(1.57079632679489662) - r, r)
    r = np.where(x < 0, np.float32(3.14159265358979324) - r, r)
    return np.copysign(r, y).astype(np.float32)


def _refine(X, Y, inv_h, est, cs, step, inv_step):
    n = len(cs)
    m = np.rint(est.astype(np.float32) * np.float32(inv_step)).astype(np.int64) & (n - 1)
    t = (Y * cs[m, 0] - X * cs[m, 1]) * inv_h
    t2 = t * t
    p = t2 * (5.0 / 112.0) + 3.0 / 40.0
    p = t2 * p + 1.0 / 6.0
    d = t * t2 * p + t
    return m.astype(np.float64) * step + d


def test_header_is_the_generators_output():
    import sys
    sys.path.insert(0, CSRC)
    try:
        pytest.importorskip("mpmath")
        import unit_circle_table
    finally:
        sys.path.remove(CSRC)
    assert open(os.path.join(CSRC, "unit_circle_table.h")).read() == unit_circle_table.header_text()


def test_table_is_the_unit_circle_at_the_reference_angles():
    cs, step, inv_step = _table()
    n = len(cs)
    assert n & (n - 1) == 0
    assert step == 2 * math.pi / n and inv_step == n / (2 * math.pi)
    a = np.arange(n) * step
    # numpy's cos/sin (an independent libm) agree to within one ulp of the correctly rounded values
    assert np.all(np.abs(cs[:, 0] - np.cos(a)) <= np.spacing(np.abs(np.cos(a))) + 1e-300)
    assert np.all(np.abs(cs[:, 1] - np.sin(a)) <= np.spacing(np.abs(np.sin(a))) + 1e-300)
    np.testing.assert_allclose(np.hypot(cs[:, 0], cs[:, 1]), 1.0, rtol=0, atol=3e-16)
    # exact values where they are exact
    assert cs[0, 0] == 1.0 and cs[0, 1] == 0.0
    assert cs[n // 4, 1] == 1.0 and cs[n // 2, 0] == -1.0 and cs[3 * n // 4, 1] == -1.0


def test_fp32_atan_polynomial_meets_its_stated_bound():
    """atan(t) ~ t p(t^2) on [0, 1] with the kernel's float coefficients, evaluated in float64:
    within the 7.1e-8 the kernel's comment states (4e-8 before the coefficients are rounded to
    float), and exact at t = 0."""
    c = np.array(_atan2_f32_coeffs(), dtype=np.float64)  # highest power first
    t = np.linspace(0.0, 1.0, 400_001)
    approx = t * np.polyval(c, t * t)
    assert np.abs(approx - np.arctan(t)).max() < 7.1e-8
    assert approx[0] == 0.0


def test_fp32_estimate_is_within_the_refinements_margin():
    coeffs = _atan2_f32_coeffs()
    assert len(coeffs) == 8
    rng = np.random.default_rng(11)
    ang = rng.uniform(-math.pi, math.pi, 400_000)
    r = 10 ** rng.uniform(9.5, 11.6, ang.size)
    y, x = r * np.sin(ang), r * np.cos(ang)
    est = _atan2_f32(y, x, coeffs).astype(np.float64)
    err = np.abs(np.angle(np.exp(1j * (est - np.arctan2(y, x)))))
    assert err.max() < 1e-6


@pytest.mark.parametrize("kind", ["theta", "phi"])
def test_refined_angle_matches_atan2(kind):
    cs, step, inv_step = _table()
    coeffs = _atan2_f32_coeffs()
    rng = np.random.default_rng(5 if kind == "theta" else 6)
    n = 300_000
    half = step / 2
    if kind == "theta":
        ang = np.concatenate([rng.uniform(0, math.pi, n),
                              np.arange(129) * step + half * rng.choice([-1, 1], 129) * (1 - 1e-12),
                              [0.0, math.pi, 1e-9, math.pi - 1e-9]])
        ang = np.clip(ang, 0, math.pi)
    else:
        ang = np.concatenate([rng.uniform(-math.pi, math.pi, n),
                              np.arange(-128, 129) * step + half * (1 - 1e-12),
                              np.arange(-128, 129) * step - half * (1 - 1e-12),
                              [0.0, -1e-12, 1e-12, math.pi, -math.pi + 1e-12]])
    r = 10 ** rng.uniform(9.5, 11.6, ang.size)
    Y, X = r * np.sin(ang), r * np.cos(ang)
    inv_h = 1.0 / np.hypot(X, Y)
    want = np.arctan2(Y, X)
    est = _atan2_f32(Y, X, coeffs)
    # the kernel's estimate, and the same estimate pushed 1e-6 rad either way (the margin the
    # series is sized for)
    for e in (est, est + np.float32(1e-6), est - np.float32(1e-6)):
        got = _refine(X, Y, inv_h, e.astype(np.float32), cs, step, inv_step)
        diff = np.angle(np.exp(1j * (got - want)))
        assert np.abs(diff).max() < 2e-15
        # the range the push folds: theta in [0, pi]; phi in (-0.0123, 2 pi)
        if kind == "theta":
            assert got.min() > -1e-15 and got.max() < math.pi + 1e-15
        else:
            assert got.min() > -0.0123 and got.max() < 2 * math.pi
