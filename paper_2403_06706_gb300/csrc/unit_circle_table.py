"""Writes unit_circle_table.h: cosine and sine of the 256 reference angles of the FP64 path's
angle refinement (gc_device.cuh, `refine_angle`).

The reference angles are a_m = m * (2 pi / 256) for m = 0..255, each product rounded to double
exactly as the kernel forms it (`__dmul_rn(m, kCircleStep)` with kCircleStep the double
nearest 2 pi, divided by 256, which is exact). Each cosine and sine is evaluated at that double
in 60-digit arithmetic and rounded once to double, so the table holds correctly rounded values.

Run from this directory: `python unit_circle_table.py` (rewrites the header; a CPU test checks
that the committed header matches this script's output).
"""
import math
import os

import mpmath

N = 256


def entries():
    step = 2.0 * math.pi / N  # exact: a power-of-two scaling of the double nearest 2 pi
    mpmath.mp.dps = 60
    out = []
    for m in range(N):
        a = float(m) * step  # IEEE round-to-nearest product, as on the device
        x = mpmath.mpf(a)
        out.append((a, float(mpmath.cos(x)), float(mpmath.sin(x))))
    return step, out


def header_text() -> str:
    step, rows = entries()
    lines = [
        "// unit_circle_table.h -- written by unit_circle_table.py; do not edit by hand.",
        f"// cos and sin of a_m = m * (2 pi / {N}), m = 0..{N - 1} (the product rounded to double, as the",
        "// kernel forms it), each correctly rounded to double.",
        "#pragma once",
        f"#define GC_CIRCLE_N {N}",
        f"static constexpr double kCircleStep = {step.hex()};  // 2 pi / {N}",
        f"static constexpr double kCircleInvStep = {(N / (2.0 * math.pi)).hex()};  // {N} / (2 pi)",
        "static __device__ const double2 kUnitCircle[GC_CIRCLE_N] = {",
    ]
    for m, (_, c, s) in enumerate(rows):
        lines.append(f"    {{{c.hex()}, {s.hex()}}},  // m = {m}")
    lines.append("};")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "unit_circle_table.h")
    with open(path, "w") as f:
        f.write(header_text())
    print("wrote", path)
