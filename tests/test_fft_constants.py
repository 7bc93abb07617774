"""The radix-16 rotation constants of the FP32 line FFT (csrc/fft_core.cuh,
Rot16Const<float>): each literal is an exact float, the rotation it encodes,
(1 + (cos - 1)) + i sin, lies within 1e-8 of the unit circle and within 3e-8
rad of its angle, and for pi/8 and pi/4 it is the best such float pair among
the neighbours of the nearest roundings.  The rounded (cos, sin) pairs lie
5.7e-8 and 3.4e-8 inside the circle, which is checked too, since that gap is
what the (cos - 1, sin) form exists to close.  Exact rational arithmetic.
The FP64 constants (Rot16Const<double>) are the correctly rounded doubles."""
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1410_2855_gb300", "csrc",
                   "fft_core.cuh")


def float_constants():
    text = open(SRC).read()
    body = text[text.index("template <> struct Rot16Const<float>"):]
    body = body[:body.index("};")]
    vals = dict(re.findall(r"(cm8|s8|cm4|s4)\s*=\s*(-?[0-9.]+)f", body))
    assert set(vals) == {"cm8", "s8", "cm4", "s4"}, vals
    return {k: Fraction(v) for k, v in vals.items()}


def is_float32(q: Fraction) -> bool:
    return Fraction(float(np.float32(float(q)))) == q


def norm_err(cm: Fraction, s: Fraction) -> float:
    return float((1 + cm) ** 2 + s ** 2 - 1)


def neighbours(x: float, k: int):
    f = np.float32(x)
    out = [f]
    up = down = f
    for _ in range(k):
        up, down = np.nextafter(up, np.float32(2)), np.nextafter(down, np.float32(-2))
        out += [up, down]
    return [Fraction(float(v)) for v in out]


def test_literals_are_exact_floats():
    for name, q in float_constants().items():
        assert is_float32(q), name


def test_rotations_lie_near_the_unit_circle_and_their_angles():
    c = float_constants()
    for cm, s, theta in ((c["cm8"], c["s8"], math.pi / 8), (c["cm4"], c["s4"], math.pi / 4)):
        assert abs(norm_err(cm, s)) <= 1e-8
        assert abs(math.atan2(float(s), float(1 + cm)) - theta) <= 3e-8


def test_pairs_are_the_best_among_neighbouring_floats():
    c = float_constants()
    for cm, s, theta in ((c["cm8"], c["s8"], math.pi / 8), (c["cm4"], c["s4"], math.pi / 4)):
        best = min(abs(norm_err(a, b)) for a in neighbours(math.cos(theta) - 1, 2)
                   for b in neighbours(math.sin(theta), 2)
                   if abs(math.atan2(float(b), float(1 + a)) - theta) <= 3e-8)
        assert abs(norm_err(cm, s)) <= best * (1 + 1e-9)


def test_rounded_cos_sin_pairs_fall_inside_the_circle():
    # The form these constants replace: (cos, sin) rounded to nearest.
    for theta, gap in ((math.pi / 8, 5.7e-8), (math.pi / 4, 3.4e-8)):
        cf, sf = Fraction(float(np.float32(math.cos(theta)))), Fraction(float(np.float32(math.sin(theta))))
        e = float(cf ** 2 + sf ** 2 - 1)
        assert e < 0 and abs(abs(e) - gap) < 0.1e-8


def test_double_constants_are_correctly_rounded():
    # Rot16Const<double>: cos(theta) - 1 and sin(theta) for pi/8 and pi/4,
    # each the double nearest the exact value (50-digit reference).
    mpmath = pytest.importorskip("mpmath")
    text = open(SRC).read()
    body = text[text.index("template <> struct Rot16Const<double>"):]
    body = body[:body.index("};")]
    vals = dict(re.findall(r"(cm8|s8|cm4|s4)\s*=\s*(-?[0-9.]+)", body))
    mpmath.mp.dps = 50
    exact = {"cm8": mpmath.cos(mpmath.pi / 8) - 1, "s8": mpmath.sin(mpmath.pi / 8),
             "cm4": mpmath.cos(mpmath.pi / 4) - 1, "s4": mpmath.sin(mpmath.pi / 4)}
    for k, v in exact.items():
        d = float(vals[k])                                  # the literal as the compiler rounds it
        assert d == float(v), (k, d, float(v))              # float(mpf) rounds to nearest
