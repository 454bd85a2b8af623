"""Host checks of the body-frame range reduction in csrc/step.cuh.

The kernels' cos/sin of a body angle (the frames of the narrow phase, Eq. 2's
contact geometry) reduce th by k pi/2 with fused multiply-adds against a
two-float split of pi/2.  These tests read the two constants from the source
and check them against pi itself, and check the claim the reduction rests on:
th - k P1 is exactly a float32 for every angle up to 2e6 rad, so the first
fma is exact.
"""
import os
import re
from fractions import Fraction

import mpmath
import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2207_03530_b300", "csrc", "step.cuh")


def _split():
    text = open(SRC).read()
    body = text[text.index("void body_axes(float th"):]
    consts = re.findall(r"fmaf\(-k, (-?[0-9.e+-]+)f, (?:th|r)\)", body)[:2]
    assert len(consts) == 2, consts
    return [np.float32(float(c)) for c in consts]


def test_split_is_pi_over_two():
    mpmath.mp.prec = 200
    hp = mpmath.pi / 2
    p1, p2 = _split()
    assert p1 == np.float32(float(hp))  # P1 = fl(pi/2)
    assert p2 == np.float32(float(hp - mpmath.mpf(float(p1))))  # P2 = fl(pi/2 - P1)
    # together they carry pi/2 to about 2^-48 relative
    assert abs(mpmath.mpf(float(p1)) + mpmath.mpf(float(p2)) - hp) < mpmath.mpf(2) ** -48


def test_first_reduction_step_is_exact():
    p1 = Fraction(float(_split()[0]))
    rng = np.random.default_rng(1)
    th = np.concatenate([rng.uniform(-2e6, 2e6, 4000), rng.uniform(-8, 8, 2000),
                         np.array([0.7853982, -0.7853982, 1.0, 2e6, -2e6])]).astype(np.float32)
    c = np.float32(0.63661977236758134)
    for t in th:
        k = np.rint(np.float32(t * c))  # the kernel's float32 product, rounded
        d = Fraction(float(t)) - Fraction(float(k)) * p1
        assert Fraction(float(np.float32(float(d)))) == d, (t, k)
        assert abs(d) < 1.0  # |r| stays below the clamp
