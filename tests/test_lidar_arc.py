"""Host checks of the culled LIDAR kernel's arc bounds (csrc/lidar.cuh).

Each (body, caster) pair tests only the rays inside the body's angular arc,
widened by the angle errors.  These tests hold the bounds the widening rests
on: the arctangent approximation's error (constants read from the source),
the linear upper bound of asin, and the ray-index arithmetic that turns an
arc into a start index in [0, R)."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2207_03530_b300", "csrc", "lidar.cuh")
f = np.float32


def _atan_consts():
    text = open(SRC).read()
    body = text[text.index("float lidar_atan2_approx(float y, float x)"):]
    m = re.search(r"z \* \(([0-9.]+)f - \(z - 1\.f\) \* \(([0-9.]+)f \+ ([0-9.]+)f \* z\)\)", body)
    assert m, "approximation not found"
    return [f(float(g)) for g in m.groups()]


def _atan2_approx(y, x):
    c0, c1, c2 = _atan_consts()
    ax, ay = np.abs(x), np.abs(y)
    sw = ay > ax
    z = (np.where(sw, ax, ay) / np.maximum(np.where(sw, ay, ax), f(1e-30))).astype(f)
    a = (z * (c0 - (z - f(1)) * (c1 + c2 * z))).astype(f)
    a = np.where(sw, f(1.57079633) - a, a)
    a = np.where(x < 0, f(3.14159265) - a, a)
    return np.where(y < 0, -a, a).astype(f)


def test_arctangent_within_the_widening():
    rng = np.random.default_rng(0)
    y = rng.normal(size=400000).astype(f)
    x = rng.normal(size=400000).astype(f)
    y[:4], x[:4] = [0, 1, -1, 0], [1, 0, 0, -1]  # axis directions
    d = np.abs(_atan2_approx(y, x).astype(np.float64) - np.arctan2(y.astype(np.float64), x))
    d = np.minimum(d, 2 * np.pi - d)
    assert d.max() <= 0.0016  # the 0.0016 rad per arc edge of the widening
    assert np.abs(_atan2_approx(y, x)).max() <= np.float32(3.1415927)


def test_linear_asin_bound():
    xs = np.linspace(0, 1, 200001)
    bound = xs * np.where(xs <= 0.5, 1.0473, 1.5708)
    assert (bound >= np.arcsin(xs)).all()


def test_arc_start_index_in_range():
    """u = (phi - phi0) R / 2pi with |phi| <= 3pi/2 and |phi0| <= pi, reduced
    modulo R; the start index of every arc narrower than R rays lies in
    [0, R) (an index of R once wrote past the caster's row)."""
    for R in (1, 2, 7, 32, 96, 3072):
        inv = f(R) / f(2 * np.pi)
        phi = np.linspace(-1.5 * np.pi, 1.5 * np.pi, 20001).astype(f)
        for phi0 in (f(-np.pi), f(-1.0), f(0.0), f(2.5), f(np.pi)):
            u = ((phi - phi0) * inv).astype(f)
            u = (u - f(R) * np.floor(u * f(1.0 / R))).astype(f)
            u = np.minimum(np.maximum(u, f(0)), f(R))
            for half in (f(0.0), f(0.05), f(1.0)):
                w = f(half * inv + f(0.0025) * inv + f(0.01))
                if not w < 0.5 * R:
                    continue
                lo = np.ceil(u - w).astype(np.int64)
                hi = np.floor(u + w).astype(np.int64)
                r0 = np.where(hi - lo + 1 < R, lo, 0)
                idx = np.where(r0 < 0, r0 + R, np.where(r0 >= R, r0 - R, r0))
                assert ((idx >= 0) & (idx < R)).all(), (R, float(phi0), float(half))
