"""Pins of the oracle's LIDAR ray casts: hand-worked distances, brute-force
ray marching with an independent inside-test, and rotation invariance."""
import math

import numpy as np
import pytest

from conftest import make_scene
from paper_2207_03530_b300 import scenes

S_, B_, L_ = scenes.SPHERE, scenes.BOX, scenes.LINE
MOV, ROT, COL, ACT = scenes.MOVABLE, scenes.ROTATABLE, scenes.COLLIDABLE, scenes.ACTUATED


def _agent(th=0.0, x=0.0, y=0.0):
    return dict(shape=S_, x=x, y=y, th=th, a=0.05, flags=MOV | COL | ACT)


def test_hand_worked_distances(orc):
    """Ray 0 points along +x (theta 0), ray 2 of 4 along -x, ray 1 along +y.
    Sphere r=0.25 centred 1.0 ahead: 0.75.  Box 0.5 wide centred at y=0.75:
    face at 0.5.  Segment crossing -x at x=-0.625: 0.625.  Nothing along -y:
    the range, 2.0."""
    bodies = [_agent(),
              dict(shape=S_, x=1.0, y=0.0, a=0.25, flags=COL),
              dict(shape=B_, x=0.0, y=0.75, a=0.5, b=0.5, flags=COL),
              dict(shape=L_, x=-0.625, y=0.0, th=math.pi / 2, a=1.0, flags=COL)]
    sc = make_scene(bodies)
    out = orc.lidar(sc, sc.init_state, 4, 2.0)[0, 0]
    np.testing.assert_allclose(out, [0.75, 0.5, 0.625, 2.0], atol=1e-7)


def test_origin_inside_and_excluded_caster(orc):
    """An agent overlapping a box reads 0 on every ray; it never sees itself;
    non-collidable bodies are invisible."""
    bodies = [_agent(), dict(shape=B_, x=0.1, y=0.0, a=0.5, b=0.5, flags=COL),
              dict(shape=S_, x=-0.5, y=0.0, a=0.1, flags=0)]
    sc = make_scene(bodies)
    np.testing.assert_array_equal(orc.lidar(sc, sc.init_state, 8, 3.0), 0.0)
    sc2 = make_scene([_agent(), dict(shape=S_, x=-0.5, y=0.0, a=0.1, flags=0)])
    np.testing.assert_array_equal(orc.lidar(sc2, sc2.init_state, 8, 3.0), 3.0)


def _inside(shape, b, px, py):
    x, y, th, a, bb = b
    c, s = math.cos(th), math.sin(th)
    lx = c * (px - x) + s * (py - y)
    ly = -s * (px - x) + c * (py - y)
    if shape == S_:
        return lx * lx + ly * ly <= a * a
    if shape == B_:
        return (np.abs(lx) <= a / 2) & (np.abs(ly) <= bb / 2)
    return np.zeros_like(lx, bool)


def _march(shape, b, ox, oy, dx, dy, rng_max, n=200001):
    t = np.linspace(0, rng_max, n)
    px, py = ox + t * dx, oy + t * dy
    if shape == L_:
        x, y, th, a, _ = b
        c, s = math.cos(th), math.sin(th)
        ly = -s * (px - x) + c * (py - y)
        lx = c * (px - x) + s * (py - y)
        cross = np.nonzero((np.sign(ly[:-1]) != np.sign(ly[1:])) & (np.abs(lx[:-1]) <= a / 2))[0]
        return t[cross[0]] if len(cross) else rng_max
    ins = np.nonzero(_inside(shape, b, px, py))[0]
    return t[ins[0]] if len(ins) else rng_max


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_marching(orc, seed):
    """Random casters and shapes: every ray's distance equals the first
    marched point inside the shape (or the segment crossing), to the step."""
    rng = np.random.default_rng(seed)
    R = 1.5
    for shape in (S_, B_, L_):
        body = [rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(-3, 3),
                rng.uniform(0.1, 0.5), rng.uniform(0.1, 0.5)]
        ox, oy = rng.uniform(-1, 1), rng.uniform(-1, 1)
        sc = make_scene([_agent(th=rng.uniform(-3, 3), x=ox, y=oy),
                         dict(shape=shape, x=body[0], y=body[1], th=body[2], a=body[3],
                              b=body[4], flags=COL)])
        st = sc.init_state.astype(np.float64)
        out = orc.lidar(sc, st, 16, R)[0, 0]
        b32 = [float(np.float32(v)) for v in body]
        for k in range(16):
            ang = st[0, 0, 4] + 2 * math.pi * k / 16
            ref = _march(shape, b32, st[0, 0, 0], st[0, 0, 1], math.cos(ang), math.sin(ang), R)
            assert out[k] == pytest.approx(ref, abs=2 * R / 200000 + 1e-12)


def test_rotation_invariance(orc):
    """Turning the whole scene (and every angle) by phi leaves every reading
    unchanged."""
    sc = scenes.paper_scene(8, 3, dense=True)
    a = orc.lidar(sc, sc.init_state, 24, 1.0)
    phi = 0.9
    c, s = math.cos(phi), math.sin(phi)
    st = sc.init_state.astype(np.float64).copy()
    x, y = st[..., 0].copy(), st[..., 1].copy()
    st[..., 0], st[..., 1] = c * x - s * y, s * x + c * y
    st[..., 4] += phi
    b = orc.lidar(sc, st, 24, 1.0)
    np.testing.assert_allclose(a, b, atol=1e-9)
