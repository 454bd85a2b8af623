"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each checks it against a
closed form of the semi-implicit Euler recurrence (Eq. 1, Eq. 3), a
conservation law the pair forces imply, an exact symmetry, a brute-force
geometric search, a textbook routine, or a hand-derived golden case.
"""
import math
import os

import numpy as np
import pytest

from conftest import make_scene
from paper_2207_03530_b300 import scenes

S_, B_, L_ = scenes.SPHERE, scenes.BOX, scenes.LINE
MOV, ROT, COL, ACT = scenes.MOVABLE, scenes.ROTATABLE, scenes.COLLIDABLE, scenes.ACTUATED
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "contact_cases.txt")


# --------------------------------------------------------------- closed forms
def _closed_form(x0, v0, b, zeta, h, n):
    """x_n, v_n of v <- (1-zeta) v + b ; x <- x + v h after n substeps."""
    if zeta == 0:
        return x0 + h * (n * v0 + b * n * (n + 1) / 2), v0 + n * b
    a = 1 - zeta
    an = a ** n
    v = an * v0 + b * (1 - an) / zeta
    x = x0 + h * (v0 * a * (1 - an) / zeta + (b / zeta) * (n - a * (1 - an) / zeta))
    return x, v


@pytest.mark.parametrize("zeta", [0.25, 0.0])
@pytest.mark.parametrize("substeps,steps", [(1, 7), (5, 3)])
def test_free_body_linear_closed_form(orc, zeta, substeps, steps):
    """Eq. 1 for a lone body under a constant action + gravity force."""
    m, f, g = 1.75, (0.6, -0.3), (0.1, -0.4)
    sc = make_scene([dict(shape=S_, x=0.25, y=-0.5, vx=0.125, vy=0.5, a=0.05, m=m,
                          flags=MOV | ACT)], substeps=substeps, dt=0.1, drag=zeta, g=g)
    act = np.zeros((steps, 1, 1, 3), np.float32)
    act[..., 0], act[..., 1] = f
    out = orc.step(sc, sc.init_state, act)
    h = 0.1 / substeps
    n = steps * substeps
    for ax, (x0, v0) in enumerate([(0.25, 0.125), (-0.5, 0.5)]):
        force = float(np.float32(f[ax])) + m * g[ax]
        b = force / float(np.float32(m)) * h
        x, v = _closed_form(float(np.float32(x0)), float(np.float32(v0)), b, zeta, h, n)
        assert out[0, 0, ax] == pytest.approx(x, rel=1e-12, abs=1e-14)
        assert out[0, 0, 2 + ax] == pytest.approx(v, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("zeta", [0.25, 0.0])
def test_free_body_angular_closed_form(orc, zeta):
    """Eq. 3 for a lone box under a constant action torque, with the default
    moment of inertia m (w^2 + h^2) / 12."""
    m, w, hgt, tau = 5.0, 0.1, 0.2, -0.7
    sc = make_scene([dict(shape=B_, th=0.3, om=0.5, a=w, b=hgt, m=m, flags=MOV | ROT | ACT)],
                    substeps=5, dt=0.1, drag=zeta)
    act = np.zeros((4, 1, 1, 3), np.float32)
    act[..., 2] = tau
    out = orc.step(sc, sc.init_state, act)
    I = m * (float(np.float32(w)) ** 2 + float(np.float32(hgt)) ** 2) / 12
    b = float(np.float32(tau)) / I * 0.02
    th, om = _closed_form(float(np.float32(0.3)), 0.5, b, zeta, 0.02, 20)
    assert out[0, 0, 4] == pytest.approx(th, rel=1e-12)
    assert out[0, 0, 5] == pytest.approx(om, rel=1e-12)
    # position untouched: no force
    assert out[0, 0, 0] == 0 and out[0, 0, 1] == 0


def test_default_inertia(orc):
    assert orc.inertia(B_, 5.0, 0.1, 0.2) == pytest.approx(5 * 0.05 / 12, rel=1e-15)
    assert orc.inertia(L_, 2.0, 3.0, 0.0) == pytest.approx(2 * 9 / 12, rel=1e-15)
    assert orc.inertia(S_, 2.0, 0.5, 0.0) == pytest.approx(0.25, rel=1e-15)
    assert orc.inertia(S_, 2.0, 0.5, 0.0, 7.0) == 7.0


def test_max_speed_saturates(orc):
    """The maximum speed (section 3, entity parameters) caps |v|; a constant
    force from rest drives the speed to exactly the cap, along the force."""
    sc = make_scene([dict(shape=S_, a=0.05, m=1.0, flags=MOV | ACT)], substeps=2, drag=0.25,
                    max_speed=0.05)
    act = np.zeros((30, 1, 1, 3), np.float32)
    act[..., 0], act[..., 1] = 0.6, 0.8
    out = orc.step(sc, sc.init_state, act)
    v = out[0, 0, 2:4]
    assert np.hypot(*v) == pytest.approx(0.05, rel=1e-12)
    assert v[0] / v[1] == pytest.approx(float(np.float32(0.6)) / float(np.float32(0.8)), rel=1e-12)


# ------------------------------------------------------------ contact law
def test_contact_magnitude_values(orc):
    """Eq. 2 magnitude c k log(1 + e^{-g/k}); at g = 0 with c = 100,
    k = 1e-3 it is 0.1 ln 2 = 0.0693147..."""
    assert orc.contact_magnitude(100.0, 1e-3, 0.0) == pytest.approx(0.06931471805599453, rel=1e-15)
    for g in [-0.05, -0.02, -1e-3, -1e-4, 0.0, 1e-4, 5e-3]:
        z = np.longdouble(-g) / np.longdouble(1e-3)
        ref = np.longdouble(100.0) * np.longdouble(1e-3) * np.log1p(np.exp(z))
        assert orc.contact_magnitude(100.0, 1e-3, g) == pytest.approx(float(ref), rel=1e-14)


@pytest.mark.parametrize("gap", [-0.015, -1e-3, -2e-4])
@pytest.mark.parametrize("other", ["sphere", "line", "box"])
def test_single_contact_velocity(orc, gap, other):
    """A resting movable sphere against a fixed body at a chosen gap: after
    one substep (zeta = 0) its velocity is f/m dt along the outward normal,
    |f| = c k ln(1 + e^{-gap/k})."""
    r, m, dt = 0.0625, 1.5, 0.1
    # the contact normal is (0.6, 0.8) in every case; the sphere sits at
    # distance d from the fixed body's closest point along it.
    nx, ny = 0.6, 0.8
    if other == "sphere":
        R = 0.125
        fixed = dict(shape=S_, x=0.0, y=0.0, a=R, flags=COL)
        cx, cy = (r + R + gap) * nx, (r + R + gap) * ny
    elif other == "line":
        # line through the origin along (0.8, -0.6): normal (0.6, 0.8)
        th = math.atan2(-0.6, 0.8)
        fixed = dict(shape=L_, x=0.0, y=0.0, th=th, a=1.0, flags=COL)
        cx, cy = (r + gap) * nx, (r + gap) * ny
    else:
        th = math.atan2(0.8, 0.6)  # box local +x face normal = (0.6, 0.8)
        fixed = dict(shape=B_, x=0.0, y=0.0, th=th, a=0.5, b=0.25, flags=COL)
        cx, cy = (0.25 + r + gap) * nx, (0.25 + r + gap) * ny
    sc = make_scene([dict(shape=S_, x=cx, y=cy, a=r, m=m, flags=MOV | COL), fixed],
                    dt=dt, drag=0.0)
    out = orc.step(sc, sc.init_state, np.zeros((1, 1, 0, 3), np.float32))
    v = out[0, 0, 2:4]
    fmag = 100.0 * 1e-3 * math.log1p(math.exp(-gap / 1e-3))
    # inputs are rounded to FP32, so the realised gap differs by ~1e-8
    assert np.hypot(*v) * m / dt == pytest.approx(fmag, rel=2e-4 if gap > -1e-3 else 2e-5)
    assert v[0] / np.hypot(*v) == pytest.approx(nx, abs=1e-6)
    assert v[1] / np.hypot(*v) == pytest.approx(ny, abs=1e-6)
    # the fixed body never moves (forces on immovable entities are dropped)
    assert np.array_equal(out[0, 1], sc.init_state[0, 1].astype(np.float64))


def test_contact_cutoff_is_inclusive_and_one_sided(orc):
    """Eq. 2 acts for |x_ij| <= d_min only: an exactly touching pair (gap
    exactly 0 in binary) is pushed with c k ln 2, a pair apart by 2^-20 is
    not pushed at all."""
    for gap, expect in [(0.0, 100 * 1e-3 * math.log(2)), (2.0 ** -20, 0.0)]:
        sc = make_scene([dict(shape=S_, x=0.25 + gap, y=0.0, a=0.125, m=1.0, flags=MOV | COL),
                         dict(shape=S_, x=0.0, y=0.0, a=0.125, flags=COL)], dt=0.1)
        out = orc.step(sc, sc.init_state, np.zeros((1, 1, 0, 3), np.float32))
        assert out[0, 0, 2] * 1.0 / 0.1 == pytest.approx(expect, rel=1e-12, abs=1e-300)
        assert out[0, 0, 3] == 0.0


def test_coincident_centres_no_force(orc):
    """Reading R8: coincident sphere centres have no normal and exert no force."""
    sc = make_scene([dict(shape=S_, x=0.1, y=0.1, a=0.1, flags=MOV | COL),
                     dict(shape=S_, x=0.1, y=0.1, a=0.1, flags=MOV | COL)], dt=0.1)
    out = orc.step(sc, sc.init_state, np.zeros((1, 1, 0, 3), np.float32))
    assert np.all(out[0, :, 2:4] == 0)


def test_non_collidable_and_static_pairs_are_inactive(orc):
    sc = make_scene([dict(shape=S_, x=0.0, y=0.0, a=0.1, flags=MOV),
                     dict(shape=S_, x=0.05, y=0.0, a=0.1, flags=MOV | COL),
                     dict(shape=S_, x=0.5, y=0.0, a=0.1, flags=COL),
                     dict(shape=S_, x=0.55, y=0.0, a=0.1, flags=COL)], dt=0.1)
    mask, gap = orc.pairs(sc, sc.init_state)
    assert mask.tolist() == [[0, 0, 0, 0, 0, 0]]
    assert np.isinf(gap[0, 0]) and np.isinf(gap[0, 5])  # pair (0,1), pair (2,3)


# ------------------------------------------------------- golden contact cases
def _parse_golden():
    cases = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        f = [p.split() for p in line.split("|")]

        def num(t):
            t = t.replace("pi", str(math.pi))
            return float(eval(t, {"__builtins__": {}})) if t != "-" else None

        name = f[0][0]
        bi = [num(t) for t in f[1]]
        bj = [num(t) for t in f[2]]
        cases.append((name, bi, bj, num(f[3][0]), [num(t) for t in f[4]],
                      [num(t) for t in f[5]], [num(t) for t in f[6]]))
    return cases


@pytest.mark.parametrize("case", _parse_golden(), ids=lambda c: c[0])
def test_golden_contact_cases(orc, case):
    name, bi, bj, g, n, pi, pj = case
    r = orc.pair_geometry(bi, bj)
    assert r["g"] == pytest.approx(g, abs=1e-12)
    if n[0] is None:
        assert not r["has_normal"]
        return
    assert r["has_normal"]
    np.testing.assert_allclose(r["n"], n, atol=1e-12)
    np.testing.assert_allclose(r["p_i"], pi, atol=1e-12)
    np.testing.assert_allclose(r["p_j"], pj, atol=1e-12)


# ----------------------------------------------------- brute-force geometry
def _corners(shape, x, y, th, a, b):
    c, s = math.cos(th), math.sin(th)
    if shape == B_:
        loc = [(-a / 2, -b / 2), (a / 2, -b / 2), (a / 2, b / 2), (-a / 2, b / 2)]
    else:
        loc = [(-a / 2, 0.0), (a / 2, 0.0)]
    return np.array([(x + c * u - s * v, y + s * u + c * v) for u, v in loc])


def _boundary_samples(shape, x, y, th, a, b, per_edge):
    """Points along the boundary; the grid is offset so it skips the corners."""
    V = _corners(shape, x, y, th, a, b)
    edges = [(V[q], V[(q + 1) % 4]) for q in range(4)] if shape == B_ else [(V[0], V[1])]
    t = (np.arange(per_edge) + 0.37) / per_edge
    return np.concatenate([p0 + t[:, None] * (p1 - p0) for p0, p1 in edges])


def _dist_point_poly(P, V, closed):
    """Distance of points P to a polyline V by the textbook projection."""
    n = len(V)
    segs = [(V[q], V[(q + 1) % n]) for q in range(n if closed else n - 1)]
    best = np.full(len(P), np.inf)
    for a, b in segs:
        e = b - a
        t = np.clip(((P - a) @ e) / (e @ e), 0, 1)
        q = a + t[:, None] * e
        best = np.minimum(best, np.hypot(*(P - q).T))
    return best


def _inside_convex(P, V):
    """Points strictly inside a CCW convex polygon."""
    ok = np.ones(len(P), bool)
    for q in range(len(V)):
        a, b = V[q], V[(q + 1) % len(V)]
        ok &= (b[0] - a[0]) * (P[:, 1] - a[1]) - (b[1] - a[1]) * (P[:, 0] - a[0]) > 0
    return ok


def _random_poly(rng, shape):
    if shape == B_:
        return [B_, rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(-3, 3),
                rng.uniform(0.1, 0.4), rng.uniform(0.1, 0.4)]
    return [L_, rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(-3, 3),
            rng.uniform(0.2, 0.6), 0.0]


@pytest.mark.parametrize("seed", range(12))
def test_sphere_geometry_brute_force(orc, seed):
    """Sphere against line / box: the gap equals the sampled distance from the
    centre to the shape's boundary minus r (centre outside), or minus the
    depth minus r (centre inside a box)."""
    rng = np.random.default_rng(seed)
    for shape in (L_, B_):
        body = _random_poly(rng, shape)
        cx, cy, r = rng.uniform(-0.45, 0.45), rng.uniform(-0.45, 0.45), rng.uniform(0.02, 0.1)
        res = orc.pair_geometry([S_, cx, cy, 0.0, r, 0.0], body)
        V = _corners(*body)
        P = _boundary_samples(*body, per_edge=20000)
        d = np.hypot(P[:, 0] - cx, P[:, 1] - cy).min()
        inside = shape == B_ and _inside_convex(np.array([[cx, cy]]), V)[0]
        expect = (-d if inside else d) - r
        assert res["g"] == pytest.approx(expect, abs=1e-4)
        # p_i - p_j is along n and has length |gap| (closest points)
        diff = res["p_i"] - res["p_j"]
        np.testing.assert_allclose(diff, res["g"] * res["n"], atol=1e-12)


@pytest.mark.parametrize("seed", range(40))
def test_polygon_geometry_brute_force(orc, seed):
    """Box/line pairs.  Apart: the gap equals the sampled boundary-to-boundary
    distance.  Overlapping: the gap is minus the minimum translation distance,
    found by scanning 3600 directions of the support functions of the two
    vertex sets; the normal is the best scanned direction."""
    rng = np.random.default_rng(1000 + seed)
    shapes = [(B_, B_), (B_, L_), (L_, B_), (L_, L_)][seed % 4]
    bi = _random_poly(rng, shapes[0])
    bj = _random_poly(rng, shapes[1])
    res = orc.pair_geometry(bi, bj)
    Vi, Vj = _corners(*bi), _corners(*bj)
    ang = np.arange(3600) * (2 * math.pi / 3600)
    U = np.stack([np.cos(ang), np.sin(ang)], 1)
    # translation of i along u that separates it from j
    sep = (Vj @ U.T).max(0) - (Vi @ U.T).min(0)
    overlap = sep.min() > 0 and not _separated_by_sampling(bi, bj)
    diff = res["p_i"] - res["p_j"]
    if res["g"] <= 0:
        assert overlap
        k = sep.argmin()
        assert -res["g"] == pytest.approx(sep[k], abs=2e-4)
        assert -res["g"] <= sep[k] + 1e-12  # the exact minimum is below the scan
        assert res["n"] @ U[k] > 0.999
        np.testing.assert_allclose(diff, res["g"] * res["n"], atol=1e-12)
    else:
        assert not overlap
        Pi = _boundary_samples(*bi, per_edge=4000)
        d = min(_dist_point_poly(Pi, Vj, shapes[1] == B_).min(),
                _dist_point_poly(_boundary_samples(*bj, per_edge=4000), Vi, shapes[0] == B_).min())
        assert res["g"] == pytest.approx(d, abs=2e-4)
        assert res["g"] <= d + 1e-12
        assert np.hypot(*diff) == pytest.approx(res["g"], rel=1e-12)


def _separated_by_sampling(bi, bj):
    """Disjointness of two boxes/lines by dense boundary sampling: they touch
    iff some boundary point of one is inside the other or edges cross."""
    Vi, Vj = _corners(*bi), _corners(*bj)
    Pi = _boundary_samples(*bi, per_edge=4000)
    Pj = _boundary_samples(*bj, per_edge=4000)
    di = _dist_point_poly(Pi, Vj, bj[0] == B_).min()
    dj = _dist_point_poly(Pj, Vi, bi[0] == B_).min()
    if min(di, dj) < 1e-3:
        return False
    if bj[0] == B_ and _inside_convex(Pi, Vj).any():
        return False
    if bi[0] == B_ and _inside_convex(Pj, Vi).any():
        return False
    return True


@pytest.mark.parametrize("seed", range(6))
def test_polygon_contact_point_on_incident_boundary(orc, seed):
    """Overlapping polygons: the contact point on one body lies on that
    body's boundary (the incident edge) and the other is displaced from it
    by gap * n."""
    rng = np.random.default_rng(77 + seed)
    found = 0
    while found < 5:
        shapes = [(B_, B_), (B_, L_), (L_, B_)][rng.integers(3)]
        bi, bj = _random_poly(rng, shapes[0]), _random_poly(rng, shapes[1])
        res = orc.pair_geometry(bi, bj)
        if res["g"] > 0:
            continue
        found += 1
        Vi, Vj = _corners(*bi), _corners(*bj)
        on_i = _dist_point_poly(res["p_i"][None], Vi, bi[0] == B_)[0]
        on_j = _dist_point_poly(res["p_j"][None], Vj, bj[0] == B_)[0]
        assert min(on_i, on_j) < 1e-12


# ------------------------------------------------------ invariants of a step
def _closed_world(seed, n_envs=8):
    """Mixed scene with every body movable and rotatable, no drag, gravity
    or actions: total momentum and angular momentum must be conserved."""
    sc = scenes.mixed_scene(n_envs, seed, substeps=4)
    sc.flags[:] = MOV | ROT | COL | ACT
    sc.gx = sc.gy = 0.0
    sc.drag = 0.0
    sc.n_actuated = sc.n_entities
    return sc


def _inertia_all(orc, sc):
    I = np.zeros(sc.shape.shape)
    for e in range(sc.n_envs):
        for i in range(sc.n_entities):
            I[e, i] = orc.inertia(int(sc.shape[e, i]), float(sc.mass[e, i]), float(sc.size_a[e, i]),
                                  float(sc.size_b[e, i]), float(sc.inertia[e, i]))
    return I


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_newton_third_law_momentum(orc, seed):
    """Equal and opposite pair forces: sum_i m_i v_i is conserved exactly (to
    FP64 rounding) with drag, gravity and actions off."""
    sc = _closed_world(seed)
    act = np.zeros((5, sc.n_envs, sc.n_actuated, 3), np.float32)
    out = orc.step(sc, sc.init_state, act)
    m = sc.mass.astype(np.float64)
    p0 = (m[..., None] * sc.init_state[..., 2:4].astype(np.float64)).sum(1)
    p1 = (m[..., None] * out[..., 2:4]).sum(1)
    moved = np.abs(out[..., 2:4] - sc.init_state[..., 2:4]).max()
    assert moved > 0.1  # contacts really happened
    np.testing.assert_allclose(p1, p0, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_angular_momentum_conserved(orc, seed):
    """sum_i m_i x_i x v_i + I_i omega_i is conserved per step: the pair
    forces act along p_i - p_j, so with the signed torque r x f of Eq. 3 the
    moments cancel.  A wrong torque sign or contact point breaks this."""
    sc = _closed_world(seed)
    I = _inertia_all(orc, sc)
    act = np.zeros((5, sc.n_envs, sc.n_actuated, 3), np.float32)
    m = sc.mass.astype(np.float64)

    def L(st):
        st = st.astype(np.float64)
        return (m * (st[..., 0] * st[..., 3] - st[..., 1] * st[..., 2]) + I * st[..., 5]).sum(1)

    out = orc.step(sc, sc.init_state, act)
    spun = np.abs(out[..., 5] - sc.init_state[..., 5]).max()
    assert spun > 0.1
    np.testing.assert_allclose(L(out), L(sc.init_state), atol=1e-12)


def test_permutation_equivariance(orc):
    """Relabelling entities (with their actions) relabels the result."""
    sc = scenes.mixed_scene(16, 5)
    act = np.random.default_rng(3).uniform(-1, 1, (3, sc.n_envs, sc.n_actuated, 3)).astype(np.float32)
    out = orc.step(sc, sc.init_state, act)
    rng = np.random.default_rng(9)
    perm = rng.permutation(sc.n_entities)
    sp = sc.subset(np.arange(sc.n_envs))
    for key in ("shape", "flags", "size_a", "size_b", "mass", "inertia"):
        getattr(sp, key)[:] = getattr(sc, key)[:, perm]
    sp.init_state[:] = sc.init_state[:, perm]
    # actions follow the actuated entities in their new order
    act_idx = np.cumsum(sc.flags[0] & ACT > 0) - 1
    new_rows = [act_idx[p] for p in perm if sc.flags[0, p] & ACT]
    outp = orc.step(sp, sp.init_state, act[:, :, new_rows])
    np.testing.assert_allclose(outp, out[:, perm], rtol=0, atol=1e-11)


def _rot90(st):
    r = st.copy()
    r[..., 0], r[..., 1] = -st[..., 1], st[..., 0]
    r[..., 2], r[..., 3] = -st[..., 3], st[..., 2]
    return r


def test_rotation_and_mirror_are_bitwise_for_spheres(orc):
    """A quarter turn or a mirror of a sphere scene maps every floating-point
    operation of the step onto the same operation on swapped / negated
    operands, so the result must map bitwise."""
    sc = scenes.small_scene(32, 4, dense=True)
    sc.gx, sc.gy = 0.0, 0.0
    act = np.random.default_rng(1).uniform(-1, 1, (4, sc.n_envs, sc.n_actuated, 3)).astype(np.float32)
    out = orc.step(sc, sc.init_state, act)
    # quarter turn
    sr = sc.with_state(_rot90(sc.init_state))
    ar = act.copy()
    ar[..., 0], ar[..., 1] = -act[..., 1], act[..., 0]
    assert np.array_equal(orc.step(sr, sr.init_state, ar), _rot90(out))
    # mirror y -> -y
    sm_state = sc.init_state.copy()
    sm_state[..., 1] *= -1
    sm_state[..., 3] *= -1
    am = act.copy()
    am[..., 1] *= -1
    outm = orc.step(sc.with_state(sm_state), sm_state, am)
    expect = out.copy()
    expect[..., 1] *= -1
    expect[..., 3] *= -1
    assert np.array_equal(outm, expect)


def test_rigid_motion_equivariance_mixed(orc):
    """Rotating and translating a mixed scene (angles shift by phi) rotates
    and translates the result, to rounding."""
    sc = scenes.mixed_scene(16, 11)
    sc.gx, sc.gy = 0.0, 0.0
    act = np.random.default_rng(2).uniform(-1, 1, (2, sc.n_envs, sc.n_actuated, 3))
    out = orc.step(sc, sc.init_state.astype(np.float64), act)
    phi, t = 0.7, np.array([0.3, -0.2])
    c, s = math.cos(phi), math.sin(phi)
    R = np.array([[c, -s], [s, c]])
    st = sc.init_state.astype(np.float64).copy()
    st[..., :2] = st[..., :2] @ R.T + t
    st[..., 2:4] = st[..., 2:4] @ R.T
    st[..., 4] += phi
    ar = act.copy()
    ar[..., :2] = act[..., :2] @ R.T
    out2 = orc.step(sc, st, ar)
    exp = out.copy()
    exp[..., :2] = out[..., :2] @ R.T + t
    exp[..., 2:4] = out[..., 2:4] @ R.T
    exp[..., 4] += phi
    np.testing.assert_allclose(out2, exp, atol=1e-9)


# ------------------------------------------------------------- enumeration
@pytest.mark.parametrize("n", [0, 1, 2, 6, 24, 77])
def test_pair_list_matches_index_formula(orc, n):
    """Canonical pairs (i < j, row-major) at index i N - i(i+1)/2 + j-i-1."""
    pi, pj = orc.pair_list(n)
    assert len(pi) == n * (n - 1) // 2
    for p, (i, j) in enumerate(zip(pi, pj)):
        assert i < j < n
        assert i * n - i * (i + 1) // 2 + (j - i - 1) == p


def test_mask_matches_brute_force_sphere_overlap(orc):
    """For sphere scenes the mask is exactly 'centre distance <= r_i + r_j'
    over active pairs, computed here directly."""
    sc = scenes.small_scene(64, 2, dense=True)
    mask, gap = orc.pairs(sc, sc.init_state)
    st = sc.init_state.astype(np.float64)
    pi, pj = orc.pair_list(sc.n_entities)
    d = np.hypot(st[:, pi, 0] - st[:, pj, 0], st[:, pi, 1] - st[:, pj, 1])
    rsum = sc.size_a[:, pi].astype(np.float64) + sc.size_a[:, pj]
    movable = ((sc.flags[:, pi] | sc.flags[:, pj]) & (MOV | ROT)) > 0
    assert np.array_equal(mask.astype(bool), (d <= rsum) & movable)
    assert mask.sum() > 0


def test_degenerate_worlds(orc):
    """Zero envs, one entity, no actuated entities all run."""
    sc = scenes.small_scene(4, 0).subset([])
    out = orc.step(sc, sc.init_state, np.zeros((1, 0, 4, 3), np.float32))
    assert out.shape == (0, 6, 6)
    one = make_scene([dict(shape=S_, vx=1.0, a=0.1, flags=MOV | COL)], drag=0.5)
    out = orc.step(one, one.init_state, np.zeros((2, 1, 0, 3), np.float32))
    assert out[0, 0, 2] == pytest.approx(0.25, rel=1e-15)


# ---- decision margins and ray sensitivity (the near-tie certificates) ----

def test_step_margin_leaves_the_step_unchanged(orc):
    """ow_step_margin is ow_step plus bookkeeping: bitwise the same state."""
    from paper_2207_03530_b300 import scenes

    sc = scenes.mixed_scene(64, 5)
    act = scenes.make_actions(sc, 2, 1)
    a = orc.step(sc, sc.init_state, act)
    b, m = orc.step_margin(sc, sc.init_state, act)
    assert np.array_equal(a, b)
    assert m.shape == (64,) and (m >= 0).all() and np.isfinite(m).all()


def test_step_margin_sphere_inside_box_runner_up_face(orc):
    """A sphere (r = 0.01) whose centre sits at (0.03, 0.01) inside a fixed
    0.2 x 0.1 box: face depths +x 0.07, -x 0.13, +y 0.04, -y 0.06, so the
    contact leaves through +y and the runner-up face is 0.02 deeper; the
    gap is -0.05.  One substep: the margin is min(|gap|, 0.02) = 0.02, i.e.
    2 y in the box frame (the -y face depth minus the +y one), with y the
    FP32 value the scene holds."""
    sc = make_scene([dict(shape=S_, x=0.03, y=0.01, a=0.01, flags=MOV | COL),
                     dict(shape=B_, a=0.2, b=0.1, flags=COL)], substeps=1)
    _, m = orc.step_margin(sc, sc.init_state, np.zeros((1, 1, 0, 3)))
    assert m[0] == pytest.approx(2 * float(np.float32(0.01)), abs=1e-15)


def test_step_margin_box_box_runner_up_axis(orc):
    """Two axis-aligned 0.2 x 0.2 boxes, centres 0.15 apart in x and 0.17 in
    y: overlap depths 0.05 along x and 0.03 along y (on both boxes' axes),
    so the least axis is y (i's own, found first) with i's x-axis and
    both of j's axes as runners-up; the nearest runner-up is j's y-axis at
    the same depth: margin 0 (an exact tie, resolved by order), and the
    scene with j turned by 0.1 rad has a positive margin."""
    bodies = [dict(shape=B_, a=0.2, b=0.2, flags=MOV | ROT | COL),
              dict(shape=B_, x=0.15, y=0.17, a=0.2, b=0.2, flags=COL)]
    sc = make_scene(bodies, substeps=1)
    _, m = orc.step_margin(sc, sc.init_state, np.zeros((1, 1, 0, 3)))
    assert m[0] == 0.0
    bodies[1]["th"] = 0.1
    sc = make_scene(bodies, substeps=1)
    _, m = orc.step_margin(sc, sc.init_state, np.zeros((1, 1, 0, 3)))
    assert m[0] > 1e-3


def test_lidar_sensitivity_separates_grazing_from_central_rays(orc):
    """A disc of radius 0.1 centred 0.5 ahead of the caster: ray 0 hits it
    head on (entry at 0.4, well conditioned); a second caster's ray passes
    the disc 0.1 - 1e-7 from its centre (a graze: the entry distance moves
    with the square root of the discriminant).  The central ray's
    sensitivity is about its input perturbation, the grazing one's far
    larger."""
    act = MOV | COL | ACT
    sc = make_scene([dict(shape=S_, x=0.0, y=0.0, a=0.01, flags=act),
                     dict(shape=S_, x=0.0, y=0.3 - 1e-7, a=0.01, flags=act),
                     dict(shape=S_, x=0.5, y=0.2, a=0.1, flags=COL),
                     dict(shape=S_, x=0.5, y=0.0, a=0.1, flags=COL)])
    ref = orc.lidar(sc, sc.init_state, 1, 2.0)
    sens = orc.lidar_sensitivity(sc, sc.init_state, 1, 2.0)
    assert ref[0, 0, 0] == 0.5 - float(np.float32(0.1))  # the scene's FP32 radius
    assert sens[0, 0, 0] < 1e-5
    assert sens[0, 1, 0] > 1e-4
