"""Seeded synthetic scenes and action streams for the VMAS world step.

This module only places bodies and draws random numbers.  It holds none of the
step's arithmetic (no forces, no contact geometry, no integration), so both
the CUDA path and the FP64 oracle can be fed from it without sharing any of
the method.

The scenes stand in for the paper's workloads (section 5 times MPE's
``simple_spread`` and section 4 lists scenarios with agent spheres, box
packages, walls and gravity); those task definitions are not reproduced.

Entity order inside an env is fixed per scene family and documented below.
Every array is FP32 (or uint8), so the GPU and the oracle read identical
inputs; the oracle widens them to FP64 exactly.

Placement rule: bodies are rejection-sampled so that their bounding circles
keep a clearance of ``CLEARANCE`` from each other.  A shape lies inside its
bounding circle, so such a pair is apart by at least the clearance.  The
"dense" variants additionally place bodies *against* a previously placed
body at a drawn signed offset u in [-0.02, -1e-3] (u < 0 = overlap), either
centre-to-centre for two spheres or against a face for a sphere and a box.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SPHERE, BOX, LINE = 0, 1, 2
MOVABLE, ROTATABLE, COLLIDABLE, ACTUATED = 1, 2, 4, 8

CLEARANCE = 1e-3
DENSE_FRACTION = 0.3
DENSE_OFFSET = (-0.02, -1e-3)


@dataclasses.dataclass
class Scene:
    """A batch of environments with the same entity count.

    Per-entity arrays are [n_envs, n_entities]; init_state is
    [n_envs, n_entities, 6] holding (x, y, vx, vy, theta, omega).
    size_a is a sphere's radius, a box's width or a line's length; size_b is
    a box's height.  inertia 0 selects the default moment of inertia.
    """

    name: str
    n_envs: int
    n_entities: int
    n_actuated: int
    substeps: int
    dt: float
    drag: float
    gx: float
    gy: float
    c: float
    k: float
    max_speed: float
    shape: np.ndarray
    flags: np.ndarray
    size_a: np.ndarray
    size_b: np.ndarray
    mass: np.ndarray
    inertia: np.ndarray
    init_state: np.ndarray

    @property
    def n_pairs(self) -> int:
        return self.n_entities * (self.n_entities - 1) // 2

    def subset(self, envs) -> "Scene":
        """The same scene restricted to the given env indices (a copy)."""
        idx = np.asarray(envs, dtype=np.int64)
        kw = dataclasses.asdict(self)
        for key in ("shape", "flags", "size_a", "size_b", "mass", "inertia", "init_state"):
            kw[key] = np.ascontiguousarray(getattr(self, key)[idx])
        kw["n_envs"] = int(len(idx))
        return Scene(**kw)

    def with_state(self, state) -> "Scene":
        kw = dataclasses.asdict(self)
        kw["init_state"] = np.ascontiguousarray(np.asarray(state, dtype=np.float32))
        return Scene(**kw)


def _empty(name, E, N, A, S, dt, drag, gx=0.0, gy=0.0, c=100.0, k=1e-3, max_speed=0.0):
    return Scene(
        name=name, n_envs=E, n_entities=N, n_actuated=A, substeps=S, dt=dt, drag=drag,
        gx=gx, gy=gy, c=c, k=k, max_speed=max_speed,
        shape=np.zeros((E, N), np.uint8), flags=np.zeros((E, N), np.uint8),
        size_a=np.zeros((E, N), np.float32), size_b=np.zeros((E, N), np.float32),
        mass=np.ones((E, N), np.float32), inertia=np.zeros((E, N), np.float32),
        init_state=np.zeros((E, N, 6), np.float32),
    )


class _Placer:
    """Vectorised rejection sampling of bounding circles for all envs at once."""

    def __init__(self, rng, n_envs, n_slots):
        self.rng = rng
        self.E = n_envs
        self.cx = np.zeros((n_envs, n_slots))
        self.cy = np.zeros((n_envs, n_slots))
        self.R = np.zeros((n_envs, n_slots))
        self.n = 0

    def _clear(self, x, y, R, envs, skip=None):
        """True where a circle (x, y, R) keeps CLEARANCE to every placed one."""
        if self.n == 0:
            return np.ones(len(envs), bool)
        dx = x[:, None] - self.cx[envs, : self.n]
        dy = y[:, None] - self.cy[envs, : self.n]
        need = R[:, None] + self.R[envs, : self.n] + CLEARANCE
        ok = dx * dx + dy * dy >= need * need
        if skip is not None:
            ok[np.arange(len(envs)), skip] = True
        return ok.all(axis=1)

    def place_free(self, R, lo, hi, envs=None):
        """Uniform centres in [lo+R, hi-R]^2, clear of everything placed."""
        envs = np.arange(self.E) if envs is None else envs
        R = np.broadcast_to(np.asarray(R, float), (self.E,))[envs]
        x = np.empty(len(envs))
        y = np.empty(len(envs))
        todo = np.arange(len(envs))
        for _ in range(10000):
            if len(todo) == 0:
                break
            rr = R[todo]
            x[todo] = self.rng.uniform(lo + rr, hi - rr)
            y[todo] = self.rng.uniform(lo + rr, hi - rr)
            ok = self._clear(x[todo], y[todo], rr, envs[todo])
            todo = todo[~ok]
        if len(todo):
            raise RuntimeError("scene placement did not converge")
        return x, y

    def commit(self, x, y, R, envs=None):
        envs = np.arange(self.E) if envs is None else envs
        self.cx[envs, self.n] = x
        self.cy[envs, self.n] = y
        self.R[envs, self.n] = np.broadcast_to(np.asarray(R, float), (self.E,))[envs]

    def advance(self):
        self.n += 1


def _f32(a):
    return np.asarray(a, dtype=np.float32)


def small_scene(n_envs: int = 32, seed: int = 0, dense: bool = False) -> Scene:
    """Plain-step small workload: per env 4 agent spheres (r=0.05, mass 1,
    movable, actuated) then 2 static landmark spheres (r=0.1, collidable,
    immovable); centres uniform in [-1,1]^2, zero initial velocity; dt=0.1,
    drag 0.25, 1 substep.  Landmarks are collidable so that the immovable
    path is exercised.

    dense: each body after the first is, with probability 0.3, placed against
    an earlier body at a drawn centre-distance offset u (the signed gap of two
    spheres) instead of freely.
    """
    E, N = n_envs, 6
    sc = _empty("small" + ("-dense" if dense else ""), E, N, 4, 1, 0.1, 0.25)
    rng = np.random.default_rng(seed)
    radii = np.array([0.05] * 4 + [0.1] * 2)
    sc.shape[:] = SPHERE
    sc.flags[:, :4] = MOVABLE | COLLIDABLE | ACTUATED
    sc.flags[:, 4:] = COLLIDABLE
    sc.size_a[:] = _f32(radii)
    sc.mass[:] = 1.0
    P = _Placer(rng, E, N)
    # The landmarks are placed first (they are larger), then the agents.
    order = [4, 5, 0, 1, 2, 3]
    for slot, ent in enumerate(order):
        x, y = _place_sphere(P, rng, radii[ent], dense and slot > 0)
        sc.init_state[:, ent, 0] = x
        sc.init_state[:, ent, 1] = y
    return sc


def _place_sphere(P, rng, R, dense):
    """Place one sphere of radius R in every env: freely inside [-1, 1]^2 or,
    in dense mode for a random subset of envs, against an earlier sphere."""
    E = P.E
    x, y = P.place_free(R, -1.0, 1.0)
    if dense and P.n > 0:
        pick = rng.random(E) < DENSE_FRACTION
        envs = np.nonzero(pick)[0]
        todo = np.arange(len(envs))
        for _ in range(200):
            if len(todo) == 0:
                break
            ee = envs[todo]
            partner = rng.integers(0, P.n, size=len(ee))
            u = rng.uniform(*DENSE_OFFSET, size=len(ee))
            phi = rng.uniform(0, 2 * math.pi, size=len(ee))
            d = P.R[ee, partner] + R + u
            cx = P.cx[ee, partner] + d * np.cos(phi)
            cy = P.cy[ee, partner] + d * np.sin(phi)
            ok = P._clear(cx, cy, np.full(len(ee), R), ee, skip=partner)
            x[todo[ok]] = cx[ok]
            y[todo[ok]] = cy[ok]
            todo = todo[~ok]
    P.commit(x, y, R)
    P.advance()
    return x, y


def paper_scene(n_envs: int = 30000, seed: int = 0, dense: bool = False,
                substeps: int = 5) -> Scene:
    """Plain step at paper scale.  Per env, in entity order:

    * 0..15  agent spheres, r ~ U[0.03, 0.08], mass ~ U[1, 2]; movable,
             collidable, actuated (force only: agents do not rotate);
    * 16..19 boxes 0.1 x 0.2, mass 5, theta ~ U[0, 2 pi); movable, rotatable,
             collidable, actuated (force and torque);
    * 20..23 fixed walls: lines of length 2 centred at (+1, 0), (-1, 0) with
             theta = pi/2 and (0, +1), (0, -1) with theta = 0; collidable only.

    Bodies are rejection-sampled inside [-0.9, 0.9]^2; dt = 0.1, drag 0.25,
    5 substeps.  dense: each sphere is, with probability 0.3, placed against an
    earlier sphere (centre distance r1 + r2 + u) or against a face of an
    earlier box (its centre at half-extent + r + u from the face plane, within
    the middle 80% of the face), and each box, with probability 0.3, is
    pushed against a wall by u along the wall normal.
    """
    E, NS, NB, NW = n_envs, 16, 4, 4
    N = NS + NB + NW
    sc = _empty("paper" + ("-dense" if dense else ""), E, N, NS + NB, substeps, 0.1, 0.25)
    rng = np.random.default_rng(seed)
    s_idx = np.arange(NS)
    b_idx = np.arange(NS, NS + NB)
    w_idx = np.arange(NS + NB, N)
    sc.shape[:, s_idx] = SPHERE
    sc.shape[:, b_idx] = BOX
    sc.shape[:, w_idx] = LINE
    sc.flags[:, s_idx] = MOVABLE | COLLIDABLE | ACTUATED
    sc.flags[:, b_idx] = MOVABLE | ROTATABLE | COLLIDABLE | ACTUATED
    sc.flags[:, w_idx] = COLLIDABLE
    sc.size_a[:, s_idx] = _f32(rng.uniform(0.03, 0.08, size=(E, NS)))
    sc.mass[:, s_idx] = _f32(rng.uniform(1.0, 2.0, size=(E, NS)))
    sc.size_a[:, b_idx] = 0.1
    sc.size_b[:, b_idx] = 0.2
    sc.mass[:, b_idx] = 5.0
    sc.size_a[:, w_idx] = 2.0
    sc.mass[:, w_idx] = 1.0
    half_pi = np.float32(math.pi / 2)
    walls = [(1.0, 0.0, half_pi), (-1.0, 0.0, half_pi), (0.0, 1.0, 0.0), (0.0, -1.0, 0.0)]
    for q, (wx, wy, wt) in enumerate(walls):
        sc.init_state[:, NS + NB + q, 0] = wx
        sc.init_state[:, NS + NB + q, 1] = wy
        sc.init_state[:, NS + NB + q, 4] = wt

    P = _Placer(rng, E, NS + NB)
    Rb = math.hypot(0.05, 0.1)
    box_th = rng.uniform(0, 2 * math.pi, size=(E, NB)).astype(np.float32)
    sc.init_state[:, b_idx, 4] = box_th
    for q in range(NB):
        x, y = P.place_free(Rb, -0.9, 0.9)
        if dense:
            x, y = _push_box_to_wall(P, rng, x, y, box_th[:, q].astype(float))
        P.commit(x, y, Rb)
        P.advance()
        sc.init_state[:, NS + q, 0] = x
        sc.init_state[:, NS + q, 1] = y
    box_xy = sc.init_state[:, NS:NS + NB, :2].astype(float)
    radii = sc.size_a[:, s_idx].astype(float)
    for q in range(NS):
        r = radii[:, q]
        x, y = P.place_free(r, -0.9, 0.9)
        if dense:
            x, y = _dense_sphere(P, rng, x, y, r, box_xy, box_th.astype(float), NB, q)
        P.commit(x, y, r)
        P.advance()
        sc.init_state[:, q, 0] = x
        sc.init_state[:, q, 1] = y
    return sc


def _push_box_to_wall(P, rng, x, y, th):
    """Dense mode: with probability 0.3 move a box so that its extent along a
    random wall's normal crosses the wall plane by -u."""
    E = P.E
    pick = np.nonzero(rng.random(E) < DENSE_FRACTION)[0]
    if len(pick) == 0:
        return x, y
    wall = rng.integers(0, 4, size=len(pick))
    u = rng.uniform(*DENSE_OFFSET, size=len(pick))
    t = th[pick]
    ext_x = 0.05 * np.abs(np.cos(t)) + 0.1 * np.abs(np.sin(t))
    ext_y = 0.05 * np.abs(np.sin(t)) + 0.1 * np.abs(np.cos(t))
    along = rng.uniform(-0.6, 0.6, size=len(pick))
    nx = np.where(wall == 0, 1.0, np.where(wall == 1, -1.0, 0.0))
    ny = np.where(wall == 2, 1.0, np.where(wall == 3, -1.0, 0.0))
    ext = np.where(wall < 2, ext_x, ext_y)
    cx = np.where(wall < 2, nx * (1.0 - ext - u), along)
    cy = np.where(wall < 2, along, ny * (1.0 - ext - u))
    Rb = math.hypot(0.05, 0.1)
    ok = P._clear(cx, cy, np.full(len(pick), Rb), pick)
    x = x.copy()
    y = y.copy()
    x[pick[ok]] = cx[ok]
    y[pick[ok]] = cy[ok]
    return x, y


def _dense_sphere(P, rng, x, y, r, box_xy, box_th, NB, q):
    """Dense mode for sphere q: with probability 0.3 put it against an earlier
    sphere or against a face of a box."""
    E = P.E
    pick = np.nonzero(rng.random(E) < DENSE_FRACTION)[0]
    x = x.copy()
    y = y.copy()
    todo = np.arange(len(pick))
    for _ in range(200):
        if len(todo) == 0:
            break
        ee = pick[todo]
        n_placed = P.n  # boxes occupy slots 0..NB-1 of the placer
        partner = rng.integers(0, n_placed, size=len(ee))
        u = rng.uniform(*DENSE_OFFSET, size=len(ee))
        rr = r[ee]
        is_box = partner < NB
        # sphere partner: centre distance r1 + r2 + u along a random direction
        phi = rng.uniform(0, 2 * math.pi, size=len(ee))
        d = P.R[ee, partner] + rr + u
        cx = P.cx[ee, partner] + d * np.cos(phi)
        cy = P.cy[ee, partner] + d * np.sin(phi)
        # box partner: face f in (+x, -x, +y, -y) of the box frame
        bi = np.minimum(partner, NB - 1)
        face = rng.integers(0, 4, size=len(ee))
        hw, hh = 0.05, 0.1
        off = rng.uniform(-0.8, 0.8, size=len(ee))
        lx = np.where(face == 0, hw + rr + u, np.where(face == 1, -(hw + rr + u), off * hw))
        ly = np.where(face == 2, hh + rr + u, np.where(face == 3, -(hh + rr + u), off * hh))
        t = box_th[ee, bi]
        bx = box_xy[ee, bi, 0] + np.cos(t) * lx - np.sin(t) * ly
        by = box_xy[ee, bi, 1] + np.sin(t) * lx + np.cos(t) * ly
        cx = np.where(is_box, bx, cx)
        cy = np.where(is_box, by, cy)
        ok = P._clear(cx, cy, rr, ee, skip=partner)
        # keep well clear of the walls at +-1
        ok &= (np.abs(cx) + rr <= 0.95) & (np.abs(cy) + rr <= 0.95)
        x[ee[ok]] = cx[ok]
        y[ee[ok]] = cy[ok]
        todo = todo[~ok]
    return x, y


def mixed_scene(n_envs: int = 64, seed: int = 0, spread: float = 0.35,
                substeps: int = 3) -> Scene:
    """Test scene with every pair type in contact: per env 6 spheres, 3 boxes,
    2 movable lines and 1 fixed line, centres uniform in [-spread, spread]^2
    with random orientations, sizes and masses, random initial velocities,
    most bodies movable and rotatable, gravity (0, -1).  Overlaps are left
    as they fall (no clearance), so contacts of all kinds occur."""
    E, NS, NB, NL = n_envs, 6, 3, 3
    N = NS + NB + NL
    sc = _empty("mixed", E, N, NS + NB + 2, substeps, 0.05, 0.1, gx=0.0, gy=-1.0)
    rng = np.random.default_rng(seed)
    s = slice(0, NS)
    b = slice(NS, NS + NB)
    ln = slice(NS + NB, N)
    sc.shape[:, s] = SPHERE
    sc.shape[:, b] = BOX
    sc.shape[:, ln] = LINE
    allf = MOVABLE | ROTATABLE | COLLIDABLE | ACTUATED
    sc.flags[:, : N - 1] = allf
    sc.flags[:, N - 1] = COLLIDABLE
    sc.size_a[:, s] = _f32(rng.uniform(0.04, 0.1, size=(E, NS)))
    sc.size_a[:, b] = _f32(rng.uniform(0.08, 0.25, size=(E, NB)))
    sc.size_b[:, b] = _f32(rng.uniform(0.08, 0.25, size=(E, NB)))
    sc.size_a[:, ln] = _f32(rng.uniform(0.15, 0.5, size=(E, NL)))
    sc.mass[:] = _f32(rng.uniform(0.5, 3.0, size=(E, N)))
    st = sc.init_state
    st[:, :, 0] = _f32(rng.uniform(-spread, spread, size=(E, N)))
    st[:, :, 1] = _f32(rng.uniform(-spread, spread, size=(E, N)))
    st[:, :, 2] = _f32(rng.uniform(-0.5, 0.5, size=(E, N)))
    st[:, :, 3] = _f32(rng.uniform(-0.5, 0.5, size=(E, N)))
    st[:, :, 4] = _f32(rng.uniform(-math.pi, math.pi, size=(E, N)))
    st[:, :, 5] = _f32(rng.uniform(-1.0, 1.0, size=(E, N)))
    st[:, N - 1, 2:] = 0.0
    st[:, N - 1, 5] = 0.0
    return sc


def diff_scene(n_envs: int = 4096, seed: int = 0, dense: bool = False) -> Scene:
    """Differentiable-rollout workload: per env 8 agent spheres (r=0.05,
    mass 1, movable, actuated) then 2 static landmark spheres (r=0.1); centres
    uniform in [-1,1]^2 with bounding circles apart (or, dense, 30% placed
    against an earlier body); dt=0.1, drag 0.25, 3 substeps."""
    E, N = n_envs, 10
    sc = _empty("diff" + ("-dense" if dense else ""), E, N, 8, 3, 0.1, 0.25)
    rng = np.random.default_rng(seed)
    radii = np.array([0.05] * 8 + [0.1] * 2)
    sc.shape[:] = SPHERE
    sc.flags[:, :8] = MOVABLE | COLLIDABLE | ACTUATED
    sc.flags[:, 8:] = COLLIDABLE
    sc.size_a[:] = _f32(radii)
    P = _Placer(rng, E, N)
    order = [8, 9] + list(range(8))
    for slot, ent in enumerate(order):
        x, y = _place_sphere(P, rng, radii[ent], dense and slot > 0)
        sc.init_state[:, ent, 0] = x
        sc.init_state[:, ent, 1] = y
    return sc


def ragged_scene(n_envs: int = 65536, seed: int = 0, max_agents: int = 64,
                 max_boxes: int = 8, max_lines: int = 4):
    """Ragged workload: per env U{2..max_agents} agent spheres (r=0.05, mass
    1, actuated), U{0..max_boxes} boxes (0.1 x 0.2, mass 5, rotatable,
    actuated) and U{0..max_lines} fixed walls (the walls at x = +1, x = -1,
    y = +1, y = -1, in that order); bodies rejection-sampled inside
    [-0.9, 0.9]^2; dt 0.1, drag 0.25, 5 substeps.

    Returns (scene, counts): the scene padded to the largest count with inert
    entities (no flags) after each env's real ones, and counts [E] of real
    entities (agents, then boxes, then walls)."""
    rng = np.random.default_rng(seed)
    na = rng.integers(2, max_agents + 1, size=n_envs)
    nb = rng.integers(0, max_boxes + 1, size=n_envs)
    nl = rng.integers(0, max_lines + 1, size=n_envs)
    counts = na + nb + nl
    N = int(counts.max()) if n_envs else 1
    A = int((na + nb).max()) if n_envs else 0
    sc = _empty("ragged", n_envs, N, A, 5, 0.1, 0.25)
    sc.shape[:] = SPHERE
    sc.size_a[:] = 0.05
    walls = [(1.0, 0.0, np.float32(math.pi / 2)), (-1.0, 0.0, np.float32(math.pi / 2)),
             (0.0, 1.0, 0.0), (0.0, -1.0, 0.0)]
    P = _Placer(rng, n_envs, max_agents + max_boxes)
    Rb = math.hypot(0.05, 0.1)
    envs_all = np.arange(n_envs)
    for q in range(max_boxes):
        envs = envs_all[nb > q]
        idx = na[envs] + q
        x, y = P.place_free(np.full(n_envs, Rb), -0.9, 0.9, envs=envs)
        P.cx[envs, P.n], P.cy[envs, P.n], P.R[envs, P.n] = x, y, Rb
        P.advance()
        sc.shape[envs, idx] = BOX
        sc.flags[envs, idx] = MOVABLE | ROTATABLE | COLLIDABLE | ACTUATED
        sc.size_a[envs, idx] = 0.1
        sc.size_b[envs, idx] = 0.2
        sc.mass[envs, idx] = 5.0
        sc.init_state[envs, idx, 0] = x
        sc.init_state[envs, idx, 1] = y
        sc.init_state[envs, idx, 4] = rng.uniform(0, 2 * math.pi, size=len(envs)).astype(np.float32)
    for q in range(int(na.max()) if n_envs else 0):
        envs = envs_all[na > q]
        x, y = P.place_free(np.full(n_envs, 0.05), -0.9, 0.9, envs=envs)
        P.cx[envs, P.n], P.cy[envs, P.n], P.R[envs, P.n] = x, y, 0.05
        P.advance()
        sc.flags[envs, q] = MOVABLE | COLLIDABLE | ACTUATED
        sc.init_state[envs, q, 0] = x
        sc.init_state[envs, q, 1] = y
    # agents occupy [0, na), boxes were written at [na, na + nb): move boxes
    # after agents is already their index; walls follow
    for q in range(max_lines):
        envs = envs_all[nl > q]
        idx = na[envs] + nb[envs] + q
        wx, wy, wt = walls[q]
        sc.shape[envs, idx] = LINE
        sc.flags[envs, idx] = COLLIDABLE
        sc.size_a[envs, idx] = 2.0
        sc.init_state[envs, idx, 0] = wx
        sc.init_state[envs, idx, 1] = wy
        sc.init_state[envs, idx, 4] = wt
    return sc, counts


def pack_ragged(scene: Scene, counts):
    """Packed per-entity arrays (dict of [total] / [total, 6]) of the first
    counts[e] entities of every env."""
    sel = np.arange(scene.n_entities)[None, :] < np.asarray(counts)[:, None]
    out = {k: np.ascontiguousarray(getattr(scene, k)[sel])
           for k in ("shape", "flags", "size_a", "size_b", "mass", "inertia")}
    out["init_state"] = np.ascontiguousarray(scene.init_state[sel])
    return out


def surrogate_scene(n_envs: int = 65536, seed: int = 0, substeps: int = 5) -> Scene:
    """The walled sphere world of the learned surrogate: ``paper_scene``
    without its boxes, i.e. per env the 16 agent spheres (entities 0..15,
    actuated, action rows 0..15) then the 4 walls (entities 16..19)."""
    sc = paper_scene(n_envs, seed, dense=False, substeps=substeps)
    keep = np.r_[0:16, 20:24]
    kw = dataclasses.asdict(sc)
    for key in ("shape", "flags", "size_a", "size_b", "mass", "inertia", "init_state"):
        kw[key] = np.ascontiguousarray(getattr(sc, key)[:, keep])
    kw.update(name="surrogate", n_entities=20, n_actuated=16)
    return Scene(**kw)


def make_goals(scene: Scene, seed: int = 0) -> np.ndarray:
    """Goal positions [n_envs, n_actuated, 2], uniform in [-1, 1]^2, FP32."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x60A1]))
    return rng.uniform(-1.0, 1.0, size=(scene.n_envs, scene.n_actuated, 2)).astype(np.float32)


def make_actions(scene: Scene, n_steps: int, seed: int = 0) -> np.ndarray:
    """Per-step actions [n_steps, n_envs, n_actuated, 3] (fx, fy, torque),
    uniform in [-1, 1], FP32."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xAC7]))
    shape = (n_steps, scene.n_envs, scene.n_actuated, 3)
    return rng.uniform(-1.0, 1.0, size=shape).astype(np.float32)


CONFIGS = {
    "small": small_scene,
    "paper": paper_scene,
    "mixed": mixed_scene,
    "diff": diff_scene,
    "surrogate": surrogate_scene,
}
