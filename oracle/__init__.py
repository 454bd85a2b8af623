"""FP64 CPU oracle of the VMAS world step -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The CUDA product path never does,
and the two share no code: the oracle is plain C in ``vmas_oracle.c``
(section 3 of the VMAS paper, Eqs. 1-3, with the readings listed in that
file's header), compiled with gcc, loaded here through ctypes.

Inputs are duck-typed: any object with the attributes of a scene
(n_envs, n_entities, n_actuated, substeps, dt, drag, gx, gy, c, k,
max_speed, shape, flags, size_a, size_b, mass, inertia) works.  Arrays are
widened to float64 exactly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vmas_oracle.c")
_LIB = os.path.join(_HERE, "libvmas_oracle.so")
_handle = None

SPHERE, BOX, LINE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _World(ctypes.Structure):
    _fields_ = [
        ("n_envs", ctypes.c_int32), ("n_entities", ctypes.c_int32),
        ("n_actuated", ctypes.c_int32), ("substeps", ctypes.c_int32),
        ("dt", ctypes.c_double), ("drag", ctypes.c_double), ("gx", ctypes.c_double),
        ("gy", ctypes.c_double), ("c", ctypes.c_double), ("k", ctypes.c_double),
        ("max_speed", ctypes.c_double),
        ("shape", ctypes.c_void_p), ("flags", ctypes.c_void_p),
        ("size_a", ctypes.c_void_p), ("size_b", ctypes.c_void_p),
        ("mass", ctypes.c_void_p), ("inertia", ctypes.c_void_p),
    ]


def _lib():
    global _handle
    if _handle is None:
        h = ctypes.CDLL(build())
        h.ow_step.argtypes = [ctypes.POINTER(_World), ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_int, ctypes.c_int]
        h.ow_step.restype = ctypes.c_int
        h.ow_step_margin.argtypes = [ctypes.POINTER(_World), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        h.ow_step_margin.restype = ctypes.c_int
        h.ow_pairs.argtypes = [ctypes.POINTER(_World), ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p]
        h.ow_pairs.restype = ctypes.c_int
        h.ow_pair_list.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        h.ow_pair_list.restype = ctypes.c_int
        h.ow_pair_geometry.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        h.ow_pair_geometry.restype = ctypes.c_int
        h.ow_contact_magnitude.argtypes = [ctypes.c_double] * 3
        h.ow_contact_magnitude.restype = ctypes.c_double
        h.ow_inertia.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4
        h.ow_inertia.restype = ctypes.c_double
        h.ow_max_threads.restype = ctypes.c_int
        h.ow_rollout_grad.argtypes = [ctypes.POINTER(_World), ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]
        h.ow_rollout_grad.restype = ctypes.c_int
        h.ow_lidar.argtypes = [ctypes.POINTER(_World), ctypes.c_void_p, ctypes.c_int,
                               ctypes.c_double, ctypes.c_void_p]
        h.ow_lidar.restype = ctypes.c_int
        _handle = h
    return _handle


class _Packed:
    """Keeps the float64 copies alive while the C side reads them."""

    def __init__(self, sc):
        E, N = int(sc.n_envs), int(sc.n_entities)
        self.shape = np.ascontiguousarray(np.asarray(sc.shape, np.uint8).reshape(E, N))
        self.flags = np.ascontiguousarray(np.asarray(sc.flags, np.uint8).reshape(E, N))
        self.arrs = [np.ascontiguousarray(np.asarray(getattr(sc, k), np.float64).reshape(E, N))
                     for k in ("size_a", "size_b", "mass", "inertia")]
        self.w = _World(E, N, int(sc.n_actuated), int(sc.substeps), float(sc.dt), float(sc.drag),
                        float(sc.gx), float(sc.gy), float(sc.c), float(sc.k), float(sc.max_speed),
                        self.shape.ctypes.data, self.flags.ctypes.data,
                        *[a.ctypes.data for a in self.arrs])


def step(scene, state, actions, threads: int = 1) -> np.ndarray:
    """Run len(actions) world steps from ``state`` ([E, N, 6]).

    actions: [T, E, n_actuated, 3] (or [E, n_actuated, 3] for one step).
    Returns the new state as float64 [E, N, 6]; the inputs are not modified.
    """
    pk = _Packed(scene)
    E, N, A = int(scene.n_envs), int(scene.n_entities), int(scene.n_actuated)
    st = np.array(np.asarray(state, np.float64).reshape(E, N, 6), order="C", copy=True)
    act = np.asarray(actions, np.float64)
    if act.ndim == 3:
        act = act[None]
    act = np.ascontiguousarray(act.reshape(act.shape[0], E, A, 3))
    rc = _lib().ow_step(ctypes.byref(pk.w), st.ctypes.data, act.ctypes.data, act.shape[0], threads)
    if rc != 0:
        raise ValueError("oracle rejected the world description")
    return st


def step_margin(scene, state, actions, threads: int = 1):
    """As ``step``, and also the smallest decision margin [E] each env met
    over all its substeps (Reading R9 of the C file): the least |gap| of an
    active pair and, for pairs in contact, how far the chosen face, axis,
    incident edge, clip or normal orientation was from its runner-up.  Two
    correct implementations in different precisions can only disagree
    beyond rounding where that margin is within their rounding difference."""
    pk = _Packed(scene)
    E, N, A = int(scene.n_envs), int(scene.n_entities), int(scene.n_actuated)
    st = np.array(np.asarray(state, np.float64).reshape(E, N, 6), order="C", copy=True)
    act = np.asarray(actions, np.float64)
    if act.ndim == 3:
        act = act[None]
    act = np.ascontiguousarray(act.reshape(act.shape[0], E, A, 3))
    margin = np.zeros(E, np.float64)
    rc = _lib().ow_step_margin(ctypes.byref(pk.w), st.ctypes.data, act.ctypes.data,
                               act.shape[0], threads, margin.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the world description")
    return st, margin


def pairs(scene, state):
    """First-substep contact mask (uint8 [E, P]) and signed gap (float64
    [E, P], +inf where a pair is not active) from ``state``."""
    pk = _Packed(scene)
    E, N = int(scene.n_envs), int(scene.n_entities)
    P = N * (N - 1) // 2
    st = np.ascontiguousarray(np.asarray(state, np.float64).reshape(E, N, 6))
    mask = np.zeros((E, P), np.uint8)
    gap = np.zeros((E, P), np.float64)
    _lib().ow_pairs(ctypes.byref(pk.w), st.ctypes.data, mask.ctypes.data, gap.ctypes.data)
    return mask, gap


def pair_list(n: int):
    """Canonical pair list (i < j, row-major) as two int32 arrays."""
    P = n * (n - 1) // 2
    pi = np.zeros(max(P, 1), np.int32)
    pj = np.zeros(max(P, 1), np.int32)
    _lib().ow_pair_list(n, pi.ctypes.data, pj.ctypes.data)
    return pi[:P], pj[:P]


def pair_geometry(body_i, body_j):
    """Closest points of one ordered pair.  body = (shape, x, y, theta, a, b).

    Returns dict(g, n=(nx, ny), p_i=(x, y), p_j=(x, y), has_normal)."""
    bi = np.ascontiguousarray(np.asarray(body_i, np.float64))
    bj = np.ascontiguousarray(np.asarray(body_j, np.float64))
    out = np.zeros(7, np.float64)
    hn = _lib().ow_pair_geometry(bi.ctypes.data, bj.ctypes.data, out.ctypes.data)
    return {"g": out[0], "n": out[1:3].copy(), "p_i": out[3:5].copy(),
            "p_j": out[5:7].copy(), "has_normal": bool(hn)}


def contact_magnitude(c: float, k: float, gap: float) -> float:
    """Eq. 2 magnitude c*k*log(1+exp(-gap/k)) (applied when gap <= 0)."""
    return _lib().ow_contact_magnitude(c, k, gap)


def inertia(shape: int, m: float, a: float, b: float, given: float = 0.0) -> float:
    return _lib().ow_inertia(shape, m, a, b, given)


def max_threads() -> int:
    return _lib().ow_max_threads()


def rollout_grad(scene, state, actions, goals, with_grad=True):
    """Differentiable rollout of a sphere world (FP64): per-env loss
    sum_k |x_k(T) - goal_k|^2 over the actuated entities after len(actions)
    steps, and its gradient with respect to the actions (reverse mode).

    actions [T, E, A, 3], goals [E, A, 2].  Returns (loss [E], grad [T, E, A, 3]
    or None)."""
    pk = _Packed(scene)
    E, N, A = int(scene.n_envs), int(scene.n_entities), int(scene.n_actuated)
    st = np.ascontiguousarray(np.asarray(state, np.float64).reshape(E, N, 6))
    act = np.ascontiguousarray(np.asarray(actions, np.float64))
    T = act.shape[0]
    act = act.reshape(T, E, A, 3)
    gl = np.ascontiguousarray(np.asarray(goals, np.float64).reshape(E, A, 2))
    loss = np.zeros(E, np.float64)
    grad = np.zeros((T, E, A, 3), np.float64) if with_grad else None
    rc = _lib().ow_rollout_grad(ctypes.byref(pk.w), st.ctypes.data, act.ctypes.data, T,
                                gl.ctypes.data, loss.ctypes.data,
                                grad.ctypes.data if with_grad else None)
    if rc != 0:
        raise ValueError("rollout_grad needs a sphere world without a speed cap")
    return loss, grad


def lidar(scene, state, n_rays: int, max_range: float) -> np.ndarray:
    """Ray-cast distances [E, n_actuated, n_rays] from every actuated entity
    (angles theta + 2 pi k / n_rays), FP64."""
    pk = _Packed(scene)
    E, N, A = int(scene.n_envs), int(scene.n_entities), int(scene.n_actuated)
    st = np.ascontiguousarray(np.asarray(state, np.float64).reshape(E, N, 6))
    out = np.zeros((E, A, n_rays), np.float64)
    _lib().ow_lidar(ctypes.byref(pk.w), st.ctypes.data, n_rays, float(max_range), out.ctypes.data)
    return out


def lidar_sensitivity(scene, state, n_rays: int, max_range: float, trials: int = 24,
                      rel: float = 2.0 ** -20, seed: int = 0) -> np.ndarray:
    """How much each ray's FP64 result moves when the inputs are perturbed
    at the size of single-precision rounding: the largest |t' - t| [E, A,
    n_rays] over ``trials`` copies of the scene whose positions, angles and
    sizes are each moved by a uniform random amount of at most ``rel`` times
    max(1, |value|) (2^-20: eight FP32 units in the last place at 1).  A ray
    that grazes a disc (the entry distance goes as the square root of the
    discriminant), clips a box corner or a segment end, or starts on a
    surface moves by far more than its inputs; a well-conditioned ray moves
    by about as much as they do."""
    import dataclasses

    rng = np.random.default_rng(seed)
    st0 = np.asarray(state, np.float64)
    ref = lidar(scene, st0, n_rays, max_range)
    spread = np.zeros_like(ref)

    def jig(a):
        a = np.asarray(a, np.float64)
        return a + rng.uniform(-rel, rel, a.shape) * np.maximum(1.0, np.abs(a))

    for _ in range(trials):
        st = st0.copy()
        st[..., 0] = jig(st[..., 0])
        st[..., 1] = jig(st[..., 1])
        st[..., 4] = jig(st[..., 4])
        sa = np.asarray(scene.size_a, np.float64)
        sb = np.asarray(scene.size_b, np.float64)
        sc = _Jiggled(scene, sa * (1 + rng.uniform(-rel, rel, sa.shape)),
                      sb * (1 + rng.uniform(-rel, rel, sb.shape)))
        spread = np.maximum(spread, np.abs(lidar(sc, st, n_rays, max_range) - ref))
    return spread


class _Jiggled:
    """A scene with its sizes replaced (every other attribute delegated)."""

    def __init__(self, base, size_a, size_b):
        self._base, self.size_a, self.size_b = base, size_a, size_b

    def __getattr__(self, name):
        return getattr(self._base, name)
