"""Python binding of the VMAS world step: argument marshalling over the C ABI.

Every step of the physics runs in the CUDA library (libvmas.so); this module
only builds the world description from numpy arrays, passes torch tensors'
device pointers and torch's current CUDA stream, and turns status codes into
exceptions.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


def _stream_handle(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


class World:
    """A batch of VMAS worlds resident on one CUDA device.

    scene: any object with the attributes of ``scenes.Scene`` (n_envs,
    n_entities, n_actuated, substeps, dt, drag, gx, gy, c, k, max_speed and
    the per-entity arrays shape, flags, size_a, size_b, mass, inertia,
    init_state).  The world is created on the current CUDA device.
    """

    def __init__(self, scene, device=None):
        L = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        E, N = int(scene.n_envs), int(scene.n_entities)
        self.n_envs, self.n_entities = E, N
        self.n_actuated, self.substeps = int(scene.n_actuated), int(scene.substeps)
        self.n_pairs = N * (N - 1) // 2
        keep = {
            "shape": np.ascontiguousarray(np.asarray(scene.shape, np.uint8).reshape(E, N)),
            "flags": np.ascontiguousarray(np.asarray(scene.flags, np.uint8).reshape(E, N)),
        }
        for key in ("size_a", "size_b", "mass", "inertia"):
            keep[key] = np.ascontiguousarray(np.asarray(getattr(scene, key), np.float32).reshape(E, N))
        keep["init_state"] = np.ascontiguousarray(
            np.asarray(scene.init_state, np.float32).reshape(E, N, 6))
        d = _lib.WorldDesc(E, N, self.n_actuated, self.substeps, scene.dt, scene.drag, scene.gx,
                           scene.gy, scene.c, scene.k, scene.max_speed,
                           *[keep[k].ctypes.data for k in ("shape", "flags", "size_a", "size_b",
                                                           "mass", "inertia", "init_state")])
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(L.vmas_world_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self._L = L

    # ---------------------------------------------------------------- steps
    def _handle(self):
        if self._h is None:
            raise RuntimeError("world is closed")
        return self._h

    def _actions(self, actions, steps=None):
        shape = (self.n_envs, self.n_actuated, 3) if steps is None else \
            (steps, self.n_envs, self.n_actuated, 3)
        if tuple(actions.shape) != shape:
            raise ValueError("actions must have shape %s, got %s" % (shape, tuple(actions.shape)))
        if actions.dtype != torch.float32 or not actions.is_contiguous():
            raise ValueError("actions must be contiguous float32")
        return actions

    def step(self, actions: torch.Tensor, stream=None) -> None:
        """One world step.  actions: CUDA float32 [E, n_actuated, 3]."""
        a = self._actions(actions)
        if not a.is_cuda:
            raise ValueError("step() takes a CUDA tensor; use step_host() for host actions")
        _lib.check(self._L.vmas_step(self._handle(), _ptr(a) if a.numel() else None,
                                     _stream_handle(stream)))

    def step_host(self, actions, stream=None) -> None:
        """One world step from HOST actions [E, n_actuated, 3] (numpy or CPU
        tensor; pinned memory keeps the upload asynchronous)."""
        if isinstance(actions, np.ndarray):
            actions = torch.from_numpy(np.ascontiguousarray(actions, np.float32))
        a = self._actions(actions)
        if a.is_cuda:
            raise ValueError("step_host() takes host actions")
        _lib.check(self._L.vmas_step_host(self._handle(), _ptr(a) if a.numel() else None,
                                          _stream_handle(stream)))
        if a.numel() and a.is_pinned():
            # the upload is asynchronous: hold the buffer until it has run, so
            # that the pinned-memory cache cannot hand it out again earlier
            ev = torch.cuda.Event()
            ev.record(torch.cuda.current_stream() if stream is None else stream)
            self._in_flight = [(e, t) for e, t in getattr(self, "_in_flight", []) if not e.query()]
            self._in_flight.append((ev, a))

    def rollout(self, actions: torch.Tensor, stream=None) -> None:
        """len(actions) consecutive steps; actions: CUDA float32 [T, E, A, 3]."""
        T = int(actions.shape[0])
        a = self._actions(actions, T)
        _lib.check(self._L.vmas_rollout(self._handle(), _ptr(a) if a.numel() else None, T,
                                        _stream_handle(stream)))

    def set_rollout_tile(self, steps_per_launch: int) -> None:
        """World steps per kernel launch in rollout() (1..1024): state and
        candidate lists stay on chip between them; results are bitwise the
        same for any value."""
        _lib.check(self._L.vmas_world_set_rollout_tile(self._handle(), int(steps_per_launch)))

    def rollout_host(self, actions, states_out=None, stream=None) -> torch.Tensor:
        """len(actions) steps between host buffers: actions [T, E, A, 3] (host;
        pinned keeps the uploads asynchronous), every step's state into
        states_out [T, E, N, 6] (host, allocated pinned if None).  Uploads,
        steps and downloads overlap; returns states_out once all have arrived."""
        if isinstance(actions, np.ndarray):
            actions = torch.from_numpy(np.ascontiguousarray(actions, np.float32))
        T = int(actions.shape[0])
        a = self._actions(actions, T)
        if a.is_cuda:
            raise ValueError("rollout_host() takes host actions")
        shape = (T, self.n_envs, self.n_entities, 6)
        if states_out is None:
            states_out = torch.empty(shape, dtype=torch.float32).pin_memory()
        if (tuple(states_out.shape) != shape or states_out.dtype != torch.float32
                or states_out.is_cuda or not states_out.is_contiguous()):
            raise ValueError("states_out must be a contiguous host float32 %s" % (shape,))
        _lib.check(self._L.vmas_rollout_host(self._handle(), _ptr(a) if a.numel() else None, T,
                                             _ptr(states_out) if states_out.numel() else None,
                                             _stream_handle(stream)))
        return states_out

    # ---------------------------------------------------------------- state
    def state(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """State [E, N, 6] (x, y, vx, vy, theta, omega).  Into ``out`` when
        given (CUDA or CPU float32); otherwise a new CUDA tensor."""
        if out is None:
            out = torch.empty((self.n_envs, self.n_entities, 6), dtype=torch.float32,
                              device=self.device)
        if tuple(out.shape) != (self.n_envs, self.n_entities, 6) or out.dtype != torch.float32 \
                or not out.is_contiguous():
            raise ValueError("out must be contiguous float32 [E, N, 6]")
        _lib.check(self._L.vmas_state(self._handle(), _ptr(out) if out.numel() else None,
                                      1 if out.is_cuda else 0, _stream_handle(stream)))
        return out

    def set_state(self, state, env_mask=None, stream=None) -> None:
        """Overwrite the state of the envs selected by env_mask (bool/uint8
        [E], None = all).  state: [E, N, 6] CUDA or host."""
        if isinstance(state, np.ndarray):
            state = torch.from_numpy(np.ascontiguousarray(state, np.float32))
        if tuple(state.shape) != (self.n_envs, self.n_entities, 6) or state.dtype != torch.float32:
            raise ValueError("state must be float32 [E, N, 6]")
        state = state.contiguous()
        m = None
        if env_mask is not None:
            m = np.ascontiguousarray(np.asarray(
                env_mask.cpu() if isinstance(env_mask, torch.Tensor) else env_mask).astype(np.uint8))
            if m.shape != (self.n_envs,):
                raise ValueError("env_mask must have shape [E]")
        _lib.check(self._L.vmas_set_state(self._handle(), _ptr(state) if state.numel() else None,
                                          1 if state.is_cuda else 0,
                                          m.ctypes.data if m is not None else None,
                                          _stream_handle(stream)))

    def debug_pairs(self, stream=None) -> torch.Tensor:
        """First-substep contact mask of the current state, uint8 [E, P]."""
        out = torch.zeros((self.n_envs, self.n_pairs), dtype=torch.uint8, device=self.device)
        _lib.check(self._L.vmas_debug_pairs(self._handle(), _ptr(out) if out.numel() else None,
                                            _stream_handle(stream)))
        return out

    def lidar(self, n_rays: int, max_range: float, stream=None) -> torch.Tensor:
        """LIDAR distances [E, n_actuated, n_rays] from the current state."""
        out = torch.empty((self.n_envs, self.n_actuated, n_rays), dtype=torch.float32,
                          device=self.device)
        _lib.check(self._L.vmas_lidar(self._handle(), int(n_rays), float(max_range),
                                      out.data_ptr() if out.numel() else None,
                                      _stream_handle(stream)))
        return out

    def pair_table(self):
        pi = np.zeros(max(self.n_pairs, 1), np.int32)
        pj = np.zeros(max(self.n_pairs, 1), np.int32)
        _lib.check(self._L.vmas_pair_table(self._handle(), pi.ctypes.data, pj.ctypes.data))
        return pi[: self.n_pairs], pj[: self.n_pairs]

    @property
    def skin(self) -> float:
        """Margin of the per-step contact-candidate list (speed only)."""
        v = ctypes.c_float()
        _lib.check(self._L.vmas_world_get_skin(self._handle(), ctypes.byref(v)))
        return v.value

    @skin.setter
    def skin(self, value: float) -> None:
        _lib.check(self._L.vmas_world_set_skin(self._handle(), float(value)))

    def enable_stats(self, on: bool = True) -> None:
        """Turn the step counters on or off (tuning aid; costs atomics)."""
        _lib.check(self._L.vmas_world_set_stats(self._handle(), 1 if on else 0))

    def stats(self, reset: bool = False, stream=None) -> dict:
        """The step counters as a dict (see include/vmas.h)."""
        out = np.zeros(_lib.STATS_COUNT, np.uint64)
        _lib.check(self._L.vmas_world_get_stats(self._handle(), out.ctypes.data, 1 if reset else 0,
                                                _stream_handle(stream)))
        return dict(zip(_lib.STATS_NAMES, (int(v) for v in out)))

    def check(self, stream=None) -> int:
        """Wait for the stream; raise if a kernel set the device error word."""
        bits = ctypes.c_int32(0)
        rc = self._L.vmas_check(self._handle(), _stream_handle(stream), ctypes.byref(bits))
        if rc == _lib.VMAS_EDEVICE:
            raise _lib.VmasError(rc, "device error bits %d" % bits.value)
        _lib.check(rc)
        return bits.value

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            self._L.vmas_world_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
