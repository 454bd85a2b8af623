"""Python binding of packed ragged worlds (argument marshalling only).

A ragged world holds environments with different entity counts, packed
without padding; the CUDA library sorts them into size classes, steps each
class with the kernel compiled for it, runs rollouts as captured CUDA graphs
and autotunes its launch choices (see include/vmas.h).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


def _stream():
    return torch.cuda.current_stream().cuda_stream


class RaggedWorld:
    """counts [E] entities per env; per-entity arrays are packed [total] (or
    [total, 6] for init_state) in env order."""

    def __init__(self, counts, shape, flags, size_a, size_b, mass, inertia, init_state, *,
                 substeps, dt, drag, gx=0.0, gy=0.0, c=100.0, k=1e-3, max_speed=0.0):
        L = _lib.load()
        counts = np.asarray(counts, np.int64)
        offs = np.zeros(len(counts) + 1, np.int32)
        offs[1:] = np.cumsum(counts)
        keep = [np.ascontiguousarray(offs),
                np.ascontiguousarray(shape, np.uint8), np.ascontiguousarray(flags, np.uint8)]
        keep += [np.ascontiguousarray(a, np.float32) for a in (size_a, size_b, mass, inertia)]
        keep.append(np.ascontiguousarray(np.asarray(init_state, np.float32).reshape(-1, 6)))
        d = _lib.RaggedDesc(len(counts), substeps, dt, drag, gx, gy, c, k, max_speed,
                            *[a.ctypes.data for a in keep])
        h = ctypes.c_void_p()
        _lib.check(L.vmas_ragged_create(ctypes.byref(d), ctypes.byref(h)))
        self._h, self._L = h, L
        ne, nt, na = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        self.class_envs = np.zeros(5, np.int32)
        _lib.check(L.vmas_ragged_info(h, ctypes.byref(ne), ctypes.byref(nt), ctypes.byref(na),
                                      self.class_envs.ctypes.data))
        self.n_envs, self.n_entities, self.n_action_rows = ne.value, nt.value, na.value
        self.action_offsets = np.zeros(self.n_envs + 1, np.int32)
        _lib.check(L.vmas_ragged_action_offsets(h, self.action_offsets.ctypes.data))
        self.entity_offsets = offs

    def step(self, actions: torch.Tensor) -> None:
        _lib.check(self._L.vmas_ragged_step(self._h, actions.data_ptr() if actions.numel() else None,
                                            _stream()))

    def rollout(self, actions: torch.Tensor) -> None:
        """actions [T, n_action_rows, 3] (CUDA float32); a CUDA graph replay."""
        _lib.check(self._L.vmas_ragged_rollout(self._h, actions.data_ptr() if actions.numel() else None,
                                               int(actions.shape[0]), _stream()))

    def state(self) -> torch.Tensor:
        out = torch.empty((self.n_entities, 6), dtype=torch.float32, device="cuda")
        _lib.check(self._L.vmas_ragged_state(self._h, out.data_ptr() if out.numel() else None, 1,
                                             _stream()))
        return out

    def set_state(self, state: torch.Tensor) -> None:
        _lib.check(self._L.vmas_ragged_set_state(self._h, state.contiguous().data_ptr(), _stream()))

    def check(self) -> int:
        """Wait for the stream; raise if a kernel set the device error word."""
        bits = ctypes.c_int32(0)
        rc = self._L.vmas_ragged_check(self._h, _stream(), ctypes.byref(bits))
        if rc == _lib.VMAS_EDEVICE:
            raise _lib.VmasError(rc, "device error bits %d" % bits.value)
        _lib.check(rc)
        return bits.value

    def tuning(self):
        lanes = np.zeros(5, np.int32)
        tile = ctypes.c_int32()
        _lib.check(self._L.vmas_ragged_get_tuning(self._h, lanes.ctypes.data, ctypes.byref(tile)))
        return lanes, tile.value

    def set_tuning(self, lanes=None, steps_per_launch: int = 1) -> None:
        arr = None if lanes is None else np.ascontiguousarray(lanes, np.int32)
        _lib.check(self._L.vmas_ragged_set_tuning(self._h, arr.ctypes.data if arr is not None else None,
                                                  int(steps_per_launch)))

    @property
    def schedule(self) -> int:
        """0: one launch per size class; 1, 2: every class in one persistent
        launch with an atomic work queue (128- or 96-register build)."""
        v = ctypes.c_int32()
        _lib.check(self._L.vmas_ragged_get_schedule(self._h, ctypes.byref(v)))
        return v.value

    @schedule.setter
    def schedule(self, value: int) -> None:
        _lib.check(self._L.vmas_ragged_set_schedule(self._h, int(value)))

    @property
    def persistent(self) -> bool:
        """True when every size class runs in one persistent launch."""
        return self.schedule != 0

    @persistent.setter
    def persistent(self, on: bool) -> None:
        self.schedule = 1 if on else 0

    def autotune(self, actions: torch.Tensor) -> None:
        _lib.check(self._L.vmas_ragged_autotune(self._h, actions.data_ptr(), int(actions.shape[0]),
                                                _stream()))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            self._L.vmas_ragged_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
