"""ctypes declarations of the C ABI in include/vmas.h (argument marshalling only).

Loading fails loudly when libvmas.so is missing: there is no CPU fallback.
With VMAS_CHECKED=1 in the environment the bounds-checked build
libvmas_checked.so is loaded instead (see build.py).
"""
from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "libvmas_checked.so" if os.environ.get("VMAS_CHECKED") == "1" else "libvmas.so")

VMAS_OK, VMAS_EINVAL, VMAS_ENOMEM, VMAS_ECUDA, VMAS_EDEVICE = 0, -1, -2, -3, -4
MAX_ENTITIES = 128
ABI_VERSION = 1

# Every symbol include/vmas.h declares.
SYMBOLS = (
    "vmas_world_create", "vmas_world_destroy", "vmas_world_info", "vmas_step",
    "vmas_step_host", "vmas_rollout", "vmas_rollout_host", "vmas_state", "vmas_set_state", "vmas_debug_pairs",
    "vmas_pair_table", "vmas_check", "vmas_last_error", "vmas_abi_version",
    "vmas_world_set_skin", "vmas_world_get_skin", "vmas_world_set_stats", "vmas_world_get_stats",
    "vmas_debug_body_axes", "vmas_debug_stage_timeout", "vmas_step_noalloc",
    "vmas_diff_rollout", "vmas_diff_backward",
    "vmas_lidar", "vmas_world_set_rollout_tile",
    "vmas_ragged_create", "vmas_ragged_destroy", "vmas_ragged_info", "vmas_ragged_action_offsets",
    "vmas_ragged_step", "vmas_ragged_rollout", "vmas_ragged_state", "vmas_ragged_set_state",
    "vmas_ragged_check",
    "vmas_ragged_set_tuning", "vmas_ragged_get_tuning", "vmas_ragged_autotune",
    "vmas_ragged_set_schedule", "vmas_ragged_get_schedule",
    "vmas_sur_param_count", "vmas_sur_create", "vmas_sur_destroy", "vmas_sur_set_params",
    "vmas_sur_get_params", "vmas_sur_set_mode", "vmas_sur_forward", "vmas_sur_loss_grad", "vmas_sur_adam",
    "vmas_sur_train_grad", "vmas_sur_train_step", "vmas_sur_step", "vmas_sur_debug_features", "vmas_debug_gemm_bf16",
    "vmas_sur_check", "vmas_debug_gemm_engine", "vmas_debug_diff_split",
    "vmas_debug_gemm_timeout", "vmas_debug_lidar_cull",
)
STATS_COUNT = 16
STATS_NAMES = ("env_steps", "rebuilds", "candidates",
               "eval_ss", "eval_sb", "eval_sl", "eval_bb", "eval_bl", "eval_ll",
               "hits_ss", "hits_sb", "hits_sl", "hits_bb", "hits_bl", "hits_ll", "full_scan")


class WorldDesc(ctypes.Structure):
    _fields_ = [
        ("n_envs", ctypes.c_int32), ("n_entities", ctypes.c_int32),
        ("n_actuated", ctypes.c_int32), ("substeps", ctypes.c_int32),
        ("dt", ctypes.c_float), ("drag", ctypes.c_float), ("gx", ctypes.c_float),
        ("gy", ctypes.c_float), ("contact_force", ctypes.c_float),
        ("contact_margin", ctypes.c_float), ("max_speed", ctypes.c_float),
        ("shape", ctypes.c_void_p), ("flags", ctypes.c_void_p), ("size_a", ctypes.c_void_p),
        ("size_b", ctypes.c_void_p), ("mass", ctypes.c_void_p), ("inertia", ctypes.c_void_p),
        ("init_state", ctypes.c_void_p),
    ]


class StepNoallocArgs(ctypes.Structure):
    """vmas_step_noalloc_args: sizes, parameters and caller-owned device buffers."""

    _fields_ = [
        ("n_envs", ctypes.c_int32), ("n_entities", ctypes.c_int32),
        ("n_actuated", ctypes.c_int32), ("substeps", ctypes.c_int32),
        ("dt", ctypes.c_float), ("drag", ctypes.c_float), ("gx", ctypes.c_float),
        ("gy", ctypes.c_float), ("contact_force", ctypes.c_float),
        ("contact_margin", ctypes.c_float), ("max_speed", ctypes.c_float),
        ("skin", ctypes.c_float),
        ("shape", ctypes.c_void_p), ("flags", ctypes.c_void_p), ("size_a", ctypes.c_void_p),
        ("size_b", ctypes.c_void_p), ("mass", ctypes.c_void_p), ("inertia", ctypes.c_void_p),
        ("state", ctypes.c_void_p), ("actions", ctypes.c_void_p), ("status", ctypes.c_void_p),
    ]


class RaggedDesc(ctypes.Structure):
    _fields_ = [
        ("n_envs", ctypes.c_int32), ("substeps", ctypes.c_int32),
        ("dt", ctypes.c_float), ("drag", ctypes.c_float), ("gx", ctypes.c_float),
        ("gy", ctypes.c_float), ("contact_force", ctypes.c_float),
        ("contact_margin", ctypes.c_float), ("max_speed", ctypes.c_float),
        ("env_offsets", ctypes.c_void_p),
        ("shape", ctypes.c_void_p), ("flags", ctypes.c_void_p), ("size_a", ctypes.c_void_p),
        ("size_b", ctypes.c_void_p), ("mass", ctypes.c_void_p), ("inertia", ctypes.c_void_p),
        ("init_state", ctypes.c_void_p),
    ]


class VmasError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("vmas error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load():
    """The loaded library (ctypes.CDLL) with prototypes set."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("%s is not built (expected at %s); build it with "
                          "paper_2207_03530_b300.build.build()"
                          % (os.path.basename(LIB_PATH), LIB_PATH))
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, P = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER
    sig = {
        "vmas_world_create": ([P(WorldDesc), P(vp)], ctypes.c_int),
        "vmas_world_destroy": ([vp], ctypes.c_int),
        "vmas_world_info": ([vp, P(i32), P(i32), P(i32), P(i32), P(i32)], ctypes.c_int),
        "vmas_step": ([vp, vp, vp], ctypes.c_int),
        "vmas_step_host": ([vp, vp, vp], ctypes.c_int),
        "vmas_rollout": ([vp, vp, i32, vp], ctypes.c_int),
        "vmas_rollout_host": ([vp, vp, i32, vp, vp], ctypes.c_int),
        "vmas_state": ([vp, vp, i32, vp], ctypes.c_int),
        "vmas_set_state": ([vp, vp, i32, vp, vp], ctypes.c_int),
        "vmas_debug_pairs": ([vp, vp, vp], ctypes.c_int),
        "vmas_pair_table": ([vp, vp, vp], ctypes.c_int),
        "vmas_check": ([vp, vp, P(i32)], ctypes.c_int),
        "vmas_last_error": ([], ctypes.c_char_p),
        "vmas_abi_version": ([], ctypes.c_int),
        "vmas_world_set_skin": ([vp, ctypes.c_float], ctypes.c_int),
        "vmas_world_get_skin": ([vp, P(ctypes.c_float)], ctypes.c_int),
        "vmas_world_set_stats": ([vp, i32], ctypes.c_int),
        "vmas_world_get_stats": ([vp, vp, i32, vp], ctypes.c_int),
        "vmas_debug_body_axes": ([vp, vp, i32, vp], ctypes.c_int),
        "vmas_debug_stage_timeout": ([vp, i32], ctypes.c_int),
        "vmas_step_noalloc": ([P(StepNoallocArgs), vp], ctypes.c_int),
        "vmas_diff_rollout": ([vp, vp, i32, vp, i32, vp, vp, vp], ctypes.c_int),
        "vmas_diff_backward": ([vp, vp, i32, vp, i32, vp, vp, vp, vp], ctypes.c_int),
        "vmas_lidar": ([vp, i32, ctypes.c_float, vp, vp], ctypes.c_int),
        "vmas_world_set_rollout_tile": ([vp, i32], ctypes.c_int),
        "vmas_ragged_create": ([P(RaggedDesc), P(vp)], ctypes.c_int),
        "vmas_ragged_destroy": ([vp], ctypes.c_int),
        "vmas_ragged_info": ([vp, P(i32), P(ctypes.c_int64), P(ctypes.c_int64), vp], ctypes.c_int),
        "vmas_ragged_action_offsets": ([vp, vp], ctypes.c_int),
        "vmas_ragged_step": ([vp, vp, vp], ctypes.c_int),
        "vmas_ragged_rollout": ([vp, vp, i32, vp], ctypes.c_int),
        "vmas_ragged_state": ([vp, vp, i32, vp], ctypes.c_int),
        "vmas_ragged_check": ([vp, vp, P(i32)], ctypes.c_int),
        "vmas_ragged_set_state": ([vp, vp, vp], ctypes.c_int),
        "vmas_ragged_set_tuning": ([vp, vp, i32], ctypes.c_int),
        "vmas_ragged_get_tuning": ([vp, vp, vp], ctypes.c_int),
        "vmas_ragged_autotune": ([vp, vp, i32, vp], ctypes.c_int),
        "vmas_ragged_set_schedule": ([vp, i32], ctypes.c_int),
        "vmas_ragged_get_schedule": ([vp, vp], ctypes.c_int),
        "vmas_sur_param_count": ([], ctypes.c_int),
        "vmas_sur_create": ([i32, P(vp)], ctypes.c_int),
        "vmas_sur_destroy": ([vp], ctypes.c_int),
        "vmas_sur_set_params": ([vp, vp], ctypes.c_int),
        "vmas_sur_get_params": ([vp, vp], ctypes.c_int),
        "vmas_sur_set_mode": ([vp, i32], ctypes.c_int),
        "vmas_sur_forward": ([vp, vp, vp, vp, vp], ctypes.c_int),
        "vmas_sur_loss_grad": ([vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "vmas_sur_adam": ([vp, ctypes.c_float, vp, vp], ctypes.c_int),
        "vmas_sur_train_grad": ([vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "vmas_sur_train_step": ([vp, vp, vp, ctypes.c_float, vp, vp], ctypes.c_int),
        "vmas_sur_step": ([vp, vp, vp, ctypes.c_float, vp, vp], ctypes.c_int),
        "vmas_sur_debug_features": ([vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "vmas_sur_check": ([vp, vp, vp], ctypes.c_int),
        "vmas_debug_gemm_engine": ([i32, vp], ctypes.c_int),
        "vmas_debug_diff_split": ([i32], ctypes.c_int),
        "vmas_debug_gemm_timeout": ([i32], ctypes.c_int),
        "vmas_debug_lidar_cull": ([i32], ctypes.c_int),
        "vmas_debug_gemm_bf16": ([i32, i32, i32, i32, i32, vp, i32, vp, i32, vp, i32, vp, vp,
                                  i32, vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    if L.vmas_abi_version() != ABI_VERSION:
        raise ImportError("libvmas.so ABI %d, binding expects %d" % (L.vmas_abi_version(), ABI_VERSION))
    _lib = L
    return L


def check(rc):
    if rc != VMAS_OK:
        raise VmasError(rc, load().vmas_last_error().decode())
    return rc
