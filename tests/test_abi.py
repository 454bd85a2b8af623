"""The C-ABI library loads and exports every symbol include/vmas.h declares;
host-side validation rejects malformed world descriptions before any CUDA
call (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2207_03530_b300 import _lib, build, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "vmas.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vmas_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_lib.SYMBOLS)


def test_abi_version(L):
    assert L.vmas_abi_version() == _lib.ABI_VERSION


def test_nvcc_targets_sm103a():
    flags = " ".join(build.NVCC_FLAGS)
    assert "arch=compute_103a,code=sm_103a" in flags


def _desc(sc, **over):
    E, N = sc.n_envs, sc.n_entities
    keep = [np.ascontiguousarray(a) for a in (sc.shape, sc.flags, sc.size_a, sc.size_b, sc.mass,
                                              sc.inertia, sc.init_state)]
    fields = dict(n_envs=E, n_entities=N, n_actuated=sc.n_actuated, substeps=sc.substeps,
                  dt=sc.dt, drag=sc.drag, gx=sc.gx, gy=sc.gy, contact_force=sc.c,
                  contact_margin=sc.k, max_speed=sc.max_speed)
    fields.update(over)
    d = _lib.WorldDesc(**fields)
    for name, a in zip(("shape", "flags", "size_a", "size_b", "mass", "inertia", "init_state"), keep):
        setattr(d, name, a.ctypes.data)
    return d, keep


def _create(L, d):
    h = ctypes.c_void_p()
    rc = L.vmas_world_create(ctypes.byref(d), ctypes.byref(h))
    return rc, h, L.vmas_last_error().decode()


@pytest.mark.parametrize("over,needle", [
    (dict(n_envs=-1), "n_envs"),
    (dict(n_entities=0), "n_entities"),
    (dict(n_entities=129), "n_entities"),
    (dict(substeps=0), "substeps"),
    (dict(dt=0.0), "dt"),
    (dict(contact_margin=0.0), "contact_margin"),
    (dict(contact_force=-1.0), "contact_force"),
    (dict(max_speed=-1.0), "max_speed"),
    (dict(n_actuated=3), "actuated"),
])
def test_create_rejects_bad_descriptions(L, over, needle):
    sc = scenes.small_scene(4, 0)
    d, keep = _desc(sc, **over)
    rc, h, msg = _create(L, d)
    assert rc == _lib.VMAS_EINVAL
    assert needle in msg
    assert not h.value


@pytest.mark.parametrize("field,value,needle", [
    ("shape", 7, "shape"), ("flags", 64, "flag"), ("size_a", 0.0, "size_a"),
    ("mass", 0.0, "mass"), ("size_b", -1.0, "size_b"),
])
def test_create_rejects_bad_entities(L, field, value, needle):
    sc = scenes.paper_scene(3, 0)
    arr = getattr(sc, field)
    arr[1, 17] = value  # a box
    d, keep = _desc(sc)
    rc, h, msg = _create(L, d)
    assert rc == _lib.VMAS_EINVAL
    assert needle in msg


def test_create_rejects_nonfinite_state(L):
    sc = scenes.small_scene(2, 0)
    sc.init_state[1, 2, 3] = np.nan
    d, keep = _desc(sc)
    rc, h, msg = _create(L, d)
    assert rc == _lib.VMAS_EINVAL and "finite" in msg


def test_null_arguments(L):
    h = ctypes.c_void_p()
    assert L.vmas_world_create(None, ctypes.byref(h)) == _lib.VMAS_EINVAL
    assert L.vmas_step(None, None, None) == _lib.VMAS_EINVAL
    assert L.vmas_state(None, None, 0, None) == _lib.VMAS_EINVAL
    assert L.vmas_world_destroy(None) == _lib.VMAS_OK
    assert "NULL" in L.vmas_last_error().decode()
    assert L.vmas_rollout_host(None, None, 1, None, None) == _lib.VMAS_EINVAL
    assert L.vmas_check(None, None, None) == _lib.VMAS_EINVAL
    assert L.vmas_ragged_check(None, None, None) == _lib.VMAS_EINVAL


def test_surrogate_null_and_bad_arguments(L):
    """The surrogate entry points reject bad arguments before any CUDA call."""
    E = _lib.VMAS_EINVAL
    h = ctypes.c_void_p()
    assert L.vmas_sur_param_count() == 33160
    assert L.vmas_sur_create(5, None) == E
    assert L.vmas_sur_create(-1, ctypes.byref(h)) == E
    assert L.vmas_sur_create(1 << 23, ctypes.byref(h)) == E
    assert L.vmas_sur_destroy(None) == E
    assert L.vmas_sur_set_params(None, None) == E
    assert L.vmas_sur_get_params(None, None) == E
    assert L.vmas_sur_set_mode(None, 0) == E
    assert L.vmas_sur_forward(None, None, None, None, None) == E
    assert L.vmas_sur_loss_grad(None, None, None, None, None, None, None) == E
    assert L.vmas_sur_adam(None, 1e-3, None, None) == E
    assert L.vmas_sur_train_grad(None, None, None, None, None, None) == E
    assert L.vmas_sur_train_step(None, None, None, 1e-3, None, None) == E
    assert L.vmas_sur_step(None, None, None, 0.01, None, None) == E
    assert L.vmas_sur_debug_features(None, None, None, None, None, None, None) == E
    assert "NULL" in L.vmas_last_error().decode()
    # GEMM diagnostic: sizes and combinations are checked first
    assert L.vmas_debug_gemm_bf16(0, 0, -1, 8, 8, None, 8, None, 8, None, 0, None, None, 1,
                                  None) == E
    assert L.vmas_debug_gemm_bf16(0, 0, 8, 8, 8, None, 8, None, 8, None, 1, None, None, 2,
                                  None) == E
    assert L.vmas_debug_gemm_bf16(0, 0, 8, 8, 8, None, 4, None, 8, None, 0, None, None, 1,
                                  None) == E


def test_binding_refuses_to_run_without_library(monkeypatch):
    """The product path has no CPU fallback: a missing library is an error."""
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/libvmas.so")
    with pytest.raises(ImportError):
        _lib.load()


def test_no_conditionally_skipped_warp_votes():
    """A full-warp vote or shuffle that some lanes skip (because it sits on
    the right of && / || or in a ?: branch) is undefined behaviour and can
    hang or corrupt a warp; the sources must not contain that pattern."""
    import glob

    pat = re.compile(r"(&&|\|\||\?|:)\s*\(*\s*__(ballot|any|all|shfl|reduce|match)\w*_sync")
    bad = []
    for f in glob.glob(os.path.join(ROOT, "paper_2207_03530_b300", "csrc", "*")):
        for n, line in enumerate(open(f), 1):
            if pat.search(line.split("//")[0]):
                bad.append("%s:%d: %s" % (os.path.basename(f), n, line.strip()))
    assert not bad, bad


@pytest.mark.parametrize("field", ["drag", "gx", "gy", "contact_force", "max_speed"])
@pytest.mark.parametrize("value", [float("nan"), float("inf")])
def test_noalloc_step_rejects_non_finite_parameters(L, field, value):
    """vmas_step_noalloc checks its world parameters on the host, as
    vmas_world_create does, before it enqueues anything (no GPU needed)."""
    a = _lib.StepNoallocArgs()
    a.n_envs, a.n_entities, a.n_actuated, a.substeps = 4, 6, 0, 1
    a.dt, a.contact_margin, a.contact_force = 0.1, 1e-3, 100.0
    setattr(a, field, value)
    rc = L.vmas_step_noalloc(ctypes.byref(a), None)
    assert rc == _lib.VMAS_EINVAL
    assert "finite" in L.vmas_last_error().decode() or field in L.vmas_last_error().decode()
