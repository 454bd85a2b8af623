"""The allocation-free world step (vmas_step_noalloc) against the regular step.

Some callers cannot let a library allocate device memory: code whose device
memory all belongs to its own allocator (a framework's pool, an arena
reserved up front), loops that must not stall on the device synchronisation
that cudaMalloc and cudaFree can cause, and code running under stream
capture, where those calls are not allowed.  vmas_step_noalloc serves them:
the caller passes every buffer (entity arrays, state, actions) and the
library uses only a fixed scratch array of its own.

This test calls it through the C ABI twice in a row on the same buffers and
checks each result against the regular step (vmas_step on a world created
from the same scene) within the parity tolerance the other GPU tests use.
It lives in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest
import torch

from conftest import normwise_err
from paper_2207_03530_b300 import _lib, scenes

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _args(sc, skin, state, actions, status, keep):
    """vmas_step_noalloc_args over device copies of the scene's arrays."""
    dev = {}
    for key, dt in (("shape", torch.uint8), ("flags", torch.uint8), ("size_a", torch.float32),
                    ("size_b", torch.float32), ("mass", torch.float32), ("inertia", torch.float32)):
        dev[key] = torch.from_numpy(np.ascontiguousarray(getattr(sc, key))).to("cuda", dt)
    keep.append(dev)
    return _lib.StepNoallocArgs(
        sc.n_envs, sc.n_entities, sc.n_actuated, sc.substeps, sc.dt, sc.drag, sc.gx, sc.gy,
        sc.c, sc.k, sc.max_speed, skin,
        *[dev[k].data_ptr() for k in ("shape", "flags", "size_a", "size_b", "mass", "inertia")],
        state.data_ptr(), actions.data_ptr(), status.data_ptr())


def _padded_ragged(n_envs, seed, n_total, max_agents):
    """A mixed scene of spheres, boxes and walls (the ragged generator's), every
    env padded with inert entities to exactly n_total entities."""
    sc, _ = scenes.ragged_scene(n_envs, seed, max_agents=max_agents)
    pad = n_total - sc.n_entities
    assert pad >= 0
    kw = {}
    for key, fill in (("shape", 0), ("flags", 0), ("size_a", 0.05), ("size_b", 0.0),
                      ("mass", 1.0), ("inertia", 0.0)):
        a = getattr(sc, key)
        kw[key] = np.ascontiguousarray(np.concatenate(
            [a, np.full((sc.n_envs, pad), fill, a.dtype)], axis=1))
    kw["init_state"] = np.ascontiguousarray(np.concatenate(
        [sc.init_state, np.zeros((sc.n_envs, pad, 6), np.float32)], axis=1))
    import dataclasses

    return dataclasses.replace(sc, n_entities=n_total, **kw)


@pytest.mark.parametrize("make", [lambda: scenes.paper_scene(203, 5, dense=True),
                                  lambda: scenes.small_scene(37, 2, dense=True),
                                  lambda: _padded_ragged(45, 11, 48, 36),
                                  lambda: _padded_ragged(21, 12, 128, 116)],
                         ids=["paper-203envs", "small-37envs", "mixed-48ent-45envs",
                              "mixed-128ent-21envs"])
def test_noalloc_step_matches_regular_step_twice(vmas_lib, make):
    from paper_2207_03530_b300 import World

    sc = make()
    act = torch.from_numpy(scenes.make_actions(sc, 2, 4)).cuda()
    stream = torch.cuda.current_stream().cuda_stream

    w = World(sc)
    skin = w.skin
    ref = []
    for t in range(2):
        w.step(act[t])
        ref.append(w.state().cpu().numpy())
    w.check()
    w.close()

    keep = []
    state = torch.from_numpy(np.ascontiguousarray(sc.init_state)).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for t in range(2):
        args = _args(sc, skin, state, act[t], status, keep)
        _lib.check(vmas_lib.vmas_step_noalloc(ctypes.byref(args), stream))
        got = state.cpu().numpy()
        err = normwise_err(got, ref[t])
        assert err.max() <= TOL, (t, err)
    assert int(status.item()) == 0


def test_noalloc_step_rejects_too_many_entities(vmas_lib):
    """Sizes beyond the scratch array's capacity fail before any GPU work."""
    a = _lib.StepNoallocArgs()
    a.n_envs, a.n_entities, a.n_actuated, a.substeps = 4, 129, 0, 1
    a.dt, a.contact_margin, a.contact_force = 0.1, 1e-3, 100.0
    rc = vmas_lib.vmas_step_noalloc(ctypes.byref(a), None)
    assert rc == _lib.VMAS_EINVAL
    assert "128" in vmas_lib.vmas_last_error().decode()
