"""Failure detection without a GPU fault: a bounded wait in the step kernel
runs out, the kernel reports it through the device error word, and the
context stays usable.

The step kernel's staging copies complete on an mbarrier whose wait is
bounded (about a second).  vmas_debug_stage_timeout makes the barrier expect
16 bytes that no copy delivers, so the wait runs out: the CTA sets
VMAS_DEVERR_TIMEOUT and leaves its envs unchanged.  With the hook off again
the same world steps normally."""
import ctypes

import pytest
import torch

from paper_2207_03530_b300 import _lib, scenes

pytestmark = pytest.mark.gpu


def test_staging_wait_runs_out_and_context_survives(vmas_lib):
    from paper_2207_03530_b300 import World

    sc = scenes.paper_scene(16, 3)  # exactly one full CTA: staged
    act = torch.from_numpy(scenes.make_actions(sc, 2, 1)).cuda()
    w, ref = World(sc), World(sc)
    before = w.state().clone()
    _lib.check(vmas_lib.vmas_debug_stage_timeout(w._h, 1))
    w.step(act[0])
    bits = ctypes.c_int32(0)
    rc = vmas_lib.vmas_check(w._h, None, ctypes.byref(bits))
    assert rc == _lib.VMAS_EDEVICE and bits.value & 8, (rc, bits.value)
    assert torch.equal(w.state(), before)  # the CTA left its envs unchanged
    _lib.check(vmas_lib.vmas_debug_stage_timeout(w._h, 0))
    w.step(act[1])
    ref.step(act[1])
    w.check()
    assert torch.equal(w.state(), ref.state())
    w.close()
    ref.close()
