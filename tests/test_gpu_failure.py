"""Failure detection without a GPU fault: a bounded wait in the step kernel
runs out, the kernel reports it through the device error word, and the
context stays usable.

The step kernel's staging copies complete on an mbarrier whose wait is
bounded (about a second).  vmas_debug_stage_timeout makes the barrier expect
16 bytes that no copy delivers, so the wait runs out: the CTA sets
VMAS_DEVERR_TIMEOUT and leaves its envs unchanged.  With the hook off again
the same world steps normally.

The surrogate's tcgen05 GEMM waits (bounded) on mbarriers for its TMA
copies and its MMAs.  vmas_debug_gemm_timeout makes every A-tile barrier
expect 16 bytes that no copy delivers: the CTAs' waits run out, they set
VMAS_DEVERR_TIMEOUT, free their tensor memory and return, and the next GEMM
(which allocates tensor memory again) runs normally."""
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


def test_tcgen05_gemm_wait_runs_out_and_context_survives(vmas_lib):
    import numpy as np

    from paper_2207_03530_b300.surrogate import gemm_bf16, tcgen05_gemm_launches

    rng = np.random.default_rng(0)
    a = torch.tensor(rng.normal(0, 1, (300, 64)), dtype=torch.bfloat16, device="cuda")
    bt = torch.tensor(rng.normal(0, 1, (64, 64)), dtype=torch.bfloat16, device="cuda")
    n0 = tcgen05_gemm_launches()
    _lib.check(vmas_lib.vmas_debug_gemm_timeout(1))
    try:
        with pytest.raises(_lib.VmasError) as ei:
            gemm_bf16(a, bt, trans_b=True)
        assert ei.value.code == _lib.VMAS_EDEVICE
        assert "bits 8" in str(ei.value), str(ei.value)
    finally:
        _lib.check(vmas_lib.vmas_debug_gemm_timeout(0))
    assert tcgen05_gemm_launches() == n0 + 1  # the tensor-core kernel was the one that timed out
    out, _ = gemm_bf16(a, bt, trans_b=True)
    ref = a.double() @ bt.double().T
    assert torch.allclose(out.double(), ref, rtol=0, atol=1e-4 * float(ref.abs().max()))
    assert tcgen05_gemm_launches() == n0 + 2


def test_tcgen05_weight_gradient_wait_runs_out_and_context_survives(vmas_lib):
    """The split-K weight-gradient kernel under the same hook: every CTA's
    first copy barrier waits for 16 bytes that never come, its bounded wait
    runs out, the error word is set, and the next call is correct."""
    import numpy as np

    from paper_2207_03530_b300.surrogate import gemm_bf16, tcgen05_gemm_launches

    rng = np.random.default_rng(1)
    a = torch.tensor(rng.normal(0, 1, (4096, 64)), dtype=torch.bfloat16, device="cuda")
    b = torch.tensor(rng.normal(0, 1, (4096, 64)), dtype=torch.bfloat16, device="cuda")
    n0 = tcgen05_gemm_launches()
    _lib.check(vmas_lib.vmas_debug_gemm_timeout(1))
    try:
        with pytest.raises(_lib.VmasError) as ei:
            gemm_bf16(a, b, trans_a=True, splits=64)
        assert ei.value.code == _lib.VMAS_EDEVICE
        assert "bits 8" in str(ei.value), str(ei.value)
    finally:
        _lib.check(vmas_lib.vmas_debug_gemm_timeout(0))
    assert tcgen05_gemm_launches() == n0 + 1
    out, _ = gemm_bf16(a, b, trans_a=True, splits=64)
    ref = a.double().T @ b.double()
    assert torch.allclose(out.double(), ref, rtol=0, atol=1e-4 * float(ref.abs().max()))
    assert tcgen05_gemm_launches() == n0 + 2

