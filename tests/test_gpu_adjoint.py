"""Differentiable rollout on the GPU (hand-written adjoint) against the FP64
oracle's loss and reverse-mode gradient (itself pinned to central
differences), through the C ABI and torch.autograd."""
import numpy as np
import pytest
import torch

from paper_2207_03530_b300 import scenes

pytestmark = pytest.mark.gpu


def _setup(n_envs, seed, dense=True, T=50):
    from paper_2207_03530_b300 import World

    sc = scenes.diff_scene(n_envs, seed, dense=dense)
    act = scenes.make_actions(sc, T, seed + 1)
    goals = scenes.make_goals(sc, seed + 2)
    return sc, World(sc), act, goals


# Gates.  The gradient is a chain of ~150 substep Jacobians evaluated in
# FP32: rounding of 6e-8 per operation, accumulated as a random walk over
# the substeps, gives about 7e-7 of the largest gradient entry; contact
# Jacobians (stiffness c / k times h^2 / m) amplify it where contacts
# cluster, measured up to 4.6e-6 in the dense 64-env scene.  GRAD_TOL
# leaves a factor of 2 over that.  The loss is a sum of squares of FP32
# positions: relative error a few times 1e-7.
GRAD_TOL = 1e-5
LOSS_TOL = 1e-6


def _relerr(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-12)


@pytest.fixture(params=[1, 2], ids=["split1", "split2"])
def split(request, vmas_lib):
    """Lanes per env of the differentiable rollout: one group (the default),
    or two half-groups that each sum half of every entity's pairs."""
    from paper_2207_03530_b300 import _lib

    _lib.check(vmas_lib.vmas_debug_diff_split(request.param))
    yield request.param
    _lib.check(vmas_lib.vmas_debug_diff_split(0))


@pytest.mark.parametrize("dense", [False, True])
def test_loss_and_gradient_match_oracle(vmas_lib, orc, dense, split):
    """64 envs x 50 steps x 3 substeps: loss and gradient against the
    oracle's (normwise, per tensor); FP32 through 150 substeps of stiff
    contacts."""
    from paper_2207_03530_b300.diff import rollout_loss

    sc, w, act, goals = _setup(64, 3, dense)
    a = torch.from_numpy(act).cuda().requires_grad_(True)
    g = torch.from_numpy(goals).cuda()
    loss = rollout_loss(w, a, g, ckpt_every=10)
    loss.sum().backward()
    ref_loss, ref_grad = orc.rollout_grad(sc, sc.init_state, act, goals)
    assert _relerr(loss.detach().cpu().numpy(), ref_loss) <= LOSS_TOL
    err = _relerr(a.grad.cpu().numpy(), ref_grad)
    print("\n[adjoint] 64 envs dense=%s split=%d: loss err %.2e, gradient err %.2e"
          % (dense, split, _relerr(loss.detach().cpu().numpy(), ref_loss), err))
    assert err <= GRAD_TOL, err
    # the world's own state is untouched by the differentiable rollout
    assert np.array_equal(w.state().cpu().numpy(), sc.init_state)
    w.close()


def test_full_config_gradient_on_sampled_envs(vmas_lib, orc):
    """4,096 envs x (8 agents + 2 landmarks), 50 steps, checkpoint every 10:
    4 sampled envs checked against the oracle's gradient."""
    from paper_2207_03530_b300.diff import rollout_loss

    sc, w, act, goals = _setup(4096, 0, dense=False)
    a = torch.from_numpy(act).cuda().requires_grad_(True)
    loss = rollout_loss(w, a, torch.from_numpy(goals).cuda())
    loss.sum().backward()
    pick = np.array([0, 1234, 2047, 4095])
    sub = sc.subset(pick)
    ref_loss, ref_grad = orc.rollout_grad(sub, sub.init_state, act[:, pick], goals[pick])
    assert _relerr(loss.detach().cpu().numpy()[pick], ref_loss) <= LOSS_TOL
    print("\n[adjoint] 4,096 envs sampled: gradient err %.2e"
          % _relerr(a.grad.cpu().numpy()[:, pick], ref_grad))
    assert _relerr(a.grad.cpu().numpy()[:, pick], ref_grad) <= GRAD_TOL
    w.close()


def test_checkpoint_interval_does_not_change_gradient(vmas_lib):
    """Segments are replayed bit for bit, so the gradient is the same for any
    checkpoint interval."""
    from paper_2207_03530_b300.diff import rollout_loss

    sc, w, act, goals = _setup(48, 9, T=23)
    g = torch.from_numpy(goals).cuda()
    grads = []
    for k in (1, 4, 10, 23, 40):
        a = torch.from_numpy(act).cuda().requires_grad_(True)
        rollout_loss(w, a, g, ckpt_every=k).sum().backward()
        grads.append(a.grad.cpu().numpy())
    for gr in grads[1:]:
        assert np.array_equal(gr, grads[0])
    w.close()


@pytest.mark.parametrize("dense,push", [(False, 1.0), (True, 1.0), (True, 6.0)])
def test_candidate_skin_does_not_change_gradient(vmas_lib, dense, push):
    """The pair sums visit each entity's candidate partners (pairs within
    r_i + r_j + skin, rebuilt when a body may have moved half the skin) in
    ascending order.  A pair left out cannot touch, so every skin gives
    bitwise the loss and gradient of all pairs (skin 1e4: every pair, never
    rebuilt); skin 0 and 1e-4 rebuild at almost every substep, and the
    pushed scene (actions x 6) moves bodies through many rebuilds."""
    from paper_2207_03530_b300.diff import rollout_loss

    sc, w, act, goals = _setup(96, 21, dense, T=30)
    g = torch.from_numpy(goals).cuda()
    out = []
    for skin in (1e4, None, 0.0, 1e-4, 0.05):
        if skin is not None:
            w.skin = skin
        a = torch.from_numpy(act * np.float32(push)).cuda().requires_grad_(True)
        loss = rollout_loss(w, a, g, ckpt_every=7)
        loss.sum().backward()
        out.append((loss.detach().cpu().numpy(), a.grad.cpu().numpy()))
    for loss, grad in out[1:]:
        assert np.array_equal(loss, out[0][0])
        assert np.array_equal(grad, out[0][1])
    assert np.abs(out[0][1]).max() > 0
    w.close()


def test_upstream_weights_scale_env_gradients(vmas_lib):
    """d(sum_e w_e loss_e)/d a = w_e d loss_e / d a, env by env."""
    from paper_2207_03530_b300.diff import rollout_loss

    sc, w, act, goals = _setup(16, 4, T=12)
    g = torch.from_numpy(goals).cuda()
    a1 = torch.from_numpy(act).cuda().requires_grad_(True)
    rollout_loss(w, a1, g).sum().backward()
    wts = torch.linspace(-2, 3, 16, device="cuda")
    a2 = torch.from_numpy(act).cuda().requires_grad_(True)
    (rollout_loss(w, a2, g) * wts).sum().backward()
    expect = a1.grad * wts[None, :, None, None]
    torch.testing.assert_close(a2.grad, expect, rtol=1e-6, atol=1e-7)
    w.close()


def test_rejects_non_sphere_worlds(vmas_lib):
    from paper_2207_03530_b300 import World, _lib
    from paper_2207_03530_b300.diff import rollout_loss

    sc = scenes.paper_scene(4, 0)
    w = World(sc)
    a = torch.zeros((2, 4, sc.n_actuated, 3), device="cuda", requires_grad=True)
    with pytest.raises(_lib.VmasError):
        rollout_loss(w, a, torch.zeros((4, sc.n_actuated, 2), device="cuda"))
    w.close()


def _sphere_subset(sc, ents, A):
    import dataclasses

    kw = dataclasses.asdict(sc)
    for key in ("shape", "flags", "size_a", "size_b", "mass", "inertia", "init_state"):
        kw[key] = np.ascontiguousarray(getattr(sc, key)[:, ents])
    kw.update(n_entities=len(ents), n_actuated=A)
    return scenes.Scene(**kw)


@pytest.mark.parametrize("which,E", [("n3", 5), ("n6", 17), ("n16", 7), ("n16", 1)])
def test_lane_groups_of_every_width(vmas_lib, orc, which, E, split):
    """Envs of 3, 6 and 16 spheres take 4, 8 and 16 lanes (8, 4 and 2 envs
    per warp); env counts that leave groups of a warp empty."""
    from paper_2207_03530_b300 import World
    from paper_2207_03530_b300.diff import rollout_loss

    if which == "n6":
        sc = scenes.small_scene(E, 4, dense=True)
    else:
        base = scenes.paper_scene(E, 5, dense=True)
        n = 3 if which == "n3" else 16
        sc = _sphere_subset(base, list(range(n)), n)
    T = 20
    act = scenes.make_actions(sc, T, 6)
    goals = scenes.make_goals(sc, 7)
    w = World(sc)
    a = torch.from_numpy(act).cuda().requires_grad_(True)
    loss = rollout_loss(w, a, torch.from_numpy(goals).cuda(), ckpt_every=7)
    loss.sum().backward()
    ref_loss, ref_grad = orc.rollout_grad(sc, sc.init_state, act, goals)
    assert _relerr(loss.detach().cpu().numpy(), ref_loss) <= LOSS_TOL
    print("\n[adjoint] %s E=%d split=%d: gradient err %.2e"
          % (which, E, split, _relerr(a.grad.cpu().numpy(), ref_grad)))
    assert _relerr(a.grad.cpu().numpy(), ref_grad) <= GRAD_TOL
    w.close()
