"""Pins of the oracle's rollout gradient (the adjoint of Eqs. 1-3 for
sphere worlds) to central finite differences of its own loss, to the
closed-form gradient of a free body, and of its forward to the main step."""
import numpy as np
import pytest

from conftest import make_scene
from paper_2207_03530_b300 import scenes

S_ = scenes.SPHERE
MOV, COL, ACT = scenes.MOVABLE, scenes.COLLIDABLE, scenes.ACTUATED


def test_rollout_forward_matches_step(orc):
    """The differentiable rollout's trajectory is the plain step's."""
    sc = scenes.diff_scene(6, 3, dense=True)
    act = scenes.make_actions(sc, 12, 1)
    goals = scenes.make_goals(sc, 2)
    loss, _ = orc.rollout_grad(sc, sc.init_state, act, goals, with_grad=False)
    st = orc.step(sc, sc.init_state, act)
    ref = ((st[:, :8, :2] - goals.astype(np.float64)) ** 2).sum(axis=(1, 2))
    np.testing.assert_allclose(loss, ref, rtol=1e-13)


def test_free_body_gradient_closed_form(orc):
    """One free sphere, no contacts: x_T is linear in each step's force, with
    d x_T / d f(t) = sum over substeps q of step t of (h/m) h (1 - a^(n-q)) / zeta,
    n = T S, a = 1 - zeta (q counted from 0 over the whole rollout)."""
    T, S, dt, zeta, m = 6, 3, 0.1, 0.25, 1.5
    sc = make_scene([dict(shape=S_, x=0.1, y=-0.2, vx=0.3, a=0.05, m=m, flags=MOV | COL | ACT)],
                    substeps=S, dt=dt, drag=zeta)
    act = np.random.default_rng(0).uniform(-1, 1, (T, 1, 1, 3))
    goals = np.array([[[0.4, 0.5]]])
    loss, grad = orc.rollout_grad(sc, sc.init_state, act, goals)
    st = orc.step(sc, sc.init_state, act)
    resid = st[0, 0, :2] - goals[0, 0]
    h, a, n = dt / S, 1 - zeta, T * S
    for t in range(T):
        dxdf = sum((h / float(np.float32(m))) * h * (1 - a ** (n - q)) / zeta
                   for q in range(t * S, (t + 1) * S))
        np.testing.assert_allclose(grad[t, 0, 0, :2], 2 * resid * dxdf, rtol=1e-12)
        assert grad[t, 0, 0, 2] == 0


@pytest.mark.parametrize("dense", [False, True])
def test_gradient_matches_central_differences(orc, dense):
    """Every action component of 4 envs over a 50-step rollout: analytic
    gradient vs central differences (h = 1e-6) of the same FP64 loss.  A
    perturbation can carry a pair across the contact jump at gap 0 (Reading
    R2), which spoils that difference; at most a few such components are
    allowed and the rest must agree to 1e-6 of the gradient scale."""
    sc = scenes.diff_scene(4, 11, dense=dense)
    T = 50
    act = scenes.make_actions(sc, T, 5).astype(np.float64)
    goals = scenes.make_goals(sc, 6)
    loss, grad = orc.rollout_grad(sc, sc.init_state, act, goals)
    h = 1e-6
    fd = np.zeros_like(grad)
    for t in range(T):
        for k in range(sc.n_actuated):
            for c in range(2):
                ap = act.copy()
                am = act.copy()
                ap[t, :, k, c] += h
                am[t, :, k, c] -= h
                lp, _ = orc.rollout_grad(sc, sc.init_state, ap, goals, with_grad=False)
                lm, _ = orc.rollout_grad(sc, sc.init_state, am, goals, with_grad=False)
                fd[t, :, k, c] = (lp - lm) / (2 * h)
    scale = np.abs(grad).max()
    bad = np.abs(fd - grad) > 1e-6 * scale
    assert bad.sum() <= 4, (bad.sum(), np.argwhere(bad)[:5])
    assert scale > 1e-3
