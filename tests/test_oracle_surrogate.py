"""Pins of the surrogate's FP64 reference: its backward against central
differences of its exact (unrounded) loss, features against hand-computed
values, and bfloat16 rounding against the bit-level definition."""
import math

import numpy as np
import pytest

from oracle import surrogate as S
from paper_2207_03530_b300 import scenes


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159265, 65504.0, 1e-30])
    r = S.bf(x)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: nearest even keeps 1
    assert r[0] == 1.0 and r[1] == 1.0
    assert r[2] == 1.0078125
    assert abs(r[3] - (-3.140625)) < 1e-12
    np.testing.assert_array_equal(S.bf(r), r)  # idempotent


def test_features_hand_worked():
    E = 1
    st = np.zeros((E, 20, 6))
    st[0, :16, 0] = np.linspace(-0.8, 0.8, 16)
    st[0, :16, 1] = -0.5
    st[0, 3, 0], st[0, 3, 1], st[0, 3, 2] = 0.0, 0.0, 0.25
    st[0, 7, 0], st[0, 7, 1] = 0.1, 0.2  # 0.2236 from agent 3
    act = np.zeros((E, 16, 3))
    act[0, 3, :2] = [0.5, -1.0]
    r = np.full((E, 16), 0.05)
    m = np.full((E, 16), 2.0)
    node, edge, mask = S.features(st, act, r, m)
    n3 = node[3]
    np.testing.assert_allclose(n3[:10], [2.5, 0, 0.25, -0.5, 0.5, 0.5, 1, 1, 1, 1])
    assert mask[3].sum() == 1.0
    d = math.hypot(0.1, 0.2)
    np.testing.assert_allclose(edge[3, 0, :7], [0.1 / 0.3, 0.2 / 0.3, -2.5, 0, 0.5,
                                                (d - 0.1) / 0.3, 1.0])


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    sc = scenes.paper_scene(3, 1)
    st = sc.init_state[:, [*range(16), 20, 21, 22, 23]].astype(np.float64)
    st[:, :16, 2:4] = rng.uniform(-0.3, 0.3, (3, 16, 2))
    act = rng.uniform(-1, 1, (3, 16, 3))
    node, edge, mask = S.features(st, act, sc.size_a[:, :16], sc.mass[:, :16])
    w = S.init_weights(3)
    for k in w:
        w[k] = w[k] + rng.normal(0, 0.05, w[k].shape)  # non-zero biases / rows
    target = rng.normal(0, 1, (node.shape[0], 4))
    loss, g = S.loss_and_grad(w, node, edge, mask, target, round_bf=False)
    h = 1e-6
    for name in S.ORDER:
        flat = w[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = float(((S.forward(w, node, edge, mask, round_bf=False)[:, :4] - target) ** 2).mean())
            flat[idx] = old - h
            lm = float(((S.forward(w, node, edge, mask, round_bf=False)[:, :4] - target) ** 2).mean())
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert g[name].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), name
