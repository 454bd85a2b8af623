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


# Standard normal distribution function at the points the hand-worked network
# below visits (values of a printed normal table, to 16 digits):
PHI = {0.5: 0.6914624612740131, 1.0: 0.8413447460685429, 2.0: 0.9772498680518208,
       -1.0: 0.15865525393145707, -2.0: 0.022750131948179195, -3.0: 0.0013498980316301035}


def test_gelu_at_table_points():
    """gelu(z) = z Phi(z) (the exact erf form of the surrogate's activation)
    at normal-table points; gelu'(z) = Phi(z) + z phi(z) at z = 0 and 1."""
    for z, phi in PHI.items():
        assert S.gelu(np.array([z]))[0] == pytest.approx(z * phi, rel=1e-14)
    assert S.gelu(np.array([0.0]))[0] == 0.0
    assert S.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5, rel=1e-15)
    # phi(1) = exp(-1/2) / sqrt(2 pi) = 0.24197072451914337 (table value)
    assert S.gelu_grad(np.array([1.0]))[0] == pytest.approx(PHI[1.0] + 0.24197072451914337,
                                                            rel=1e-14)


def test_gelu_against_library_normal_cdf():
    """On a dense grid the activation equals z * scipy.special.ndtr(z) (an
    independent normal-CDF routine), and its derivative matches central
    differences of that product."""
    from scipy.special import ndtr

    z = np.linspace(-8.0, 8.0, 4001)
    np.testing.assert_allclose(S.gelu(z), z * ndtr(z), rtol=1e-13, atol=1e-15)
    h = 1e-5
    fd = ((z + h) * ndtr(z + h) - (z - h) * ndtr(z - h)) / (2 * h)
    np.testing.assert_allclose(S.gelu_grad(z), fd, rtol=1e-8, atol=1e-9)


def _hand_network():
    """A network of the surrogate's shapes whose weights are zero except for a
    few entries on the bfloat16 grid, chosen so that every pre-activation on
    the path is a normal-table point; one agent, one present edge (slot 0), an
    absent slot 1 holding the same features, slots 2-5 empty."""
    w = {name: np.zeros(shape) for name, shape in S.SHAPES.items()}
    # edge MLP, layer 1: ze1[0] = 3 * 0.5 - 0.5 = 1, ze1[1] = -2 * 1 + 1 = -1
    w["We1"][0, 0], w["be1"][0] = 3.0, -0.5
    w["We1"][1, 6], w["be1"][1] = -2.0, 1.0
    # layer 2 (on he = bf(gelu(ze1)) = [bf(Phi(1)), bf(-Phi(-1))] =
    # [0.83984375, -0.158203125]):
    #   ze2[0] = 0.83984375 + 0.5 * -0.158203125 + 0.2392578125 = 1
    #   ze2[1] = -0.158203125 - 1.841796875 = -2
    w["We2"][0, 0], w["We2"][0, 1], w["be2"][0] = 1.0, 0.5, 0.2392578125
    w["We2"][1, 1], w["be2"][1] = 1.0, -1.841796875
    # node MLP, layer 1, on z = [bf(node) (16), M (64)] with node = [1.5, -0.25]
    # and M = bf(gelu(ze2)) over the one present edge = [bf(Phi(1)),
    # bf(-2 Phi(-2))] = [0.83984375, -0.04541015625]:
    #   z1[0] = 1.5 + 2 * 0.83984375 - 1.1796875 = 2
    #   z1[1] = 4 * -0.25 - 0.04541015625 + 0.04541015625 = -1
    w["W1"][0, 0], w["W1"][0, 16], w["b1"][0] = 1.0, 2.0, -1.1796875
    w["W1"][1, 1], w["W1"][1, 17], w["b1"][1] = 4.0, 1.0, 0.04541015625
    # layer 2 on h1 = [bf(2 Phi(2)), bf(-Phi(-1))] = [1.953125, -0.158203125]:
    #   z2[0] = 0.5 * 1.953125 - 0.158203125 - 0.318359375 = 0.5
    #   z2[1] = -3 (bias only)
    w["W2"][0, 0], w["W2"][0, 1], w["b2"][0] = 0.5, 1.0, -0.318359375
    w["b2"][1] = -3.0
    # output on h2 = [bf(0.5 Phi(0.5)), bf(-3 Phi(-3))] =
    # [0.345703125, -0.004058837890625]
    w["W3"][0, 0], w["W3"][0, 1], w["b3"][0] = 2.0, 256.0, 0.25
    w["W3"][1, 1], w["b3"][1] = 1.0, 0.125
    w["b3"][2] = -0.5
    w["W3"][3, 0] = -1.0
    node = np.zeros((1, 16))
    node[0, :2] = [1.5, -0.25]
    edge = np.zeros((1, S.K, 16))
    edge[0, 0, 0], edge[0, 0, 6] = 0.5, 1.0
    edge[0, 1] = edge[0, 0]
    mask = np.zeros((1, S.K))
    mask[0, 0] = 1.0
    return w, node, edge, mask


# out[0] = 2 * 0.345703125 + 256 * -0.004058837890625 + 0.25
# out[1] = -0.004058837890625 + 0.125;  out[2] = -0.5;  out[3] = -0.345703125
HAND_OUT = [-0.09765625, 0.120941162109375, -0.5, -0.345703125, 0, 0, 0, 0]


def test_forward_hand_worked():
    """The reference network's forward pass against values worked by hand
    from the normal table and the bfloat16 grid (every rounding point of
    the definition: edge input, edge hidden, summed message, node input,
    node hidden layers).  A swapped concat order, a dropped bias or mask, a
    transposed square weight, a skipped rounding or erf(z) in place of
    erf(z / sqrt 2) each moves at least one output."""
    w, node, edge, mask = _hand_network()
    out = S.forward(w, node, edge, mask)
    np.testing.assert_array_equal(out[0], HAND_OUT)


def test_forward_hand_worked_catches_planted_mistakes():
    """The hand-worked values distinguish the definition from nearby wrong
    ones (each mistake planted in a copy of the reference's formulas)."""
    w, node, edge, mask = _hand_network()
    bf = S.bf

    def net(concat_swap=False, drop_mask=False, drop_bias=None, transpose=None, no_round=False,
            gelu=S.gelu):
        r = (lambda v: np.asarray(v, np.float64)) if no_round else bf
        ww = {k: (v.T if k == transpose else v) for k, v in w.items()}
        if drop_bias:
            ww[drop_bias] = np.zeros_like(ww[drop_bias])
        e = r(edge.reshape(S.K, 16))
        he = r(gelu(e @ ww["We1"].T + ww["be1"]))
        m = gelu(he @ ww["We2"].T + ww["be2"]) * (1.0 if drop_mask else mask.reshape(S.K, 1))
        M = r(m.sum(axis=0, keepdims=True))
        z = np.concatenate([M, r(node)] if concat_swap else [r(node), M], axis=1)
        if concat_swap:
            z = z[:, :80]
        h1 = r(gelu(z @ ww["W1"].T + ww["b1"]))
        h2 = r(gelu(h1 @ ww["W2"].T + ww["b2"]))
        return (h2 @ ww["W3"].T + ww["b3"])[0]

    def gelu_wrong(z):
        import math

        return 0.5 * z * (1.0 + np.vectorize(math.erf)(z))

    np.testing.assert_array_equal(net(), HAND_OUT)  # the copy itself is faithful
    mistakes = [dict(concat_swap=True), dict(drop_mask=True), dict(no_round=True),
                dict(gelu=gelu_wrong), dict(transpose="We2"), dict(transpose="W2")]
    mistakes += [dict(drop_bias=b) for b in ("be1", "be2", "b1", "b2", "b3")]
    for mk in mistakes:
        assert not np.array_equal(net(**mk), HAND_OUT), mk


def test_box_world_features_hand_worked():
    """Box world: the node of a box (bounding radius = half diagonal, angle,
    angular velocity, torque over inertia) and an agent's edge to it, worked
    by hand.  Box 16: 0.1 x 0.2 at (0.1, 0), theta = pi / 6, omega = 2,
    mass 5, default inertia 5 (0.1^2 + 0.2^2) / 12 = 0.0208333, action
    (0.5, -1, 0.6); agent 3 at the origin (r = 0.05, mass 2), every other
    body more than 0.3 away."""
    E, N = 1, 24
    st = np.zeros((E, N, 6))
    shape = np.zeros((E, N), int)
    sa = np.full((E, N), 0.05)
    sb = np.zeros((E, N))
    mass = np.full((E, N), 2.0)
    inertia = np.zeros((E, N))
    xs = np.linspace(-0.8, 0.8, 5)
    far = [(x, y) for y in (-0.8, 0.8) for x in xs] + [(-0.8, -0.4), (0.8, -0.4), (-0.8, 0.4),
                                                       (0.8, 0.4), (-0.4, 0.45)]
    k = 0
    for i in range(16):
        if i != 3:
            st[0, i, :2] = far[k]
            k += 1
    shape[0, 16:20] = 1
    sa[0, 16:20], sb[0, 16:20], mass[0, 16:20] = 0.1, 0.2, 5.0
    st[0, 16, :2], st[0, 16, 4], st[0, 16, 5] = (0.1, 0.0), math.pi / 6, 2.0
    for q, (x, y) in enumerate([(0.45, 0.45), (0.45, -0.45), (-0.45, -0.05)]):
        st[0, 17 + q, :2] = (x, y)
    shape[0, 20:] = 2
    act = np.zeros((E, 20, 3))
    act[0, 16] = [0.5, -1.0, 0.6]
    node, edge, mask = S.features_box(st, act, shape, sa, sb, mass, inertia)
    R = math.hypot(0.05, 0.1)  # 0.1118034
    I = 5.0 * (0.01 + 0.04) / 12.0
    np.testing.assert_allclose(node[16], [0, 0, 0.1, -0.2, 10 * R, 0.2, 1, 1, 1, 1, 1,
                                          math.sqrt(3) / 2, 0.5, 0.2, 0.01 * 0.6 / I, 0],
                               rtol=0, atol=1e-12)
    assert mask[3].sum() == 1.0 and mask[16].sum() == 1.0
    np.testing.assert_allclose(edge[3, 0, :11], [0.1 / 0.3, 0, 0, 0, 10 * R,
                                                 (0.1 - 0.05 - R) / 0.3, 1, 1, math.sqrt(3) / 2,
                                                 0.5, 0.2], rtol=0, atol=1e-12)
    # the box's edge back to the agent carries no box fields
    np.testing.assert_allclose(edge[16, 0, :8], [-0.1 / 0.3, 0, 0, 0, 0.5,
                                                 (0.1 - R - 0.05) / 0.3, 1, 0], atol=1e-12)
    # an agent's node is the sphere world's (zeros past slot 9)
    assert np.all(node[3, 10:] == 0) and node[3, 4] == 0.5


def test_box_world_loss_counts_used_outputs():
    """The loss averages over the outputs each row uses: 4 per agent, 6 per
    box (88 per env); a box's angle columns count, an agent's do not."""
    rng = np.random.default_rng(4)
    w = S.init_weights(1)
    R = 20
    node = rng.normal(0, 0.5, (R, 16))
    edge = rng.normal(0, 0.5, (R, S.K, 16))
    mask = (rng.uniform(size=(R, S.K)) < 0.5).astype(float)
    out = S.forward(w, node, edge, mask)
    tgt = rng.normal(0, 1, (R, 6))
    used = S.used_outputs(1, 20)
    assert used.sum() == 88
    loss, _ = S.loss_and_grad(w, node, edge, mask, tgt, used=used)
    se = ((out[:16, :4] - tgt[:16, :4]) ** 2).sum() + ((out[16:, :6] - tgt[16:, :6]) ** 2).sum()
    assert loss == pytest.approx(se / 88, rel=1e-12)
