"""FP64 CPU reference of the learned surrogate -- TEST INFRASTRUCTURE ONLY.

Only the test-suite and the benchmark's checks use it; the CUDA product path
never does and shares no code with it.

The surrogate predicts one world step (all substeps) of the agents of a
walled sphere world (16 agent spheres plus the 4 walls at x = +-1,
y = +-1).  It is a per-agent message-passing network:

  node features n_i (16): 10 vx, 10 vy, fx / m, fy / m, 10 r, 1 / m, and the
      gaps to the 4 walls (+x, -x, +y, -y), min(gap, 0.3) / 0.3; zeros after.
  edges: the (up to) K = 6 nearest other agents j with centre distance
      < 0.3, nearest first (ties: lower index); features e_ij (16): dx / 0.3,
      dy / 0.3 (d = x_j - x_i), 10 dvx, 10 dvy, 10 r_j, (|d| - r_i - r_j) / 0.3,
      1; zeros after.
  edge MLP: h = bf(gelu(We1 bf(e) + be1)) (16 -> 64),
            m = gelu(We2 h + be2) (64 -> 64); M_i = bf(sum over edges of m).
  node MLP: z = [bf(n_i), M_i] (80), h1 = bf(gelu(W1 z + b1)) (-> 128),
            h2 = bf(gelu(W2 h1 + b2)) (-> 128), out = W3 h2 + b3 (-> 8, the
            first 4 used).
  prediction: x' = x + 0.01 out0..1, v' = v + 0.1 out2..3.

bf() rounds to bfloat16 (nearest even); weights are held in bfloat16, biases
in FP32; gelu(z) = z (1 + erf(z / sqrt 2)) / 2 = z Phi(z).  The rounding
points are part of the network's definition (bfloat16 weights and
activations feeding every matrix product, FP32-or-better accumulation); any
implementation of the network rounds at them, and this reference evaluates
everything else in FP64.

Pins (tests/test_oracle_surrogate.py): the forward pass against a network
worked by hand from the normal table and the bfloat16 grid; gelu against
table values and a library normal CDF; the backward against central
differences of the unrounded loss; features against hand-computed values.

Training loss: mean over agents and the 4 outputs of (out - target)^2, the
target being the true step's deltas divided by (0.01, 0.01, 0.1, 0.1).

The box world (the paper-scale layout: 16 agents, 4 movable rotatable boxes,
4 walls) runs the same network on 20 nodes per env (``features_box``):

  node features of a box: as an agent's with R = its half diagonal in place
      of r (10 R in slot 4, the wall gaps of its bounding circle), and
      10: 1, 11: cos theta, 12: sin theta, 13: 0.1 omega, 14: 0.01 tau / I;
  edges: the 6 nearest other nodes (agents or boxes) within 0.3, with the
      surface gap taken between bounding circles, |d| - R_i - R_j, and for a
      box neighbour 7: 1, 8: cos theta_j, 9: sin theta_j, 10: 0.1 omega_j;
  outputs: a box uses 6 (theta' = theta + 0.1 out4, omega' = omega + out5);
  loss: the mean of (out - target)^2 over the outputs each node uses.
An agent, and an agent's edge to an agent, read the same values in both
worlds.
"""
from __future__ import annotations

import math

import numpy as np

K = 6
RADIUS = 0.3
X_SCALE, V_SCALE = 0.01, 0.1
TH_SCALE, OM_SCALE = 0.1, 1.0
AGENTS, BOXES = 16, 4
SHAPES = {"We1": (64, 16), "be1": (64,), "We2": (64, 64), "be2": (64,),
          "W1": (128, 80), "b1": (128,), "W2": (128, 128), "b2": (128,),
          "W3": (8, 128), "b3": (8,)}
ORDER = ("We1", "be1", "We2", "be2", "W1", "b1", "W2", "b2", "W3", "b3")


def bf(x):
    """Round to bfloat16 (nearest even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    z = np.asarray(z, np.float64)
    erf = np.vectorize(math.erf)(z / math.sqrt(2.0))
    return 0.5 * z * (1.0 + erf)


def gelu_grad(z):
    z = np.asarray(z, np.float64)
    erf = np.vectorize(math.erf)(z / math.sqrt(2.0))
    return 0.5 * (1.0 + erf) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def features(state, actions, radius_a, mass):
    """state [E, 20, 6] (16 agents then walls), actions [E, 16, 3], radius_a
    and mass [E, 16].  Returns node [E*16, 16], edge [E*16, K, 16], mask
    [E*16, K] (float64, unrounded)."""
    state = np.asarray(state, np.float64)
    E = state.shape[0]
    node = np.zeros((E * 16, 16))
    edge = np.zeros((E * 16, K, 16))
    mask = np.zeros((E * 16, K))
    for e in range(E):
        for i in range(16):
            row = e * 16 + i
            x, y, vx, vy = state[e, i, :4]
            r, m = float(radius_a[e, i]), float(mass[e, i])
            gaps = [1.0 - x - r, 1.0 + x - r, 1.0 - y - r, 1.0 + y - r]
            node[row, :10] = [10 * vx, 10 * vy, actions[e, i, 0] / m, actions[e, i, 1] / m,
                              10 * r, 1.0 / m] + [min(g, RADIUS) / RADIUS for g in gaps]
            cand = []
            for j in range(16):
                if j == i:
                    continue
                dx, dy = state[e, j, 0] - x, state[e, j, 1] - y
                dist = math.sqrt(dx * dx + dy * dy)
                if dist < RADIUS:
                    cand.append((dist, j, dx, dy))
            cand.sort(key=lambda c: (c[0], c[1]))
            for k, (dist, j, dx, dy) in enumerate(cand[:K]):
                rj = float(radius_a[e, j])
                edge[row, k, :7] = [dx / RADIUS, dy / RADIUS, 10 * (state[e, j, 2] - vx),
                                    10 * (state[e, j, 3] - vy), 10 * rj,
                                    (dist - r - rj) / RADIUS, 1.0]
                mask[row, k] = 1.0
    return node, edge, mask


def _bounding(shape, a, b):
    """Bounding radius: a sphere's radius, a box's half diagonal."""
    return math.hypot(0.5 * a, 0.5 * b) if shape == 1 else a


def features_box(state, actions, shape, size_a, size_b, mass, inertia):
    """Box world: state [E, 24, 6] (16 agents, 4 boxes, 4 walls), actions
    [E, >= 20, 3], per-entity arrays [E, 24].  Returns node [E*20, 16], edge
    [E*20, K, 16], mask [E*20, K] (float64, unrounded)."""
    state = np.asarray(state, np.float64)
    E = state.shape[0]
    NN = AGENTS + BOXES
    node = np.zeros((E * NN, 16))
    edge = np.zeros((E * NN, K, 16))
    mask = np.zeros((E * NN, K))
    for e in range(E):
        R = [_bounding(int(shape[e, i]), float(size_a[e, i]), float(size_b[e, i]))
             for i in range(NN)]
        box = [int(shape[e, i]) == 1 for i in range(NN)]
        for i in range(NN):
            row = e * NN + i
            x, y, vx, vy, th, om = state[e, i]
            m = float(mass[e, i])
            gaps = [1.0 - x - R[i], 1.0 + x - R[i], 1.0 - y - R[i], 1.0 + y - R[i]]
            node[row, :10] = [10 * vx, 10 * vy, actions[e, i, 0] / m, actions[e, i, 1] / m,
                              10 * R[i], 1.0 / m] + [min(g, RADIUS) / RADIUS for g in gaps]
            if box[i]:
                I = float(inertia[e, i])
                if I == 0.0:
                    I = m * (float(size_a[e, i]) ** 2 + float(size_b[e, i]) ** 2) / 12.0
                node[row, 10:15] = [1.0, math.cos(th), math.sin(th), 0.1 * om,
                                    0.01 * actions[e, i, 2] / I]
            cand = []
            for j in range(NN):
                if j == i:
                    continue
                dx, dy = state[e, j, 0] - x, state[e, j, 1] - y
                dist = math.sqrt(dx * dx + dy * dy)
                if dist < RADIUS:
                    cand.append((dist, j, dx, dy))
            cand.sort(key=lambda c: (c[0], c[1]))
            for k, (dist, j, dx, dy) in enumerate(cand[:K]):
                edge[row, k, :7] = [dx / RADIUS, dy / RADIUS, 10 * (state[e, j, 2] - vx),
                                    10 * (state[e, j, 3] - vy), 10 * R[j],
                                    (dist - R[i] - R[j]) / RADIUS, 1.0]
                if box[j]:
                    edge[row, k, 7:11] = [1.0, math.cos(state[e, j, 4]), math.sin(state[e, j, 4]),
                                          0.1 * state[e, j, 5]]
                mask[row, k] = 1.0
    return node, edge, mask


def used_outputs(n_envs, nodes):
    """Outputs each row uses: 4 for an agent (node < 16), 6 for a box."""
    return np.tile(np.where(np.arange(nodes) < AGENTS, 4, 6), n_envs)


def targets_box(state, next_state):
    """Normalised one-step deltas [E*20, 6] of the nodes of the box world
    (x, y over 0.01, vx, vy over 0.1, theta over 0.1, omega over 1; 0 in the
    angle columns of agents)."""
    s, n = np.asarray(state, np.float64), np.asarray(next_state, np.float64)
    NN = AGENTS + BOXES
    d = (n[:, :NN, :6] - s[:, :NN, :6]) / np.array(
        [X_SCALE, X_SCALE, V_SCALE, V_SCALE, TH_SCALE, OM_SCALE])
    d[:, :AGENTS, 4:] = 0.0
    return d.reshape(-1, 6)


def init_weights(seed=0):
    """Deterministic initialisation (uniform fan-in scaling), weights rounded
    to bfloat16; W3 rows 4..7 and all biases start at zero."""
    rng = np.random.default_rng(seed)
    w = {}
    for name in ORDER:
        shp = SHAPES[name]
        if name.startswith("b"):
            w[name] = np.zeros(shp)
        else:
            bound = 1.0 / math.sqrt(shp[1])
            w[name] = bf(rng.uniform(-bound, bound, size=shp))
    w["W3"][4:] = 0.0
    return w


def forward(w, node, edge, mask, round_bf=True, keep=False):
    """Network output [R, 8] (float64).  round_bf=False gives the exact
    FP64 network (for finite differences); keep=True also returns the
    intermediate values needed by backward."""
    r = bf if round_bf else (lambda v: np.asarray(v, np.float64))
    R = node.shape[0]
    e_in = r(edge.reshape(R * K, 16))
    ze1 = e_in @ w["We1"].T + w["be1"]
    he = r(gelu(ze1))
    ze2 = he @ w["We2"].T + w["be2"]
    m = gelu(ze2) * mask.reshape(R * K, 1)
    M = r(m.reshape(R, K, 64).sum(axis=1))
    z = np.concatenate([r(node), M], axis=1)
    z1 = z @ w["W1"].T + w["b1"]
    h1 = r(gelu(z1))
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = r(gelu(z2))
    out = h2 @ w["W3"].T + w["b3"]
    if keep:
        return out, dict(e_in=e_in, ze1=ze1, he=he, ze2=ze2, z=z, z1=z1, h1=h1, z2=z2, h2=h2)
    return out


def loss_and_grad(w, node, edge, mask, target, round_bf=True, used=None):
    """Loss: the mean of (out - target)^2 over the outputs each row uses
    (``used`` [R], default 4 for every row; target [R, >= max used]), and
    its gradient (FP64 backward through the stored forward values)."""
    R = node.shape[0]
    out, c = forward(w, node, edge, mask, round_bf, keep=True)
    used = np.full(R, 4) if used is None else np.asarray(used)
    cols = np.arange(8)[None, :] < used[:, None]
    tgt = np.zeros((R, 8))
    tgt[:, :target.shape[1]] = target
    diff = np.where(cols, out - tgt, 0.0)
    count = float(used.sum())
    loss = float((diff ** 2).sum() / count)
    d_out = 2.0 * diff / count
    g = {}
    g["W3"] = d_out.T @ c["h2"]
    g["b3"] = d_out.sum(0)
    d_h2 = d_out @ w["W3"]
    d_z2 = d_h2 * gelu_grad(c["z2"])
    g["W2"] = d_z2.T @ c["h1"]
    g["b2"] = d_z2.sum(0)
    d_h1 = d_z2 @ w["W2"]
    d_z1 = d_h1 * gelu_grad(c["z1"])
    g["W1"] = d_z1.T @ c["z"]
    g["b1"] = d_z1.sum(0)
    d_zin = d_z1 @ w["W1"]
    d_M = d_zin[:, 16:]
    d_m = np.repeat(d_M[:, None, :], K, axis=1).reshape(R * K, 64) * mask.reshape(R * K, 1)
    d_ze2 = d_m * gelu_grad(c["ze2"])
    g["We2"] = d_ze2.T @ c["he"]
    g["be2"] = d_ze2.sum(0)
    d_he = d_ze2 @ w["We2"]
    d_ze1 = d_he * gelu_grad(c["ze1"])
    g["We1"] = d_ze1.T @ c["e_in"]
    g["be1"] = d_ze1.sum(0)
    return loss, g


def targets(state, next_state):
    """Normalised one-step deltas [E*16, 4] of the agents."""
    s, n = np.asarray(state, np.float64), np.asarray(next_state, np.float64)
    d = n[:, :16, :4] - s[:, :16, :4]
    return (d / np.array([X_SCALE, X_SCALE, V_SCALE, V_SCALE])).reshape(-1, 4)
