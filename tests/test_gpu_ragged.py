"""Packed ragged worlds on the GPU: against the FP64 oracle run on the same
scene padded with inert entities, against the padded regular world, and
bitwise invariance of graph-captured, tiled and autotuned rollouts."""
import numpy as np
import pytest
import torch

from conftest import normwise_err
from paper_2207_03530_b300 import scenes

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _ragged(sc, counts):
    from paper_2207_03530_b300.ragged import RaggedWorld

    pk = scenes.pack_ragged(sc, counts)
    return RaggedWorld(counts, pk["shape"], pk["flags"], pk["size_a"], pk["size_b"], pk["mass"],
                       pk["inertia"], pk["init_state"], substeps=sc.substeps, dt=sc.dt,
                       drag=sc.drag, gx=sc.gx, gy=sc.gy, c=sc.c, k=sc.k, max_speed=sc.max_speed)


def _packed_actions(rw, sc, act):
    """[T, E, A, 3] padded actions -> [T, n_action_rows, 3] packed."""
    aoff = rw.action_offsets
    rows = [act[:, e, : aoff[e + 1] - aoff[e]] for e in range(sc.n_envs)]
    return np.ascontiguousarray(np.concatenate(rows, axis=1))


def _unpack_state(state, counts, N):
    out = np.zeros((len(counts), N, 6), np.float32)
    sel = np.arange(N)[None, :] < np.asarray(counts)[:, None]
    out[sel] = state
    return out, sel


@pytest.mark.parametrize("seed", [0, 1])
def test_ragged_matches_oracle(vmas_lib, orc, seed):
    sc, counts = scenes.ragged_scene(300, seed)
    rw = _ragged(sc, counts)
    assert (rw.class_envs > 0).sum() >= 4  # several size classes in play
    act = scenes.make_actions(sc, 2, seed)
    pact = torch.from_numpy(_packed_actions(rw, sc, act)).cuda()
    for t in range(2):
        rw.step(pact[t])
    got, sel = _unpack_state(rw.state().cpu().numpy(), counts, sc.n_entities)
    ref = orc.step(sc, sc.init_state, act, threads=8)
    assert normwise_err(got[sel], ref[sel]).max() <= TOL
    rw.check()
    rw.close()


@pytest.mark.parametrize("lanes", [[4, 4, 8, 16, 32], [8, 8, 16, 32, 32], [8, 16, 32, 32, 32]])
def test_every_lane_choice_matches_oracle(vmas_lib, orc, lanes):
    """Every (lanes, entities per lane) kernel a size class can run -- the
    three tunings cover them all: 4 or 8 lanes for the 8-entity class, 4, 8
    or 16 for 16, 8, 16 or 32 for 32, 16 or 32 for 64, 32 for 128 -- against
    the FP64 oracle."""
    sc, counts = scenes.ragged_scene(300, 4)
    rw = _ragged(sc, counts)
    assert (rw.class_envs > 0).all()
    rw.set_tuning(lanes, 1)
    act = scenes.make_actions(sc, 2, 4)
    pact = torch.from_numpy(_packed_actions(rw, sc, act)).cuda()
    for t in range(2):
        rw.step(pact[t])
    got, sel = _unpack_state(rw.state().cpu().numpy(), counts, sc.n_entities)
    ref = orc.step(sc, sc.init_state, act, threads=8)
    assert normwise_err(got[sel], ref[sel]).max() <= TOL
    rw.check()
    rw.close()


def test_ragged_matches_padded_world(vmas_lib):
    from paper_2207_03530_b300 import World

    sc, counts = scenes.ragged_scene(200, 7)
    rw = _ragged(sc, counts)
    w = World(sc)
    act = scenes.make_actions(sc, 5, 3)
    pact = torch.from_numpy(_packed_actions(rw, sc, act)).cuda()
    dact = torch.from_numpy(act).cuda()
    for t in range(5):
        rw.step(pact[t])
        w.step(dact[t])
    got, sel = _unpack_state(rw.state().cpu().numpy(), counts, sc.n_entities)
    ref = w.state().cpu().numpy()
    assert normwise_err(got[sel], ref[sel]).max() <= TOL
    # padding entities of the regular world never move
    assert np.array_equal(ref[~sel], sc.init_state[~sel])
    rw.check()
    rw.close()
    w.close()


def test_graph_rollout_tiles_and_autotune(vmas_lib):
    """Graph-captured rollout == step by step, bitwise, for any steps per
    launch; autotuning restores the state, and the tuned rollout agrees with
    the default one to rounding growth."""
    sc, counts = scenes.ragged_scene(400, 5)
    act = scenes.make_actions(sc, 24, 1)
    base = _ragged(sc, counts)
    pact = torch.from_numpy(_packed_actions(base, sc, act)).cuda()
    for t in range(24):
        base.step(pact[t])
    ref = base.state().cpu().numpy()
    base.check()
    base.close()
    for tile in (1, 4, 7):
        rw = _ragged(sc, counts)
        rw.set_tuning(None, tile)
        rw.rollout(pact)
        assert np.array_equal(rw.state().cpu().numpy(), ref), tile
        rw.rollout(pact[:0])  # zero steps is a no-op
        rw.check()
        rw.close()
    rw = _ragged(sc, counts)
    before = rw.state().cpu().numpy()
    rw.autotune(pact[:6])
    assert np.array_equal(rw.state().cpu().numpy(), before)
    lanes, tile = rw.tuning()
    assert tile in (1, 2, 4, 8, 16, 32, 64) and all(l in (4, 8, 16, 32) for l in lanes)
    rw.rollout(pact)
    rw.rollout(pact)  # graph replay
    got = rw.state().cpu().numpy()
    rw.check()
    rw.close()
    rw2 = _ragged(sc, counts)
    rw2.rollout(pact)
    rw2.rollout(pact)
    # another lane layout sums contacts in another order: after 48 steps of
    # contact dynamics the two agree to rounding growth, not bitwise
    assert normwise_err(got, rw2.state().cpu().numpy()).max() <= 1e-4
    rw2.check()
    rw2.close()


@pytest.mark.parametrize("schedule", [0, 1, 2])
def test_extreme_env_sizes(vmas_lib, orc, schedule):
    """Envs of 1 entity and of 128 entities (the largest class) side by side,
    under either schedule."""
    from paper_2207_03530_b300.ragged import RaggedWorld

    big = scenes.mixed_scene(1, 3)
    rng = np.random.default_rng(0)
    n_big = 128
    shape = np.concatenate([[0], rng.integers(0, 3, n_big)]).astype(np.uint8)
    flags = np.concatenate([[15], np.full(n_big, 15)]).astype(np.uint8)
    size_a = np.concatenate([[0.05], rng.uniform(0.02, 0.06, n_big)]).astype(np.float32)
    size_b = np.concatenate([[0], rng.uniform(0.02, 0.06, n_big)]).astype(np.float32)
    mass = np.ones(n_big + 1, np.float32)
    inertia = np.zeros(n_big + 1, np.float32)
    st = np.zeros((n_big + 1, 6), np.float32)
    st[:, :2] = rng.uniform(-0.6, 0.6, (n_big + 1, 2))
    st[:, 4] = rng.uniform(-3, 3, n_big + 1)
    rw = RaggedWorld([1, n_big], shape, flags, size_a, size_b, mass, inertia, st,
                     substeps=2, dt=0.05, drag=0.1)
    assert rw.class_envs[0] == 1 and rw.class_envs[4] == 1
    rw.schedule = schedule
    pact = torch.zeros((rw.n_action_rows, 3), device="cuda")
    rw.step(pact)
    got = rw.state().cpu().numpy()
    # the oracle on the same two envs, padded to 128
    sc = scenes._empty("x", 2, n_big, n_big, 2, 0.05, 0.1)
    sc.shape[0, 0], sc.flags[0, 0], sc.size_a[0, 0] = 0, 15, 0.05
    sc.init_state[0, 0] = st[0]
    sc.shape[1], sc.flags[1], sc.size_a[1], sc.size_b[1] = shape[1:], flags[1:], size_a[1:], size_b[1:]
    sc.init_state[1] = st[1:]
    sc.size_a[0, 1:] = 0.05
    ref, margin = orc.step_margin(sc, sc.init_state, np.zeros((1, 2, n_big, 3)))
    refp = np.concatenate([ref[0, :1], ref[1]])
    assert normwise_err(got[:1], refp[:1]).max() <= TOL
    # 128 overlapping bodies: held to TOL unless the oracle certifies a near
    # tie (decision margin below 1e-5, as in the regular world's parity tests)
    err_big = normwise_err(got[1:], refp[1:]).max()
    print("\n[near ties] 128-entity env: margin %.2e, error %.2e" % (margin[1], err_big))
    assert err_big <= TOL or margin[1] < 1e-5, (err_big, margin[1])
    rw.check()
    rw.close()


def test_regular_world_tiled_rollout_is_bitwise(vmas_lib):
    from paper_2207_03530_b300 import World, _lib

    sc = scenes.paper_scene(500, 4, dense=True)
    act = torch.from_numpy(scenes.make_actions(sc, 12, 2)).cuda()
    outs = []
    for tile in (1, 5, 12):
        w = World(sc)
        _lib.check(w._L.vmas_world_set_rollout_tile(w._handle(), tile))
        w.rollout(act)
        outs.append(w.state().cpu().numpy())
        w.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_full_config_sampled_envs(vmas_lib, orc):
    """65,536 ragged envs (2.55 M entities) with the benchmark's autotuned
    lanes and steps per launch: one graph step against the oracle on 32
    sampled envs, then an 8-step graph rollout bitwise equal to stepping."""
    sc, counts = scenes.ragged_scene(65536, 0)
    rw = _ragged(sc, counts)
    rw2 = _ragged(sc, counts)
    T = 9
    act = scenes.make_actions(sc, T, 1)
    pact = torch.from_numpy(_packed_actions(rw, sc, act)).cuda()
    rw.autotune(pact[:8])
    lanes, tile = rw.tuning()
    rw2.set_tuning(lanes, tile)
    rw2.schedule = rw.schedule
    rw.rollout(pact[:1])
    got = rw.state().cpu().numpy()
    full, sel = _unpack_state(got, counts, sc.n_entities)
    pick = np.random.default_rng(3).choice(sc.n_envs, 32, replace=False)
    sub = sc.subset(pick)
    ref = orc.step(sub, sub.init_state, act[:1, pick], threads=8)
    assert normwise_err(full[pick][sel[pick]], ref[sel[pick]]).max() <= TOL
    rw.rollout(pact[1:])
    for t in range(T):
        rw2.step(pact[t])
    assert np.array_equal(rw.state().cpu().numpy(), rw2.state().cpu().numpy())
    rw.check()
    rw.close()
    rw2.check()
    rw2.close()


PERSIST_LANES = [8, 8, 16, 32, 32]  # the persistent schedule's fixed lanes per class


@pytest.mark.parametrize("seed,schedule", [(0, 1), (1, 1), (0, 2)])
def test_persistent_schedule_matches_oracle_and_per_class(vmas_lib, orc, seed, schedule):
    """Every size class in one persistent launch (warps take one warp's worth
    of envs at a time from an atomic work queue, largest class first):
    against the FP64 oracle, and equal to the per-class launches with the
    same lanes per class, stepped one at a time and in tiled, graph-captured
    rollouts (replayed twice).

    The two schedules run the same step body compiled into different
    kernels, and the compiler may fuse a multiply and an add into one fma in
    one kernel and not the other, so they agree to rounding, not always
    bitwise (one env of 300 differed by 3e-8 after 14 steps; built without
    automatic fma contraction, every env agreed bitwise).  An env the queue
    skipped or stepped twice would be off by a whole step's motion, about
    1e-3, so the 1e-6 bound still checks the queue."""
    sc, counts = scenes.ragged_scene(300, seed)
    act = scenes.make_actions(sc, 8, seed)
    per, pers = _ragged(sc, counts), _ragged(sc, counts)
    assert (pers.class_envs > 0).sum() >= 4
    per.set_tuning(PERSIST_LANES, 1)
    pers.schedule = schedule
    assert pers.persistent and not per.persistent
    pact = torch.from_numpy(_packed_actions(per, sc, act)).cuda()
    for t in range(2):
        per.step(pact[t])
        pers.step(pact[t])
    a, b = per.state().cpu().numpy(), pers.state().cpu().numpy()
    assert np.abs(a - b).max() <= 1e-6
    got, sel = _unpack_state(b, counts, sc.n_entities)
    ref = orc.step(sc, sc.init_state, act[:2], threads=8)
    assert normwise_err(got[sel], ref[sel]).max() <= TOL
    for rw in (per, pers):
        rw.set_tuning(None if rw is pers else PERSIST_LANES, 3)
        rw.rollout(pact[2:])
        rw.rollout(pact[2:])  # replay of the captured graph
    assert np.abs(per.state().cpu().numpy() - pers.state().cpu().numpy()).max() <= 1e-6
    for rw in (per, pers):
        rw.check()
        rw.close()


@pytest.mark.parametrize("n_envs", [0, 1, 3, 37])
def test_persistent_schedule_small_worlds(vmas_lib, orc, n_envs):
    """Fewer work items than warps, classes left empty, and an empty world."""
    sc, counts = scenes.ragged_scene(max(n_envs, 1), 9)
    if n_envs == 0:
        sc, counts = sc.subset([]), counts[:0]
    rw = _ragged(sc, counts)
    rw.persistent = True
    act = scenes.make_actions(sc, 3, 2)
    pact = torch.from_numpy(_packed_actions(rw, sc, act)).cuda() if n_envs else \
        torch.zeros((3, 0, 3), device="cuda")
    rw.set_tuning(None, 2)
    rw.rollout(pact)
    if n_envs:
        got, sel = _unpack_state(rw.state().cpu().numpy(), counts, sc.n_entities)
        ref = orc.step(sc, sc.init_state, act, threads=8)
        assert normwise_err(got[sel], ref[sel]).max() <= TOL
    rw.check()
    rw.close()
