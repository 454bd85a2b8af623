"""CUDA world step vs the FP64 oracle, element by element, through the C ABI.

Gate (max relative state error after one step): for every state field
(x, y, vx, vy, theta, omega), max |gpu - oracle| / max(max |oracle|, 1e-6)
<= 1e-5.  Pair indexing and the first-substep contact mask must match
bit-exactly (scenes keep every active pair's gap outside +-1e-4, so FP32 and
FP64 take the same decision).  Multi-step trajectory errors are reported,
not gated: contact dynamics is chaotic.

Near ties (Reading R9).  Where bodies overlap at random, two contact
features can lie within rounding of each other, and FP32 and FP64 may then
choose differently.  Such envs are named by the oracle alone, before the GPU
result is looked at: its decision margin (the least |gap| of an active pair
and, for contacts, the distance of the chosen face, separating axis,
incident edge, clip or normal orientation from its runner-up, over all
substeps) must be below MARGIN_BOUND.  Every other env meets the 1e-5 gate.
MARGIN_BOUND = 1e-5: before a choice flips, the two implementations' states
differ by FP32 rounding (about 1e-7 of the positions and angles within one
step), and a margin moves at most about 4 times as much as the state does
(a corner moves by its position change plus half its diagonal times the
angle change), so a flip needs a margin below about 1e-6; the bound leaves
a factor of 10.
"""
import os

import numpy as np
import pytest
import torch

from conftest import make_scene, normwise_err
from paper_2207_03530_b300 import scenes

pytestmark = pytest.mark.gpu
TOL = 1e-5
MARGIN_BOUND = 1e-5
S_, B_, L_ = scenes.SPHERE, scenes.BOX, scenes.LINE
MOV, ROT, COL, ACT = scenes.MOVABLE, scenes.ROTATABLE, scenes.COLLIDABLE, scenes.ACTUATED
THREADS = os.cpu_count() or 1


def _world(sc):
    from paper_2207_03530_b300 import World

    return World(sc)


def _one_step(vmas_lib, orc, sc, seed=0, steps=1):
    act = scenes.make_actions(sc, steps, seed)
    w = _world(sc)
    d_act = torch.from_numpy(act).cuda()
    for t in range(steps):
        w.step(d_act[t])
    got = w.state().cpu().numpy()
    w.check()
    ref = orc.step(sc, sc.init_state, act, threads=THREADS)
    w.close()
    return got, ref


def _one_step_certified(vmas_lib, orc, sc, seed, steps=1, label=""):
    """GPU and oracle after `steps` steps; envs whose oracle decision margin is
    below MARGIN_BOUND are reported, every other env must meet TOL."""
    act = scenes.make_actions(sc, steps, seed)
    w = _world(sc)
    d_act = torch.from_numpy(act).cuda()
    for t in range(steps):
        w.step(d_act[t])
    got = w.state().cpu().numpy()
    w.check()
    w.close()
    ref, margin = orc.step_margin(sc, sc.init_state, act, threads=THREADS)
    tie = margin < MARGIN_BOUND
    err = normwise_err(got[~tie], ref[~tie])
    assert err.max() <= TOL, (label, err)
    ties = [(int(e), float(margin[e]), float(normwise_err(got[e:e + 1], ref[e:e + 1]).max()))
            for e in np.nonzero(tie)[0]]
    print("\n[near ties] %s: %d of %d envs below margin %.0e (env, margin, error): %s"
          % (label, len(ties), sc.n_envs, MARGIN_BOUND,
             ", ".join("(%d, %.2e, %.2e)" % t for t in ties)))
    return got, ref, margin


def _mask_compare(vmas_lib, orc, sc):
    w = _world(sc)
    mask = w.debug_pairs().cpu().numpy()
    pi, pj = w.pair_table()
    w.close()
    opi, opj = orc.pair_list(sc.n_entities)
    assert np.array_equal(pi, opi) and np.array_equal(pj, opj)
    omask, gap = orc.pairs(sc, sc.init_state)
    guard = np.abs(gap) < 1e-4
    assert np.array_equal(mask[~guard], omask[~guard])
    return mask, omask, int(guard.sum())


@pytest.mark.parametrize("dense", [False, True])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_small_config_one_step(vmas_lib, orc, dense, seed):
    """32 envs x (4 agent spheres + 2 landmarks), 1 substep."""
    sc = scenes.small_scene(32, seed, dense=dense)
    got, ref = _one_step(vmas_lib, orc, sc, seed)
    err = normwise_err(got, ref)
    assert err.max() <= TOL, err
    mask, omask, nguard = _mask_compare(vmas_lib, orc, sc)
    assert nguard == 0
    if dense:
        assert omask.sum() > 0


@pytest.mark.parametrize("n_envs", [1, 5, 33, 100])
def test_small_config_partial_ctas(vmas_lib, orc, n_envs):
    """Env counts that leave empty env groups in the last warp / CTA."""
    sc = scenes.small_scene(n_envs, 11, dense=True)
    got, ref = _one_step(vmas_lib, orc, sc, 2, steps=2)
    assert normwise_err(got, ref).max() <= TOL


@pytest.mark.parametrize("dense", [False, True])
@pytest.mark.parametrize("n_envs", [1, 7, 603])
def test_paper_config_one_step(vmas_lib, orc, dense, n_envs):
    """16 spheres + 4 boxes + 4 walls, 5 substeps; env counts with a ragged
    last CTA (8 envs per CTA)."""
    sc = scenes.paper_scene(n_envs, 7, dense=dense)
    got, ref = _one_step(vmas_lib, orc, sc, 3)
    err = normwise_err(got, ref)
    assert err.max() <= TOL, err
    mask, omask, nguard = _mask_compare(vmas_lib, orc, sc)
    assert nguard == 0
    if dense and n_envs > 100:
        assert omask.sum() > 100


@pytest.mark.parametrize("seed", range(4))
def test_mixed_scene_all_pair_types(vmas_lib, orc, seed, capsys):
    """Every pair type in contact (sphere/box/line, movable lines, gravity,
    3 substeps); envs the oracle certifies as near ties (decision margin
    below MARGIN_BOUND) are reported, every other env meets TOL."""
    sc = scenes.mixed_scene(256, seed)
    with capsys.disabled():
        got, ref, margin = _one_step_certified(vmas_lib, orc, sc, seed, label="mixed seed %d" % seed)
    assert (margin < MARGIN_BOUND).sum() < sc.n_envs // 10  # the scene still tests contacts
    mask, omask, nguard = _mask_compare(vmas_lib, orc, sc)
    pi, pj = orc.pair_list(sc.n_entities)
    kinds = {(int(sc.shape[0, pi[p]]), int(sc.shape[0, pj[p]])) for p in np.nonzero(omask.any(0))[0]}
    assert len(kinds) >= 6  # SS SB SL BB BL LL all occur


def test_paper_config_full_size(vmas_lib, orc):
    """30,000 envs, the launch configuration the benchmark times; every env
    compared with the oracle (run on all host cores)."""
    sc = scenes.paper_scene(30000, 0)
    got, ref = _one_step(vmas_lib, orc, sc, 0)
    err = normwise_err(got, ref)
    assert err.max() <= TOL, err


def test_paper_config_full_size_dense_masks(vmas_lib, orc):
    sc = scenes.paper_scene(30000, 1, dense=True)
    mask, omask, nguard = _mask_compare(vmas_lib, orc, sc)
    assert nguard == 0 and omask.sum() > 100000


@pytest.mark.parametrize("N", [1, 2, 31, 32, 33, 64, 65, 100, 128])
def test_entity_counts_span_slots(vmas_lib, orc, N, capsys):
    """Entity counts around the lane / slot boundaries (1..4 slots)."""
    rng = np.random.default_rng(N)
    bodies = []
    z = min(1.0, 3.0 / np.sqrt(N))  # keep the crowding similar across N
    for i in range(N):
        sh = [S_, S_, B_, L_][i % 4]
        bodies.append(dict(shape=sh, x=rng.uniform(-1, 1), y=rng.uniform(-1, 1),
                           th=rng.uniform(-3, 3), vx=rng.uniform(-.3, .3), vy=rng.uniform(-.3, .3),
                           a=z * (rng.uniform(0.05, 0.25) if sh != S_ else rng.uniform(0.03, 0.1)),
                           b=z * rng.uniform(0.05, 0.2), m=rng.uniform(0.5, 2),
                           flags=MOV | ROT | COL | (ACT if i % 3 else 0)))
    sc = make_scene(bodies, substeps=2, drag=0.1, n_envs=11)
    # give each env its own layout
    sc.init_state[:, :, :2] += np.random.default_rng(1).uniform(-0.05, 0.05, (11, N, 2)).astype(np.float32)
    with capsys.disabled():
        _one_step_certified(vmas_lib, orc, sc, 5, label="N=%d" % N)


def test_gravity_max_speed_and_inert_padding(vmas_lib, orc):
    """Gravity, the speed cap, fewer actuated entities than action rows and
    inert padding entities (no flags)."""
    sc = scenes.paper_scene(40, 2, dense=True)
    sc.gx, sc.gy, sc.max_speed = 0.3, -2.0, 0.05
    sc.flags[:, 3] = 0   # an inert padding entity
    sc.flags[:, 5] &= np.uint8(0xFF ^ ACT)  # one fewer actuated entity than rows
    got, ref = _one_step(vmas_lib, orc, sc, 1, steps=3)
    assert normwise_err(got, ref).max() <= TOL
    assert np.array_equal(got[:, 3], sc.init_state[:, 3])


def test_empty_world(vmas_lib):
    sc = scenes.small_scene(4, 0).subset([])
    w = _world(sc)
    w.step(torch.zeros((0, 4, 3), device="cuda"))
    assert w.state().shape == (0, 6, 6)
    assert w.debug_pairs().shape == (0, 15)
    w.check()
    w.close()


def test_host_paths_and_rollout_match_device_step(vmas_lib):
    sc = scenes.paper_scene(50, 4, dense=True)
    act = scenes.make_actions(sc, 4, 9)
    w1, w2, w3 = _world(sc), _world(sc), _world(sc)
    d_act = torch.from_numpy(act).cuda()
    for t in range(4):
        w1.step(d_act[t])
        w2.step_host(torch.from_numpy(act[t]).pin_memory())
    w3.rollout(d_act)
    s1 = w1.state().cpu()
    host = torch.empty_like(s1).pin_memory()
    w2.state(out=host)
    assert torch.equal(s1, host)
    assert torch.equal(s1, w3.state().cpu())
    for w in (w1, w2, w3):
        w.close()


def test_set_state_with_env_mask(vmas_lib):
    sc = scenes.paper_scene(20, 5)
    w = _world(sc)
    act = torch.from_numpy(scenes.make_actions(sc, 1, 0)[0]).cuda()
    w.step(act)
    moved = w.state().cpu().numpy()
    mask = np.zeros(20, bool)
    mask[[0, 7, 19]] = True
    w.set_state(sc.init_state, env_mask=mask)
    now = w.state().cpu().numpy()
    assert np.array_equal(now[mask], sc.init_state[mask])
    assert np.array_equal(now[~mask], moved[~mask])
    w.set_state(torch.from_numpy(sc.init_state).cuda())
    assert np.array_equal(w.state().cpu().numpy(), sc.init_state)
    w.close()


def test_device_error_word_reports_nonfinite_state(vmas_lib):
    """A NaN fed in through set_state makes the step raise its device error
    word; the host sees VMAS_EDEVICE once, then the word is clear."""
    from paper_2207_03530_b300 import _lib

    sc = scenes.small_scene(8, 0)
    w = _world(sc)
    bad = sc.init_state.copy()
    bad[3, 1, 2] = np.nan
    w.set_state(bad)
    w.step(torch.zeros((8, 4, 3), device="cuda"))
    with pytest.raises(_lib.VmasError) as ei:
        w.check()
    assert ei.value.code == _lib.VMAS_EDEVICE
    w.set_state(sc.init_state)
    w.step(torch.zeros((8, 4, 3), device="cuda"))
    assert w.check() == 0
    w.close()


def test_trajectory_error_reported(vmas_lib, orc, capsys):
    """100 steps of the small workload and 200 of the paper workload
    (reduced env count): the error is reported, and must stay finite."""
    for sc, T in [(scenes.small_scene(32, 0), 100), (scenes.paper_scene(64, 0), 200)]:
        got, ref = _one_step(vmas_lib, orc, sc, 0, steps=T)
        err = normwise_err(got, ref)
        pos = np.abs(got[..., :2] - ref[..., :2]).max()
        with capsys.disabled():
            print("\n[trajectory] %s %d steps: normwise err per field %s, max |dx| %.3g"
                  % (sc.name, T, np.array2string(err, precision=2), pos))
        assert np.isfinite(got).all()


def test_candidate_skin_does_not_change_results(vmas_lib):
    """The per-step candidate list only skips pairs that cannot touch, and
    its order is fixed by (lane, slot, offset), so any skin gives bitwise the
    same state; an overflowing list (full pair scan) agrees to rounding."""
    sc = scenes.paper_scene(200, 6, dense=True)
    act = torch.from_numpy(scenes.make_actions(sc, 4, 2)).cuda()
    out = []
    for skin in (None, 0.0, 0.004, 0.06, 10.0):
        w = _world(sc)
        if skin is not None:
            w.skin = skin
        w.rollout(act)
        out.append(w.state().cpu().numpy())
        w.check()
        w.close()
    for o in out[1:4]:
        assert np.array_equal(o, out[0])
    assert normwise_err(out[4], out[0]).max() <= 1e-6


def test_fast_bodies_force_list_rebuilds(vmas_lib, orc):
    """Bodies moving several radii per step: the candidate list must be
    rebuilt inside the step; the result still matches the oracle."""
    sc = scenes.paper_scene(64, 8, dense=True)
    rng = np.random.default_rng(0)
    sc.init_state[:, :20, 2:4] = rng.uniform(-3, 3, (64, 20, 2)).astype(np.float32)
    got, ref = _one_step(vmas_lib, orc, sc, 4, steps=2)
    assert normwise_err(got, ref).max() <= TOL


def test_body_axes_accuracy(vmas_lib):
    """The step's own cos/sin of body angles (range reduction + series)
    against float64 math on the same float32 angles."""
    from paper_2207_03530_b300 import _lib

    rng = np.random.default_rng(0)
    th = np.concatenate([rng.uniform(-7, 7, 50000), rng.uniform(-2000, 2000, 50000),
                         rng.uniform(-2e6, 2e6, 50000),
                         np.array([0, 1e-30, np.pi / 4, -np.pi / 4, np.pi / 2, np.pi, 4000.0,
                                   6433.0, 6434.0, 6435.0, -6435.0, 1e4, -1e5, 1e6, 1.6e6,
                                   -2e6, 2e6])])
    th = th.astype(np.float32)
    d_th = torch.from_numpy(th).cuda()
    out = torch.empty((len(th), 2), device="cuda")
    _lib.check(vmas_lib.vmas_debug_body_axes(d_th.data_ptr(), out.data_ptr(), len(th),
                                             torch.cuda.current_stream().cuda_stream))
    cs = out.cpu().numpy().astype(np.float64)
    t64 = th.astype(np.float64)
    err = max(np.abs(cs[:, 0] - np.cos(t64)).max(), np.abs(cs[:, 1] - np.sin(t64)).max())
    assert err <= 1.5e-7, err
    # beyond the stated range the result stays a defined, bounded value
    far = np.array([3e6, -1e9, 1e15, 3.4e38, -3.4e38, np.inf, -np.inf, np.nan], np.float32)
    d_far = torch.from_numpy(far).cuda()
    out = torch.empty((len(far), 2), device="cuda")
    _lib.check(vmas_lib.vmas_debug_body_axes(d_far.data_ptr(), out.data_ptr(), len(far),
                                             torch.cuda.current_stream().cuda_stream))
    o = out.cpu().numpy().astype(np.float64)
    assert np.isfinite(o).all()
    assert np.abs(np.hypot(o[:, 0], o[:, 1]) - 1.0).max() <= 1e-6


def test_rollout_host_streams_every_state(vmas_lib):
    """vmas_rollout_host overlaps uploads, steps and downloads through double
    buffers: every step's state must equal the device-side step's, bitwise."""
    sc = scenes.paper_scene(300, 6, dense=True)
    T = 7
    act = scenes.make_actions(sc, T, 2)
    w1, w2 = _world(sc), _world(sc)
    d_act = torch.from_numpy(act).cuda()
    ref = []
    for t in range(T):
        w1.step(d_act[t])
        ref.append(w1.state().cpu())
    got = w2.rollout_host(torch.from_numpy(act).pin_memory())
    for t in range(T):
        assert torch.equal(got[t], ref[t]), t
    # a second call continues from the streamed world's state
    more = scenes.make_actions(sc, 2, 3)
    got2 = w2.rollout_host(more)  # pageable actions: synchronous uploads
    for t in range(2):
        w1.step(torch.from_numpy(more[t]).cuda())
        assert torch.equal(got2[t], w1.state().cpu()), t
    for w in (w1, w2):
        w.close()


def test_bulk_staged_and_plain_loads_agree_bitwise(vmas_lib):
    """Full CTAs stage their inputs with bulk copies when every copy is
    16-byte aligned; an action array that starts 4 bytes past a 16-byte
    boundary turns staging off.  Both paths must give the same bits."""
    sc = scenes.paper_scene(1000, 8, dense=True)
    act = torch.from_numpy(scenes.make_actions(sc, 3, 4)).cuda()
    n = act[0].numel()
    raw = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
    off = raw[1:1 + n].view(act[0].shape)  # starts 4 bytes past the allocation
    assert off.data_ptr() % 16 == 4 and act[0].data_ptr() % 16 == 0
    w1, w2 = _world(sc), _world(sc)
    for t in range(3):
        w1.step(act[t])
        off.copy_(act[t])
        w2.step(off)
    assert torch.equal(w1.state(), w2.state())
    w1.check()
    w2.check()
    w1.close()
    w2.close()


def test_empty_world_streamed_rollout(vmas_lib):
    sc = scenes.small_scene(4, 0).subset([])
    w = _world(sc)
    out = w.rollout_host(np.zeros((3, 0, 4, 3), np.float32))
    assert tuple(out.shape) == (3, 0, 6, 6)
    w.close()
