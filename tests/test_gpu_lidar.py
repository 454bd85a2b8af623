"""LIDAR ray casts on the GPU against the FP64 oracle, element by element.

Every ray must agree to 2e-5 world units, or to twice the oracle's own
sensitivity to single-precision rounding, whichever is larger: the oracle
recomputes every ray on copies of the scene whose positions, angles and
sizes are moved by up to eight FP32 units in the last place
(``oracle.lidar_sensitivity``), decided before the GPU result is looked at.
A ray that grazes a disc (its entry distance goes as the square root of the
discriminant), clips a box corner or a segment end, or starts on a surface
moves by far more than its inputs and may differ between FP32 and FP64;
a well-conditioned ray may not.  The rays the allowance covers are
counted and reported."""
import numpy as np
import pytest
import torch

from paper_2207_03530_b300 import scenes

pytestmark = pytest.mark.gpu


TOL = 2e-5


def _certified(orc, sc, got, n_rays, rng_max, label):
    ref = orc.lidar(sc, sc.init_state, n_rays, rng_max)
    sens = orc.lidar_sensitivity(sc, sc.init_state, n_rays, rng_max)
    diff = np.abs(got - ref)
    allow = np.maximum(TOL, 2.0 * sens)
    assert (diff <= allow).all(), (label, diff[diff > allow][:8], sens[diff > allow][:8])
    cov = diff > TOL
    print("\n[ill-conditioned rays] %s: %d of %d rays beyond %.0e, each within twice the "
          "oracle's sensitivity (largest difference %.2e); %d rays have sensitivity > %.0e"
          % (label, int(cov.sum()), diff.size, TOL, float(diff.max()), int((sens > TOL / 2).sum()),
             TOL / 2))
    return ref, int(cov.sum())


def _compare(orc, sc, n_rays, rng_max, label=""):
    from paper_2207_03530_b300 import World

    w = World(sc)
    got = w.lidar(n_rays, rng_max).cpu().numpy()
    w.close()
    ref, nbad = _certified(orc, sc, got, n_rays, rng_max, label)
    return got, ref, nbad


@pytest.mark.parametrize("make,n_rays,rng", [
    (lambda: scenes.paper_scene(300, 2, dense=True), 32, 1.0),
    (lambda: scenes.mixed_scene(200, 3), 24, 0.8),
    (lambda: scenes.small_scene(64, 1), 12, 2.0),
])
def test_lidar_matches_oracle(vmas_lib, orc, make, n_rays, rng, capsys):
    sc = make()
    with capsys.disabled():
        got, ref, nbad = _compare(orc, sc, n_rays, rng, label=sc.name)
    assert (ref < rng).mean() > 0.05  # the rays do hit things
    assert (got == 0).sum() == (ref == 0).sum()  # inside-origin readings agree


def test_lidar_full_config_sampled(vmas_lib, orc, capsys):
    """30,000 envs, 16 rays: 64 sampled envs compared."""
    from paper_2207_03530_b300 import World

    sc = scenes.paper_scene(30000, 0)
    w = World(sc)
    got = w.lidar(16, 1.0).cpu().numpy()
    w.close()
    pick = np.random.default_rng(0).choice(30000, 64, replace=False)
    sub = sc.subset(pick)
    with capsys.disabled():
        _certified(orc, sub, got[pick], 16, 1.0, "30,000 envs, 64 sampled")


def test_lidar_rays_parallel_to_box_faces_and_walls(vmas_lib, orc):
    """Ray 0 of a caster with heading 0 is exactly (1, 0): against a box with
    angle 0 it is parallel to two faces (the slab between them bounds it
    only if it starts inside), and against a wall with angle 0 it never
    crosses the segment.  Hand-worked: from (0, 0) the box face x = 0.4 is
    hit at 0.4; from (0, 0.3), outside the box's y-slab |y| <= 0.2, the ray
    misses everything and reads the range."""
    from conftest import make_scene
    from paper_2207_03530_b300 import World

    act = scenes.MOVABLE | scenes.COLLIDABLE | scenes.ACTUATED
    sc = make_scene([
        dict(shape=scenes.SPHERE, x=0.0, y=0.0, a=0.05, flags=act),
        dict(shape=scenes.SPHERE, x=0.0, y=0.3, a=0.05, flags=act),
        dict(shape=scenes.BOX, x=0.5, y=0.0, a=0.2, b=0.4, m=5.0, flags=scenes.COLLIDABLE),
        dict(shape=scenes.LINE, x=0.0, y=-0.5, a=1.0, flags=scenes.COLLIDABLE),
    ], n_envs=3)
    w = World(sc)
    got = w.lidar(4, 2.0).cpu().numpy()
    w.close()
    ref = orc.lidar(sc, sc.init_state, 4, 2.0)
    assert np.abs(got - ref).max() <= 2e-5
    assert abs(got[0, 0, 0] - 0.4) <= 1e-6 and abs(ref[0, 0, 0] - 0.4) <= 1e-6
    assert got[0, 1, 0] == 2.0 and ref[0, 1, 0] == 2.0


def _both_kernels(sc, n_rays, rng_max, state=None):
    """The culled kernel (default) and every ray against every body."""
    from paper_2207_03530_b300 import World, _lib

    L = _lib.load()
    w = World(sc)
    if state is not None:
        w.set_state(torch.from_numpy(state).cuda())
    culled = w.lidar(n_rays, rng_max).cpu().numpy()
    _lib.check(L.vmas_debug_lidar_cull(0))
    try:
        full = w.lidar(n_rays, rng_max).cpu().numpy()
    finally:
        _lib.check(L.vmas_debug_lidar_cull(1))
    w.close()
    return culled, full


@pytest.mark.parametrize("make,n_rays,rng", [
    (lambda: scenes.paper_scene(2000, 4, dense=True), 32, 1.0),
    (lambda: scenes.paper_scene(2000, 5), 7, 3.0),
    (lambda: scenes.mixed_scene(500, 6), 64, 0.6),
    (lambda: scenes.small_scene(256, 2), 1, 2.0),
    (lambda: scenes.paper_scene(500, 7, dense=True), 96, 0.05),
    (lambda: scenes.mixed_scene(300, 9), 7, 1.0),  # odd n_actuated x n_rays (11 x 7)
    (lambda: scenes.small_scene(64, 3), 1000, 2.0),  # 4 x 1000 rays: the every-ray kernel
])
def test_culled_lidar_equals_every_ray(vmas_lib, make, n_rays, rng):
    """Each (body, caster) pair testing only the rays within the body's arc
    gives the readings of testing every ray against every body: the same
    routines on the same ray directions, so equal up to the compiler's fma
    contraction in the two kernels (measured: equal bitwise)."""
    sc = make()
    culled, full = _both_kernels(sc, n_rays, rng)
    assert np.abs(culled - full).max() <= 1e-6
    assert (culled < rng).mean() > 0.01 or rng < 0.1  # the rays do hit things
    print("\n[culled LIDAR] %s, %d rays: %.4f of readings bitwise equal"
          % (sc.name, n_rays, float((culled == full).mean())))


def test_culled_lidar_large_angles_and_overlaps(vmas_lib):
    """Casters spun to large angles (their rays are then tested in full:
    fl(th + step r) strays from the ray's nominal direction) and casters
    whose origin lies inside another body (every ray reads 0)."""
    sc = scenes.paper_scene(400, 8, dense=True)
    st = sc.init_state.copy()
    rs = np.random.default_rng(8)
    st[:, :, 4] += rs.choice([0.0, 7e3, -3e5, 2e6], size=st.shape[:2]).astype(np.float32)
    # the first agent of every fourth env sits on the second one's centre
    st[::4, 0, 0:2] = st[::4, 1, 0:2] + 0.01
    culled, full = _both_kernels(sc, 32, 1.5, state=st)
    assert np.abs(culled - full).max() <= 1e-6
    assert (culled[::4, 0] == 0).all() and (culled[::4, 1] == 0).all()
