import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


def make_scene(bodies, *, substeps=1, dt=0.1, drag=0.0, g=(0.0, 0.0), c=100.0, k=1e-3,
               max_speed=0.0, n_envs=1):
    """One-env scene (replicated n_envs times) from a list of body dicts with
    keys shape, x, y, th, vx, vy, om, a, b, m, I, flags."""
    from paper_2207_03530_b300 import scenes

    N = len(bodies)
    A = sum(1 for b in bodies if b.get("flags", 0) & scenes.ACTUATED)
    st = np.zeros((n_envs, N, 6), np.float32)
    arr = {k_: np.zeros((n_envs, N), np.float32) for k_ in ("size_a", "size_b", "mass", "inertia")}
    shape = np.zeros((n_envs, N), np.uint8)
    flags = np.zeros((n_envs, N), np.uint8)
    for i, b in enumerate(bodies):
        shape[:, i] = b["shape"]
        flags[:, i] = b.get("flags", 0)
        arr["size_a"][:, i] = b.get("a", 0.05)
        arr["size_b"][:, i] = b.get("b", 0.0)
        arr["mass"][:, i] = b.get("m", 1.0)
        arr["inertia"][:, i] = b.get("I", 0.0)
        st[:, i] = [b.get("x", 0.0), b.get("y", 0.0), b.get("vx", 0.0), b.get("vy", 0.0),
                    b.get("th", 0.0), b.get("om", 0.0)]
    return scenes.Scene(name="custom", n_envs=n_envs, n_entities=N, n_actuated=A,
                        substeps=substeps, dt=dt, drag=drag, gx=g[0], gy=g[1], c=c, k=k,
                        max_speed=max_speed, shape=shape, flags=flags, init_state=st, **arr)
