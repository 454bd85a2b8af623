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


def normwise_err(got, ref):
    """Per state field (x, y, vx, vy, theta, omega): max |got - ref| divided
    by max(max |ref|, 1e-6); returns the 6 errors."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    out = []
    for f in range(6):
        scale = max(np.abs(ref[..., f]).max(initial=0.0), 1e-6)
        out.append(np.abs(got[..., f] - ref[..., f]).max(initial=0.0) / scale)
    return np.array(out)


@pytest.fixture(scope="session")
def vmas_lib():
    """The built CUDA library; GPU tests skip when no GPU is present."""
    import torch

    from paper_2207_03530_b300 import build

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_03530_b300 import _lib

    return _lib.load()
