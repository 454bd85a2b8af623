"""B300-native VMAS world step.

The batched world step of VMAS (Bettini et al., section 3, Eqs. 1-3) as a
CUDA library for sm_103a behind a C ABI (include/vmas.h), with a thin
ctypes binding:

    from paper_2207_03530_b300 import World, scenes
    sc = scenes.paper_scene(30000)
    w = World(sc)                     # on the current CUDA device
    w.step(actions_cuda)              # [E, n_actuated, 3] float32
    state = w.state()                 # [E, N, 6] (x, y, vx, vy, theta, omega)

``scenes`` draws seeded synthetic worlds and actions; ``build`` compiles the
library in-tree.
"""
from . import scenes  # noqa: F401

__all__ = ["World", "Surrogate", "scenes", "build"]


def __getattr__(name):
    import importlib

    if name == "World":
        return importlib.import_module(__name__ + ".world").World
    if name == "Surrogate":
        return importlib.import_module(__name__ + ".surrogate").Surrogate
    if name in ("build", "world", "_lib", "surrogate", "diff", "ragged", "sharding"):
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
