"""Python binding of the learned surrogate of the world step (C ABI
vmas_sur_*): argument marshalling only; features, the network, its backward,
Adam and the fallback all run in libvmas.so.

The surrogate serves the walled sphere world (16 actuated agent spheres then
4 fixed walls per env, see ``scenes.surrogate_scene``).  Parameters are one
flat FP32 vector in the order of ``ORDER`` with the shapes of ``SHAPES``.
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np
import torch

from . import _lib
from .world import World, _stream_handle

SHAPES = {"We1": (64, 16), "be1": (64,), "We2": (64, 64), "be2": (64,),
          "W1": (128, 80), "b1": (128,), "W2": (128, 128), "b2": (128,),
          "W3": (8, 128), "b3": (8,)}
ORDER = ("We1", "be1", "We2", "be2", "W1", "b1", "W2", "b2", "W3", "b3")
K = 6
FALLBACK_LIMIT = 0.01  # world units of predicted overlap


def param_count() -> int:
    return int(_lib.load().vmas_sur_param_count())


def flatten(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[k], np.float32).reshape(-1) for k in ORDER])


def unflatten(flat) -> dict:
    flat = np.asarray(flat, np.float32)
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = flat[o:o + n].reshape(SHAPES[k]).copy()
        o += n
    return out


def init_params(seed: int = 0) -> dict:
    """Uniform fan-in initialisation (bound 1/sqrt(fan_in)), biases and the
    unused output rows 4..7 zero."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5C6]))
    p = {}
    for k in ORDER:
        shp = SHAPES[k]
        if k.startswith("b"):
            p[k] = np.zeros(shp, np.float32)
        else:
            b = 1.0 / math.sqrt(shp[1])
            p[k] = rng.uniform(-b, b, size=shp).astype(np.float32)
    p["W3"][4:] = 0.0
    return p


def _dev(x, dtype=torch.float32):
    if x is None:
        return None
    if not (isinstance(x, torch.Tensor) and x.is_cuda):
        raise ValueError("expected a CUDA tensor")
    if x.dtype != dtype or not x.is_contiguous():
        raise ValueError("expected a contiguous %s tensor" % dtype)
    return x


def _p(x):
    return None if x is None else x.data_ptr()


def nodes_of(world) -> int:
    """Network rows per env: 16 agents, or 20 (16 agents + 4 boxes) in the
    box world (the paper-scale layout of 24 entities)."""
    return 20 if world.n_entities == 24 else 16


def target_width(world) -> int:
    return 6 if world.n_entities == 24 else 4


class Surrogate:
    """The network's parameters, Adam state and activations for worlds of up
    to ``max_envs`` envs on the current CUDA device."""

    def __init__(self, max_envs: int, params: dict | None = None, seed: int = 0):
        self._L = _lib.load()
        self.max_envs = int(max_envs)
        h = ctypes.c_void_p()
        _lib.check(self._L.vmas_sur_create(self.max_envs, ctypes.byref(h)))
        self._h = h
        self.set_params(init_params(seed) if params is None else params)

    def _handle(self):
        if self._h is None:
            raise RuntimeError("surrogate is closed")
        return self._h

    def close(self):
        if self._h is not None:
            _lib.check(self._L.vmas_sur_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------- parameters
    def set_params(self, params) -> None:
        flat = flatten(params) if isinstance(params, dict) else np.asarray(params, np.float32)
        flat = np.ascontiguousarray(flat, np.float32)
        if flat.size != param_count():
            raise ValueError("expected %d parameters, got %d" % (param_count(), flat.size))
        _lib.check(self._L.vmas_sur_set_params(self._handle(), flat.ctypes.data))

    def params(self) -> dict:
        flat = np.zeros(param_count(), np.float32)
        _lib.check(self._L.vmas_sur_get_params(self._handle(), flat.ctypes.data))
        return unflatten(flat)

    def set_mode(self, mode: str) -> None:
        """Inference kernels: "fused" (default; one warp per env, all on chip)
        or "layered" (one GEMM per layer, the training path)."""
        code = {"fused": 0, "layered": 1}[mode]
        _lib.check(self._L.vmas_sur_set_mode(self._handle(), code))

    # -------------------------------------------------------------- network
    def _world(self, world: World, actions):
        _dev(actions)
        if tuple(actions.shape) != (world.n_envs, world.n_actuated, 3):
            raise ValueError("actions must have shape [E, n_actuated, 3]")
        return world._handle()

    def forward(self, world: World, actions: torch.Tensor, stream=None) -> torch.Tensor:
        """Network output [E * nodes, 8] on the world's current state (nodes:
        16 agents, or 16 agents + 4 boxes in the box world)."""
        w = self._world(world, actions)
        out = torch.empty((world.n_envs * nodes_of(world), 8), dtype=torch.float32,
                          device=actions.device)
        _lib.check(self._L.vmas_sur_forward(self._handle(), w, _p(actions), _p(out),
                                            _stream_handle(stream)))
        return out

    def loss_grad(self, world: World, actions, target, stream=None):
        """(loss [1], gradient [param_count()]) against target [E * nodes,
        tw] (tw = 4: x y vx vy; 6 in the box world: also theta omega)."""
        w = self._world(world, actions)
        _dev(target)
        shape = (world.n_envs * nodes_of(world), target_width(world))
        if tuple(target.shape) != shape:
            raise ValueError("target must have shape %s" % (shape,))
        loss = torch.zeros(1, dtype=torch.float32, device=actions.device)
        grad = torch.zeros(param_count(), dtype=torch.float32, device=actions.device)
        _lib.check(self._L.vmas_sur_loss_grad(self._handle(), w, _p(actions), _p(target),
                                              _p(loss), _p(grad), _stream_handle(stream)))
        return loss, grad

    def adam(self, lr: float, grad=None, stream=None) -> None:
        """One Adam update with ``grad`` [param_count()] (CUDA float32), or
        with the last computed gradient when None."""
        if grad is not None:
            _dev(grad)
            if grad.numel() != param_count():
                raise ValueError("grad must have %d elements" % param_count())
        _lib.check(self._L.vmas_sur_adam(self._handle(), float(lr), _p(grad),
                                         _stream_handle(stream)))

    def train_grad(self, world: World, actions, loss=None, grad=None, stream=None):
        """The gradient half of a training step on the transition the plain
        step makes from the world's current state (the world advances).
        Returns (loss [1], grad [param_count()])."""
        w = self._world(world, actions)
        dev = actions.device
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device=dev)
        if grad is None:
            grad = torch.zeros(param_count(), dtype=torch.float32, device=dev)
        _lib.check(self._L.vmas_sur_train_grad(self._handle(), w, _p(actions), _p(loss),
                                               _p(grad), _stream_handle(stream)))
        return loss, grad

    def train_step(self, world: World, actions, lr: float, loss=None, stream=None):
        """One training step on the transition the plain step makes from the
        world's current state (the world advances).  Returns the loss [1]."""
        w = self._world(world, actions)
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device=actions.device)
        _lib.check(self._L.vmas_sur_train_step(self._handle(), w, _p(actions), float(lr),
                                               _p(loss), _stream_handle(stream)))
        return loss

    def step(self, world: World, actions, limit: float = FALLBACK_LIMIT, n_fallback=None,
             stream=None):
        """One world step by the surrogate (plain step where the prediction
        overlaps by more than ``limit``).  Returns the fallback count [1]."""
        w = self._world(world, actions)
        if n_fallback is None:
            n_fallback = torch.zeros(1, dtype=torch.int32, device=actions.device)
        _dev(n_fallback, torch.int32)
        _lib.check(self._L.vmas_sur_step(self._handle(), w, _p(actions), float(limit),
                                         _p(n_fallback), _stream_handle(stream)))
        return n_fallback

    def check(self, stream=None) -> int:
        """Wait for the stream; raise if a kernel set the surrogate's device
        error word (a tensor-core GEMM's bounded wait ran out)."""
        bits = ctypes.c_int32(0)
        rc = self._L.vmas_sur_check(self._handle(), _stream_handle(stream), ctypes.byref(bits))
        if rc == _lib.VMAS_EDEVICE:
            raise _lib.VmasError(rc, "surrogate device error bits %d" % bits.value)
        _lib.check(rc)
        return bits.value

    def debug_features(self, world: World, actions, stream=None):
        """(node [E*nodes, 16], edge [6, E*nodes, 16], mask [6, E*nodes]) as
        float32 (bfloat16 values) for the world's current state."""
        w = self._world(world, actions)
        R = world.n_envs * nodes_of(world)
        dev = actions.device
        node = torch.zeros((R, 16), dtype=torch.bfloat16, device=dev)
        edge = torch.zeros((K, R, 16), dtype=torch.bfloat16, device=dev)
        mask = torch.zeros((K, R), dtype=torch.float32, device=dev)
        _lib.check(self._L.vmas_sur_debug_features(self._handle(), w, _p(actions), _p(node),
                                                   _p(edge), _p(mask), _stream_handle(stream)))
        return node.float(), edge.float(), mask


def gemm_bf16(a: torch.Tensor, b: torch.Tensor, trans_a=False, trans_b=False, bias=None,
              gelu=False, splits=1, stream=None):
    """The surrogate's tensor-core GEMM on bfloat16 matrices: returns
    (C FP32 [M, N], GELU(C) bfloat16 [M, N] or None).  a is [M, K] ([K, M]
    when trans_a), b is [K, N] ([N, K] when trans_b)."""
    L = _lib.load()
    _dev(a, torch.bfloat16)
    _dev(b, torch.bfloat16)
    M, Ka = (a.shape[1], a.shape[0]) if trans_a else (a.shape[0], a.shape[1])
    N, Kb = (b.shape[0], b.shape[1]) if trans_b else (b.shape[1], b.shape[0])
    if Ka != Kb:
        raise ValueError("inner dimensions differ")
    if bias is not None:
        _dev(bias)
    out = torch.zeros((M, N), dtype=torch.float32, device=a.device)
    obf = torch.zeros((M, N), dtype=torch.bfloat16, device=a.device) if splits == 1 else None
    _lib.check(L.vmas_debug_gemm_bf16(int(trans_a), int(trans_b), M, N, Ka, _p(a), a.shape[1],
                                      _p(b), b.shape[1], _p(bias), int(gelu), _p(out), _p(obf),
                                      int(splits), _stream_handle(stream)))
    return out, obf


def set_gemm_engine(engine: str) -> None:
    """Which GEMM the surrogate's kernels use, process-wide: "tcgen05" (the
    default: the tensor-core GEMM wherever the shape allows) or "mma" (the
    warp-level mma GEMM only, for comparisons)."""
    _lib.check(_lib.load().vmas_debug_gemm_engine({"tcgen05": 0, "mma": 1}[engine], None))


def tcgen05_gemm_launches() -> int:
    """How many tcgen05 GEMMs this process has launched so far."""
    n = ctypes.c_int64(0)
    _lib.check(_lib.load().vmas_debug_gemm_engine(-1, ctypes.byref(n)))
    return n.value


def allreduce_mean(tensors, group=None):
    """Average CUDA tensors over the ranks of a torch.distributed group in
    place: directly with NCCL, through host memory with gloo."""
    import torch.distributed as dist

    ws = dist.get_world_size(group)
    for t in tensors:
        if dist.get_backend(group) == "nccl":
            dist.all_reduce(t, group=group)
            t.div_(ws)
        else:
            h = t.cpu()
            dist.all_reduce(h, group=group)
            t.copy_(h.div_(ws))


def train_on_plain_step(sur, n_envs, n_steps, lr0, seed, reset_every=100, log=None, substeps=5,
                        group=None, envs=None, boxes=False):
    """Trains ``sur`` on the GPU on transitions the plain step makes: a world
    of the surrogate's layout (``substeps`` per step; ``boxes``: the
    paper-scale scene of 16 agents, 4 boxes and 4 walls) advanced by uniform
    random actions, reset to its start every ``reset_every`` steps; Adam with
    a cosine schedule from lr0 to lr0 / 100.  Returns (seconds, final mean
    loss, transitions).

    Data parallel: with a torch.distributed ``group`` every rank steps its
    own share ``envs`` (an index array into the n_envs of the scene, e.g.
    ``sharding.env_range``) and the gradient and loss are averaged over the
    ranks (equal shares) before each Adam update, so every rank applies the
    same update."""
    from . import scenes

    sc = (scenes.paper_scene(n_envs, seed, substeps=substeps) if boxes
          else scenes.surrogate_scene(n_envs, seed, substeps=substeps))
    if envs is not None:
        sc = sc.subset(envs)
    w = World(sc)
    init = torch.from_numpy(sc.init_state).cuda()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed + 17)
    losses = torch.zeros(n_steps, device="cuda")
    grad = torch.zeros(param_count(), device="cuda") if group is not None else None
    pick = torch.from_numpy(np.asarray(envs, np.int64)).cuda() if envs is not None else None
    torch.cuda.synchronize()
    t0 = time.time()
    for t in range(n_steps):
        if t % reset_every == 0:
            w.set_state(init)
        # the same action stream on every rank: each takes its envs' rows
        act = torch.rand((n_envs, sc.n_actuated, 3), device="cuda", generator=gen) * 2 - 1
        if pick is not None:
            act = act.index_select(0, pick).contiguous()
        lr = lr0 * (0.01 + 0.99 * 0.5 * (1 + math.cos(math.pi * t / n_steps)))
        if group is None:
            sur.train_step(w, act, lr, loss=losses[t:t + 1])
        else:
            sur.train_grad(w, act, loss=losses[t:t + 1], grad=grad)
            allreduce_mean([grad, losses[t:t + 1]], group)
            sur.adam(lr, grad)
        if log and (t % 200 == 0 or t == n_steps - 1):
            print("train step %d loss %.3e" % (t, losses[t].item()), file=log, flush=True)
    torch.cuda.synchronize()
    secs = time.time() - t0
    w.close()
    tail = max(1, n_steps // 20)
    return secs, float(losses[-tail:].mean().item()), sc.n_envs * n_steps
