"""Environment sharding across ranks (one process per GPU).

Environments are independent (VMAS section 3, "Interface": an arbitrary batch
of environments is stepped in parallel), so a multi-GPU job partitions them
into contiguous ranges with no exchange on the data path.  The only
collectives are host-side bookkeeping: a max over ranks of the timed region
and an optional gather of states for readback.
"""
from __future__ import annotations


def env_range(n_total: int, world_size: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced [start, stop) of rank's environments; the first
    n_total % world_size ranks take one extra env."""
    if world_size < 1 or not 0 <= rank < world_size or n_total < 0:
        raise ValueError("bad sharding arguments")
    base, extra = divmod(n_total, world_size)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_scene(scene, world_size: int, rank: int):
    """The rank's slice of a global scene (strong scaling)."""
    import numpy as np

    a, b = env_range(scene.n_envs, world_size, rank)
    return scene.subset(np.arange(a, b))


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over all ranks of the default process group (identity
    when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_states(state, device=None):
    """Concatenate every rank's [E_r, N, 6] state in rank order (readback
    only; ranks may hold different env counts)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return state
    ws = dist.get_world_size()
    n = torch.tensor([state.shape[0]], dtype=torch.int64, device=device)
    counts = [torch.zeros_like(n) for _ in range(ws)]
    dist.all_gather(counts, n)
    counts = [int(c.item()) for c in counts]
    m = max(counts)
    pad = torch.zeros((m,) + tuple(state.shape[1:]), dtype=state.dtype, device=state.device)
    pad[: state.shape[0]] = state
    out = [torch.empty_like(pad) for _ in range(ws)]
    dist.all_gather(out, pad)
    return torch.cat([o[:c] for o, c in zip(out, counts)])
