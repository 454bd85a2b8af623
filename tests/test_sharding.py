"""Multi-rank path on CPU: env sharding with gloo, world size 2.

Environments are independent, so stepping each rank's shard and gathering
must reproduce stepping the whole batch; the timing reduction is a max.
The per-rank step here is the oracle (no GPU on this path's tests)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2207_03530_b300 import scenes, sharding


@pytest.mark.parametrize("n,ws", [(0, 2), (1, 2), (7, 2), (30000, 4), (5, 8)])
def test_env_range_partitions(n, ws):
    ranges = [sharding.env_range(n, ws, r) for r in range(ws)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_env_range_rejects_bad_arguments():
    with pytest.raises(ValueError):
        sharding.env_range(10, 0, 0)
    with pytest.raises(ValueError):
        sharding.env_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sc = scenes.paper_scene(37, 3, dense=True)
    act = scenes.make_actions(sc, 2, 1)
    mine = sharding.shard_scene(sc, ws, rank)
    a, b = sharding.env_range(sc.n_envs, ws, rank)
    st = oracle.step(mine, mine.init_state, act[:, a:b])
    full = sharding.gather_states(torch.from_numpy(st))
    tmax = sharding.max_over_ranks(float(rank + 1))
    dist.barrier()
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), full.numpy())
        np.save(os.path.join(out_dir, "tmax.npy"), np.array([tmax]))
    dist.destroy_process_group()


def test_gloo_two_ranks_shard_and_gather(tmp_path, orc):
    ws, port = 2, _free_port()
    mp.start_processes(_worker, args=(ws, port, str(tmp_path)), nprocs=ws, start_method="spawn")
    gathered = np.load(tmp_path / "gathered.npy")
    sc = scenes.paper_scene(37, 3, dense=True)
    act = scenes.make_actions(sc, 2, 1)
    whole = orc.step(sc, sc.init_state, act)
    assert np.array_equal(gathered, whole)
    assert np.load(tmp_path / "tmax.npy")[0] == 2.0


def _mean_worker(rank, ws, port, out_dir):
    import torch
    import torch.distributed as dist

    from paper_2207_03530_b300.surrogate import allreduce_mean

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    g = torch.arange(6, dtype=torch.float32) * (rank + 1)
    loss = torch.tensor([float(rank)])
    allreduce_mean([g, loss[0:1]])
    if rank == 0:
        np.save(os.path.join(out_dir, "mean.npy"), np.concatenate([g.numpy(), loss.numpy()]))
    dist.destroy_process_group()


def test_gloo_gradient_average(tmp_path):
    """The surrogate's data-parallel update averages gradients over ranks
    (host-side reduction with gloo): two ranks, world size 2."""
    ws, port = 2, _free_port()
    mp.start_processes(_mean_worker, args=(ws, port, str(tmp_path)), nprocs=ws,
                       start_method="spawn")
    got = np.load(tmp_path / "mean.npy")
    np.testing.assert_allclose(got[:6], np.arange(6) * 1.5)
    assert got[6] == 0.5
