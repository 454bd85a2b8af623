"""Data-parallel surrogate training: two ranks (processes, gloo) on one GPU,
each stepping half of the envs, with the gradient averaged over the ranks
before every Adam update.

Checks: the averaged gradient equals the single-process gradient of the
whole batch (equal halves: the mean of the halves' means is the batch mean;
only the FP32 summation order differs), and after data-parallel training
steps both ranks hold bitwise the same parameters."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu
E = 512


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out_dir):
    import datetime

    import torch
    import torch.distributed as dist

    from paper_2207_03530_b300 import World, scenes, sharding
    from paper_2207_03530_b300.surrogate import (Surrogate, allreduce_mean, flatten,
                                                 train_on_plain_step)

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws,
                            timeout=datetime.timedelta(seconds=120))
    torch.cuda.set_device(0)
    a, b = sharding.env_range(E, ws, rank)
    sc = scenes.surrogate_scene(E, 4)
    act = torch.from_numpy(scenes.make_actions(sc, 1, 5)[0]).cuda()
    # one averaged gradient
    sur = Surrogate(E, seed=2)
    w = World(sc.subset(np.arange(a, b)))
    loss, grad = sur.train_grad(w, act[a:b].contiguous())
    allreduce_mean([grad, loss])
    w.close()
    # data-parallel training steps
    train_on_plain_step(sur, E, 4, 1e-3, 9, group=dist.group.WORLD, envs=np.arange(a, b))
    np.save(os.path.join(out_dir, "grad%d.npy" % rank), grad.cpu().numpy())
    np.save(os.path.join(out_dir, "loss%d.npy" % rank), loss.cpu().numpy())
    np.save(os.path.join(out_dir, "params%d.npy" % rank), flatten(sur.params()))
    sur.close()
    dist.destroy_process_group()


def test_two_ranks_one_gpu(vmas_lib, tmp_path):
    import torch

    from paper_2207_03530_b300 import World, scenes
    from paper_2207_03530_b300.surrogate import Surrogate

    ws, port = 2, _free_port()
    mp.start_processes(_worker, args=(ws, port, str(tmp_path)), nprocs=ws, start_method="spawn")
    g0, g1 = np.load(tmp_path / "grad0.npy"), np.load(tmp_path / "grad1.npy")
    assert np.array_equal(g0, g1)
    p0, p1 = np.load(tmp_path / "params0.npy"), np.load(tmp_path / "params1.npy")
    assert np.array_equal(p0, p1)
    # the whole batch in one process
    sc = scenes.surrogate_scene(E, 4)
    act = torch.from_numpy(scenes.make_actions(sc, 1, 5)[0]).cuda()
    sur = Surrogate(E, seed=2)
    w = World(sc)
    loss, grad = sur.train_grad(w, act)
    ref = grad.cpu().numpy()
    assert np.linalg.norm(g0 - ref) <= 1e-4 * np.linalg.norm(ref)
    assert float(np.load(tmp_path / "loss0.npy")[0]) == pytest.approx(float(loss.item()), rel=1e-5)
    w.close()
    sur.close()
