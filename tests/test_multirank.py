"""The N > 1 paths of bench.py on the CPU (gloo, world size 2): for solves
each rank takes its own seeded systems (no data-path collective), the job
time is the slowest rank's, and the whole-job value counts every rank's
systems; for training the ranks average their gradients before Adam."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2305_16432_gb300 import inputs as I
    probs = bench._problems(I, "batched_256", rank)
    first = probs[0]
    local_ms = 100.0 + 50.0 * rank                     # ranks finish at different times
    ms = bench.job_ms_per_step(local_ms, world)
    value = bench.job_value(ms, len(probs), world)
    out[rank] = (first.seed, first.nx, len(probs), ms, value)
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    (s0, nx0, n0, ms0, v0), (s1, nx1, n1, ms1, v1) = res[0], res[1]
    assert s0 != s1                                     # disjoint seeded problem sets
    assert n0 == n1 == 256
    assert ms0 == ms1 == 150.0                          # max over ranks
    assert v0 == v1 == pytest.approx(150.0 / (256 * 2))


def _train_rank(rank, world, port, out):
    # data-parallel training step: each rank's gradient (the mean over its
    # own systems) is averaged over the ranks before Adam, so the weights
    # stay identical on every rank
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    import bench
    import oracle as O
    g = torch.arange(6, dtype=torch.float64) * (1.0 + rank)      # rank-dependent gradients
    bench.grad_allreduce_mean_(g, world)
    w = np.linspace(-1.0, 1.0, 6)
    m, v = np.zeros(6), np.zeros(6)
    O.adam(w, g.numpy().copy(), m, v, 1)
    out[rank] = (g.numpy().tolist(), w.tolist())
    dist.destroy_process_group()


def test_two_ranks_average_gradients():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_train_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    (g0, w0), (g1, w1) = res[0], res[1]
    assert g0 == g1 == pytest.approx([1.5 * k for k in range(6)])
    assert w0 == w1
