"""The N > 1 paths of bench.py on the CPU (gloo, world size 2): the batch of
256 systems is split over the ranks by the greedy bin-pack on nonzeros (no
data-path collective), the job time is the slowest rank's and the
per-system statistics come back in batch order; for training the ranks
average their gradients before Adam."""
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
    # the real assignment of the one fixed batch of 256 systems
    probs, shard = bench._problems(I, "batched_256", rank, world)
    local_ms = 100.0 + 50.0 * rank                     # ranks finish at different times
    ms = bench.job_ms_per_step(local_ms, world)
    # per-system statistics as the solve returns them (iterations tagged by
    # the system's batch index and the rank that solved it)
    local = [{"iters": 3 * k + 1, "status": 0, "relres": 1e-7, "rank": rank} for k in shard]
    gathered = bench.gather_stats(local, shard, 256, world)
    out[rank] = (list(shard), [p.seed for p in probs], [bench.nnz_estimate(p) for p in probs], ms, gathered)
    dist.destroy_process_group()


def test_two_ranks_shard_one_batch():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    (sh0, seeds0, w0, ms0, g0), (sh1, seeds1, w1, ms1, g1) = res[0], res[1]
    # disjoint shards that cover the batch, each rank solving its own members
    assert not set(sh0) & set(sh1) and sorted(sh0 + sh1) == list(range(256))
    from paper_2305_16432_gb300 import inputs as I
    import bench
    batch = I.batched_mix(256, seed=0)
    assert seeds0 == [batch[k].seed for k in sh0] and seeds1 == [batch[k].seed for k in sh1]
    # balance: the greedy bin-pack keeps every shard within the largest
    # system of the mean load (the largest-first guarantee), here < 1 %
    loads = [sum(w0), sum(w1)]
    mean = sum(loads) / world
    wmax = max(bench.nnz_estimate(p) for p in batch)
    assert max(loads) - mean <= wmax and max(loads) / mean < 1.01
    # the job time is the slowest rank's
    assert ms0 == ms1 == 150.0
    # gathered statistics on every rank, in batch order, each from its solver
    for g in (g0, g1):
        assert [s["iters"] for s in g] == [3 * k + 1 for k in range(256)]
        assert all(s["rank"] == (0 if k in sh0 else 1) for k, s in enumerate(g))


def test_partition_properties():
    import bench
    w = [5, 9, 1, 7, 3, 3, 8, 2]
    for world in (1, 2, 3, 8):
        sh = bench.partition_by_nnz(w, world)
        assert len(sh) == world and sorted(sum(sh, [])) == list(range(len(w)))
        loads = [sum(w[k] for k in s) for s in sh]
        assert max(loads) - sum(w) / world <= max(w)
    # largest first into the lightest shard, ties to the lower rank
    assert bench.partition_by_nnz([4, 3, 3, 2], 2) == [[0, 3], [1, 2]]


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
