"""The committed networks: every weight file matches the parameter count of
the configuration its training record names, and the benchmark picks each
workload's own file (CPU only)."""
import json
import os

import numpy as np
import pytest

import bench
from paper_2305_16432_gb300 import inputs as I

WDIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2305_16432_gb300", "weights")
FILES = sorted(f for f in os.listdir(WDIR) if f.endswith(".npy"))


@pytest.mark.parametrize("fname", FILES)
def test_weights_match_their_config(fname):
    w = np.load(os.path.join(WDIR, fname))
    meta = json.load(open(os.path.join(WDIR, fname[:-4] + ".json")))
    cfg = I.GnnConfig(**meta["config"])
    assert w.dtype == np.float32 and w.ndim == 1 and len(w) == cfg.nparams
    assert np.all(np.isfinite(w))
    w2, kind, meta2, cfg2 = bench._load_weights(I.GnnConfig(n_mp=6, l=2, l_mp=2, h=64), os.path.join(WDIR, fname))
    assert kind == "trained" and len(w2) == len(w) and meta2["config"] == meta["config"] and cfg2 == cfg


def test_bench_picks_each_workloads_network():
    assert os.path.basename(bench.weights_for("fem2d_256")) == "gnn_6x64_fem2d.npy"
    assert os.path.basename(bench.weights_for("heat2d_256")) == "gnn_6x64_heat2d.npy"
    assert os.path.basename(bench.weights_for("batched_256")) == "gnn_6x64.npy"
    assert os.path.basename(bench.weights_for("fem2d_256", x0=True)) == "gnn_6x64_fem2d_x0.npy"
    assert os.path.basename(bench.weights_for("fd3d_128")) == "gnn_6x64_fd3d.npy"
    meta3 = json.load(open(os.path.join(WDIR, "gnn_6x64_fd3d.json")))
    assert meta3["config"]["diag_mode"] == 2 and meta3["bench_iters"]["fd3d_128"] > 0
    meta = json.load(open(os.path.join(WDIR, "gnn_6x64_fem2d_x0.json")))
    assert meta["config"]["x0_head"] == 1


def test_bench_describes_the_library_launch_mode():
    # the library launches a single system's PCG iterations one by one from
    # 2^18 rows (its triangular solves run in row blocks there), and through
    # the loop graph otherwise; --eager-pcg forces one by one
    class A:
        eager_pcg = False
    assert "one by one" in bench.pcg_launch_mode(A(), 128 ** 3, 1)
    assert "one by one" in bench.pcg_launch_mode(A(), 1 << 18, 1)
    assert "graph" in bench.pcg_launch_mode(A(), (1 << 18) - 1, 1)
    assert "graph" in bench.pcg_launch_mode(A(), 28_800_000, 256)
    assert "graph" in bench.pcg_launch_mode(A(), 128 ** 3, 1, "syncfree")
    assert "one by one" in bench.pcg_launch_mode(A(), 128 ** 3, 1, "levelmerge")
    A.eager_pcg = True
    assert "forced" in bench.pcg_launch_mode(A(), 256 * 256, 1)
