"""What training gains (behavioural, not parity): the committed 6 x 64
network, trained on the GPU by this library's own forward, adjoint and Adam
kernels (paper_2305_16432_gb300/train.py) on 128 x 128 FEM systems, needs
fewer PCG iterations than the same network untrained on held-out systems of
any size, and fewer than Jacobi on held-out systems of the training size.
(On a 96 x 96 mesh it is not better than Jacobi: 323 against 289
iterations for seed 9200.)"""
import json
import os

import numpy as np
import pytest
import torch

from paper_2305_16432_gb300 import inputs as I

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2305_16432_gb300", "weights", "fem2d_6x64.npy")


@pytest.fixture(scope="module")
def N():
    from paper_2305_16432_gb300 import build
    build.build()
    from paper_2305_16432_gb300 import npcg
    return npcg


@pytest.mark.parametrize("m,seed,vs_jacobi", [(128, 9100, True), (128, 9300, True), (96, 9200, False)])
def test_trained_beats_untrained_and_jacobi(N, m, seed, vs_jacobi):
    meta = json.load(open(os.path.splitext(WEIGHTS)[0] + ".json"))
    cfg = I.GnnConfig(**meta["config"])
    w = torch.as_tensor(np.load(WEIGHTS), device="cuda")
    w0 = torch.as_tensor(I.gnn_weights(cfg, 2023), device="cuda")
    rp, ci, v = N.assemble_system(I.fem2d(m, sigma=1.0, corr_len=0.1, seed=seed))
    P = N.analyse(rp, ci)
    b = torch.as_tensor(I.rhs(P.n, seed), device="cuda")
    it = {}
    for name, ww in (("trained", w), ("untrained", w0)):
        L = N.gnn_factor(P, v, b, cfg, ww)
        _, st = N.pcg_solve(P, v, b, N.PREC_LLT, L, rtol=1e-6)
        assert st[0]["status"] == 0
        it[name] = st[0]["iters"]
    _, sj = N.pcg_solve(P, v, b, N.PREC_JACOBI, None, rtol=1e-6)
    assert it["trained"] < it["untrained"]
    if vs_jacobi:
        assert it["trained"] < sj[0]["iters"]
