"""GPU parity at the full sizes of the method's workloads, in the launch
configuration the benchmark times (BF16 network, FP32 triangular solves
inside FP64 PCG) as well as the FP32/FP64 parity path.

What the oracle cannot run in seconds at these sizes is checked on samples
it computes one by one, or through properties that hold at any size:
  - network rows: the oracle evaluates sampled rows of L on their
    (n_mp + 1)-hop neighbourhood with the full system's input scales
    (exact by the receptive field of n_mp message-passing rounds, pinned on
    the CPU by test_gnn_rows_on_neighbourhood_balls);
  - PCG: the true residual ||b - A x|| / ||b|| of every system, evaluated by
    the oracle's SpMV, is at most rtol (1 + 1e-3): the recurrence residual
    that stops Algorithm 1 and the true one differ by rounding only;
  - sampled members of the 256-system batch are solved whole by the oracle.
Bars: FP32 L 1e-5, BF16 L 2e-2 (relative, over the sampled entries); with
IC(0), FP64 x 1e-8 and iterations +-1; with a learned factor that needs
hundreds of iterations, the oracle's own spread under another summation
order (iterations 3 %, x after the same number of updates 1e-6); BF16-network
/ FP32-apply iterations +-10 %.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2305_16432_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2305_16432_gb300", "weights", "gnn_6x64.npy")


@pytest.fixture(scope="module")
def N():
    from paper_2305_16432_gb300 import build
    build.build()
    from paper_2305_16432_gb300 import npcg
    torch.cuda.init()
    return npcg


@pytest.fixture(scope="module")
def net():
    meta = json.load(open(os.path.splitext(WEIGHTS)[0] + ".json"))
    return I.GnnConfig(**meta["config"]), np.load(WEIGHTS).astype(np.float32)


def _np(t):
    return t.detach().cpu().numpy()


def _gpu(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _sample_rows(n, k, seed):
    g = np.random.default_rng(seed)
    return sorted(set(g.choice(n, size=k, replace=False).tolist()) | {0, n - 1})


def _check_rows(Ao, Lg_val, b, cfg, w, rows, tol):
    """Sampled rows of the GPU L (values on the tril pattern) against the oracle."""
    Lo_pat, _ = O.tril(Ao, with_values=False)
    ref = O.gnn_rows(cfg, Ao, b, w.astype(np.float64), rows)
    got, exp = [], []
    for r in rows:
        s, e = Lo_pat.row_ptr[r], Lo_pat.row_ptr[r + 1]
        cols, vals = ref[r]
        assert np.array_equal(cols, Lo_pat.col_idx[s:e])
        got.append(Lg_val[s:e])
        exp.append(vals)
    got, exp = np.concatenate(got), np.concatenate(exp)
    assert np.linalg.norm(got - exp) <= tol * np.linalg.norm(exp)
    assert np.abs(got - exp).max() <= tol * np.abs(exp).max()


def _true_relres(Ao, x, b):
    return np.linalg.norm(b - O.spmv(Ao, x)) / np.linalg.norm(b)


def test_fem256_learned_full_size(N, net):
    """The 256 x 256 FEM workload with the trained network: sampled rows of L
    (FP32 and BF16), FP64 PCG with the network's L against the oracle's PCG
    on the same L, and the benchmark's configuration (BF16 network, FP32
    apply) converging within 10 % of the oracle's iterations."""
    cfg, w = net
    p = I.fem2d_256()
    Ao = O.assemble(p)
    rp, ci, v = N.assemble_system(p)
    P = N.analyse(rp, ci)
    b = I.rhs(Ao.n, 0)
    bg, wg = _gpu(b), _gpu(w, torch.float32)
    rows = _sample_rows(Ao.n, 40, 1)
    L32 = N.gnn_factor(P, v, bg, cfg, wg, precision=N.FP32)
    L16 = N.gnn_factor(P, v, bg, cfg, wg, precision=N.BF16)
    _check_rows(Ao, _np(L32), b, cfg, w, rows, 1e-5)
    _check_rows(Ao, _np(L16), b, cfg, w, rows, 2e-2)
    Lpat, _ = O.tril(Ao, with_values=False)
    Lo = O.CSR(Lpat.row_ptr, Lpat.col_idx, _np(L32))
    xo, ito, _, sto = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-6)
    assert sto == 0
    xg, st = N.pcg_solve(P, v, bg, N.PREC_LLT, L32, rtol=1e-6)
    # a learned factor needing hundreds of iterations: the bars are the
    # oracle's own spread under another summation order (3 % of the
    # iterations; x after the same number of updates within 1e-6, pinned by
    # test_pcg_iteration_spread_learned_factor)
    assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= max(1, int(np.ceil(0.03 * ito)))
    assert _true_relres(Ao, _np(xg), b) <= 1e-6 * (1 + 1e-3)
    xk, sk = N.pcg_solve(P, v, bg, N.PREC_LLT, L32, rtol=0.0, max_iter=ito)
    assert sk[0]["iters"] == ito
    assert np.linalg.norm(_np(xk) - xo) / np.linalg.norm(xo) <= 1e-6
    xb, sb = N.pcg_solve(P, v, bg, N.PREC_LLT32, L16, rtol=1e-6)
    assert sb[0]["status"] == 0 and abs(sb[0]["iters"] - ito) <= 0.1 * ito
    assert _true_relres(Ao, _np(xb), b) <= 1e-6 * (1 + 1e-3)


def test_fd3d_128_full_size(N, net):
    """128^3 variable-coefficient FD (n = 2,097,152): assembly, levels (382,
    bit-exact), IC(0), IC(0)-PCG against the oracle, sampled rows of the
    network's L, and learned / Jacobi PCG converging in true residual."""
    cfg, w = net
    p = I.fd3d_128()
    Ao = O.assemble(p)
    rp, ci, v = N.assemble_system(p)
    assert np.array_equal(_np(rp), Ao.row_ptr) and np.array_equal(_np(ci), Ao.col_idx)
    assert _rel(_np(v), Ao.val) <= 1e-12
    P = N.analyse(rp, ci)
    Lo, _ = O.tril(Ao)
    lev, nf, levb, nb = O.levels(Lo)
    assert nf == 382 and nb == 382 and P.nlev_fwd == 382
    ex = P.export()
    assert np.array_equal(_np(ex["lev_fwd"]), lev) and np.array_equal(_np(ex["lev_bwd"]), levb)
    Lic, _ = O.ic0(Ao)
    Lg, _ = N.ic0_factor(P, v)
    assert _rel(_np(Lg), Lic.val) <= 1e-12
    b = I.rhs(Ao.n, 0)
    bg = _gpu(b)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lic, rtol=1e-6)
    xg, st = N.pcg_solve(P, v, bg, N.PREC_LLT, Lg, rtol=1e-6)
    assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(_np(xg) - xo) / np.linalg.norm(xo) <= 1e-8
    wg = _gpu(w, torch.float32)
    rows = _sample_rows(Ao.n, 24, 2)
    L32 = N.gnn_factor(P, v, bg, cfg, wg, precision=N.FP32)
    _check_rows(Ao, _np(L32), b, cfg, w, rows, 1e-5)
    L16 = N.gnn_factor(P, v, bg, cfg, wg, precision=N.BF16)
    _check_rows(Ao, _np(L16), b, cfg, w, rows, 2e-2)
    del L32
    for pc, L in ((N.PREC_LLT32, L16), (N.PREC_JACOBI, None)):
        x, s = N.pcg_solve(P, v, bg, pc, L, rtol=1e-6)
        assert s[0]["status"] == 0
        assert _true_relres(Ao, _np(x), b) <= 1e-6 * (1 + 1e-3)


def test_batched_256_full_size(N, net):
    """The uneven batch of 256 systems (2-D FEM n ~ U[4k, 260k], 3-D FD
    16^3..64^3; sum n ~ 28 M) in one batched solve: IC(0) and the trained
    BF16 network, every member converging; sampled members against the
    oracle (whole solves and network rows)."""
    cfg, w = net
    probs = I.batched_mix(256, seed=0)
    rps, cis, vs, bs, sys_ptr = [], [], [], [], [0]
    off_n = off_nnz = 0
    for k, p in enumerate(probs):
        rp, ci, v = N.assemble_system(p)
        n = rp.numel() - 1
        rps.append(rp[:-1] + off_nnz)
        cis.append(ci + off_n)
        vs.append(v)
        bs.append(I.rhs(n, 700 + k))
        off_n += n
        off_nnz += ci.numel()
        sys_ptr.append(off_n)
    rp_cat = torch.cat(rps + [torch.tensor([off_nnz], dtype=torch.int32, device="cuda")])
    ci_cat, v_cat = torch.cat(cis), torch.cat(vs)
    del rps, cis, vs
    P = N.analyse(rp_cat, ci_cat, sys_ptr)
    assert P.nsys == 256 and P.n == off_n and off_n > 20_000_000
    b_cat = _gpu(np.concatenate(bs))
    Lic, _ = N.ic0_factor(P, v_cat)
    xi, sti = N.pcg_solve(P, v_cat, b_cat, N.PREC_LLT32, Lic, rtol=1e-6)
    assert all(s["status"] == 0 and s["relres"] <= 1e-6 for s in sti)
    L16 = N.gnn_factor(P, v_cat, b_cat, cfg, _gpu(w, torch.float32), precision=N.BF16)
    xl, stl = N.pcg_solve(P, v_cat, b_cat, N.PREC_LLT32, L16, rtol=1e-6)
    assert all(s["status"] == 0 and s["relres"] <= 1e-6 for s in stl)
    # true residual of every member, by the oracle's SpMV on the concatenation
    A_cat = O.CSR(_np(rp_cat), _np(ci_cat), _np(v_cat))
    bh, xih, xlh = np.concatenate(bs), _np(xi), _np(xl)
    ri, rl = bh - O.spmv(A_cat, xih), bh - O.spmv(A_cat, xlh)
    for k in range(256):
        s, e = sys_ptr[k], sys_ptr[k + 1]
        nb = np.linalg.norm(bh[s:e])
        assert np.linalg.norm(ri[s:e]) <= 1e-6 * (1 + 1e-3) * nb
        assert np.linalg.norm(rl[s:e]) <= 1e-6 * (1 + 1e-3) * nb
    # the three smallest members, solved whole by the oracle (FP64 apply)
    sizes = np.diff(sys_ptr)
    small = [int(k) for k in np.argsort(sizes, kind="stable")[:3]]
    x64, st64 = N.pcg_solve(P, v_cat, b_cat, N.PREC_LLT, Lic, rtol=1e-6)
    x64 = _np(x64)
    Lic_h = _np(Lic)
    Lpat_cat, _ = O.tril(A_cat, with_values=False)
    for k in small:
        Ao = O.assemble(probs[k])
        Lo, _ = O.ic0(Ao)
        s0 = Lpat_cat.row_ptr[sys_ptr[k]]
        assert _rel(Lic_h[s0:s0 + Lo.nnz], Lo.val) <= 1e-12
        xo, ito, _, _ = O.pcg(Ao, bs[k], O.PREC_LLT, Lo, rtol=1e-6)
        assert abs(st64[k]["iters"] - ito) <= 1
        seg = x64[sys_ptr[k]:sys_ptr[k + 1]]
        assert np.linalg.norm(seg - xo) / np.linalg.norm(xo) <= 1e-8
    # network rows of one 2-D and one 3-D member, sampled
    L16h = _np(L16)
    for k in (small[0], 0):
        Ao = O.assemble(probs[k])
        s0 = Lpat_cat.row_ptr[sys_ptr[k]]
        Lk = L16h[s0:s0 + (Ao.nnz + Ao.n) // 2]
        _check_rows(Ao, Lk, bs[k], cfg, w, _sample_rows(Ao.n, 12, 3 + k), 2e-2)
