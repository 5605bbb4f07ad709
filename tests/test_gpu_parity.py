"""GPU parity: every step of the hot path through the C ABI, element by
element against the FP64 oracle on the same seeded inputs.

Tolerances (bars of the method's parity contract):
  patterns, levels, permutations    bit-exact
  assembled A                       1e-12 relative (GPU exp/cos differ by ulps)
  SpMV / SpTRSV / IC(0) values      1e-12 relative
  PCG x (same factor)               1e-8 relative, iterations +-1
  FP32 GNN L                        ||dL||_F / ||L||_F <= 1e-5 and max|dL| <= 1e-5 max|L|
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2305_16432_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_2305_16432_gb300 import build
    build.build()
    from paper_2305_16432_gb300 import npcg
    torch.cuda.init()
    return npcg


def _np(t):
    return t.detach().cpu().numpy()


def _gpu(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


PROBLEMS = {
    "poisson2d_32": I.poisson2d_32(),
    "fd2d_var": I.fd2d(23, 17, sigma=1.0, seed=3),
    "fd3d_var": I.fd3d(9, 8, 7, sigma=1.5, corr_len=0.05, seed=4),
    "fem34": I.fem2d(34, sigma=1.0, seed=5),
    "fem_nojit": I.fem2d(20, sigma=0.0, seed=0),
}


def _assemble_both(N, prob, jitter=None):
    if prob.kind == I.FEM and jitter is None:
        jitter = I.fem_jitter(prob)
    om, ph = I.grf_features(prob)
    Ao = O.assemble(prob, om, ph, jitter)
    rp, ci, v = N.assemble_system(prob, om, ph, jitter)
    return Ao, (rp, ci, v)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_assembly_parity(N, name):
    Ao, (rp, ci, v) = _assemble_both(N, PROBLEMS[name])
    assert np.array_equal(_np(rp), Ao.row_ptr)
    assert np.array_equal(_np(ci), Ao.col_idx)
    assert _rel(_np(v), Ao.val) <= 1e-12


def test_assembly_zero_jitter_pattern(N):
    # tie case of the in-circle predicate and the dropped cot(90) edges
    p = I.fem2d(18, sigma=0.0)
    Ao, (rp, ci, v) = _assemble_both(N, p, I.zero_jitter(18))
    assert np.array_equal(_np(rp), Ao.row_ptr) and np.array_equal(_np(ci), Ao.col_idx)
    assert _rel(_np(v), Ao.val) <= 1e-12


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_pattern_and_levels_bit_exact(N, name):
    Ao, (rp, ci, v) = _assemble_both(N, PROBLEMS[name])
    P = N.analyse(rp, ci)
    ex = P.export()
    Lo, _ = O.tril(Ao)
    lev, nf, levb, nb = O.levels(Lo)
    assert np.array_equal(_np(ex["L_row_ptr"]), Lo.row_ptr)
    assert np.array_equal(_np(ex["L_col_idx"]), Lo.col_idx)
    assert np.array_equal(_np(ex["lev_fwd"]), lev)
    assert np.array_equal(_np(ex["lev_bwd"]), levb)
    assert P.nlev_fwd == nf and P.nlev_bwd == nb
    perm, _ = O.level_perm(lev, nf)
    permb, _ = O.level_perm(levb, nb)
    assert np.array_equal(_np(ex["perm_fwd"]), perm)
    assert np.array_equal(_np(ex["perm_bwd"]), permb)
    assert P.nnz_L == Lo.nnz == (Ao.nnz + Ao.n) // 2


def test_levels_closed_form_grid(N):
    # 2-D natural order: nx + ny - 1 levels; 3-D: nx + ny + nz - 2
    Ao, (rp, ci, v) = _assemble_both(N, I.fd3d(20, 15, 11))
    P = N.analyse(rp, ci)
    assert P.nlev_fwd == P.nlev_bwd == 20 + 15 + 11 - 2


@pytest.mark.parametrize("name", ["fem34", "fd3d_var"])
def test_spmv_parity(N, name):
    Ao, (rp, ci, v) = _assemble_both(N, PROBLEMS[name])
    P = N.analyse(rp, ci)
    x = np.random.default_rng(1).standard_normal(Ao.n)
    y = N.spmv(P, v, _gpu(x))
    assert _rel(_np(y), O.spmv(Ao, x)) <= 1e-12


@pytest.mark.parametrize("name", ["poisson2d_32", "fem34", "fd3d_var"])
def test_ic0_and_sptrsv_parity(N, name):
    Ao, (rp, ci, v) = _assemble_both(N, PROBLEMS[name])
    P = N.analyse(rp, ci)
    Lo, alpha_o = O.ic0(Ao)
    Lg, alpha_g = N.ic0_factor(P, v)
    assert alpha_g[0] == alpha_o
    assert _rel(_np(Lg), Lo.val) <= 1e-12
    # triangular solves with the oracle's factor
    N.factor_load(P, _gpu(Lo.val))
    r = np.random.default_rng(2).standard_normal(Ao.n)
    y = N.sptrsv(P, _gpu(r), transpose=False)
    assert _rel(_np(y), O.trsv_lower(Lo, r)) <= 1e-12
    z = N.sptrsv(P, _gpu(r), transpose=True)
    assert _rel(_np(z), O.trsv_upper(Lo, r)) <= 1e-12


def iter_tol(prec, iters):
    """Iteration-count bar: +-1 for IC(0) and Jacobi; for plain CG and for
    learned factors the spread the oracle's own recurrence shows under other
    summation orders (tests/test_oracle_solvers.py::
    test_cg_iteration_spread_under_summation_order and
    test_pcg_iteration_spread_learned_factor): 1 % and 3 % of the count."""
    if prec == "cg":
        return max(1, int(np.ceil(0.01 * iters)))
    if prec == "learned":
        return max(1, int(np.ceil(0.03 * iters)))
    return 1


@pytest.mark.parametrize("name", ["poisson2d_32", "fem34", "fd3d_var", "fd2d_var"])
@pytest.mark.parametrize("prec", ["cg", "jacobi", "ic0"])
def test_pcg_parity(N, name, prec):
    Ao, (rp, ci, v) = _assemble_both(N, PROBLEMS[name])
    P = N.analyse(rp, ci)
    b = I.rhs(Ao.n, 7)
    Lo = None
    if prec == "ic0":
        Lo, _ = O.ic0(Ao)
    pc = {"cg": O.PREC_NONE, "jacobi": O.PREC_JACOBI, "ic0": O.PREC_LLT}[prec]
    Lg = _gpu(Lo.val) if Lo is not None else None
    xo, ito, rro, sto = O.pcg(Ao, b, pc, Lo, rtol=1e-8)
    xg, st = N.pcg_solve(P, v, _gpu(b), pc, Lg, rtol=1e-8)
    assert sto == 0 and st[0]["status"] == 0
    assert abs(st[0]["iters"] - ito) <= iter_tol(prec, ito)
    assert st[0]["relres"] <= 1e-8
    true_res = np.linalg.norm(b - O.spmv(Ao, _np(xg))) / np.linalg.norm(b)
    assert true_res <= 2e-8
    # the same number of updates: the iterates agree to 1e-8
    xk, stk = N.pcg_solve(P, v, _gpu(b), pc, Lg, rtol=0.0, max_iter=ito)
    assert stk[0]["iters"] == ito
    assert np.linalg.norm(_np(xk) - xo) / np.linalg.norm(xo) <= 1e-8


def test_pcg_edge_cases(N):
    Ao, (rp, ci, v) = _assemble_both(N, I.fd2d(9, 7))
    P = N.analyse(rp, ci)
    x, st = N.pcg_solve(P, v, torch.zeros(Ao.n, dtype=torch.float64, device="cuda"), N.PREC_NONE)
    assert st[0]["iters"] == 0 and st[0]["status"] == 0 and float(x.abs().max()) == 0.0
    b = I.rhs(Ao.n, 3)
    x, st = N.pcg_solve(P, v, _gpu(b), N.PREC_NONE, rtol=1e-14, max_iter=3)
    assert st[0]["status"] == N.NPCG_EMAXITER and st[0]["iters"] == 3
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_NONE, rtol=1e-14, max_iter=3)
    assert np.allclose(_np(x), xo, rtol=1e-10, atol=1e-12)
    # x0 = exact solution: nothing to do
    xs = np.linalg.solve(Ao.dense(), b)
    x, st = N.pcg_solve(P, v, _gpu(b), N.PREC_NONE, rtol=1e-6, x0=_gpu(xs))
    assert st[0]["iters"] == 0
    # single unknown
    rp1 = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    ci1 = torch.tensor([0], dtype=torch.int32, device="cuda")
    P1 = N.analyse(rp1, ci1)
    x, st = N.pcg_solve(P1, _gpu([4.0]), _gpu([2.0]), N.PREC_JACOBI, rtol=1e-12)
    assert st[0]["iters"] == 1 and abs(float(x[0]) - 0.5) < 1e-15


def test_malformed_patterns_rejected(N):
    def csr(rows):
        rp, ci = [0], []
        for r in rows:
            ci += r
            rp.append(len(ci))
        return (torch.tensor(rp, dtype=torch.int32, device="cuda"),
                torch.tensor(ci, dtype=torch.int32, device="cuda"))
    bad = {
        "unsorted": [[0, 1], [1, 0]],
        "missing diagonal": [[0, 1], [0]],
        "asymmetric": [[0, 1], [1]],
        "out of range": [[0, 5], [1]],
    }
    for name, rows in bad.items():
        rp, ci = csr(rows)
        with pytest.raises(N.NpcgError):
            N.analyse(rp, ci)


@pytest.mark.parametrize("cfg,prob", [
    (I.GnnConfig(n_mp=2, l=2, l_mp=2, h=16), I.poisson2d_32()),
    (I.GnnConfig(n_mp=6, l=2, l_mp=2, h=64), I.fem2d(22, sigma=1.0, seed=9)),
    (I.GnnConfig(n_mp=3, l=1, l_mp=3, h=32), I.fd3d(7, 6, 5, sigma=1.0, seed=2)),
    (I.GnnConfig(n_mp=0, l=2, l_mp=2, h=16), I.fd2d(12, 9, sigma=1.0, seed=1)),
    (I.GnnConfig(n_mp=3, l=2, l_mp=2, h=64, diag_mode=1), I.fem2d(18, sigma=1.0, seed=3)),
    (I.GnnConfig(n_mp=3, l=2, l_mp=2, h=64, diag_mode=2), I.fd3d(9, 8, 7, sigma=1.5, corr_len=0.2, seed=3)),
    (I.GnnConfig(n_mp=2, l=2, l_mp=2, h=32, diag_mode=2), I.fem2d(20, sigma=1.0, seed=4)),
])
def test_gnn_fp32_parity(N, cfg, prob):
    Ao, (rp, ci, v) = _assemble_both(N, prob)
    P = N.analyse(rp, ci)
    b = I.rhs(Ao.n, 11)
    w = I.gnn_weights(cfg, 1)
    Lo = O.gnn_forward(cfg, Ao, b, w)
    Lg = _np(N.gnn_factor(P, v, _gpu(b), cfg, _gpu(w, torch.float32)))
    d = Lg - Lo.val
    assert np.linalg.norm(d) / np.linalg.norm(Lo.val) <= 1e-5
    assert np.abs(d).max() <= 1e-5 * np.abs(Lo.val).max()


def test_learned_pcg_parity(N):
    # the oracle's learned factor through the GPU PCG, and the GPU factor's
    # iteration count against the oracle's
    cfg = I.GnnConfig(n_mp=2, l=2, l_mp=2, h=16)
    Ao, (rp, ci, v) = _assemble_both(N, I.poisson2d_32())
    P = N.analyse(rp, ci)
    b = I.rhs(Ao.n, 0)
    w = I.gnn_weights(cfg, 1)
    Lo = O.gnn_forward(cfg, Ao, b, w)
    xo, ito, _, sto = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    xg, st = N.pcg_solve(P, v, _gpu(b), N.PREC_LLT, _gpu(Lo.val), rtol=1e-8)
    assert abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(_np(xg) - xo) / np.linalg.norm(xo) <= 1e-8
    Lg = N.gnn_factor(P, v, _gpu(b), cfg, _gpu(w, torch.float32))
    xg2, st2 = N.pcg_solve(P, v, _gpu(b), N.PREC_LLT, Lg, rtol=1e-8)
    assert abs(st2[0]["iters"] - ito) <= 1


def test_batched_matches_individual(N):
    probs = [I.fem2d(20, sigma=1.0, seed=1), I.fd3d(6, 5, 4, sigma=1.0, seed=2), I.fd2d(13, 11, sigma=1.0, seed=3)]
    As, rps, cis, vs, bs = [], [], [], [], []
    off = 0
    sys_ptr = [0]
    for k, p in enumerate(probs):
        Ao, (rp, ci, v) = _assemble_both(N, p)
        As.append(Ao)
        cis.append(_np(ci) + off)
        vs.append(_np(v))
        bs.append(I.rhs(Ao.n, 20 + k))
        off += Ao.n
        sys_ptr.append(off)
    nnz_off = np.cumsum([0] + [a.nnz for a in As])
    rp_cat = np.concatenate([a.row_ptr[:-1] + nnz_off[k] for k, a in enumerate(As)] + [[nnz_off[-1]]])
    P = N.analyse(_gpu(rp_cat, torch.int32), _gpu(np.concatenate(cis), torch.int32), sys_ptr)
    v_cat = _gpu(np.concatenate(vs))
    b_cat = np.concatenate(bs)
    Lg, alpha = N.ic0_factor(P, v_cat)
    for prec in (N.PREC_NONE, N.PREC_LLT):
        x, st = N.pcg_solve(P, v_cat, _gpu(b_cat), prec, Lg if prec == N.PREC_LLT else None, rtol=1e-8)
        xs = _np(x)
        for k, Ao in enumerate(As):
            Lo = O.ic0(Ao)[0] if prec == N.PREC_LLT else None
            xo, ito, _, _ = O.pcg(Ao, bs[k], prec, Lo, rtol=1e-8)
            assert st[k]["status"] == 0
            assert abs(st[k]["iters"] - ito) <= 1
            seg = xs[sys_ptr[k]:sys_ptr[k + 1]]
            assert np.linalg.norm(seg - xo) / np.linalg.norm(xo) <= 1e-8


def test_solve_host_matches_device_path(N):
    Ao, (rp, ci, v) = _assemble_both(N, PROBLEMS["fem34"])
    P = N.analyse(rp, ci)
    b = I.rhs(Ao.n, 5)
    xh, st = N.solve_host(P, Ao.val.copy(), b.copy(), method=N.METHOD_IC0, rtol=1e-8)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, O.ic0(Ao)[0], rtol=1e-8)
    assert abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(xh - xo) / np.linalg.norm(xo) <= 1e-8


def test_fem256_full_size(N):
    # the 256 x 256 FEM workload: assembly, levels and the IC(0)-PCG solve
    p = I.fem2d_256()
    Ao, (rp, ci, v) = _assemble_both(N, p)
    assert np.array_equal(_np(ci), Ao.col_idx) and _rel(_np(v), Ao.val) <= 1e-12
    P = N.analyse(rp, ci)
    Lo, _ = O.tril(Ao)
    lev, nf, levb, nb = O.levels(Lo)
    ex = P.export()
    assert np.array_equal(_np(ex["lev_fwd"]), lev) and np.array_equal(_np(ex["lev_bwd"]), levb)
    Lic, _ = O.ic0(Ao)
    Lg, _ = N.ic0_factor(P, v)
    assert _rel(_np(Lg), Lic.val) <= 1e-12
    b = I.rhs(Ao.n, 0)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lic, rtol=1e-6)
    xg, st = N.pcg_solve(P, v, _gpu(b), N.PREC_LLT, Lg, rtol=1e-6)
    assert abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(_np(xg) - xo) / np.linalg.norm(xo) <= 1e-8


_MODE = {"syncfree": "TRSV_SYNCFREE", "levelsync": "TRSV_LEVELSYNC", "levelsplit": "TRSV_LEVELSPLIT"}


def _set_mode(N, P, mode):
    P.set_trsv(getattr(N, _MODE[mode]))


@pytest.mark.parametrize("mode", ["syncfree", "levelsync", "levelsplit"])
@pytest.mark.parametrize("name", ["poisson2d_32", "fem34", "fd3d_var"])
def test_trsv_designs_parity(N, name, mode):
    # the triangular-solve designs against the oracle, alone and inside PCG
    Ao, (rp, ci, v) = _assemble_both(N, PROBLEMS[name])
    P = N.analyse(rp, ci)
    _set_mode(N, P, mode)
    Lo, _ = O.ic0(Ao)
    N.factor_load(P, _gpu(Lo.val))
    r = np.random.default_rng(5).standard_normal(Ao.n)
    assert _rel(_np(N.sptrsv(P, _gpu(r))), O.trsv_lower(Lo, r)) <= 1e-12
    assert _rel(_np(N.sptrsv(P, _gpu(r), transpose=True)), O.trsv_upper(Lo, r)) <= 1e-12
    b = I.rhs(Ao.n, 8)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    xg, st = N.pcg_solve(P, v, _gpu(b), N.PREC_LLT, _gpu(Lo.val), rtol=1e-8)
    assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(_np(xg) - xo) / np.linalg.norm(xo) <= 1e-8


@pytest.mark.parametrize("mode", ["syncfree", "levelsync", "levelsplit"])
def test_batched_trsv_designs(N, mode):
    probs = [I.fem2d(26, sigma=1.0, seed=11), I.fd3d(7, 6, 5, sigma=1.0, seed=12), I.fd2d(17, 9, sigma=1.0, seed=13),
             I.fem2d(12, sigma=1.0, seed=14)]
    As, cis, vs, bs = [], [], [], []
    off, sys_ptr = 0, [0]
    for k, p in enumerate(probs):
        Ao, (rp, ci, v) = _assemble_both(N, p)
        As.append(Ao)
        cis.append(_np(ci) + off)
        vs.append(_np(v))
        bs.append(I.rhs(Ao.n, 40 + k))
        off += Ao.n
        sys_ptr.append(off)
    nnz_off = np.cumsum([0] + [a.nnz for a in As])
    rp_cat = np.concatenate([a.row_ptr[:-1] + nnz_off[k] for k, a in enumerate(As)] + [[nnz_off[-1]]])
    P = N.analyse(_gpu(rp_cat, torch.int32), _gpu(np.concatenate(cis), torch.int32), sys_ptr)
    _set_mode(N, P, mode)
    v_cat = _gpu(np.concatenate(vs))
    Lg, _ = N.ic0_factor(P, v_cat)
    x, st = N.pcg_solve(P, v_cat, _gpu(np.concatenate(bs)), N.PREC_LLT, Lg, rtol=1e-8)
    xs = _np(x)
    for k, Ao in enumerate(As):
        xo, ito, _, _ = O.pcg(Ao, bs[k], O.PREC_LLT, O.ic0(Ao)[0], rtol=1e-8)
        assert st[k]["status"] == 0 and abs(st[k]["iters"] - ito) <= 1
        seg = xs[sys_ptr[k]:sys_ptr[k + 1]]
        assert np.linalg.norm(seg - xo) / np.linalg.norm(xo) <= 1e-8


@pytest.mark.parametrize("mode", ["syncfree", "levelsync", "levelsplit"])
@pytest.mark.parametrize("name", ["fem34", "fd3d_var"])
def test_fp32_preconditioner_apply(N, name, mode):
    # P = L' L'^T with L' = fl32(L), solves in FP32: the PCG recurrences stay
    # FP64, so the solve still reaches the FP64 tolerance; the iteration count
    # stays within 5 % of the FP64-preconditioned oracle
    Ao, (rp, ci, v) = _assemble_both(N, PROBLEMS[name])
    P = N.analyse(rp, ci)
    _set_mode(N, P, mode)
    Lo, _ = O.ic0(Ao)
    b = I.rhs(Ao.n, 9)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    xg, st = N.pcg_solve(P, v, _gpu(b), N.PREC_LLT32, _gpu(Lo.val), rtol=1e-8)
    assert st[0]["status"] == 0
    assert abs(st[0]["iters"] - ito) <= max(1, int(np.ceil(0.05 * ito)))
    assert np.linalg.norm(b - O.spmv(Ao, _np(xg))) / np.linalg.norm(b) <= 2e-8


@pytest.mark.parametrize("prob", [I.fem2d(22, sigma=1.0, seed=9), I.fd3d(9, 8, 7, sigma=1.0, seed=2),
                                  I.poisson2d_32()])
@pytest.mark.parametrize("diag_mode", [0, 1, 2])
def test_gnn_bf16_parity(N, prob, diag_mode):
    # BF16 tensor-core MLPs with FP32 accumulation: L within 2e-2 of the FP64
    # oracle in relative Frobenius norm and in max-abs relative to max |L|
    cfg = I.GnnConfig(n_mp=6, l=2, l_mp=2, h=64, diag_mode=diag_mode)
    Ao, (rp, ci, v) = _assemble_both(N, prob)
    P = N.analyse(rp, ci)
    b = I.rhs(Ao.n, 12)
    w = I.gnn_weights(cfg, 4)
    Lo = O.gnn_forward(cfg, Ao, b, w)
    Lb = _np(N.gnn_factor(P, v, _gpu(b), cfg, _gpu(w, torch.float32), precision=N.BF16))
    d = Lb - Lo.val
    assert np.linalg.norm(d) / np.linalg.norm(Lo.val) <= 2e-2
    assert np.abs(d).max() <= 2e-2 * np.abs(Lo.val).max()
    # and the preconditioner it gives: iterations within 10 % of the FP64 factor's
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-6)
    xg, st = N.pcg_solve(P, v, _gpu(b), N.PREC_LLT, _gpu(Lb), rtol=1e-6)
    assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= max(1, int(np.ceil(0.1 * ito)))


def test_batched_uneven_48_systems_sampled(N):
    # 48 systems of uneven size (2-D FEM and 3-D FD, the mix of the batched
    # workload at reduced sizes) in one batched solve under the device-side
    # loop; every member converges, and sampled members match the oracle
    probs = I.batched_mix(48, seed=3, n_lo=300, n_hi=3000, s_lo=5, s_hi=12)
    rps, cis, vs, bs, sys_ptr = [], [], [], [], [0]
    off_n = off_nnz = 0
    for k, p in enumerate(probs):
        rp, ci, v = N.assemble_system(p)
        rps.append(_np(rp)[:-1] + off_nnz)
        cis.append(_np(ci) + off_n)
        vs.append(_np(v))
        n = rp.numel() - 1
        bs.append(I.rhs(n, 500 + k))
        off_n += n
        off_nnz += ci.numel()
        sys_ptr.append(off_n)
    P = N.analyse(_gpu(np.concatenate(rps + [[off_nnz]]), torch.int32), _gpu(np.concatenate(cis), torch.int32),
                  sys_ptr)
    assert P.nsys == 48
    v_cat = _gpu(np.concatenate(vs))
    Lg, alpha = N.ic0_factor(P, v_cat)
    x, st = N.pcg_solve(P, v_cat, _gpu(np.concatenate(bs)), N.PREC_LLT, Lg, rtol=1e-8)
    assert all(s["status"] == 0 and s["relres"] <= 1e-8 for s in st)
    xs = _np(x)
    for k in (0, 1, 17, 46, 47):
        Ao = O.assemble(probs[k])
        xo, ito, _, _ = O.pcg(Ao, bs[k], O.PREC_LLT, O.ic0(Ao)[0], rtol=1e-8)
        assert abs(st[k]["iters"] - ito) <= 1
        seg = xs[sys_ptr[k]:sys_ptr[k + 1]]
        assert np.linalg.norm(seg - xo) / np.linalg.norm(xo) <= 1e-8


def test_blocked_level_synchronous_solve(N):
    # one system of 2^18 rows (64^3 FD) is laid out in per-SM row blocks:
    # dependencies inside a block use the shared window, the others are read
    # from the rows the earlier blocks publish; both solves against the
    # oracle, and PCG with IC(0) in both designs
    Ao, (rp, ci, v) = _assemble_both(N, I.fd3d(64, sigma=1.0, corr_len=0.1, seed=21))
    assert Ao.n == 1 << 18
    P = N.analyse(rp, ci)
    P.set_trsv(N.TRSV_LEVELSYNC)
    Lo, _ = O.ic0(Ao)
    N.factor_load(P, _gpu(Lo.val))
    r = np.random.default_rng(6).standard_normal(Ao.n)
    assert _rel(_np(N.sptrsv(P, _gpu(r))), O.trsv_lower(Lo, r)) <= 1e-12
    assert _rel(_np(N.sptrsv(P, _gpu(r), transpose=True)), O.trsv_upper(Lo, r)) <= 1e-12
    b = I.rhs(Ao.n, 9)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    for mode in (N.TRSV_LEVELSYNC, N.TRSV_SYNCFREE):
        P.set_trsv(mode)
        xg, st = N.pcg_solve(P, v, _gpu(b), N.PREC_LLT, _gpu(Lo.val), rtol=1e-8)
        assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= 1
        assert np.linalg.norm(_np(xg) - xo) / np.linalg.norm(xo) <= 1e-8
    # FP32 apply: the bar of test_fp32_preconditioner_apply
    P.set_trsv(N.TRSV_LEVELSYNC)
    x32, s32 = N.pcg_solve(P, v, _gpu(b), N.PREC_LLT32, _gpu(Lo.val), rtol=1e-8)
    assert s32[0]["status"] == 0 and abs(s32[0]["iters"] - ito) <= max(1, int(np.ceil(0.05 * ito)))
    assert np.linalg.norm(b - O.spmv(Ao, _np(x32))) / np.linalg.norm(b) <= 2e-8


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16", 2e-2)])
def test_x0_head_parity(N, prec, tol):
    # initial-guess head: x0 against the oracle's, the factor unchanged by the
    # head, and PCG started from x0 reaching the tolerance
    cfg = I.GnnConfig(n_mp=3, l=2, l_mp=2, h=64, diag_mode=1, x0_head=1)
    Ao, (rp, ci, v) = _assemble_both(N, I.fem2d(20, sigma=1.0, seed=15))
    P = N.analyse(rp, ci)
    b = I.rhs(Ao.n, 15)
    w = I.gnn_weights(cfg, 7)
    pc = N.FP32 if prec == "fp32" else N.BF16
    L, x0 = N.gnn_factor_x0(P, v, _gpu(b), cfg, _gpu(w, torch.float32), precision=pc)
    xo = O.gnn_x0(cfg, Ao, b, w.astype(np.float64))
    d = _np(x0) - xo
    assert np.linalg.norm(d) <= tol * np.linalg.norm(xo) and np.abs(d).max() <= tol * np.abs(xo).max()
    L_plain = N.gnn_factor(P, v, _gpu(b), cfg, _gpu(w, torch.float32), precision=pc)
    assert torch.equal(L, L_plain)
    x, st = N.pcg_solve(P, v, _gpu(b), N.PREC_LLT, L, rtol=1e-8, x0=x0)
    assert st[0]["status"] == 0
    assert np.linalg.norm(b - O.spmv(Ao, _np(x))) / np.linalg.norm(b) <= 2e-8


def _wide_spd(n, seed, kmax=7):
    # 2-D 5-point grid plus random symmetric long-range couplings, strictly
    # diagonally dominant: rows with up to ~10 lower neighbours (dependencies
    # beyond the four held in a row's packed record)
    g = np.random.default_rng(seed)
    m = int(np.sqrt(n))
    n = m * m
    rows, cols = [], []
    for i in range(n):
        x, y = i % m, i // m
        if x > 0:
            rows.append(i); cols.append(i - 1)
        if y > 0:
            rows.append(i); cols.append(i - m)
        k = int(g.integers(0, kmax))
        for j in (g.integers(max(0, i - 3 * m), i, size=k) if i > 0 else []):
            if j != i - 1 and j != i - m:
                rows.append(i); cols.append(int(j))
    adj = [dict() for _ in range(n)]
    for i, j in sorted(set(zip(rows, cols))):
        w = -float(g.uniform(0.1, 1.0))
        adj[i][j] = w
        adj[j][i] = w
    rp, ci, val = [0], [], []
    for i in range(n):
        adj[i][i] = 1.1 + sum(-w for w in adj[i].values())
        for j in sorted(adj[i]):
            ci.append(j)
            val.append(adj[i][j])
        rp.append(len(ci))
    return O.CSR(np.array(rp), np.array(ci), np.array(val))


@pytest.mark.parametrize("case", ["fem130", "fd2d_var", "wide"])
def test_flag_trsv_matches_barrier_bit_exact(N, case):
    # the flag-synchronised FP32 solve performs the barrier kernel's FP32
    # operations in the same order: both directions bit-identical, and both
    # within FP32 rounding of the FP64 oracle on fl32(L)
    if case == "wide":
        Ao = _wide_spd(4900, 3)
        P = N.analyse(_gpu(Ao.row_ptr, torch.int32), _gpu(Ao.col_idx, torch.int32))
    else:
        prob = I.fem2d(130, sigma=1.0, seed=3) if case == "fem130" else PROBLEMS[case]
        Ao, (rp, ci, v) = _assemble_both(N, prob)
        P = N.analyse(rp, ci)
    Lo, _ = O.ic0(Ao)
    N.factor_load(P, _gpu(Lo.val))
    L32 = O.CSR(Lo.row_ptr, Lo.col_idx, Lo.val.astype(np.float32).astype(np.float64))
    r = np.random.default_rng(7).standard_normal(Ao.n)
    r32 = r.astype(np.float32).astype(np.float64)
    for tr in (False, True):
        P.set_trsv(N.TRSV_LEVELSYNC)
        _, yb = N.sptrsv_timed(P, _gpu(r), transpose=tr, reps=1, f32=True)
        P.set_trsv(N.TRSV_LEVELFLAG)
        _, yf = N.sptrsv_timed(P, _gpu(r), transpose=tr, reps=1, f32=True)
        assert torch.equal(yb, yf)
        P.set_trsv(N.TRSV_LEVELSPLIT)
        _, ys = N.sptrsv_timed(P, _gpu(r), transpose=tr, reps=1, f32=True)
        assert torch.equal(yb, ys)
        yo = O.trsv_upper(L32, r32) if tr else O.trsv_lower(L32, r32)
        assert _rel(_np(yf), yo) <= 1e-4


def test_flag_trsv_batched_pcg(N):
    # one CTA per system: PCG with the FP32 apply in the flag design against
    # the oracle (the bar of test_fp32_preconditioner_apply), and the same
    # iterations as the barrier design
    probs = [I.fem2d(60, sigma=1.0, seed=31), I.fd3d(12, 10, 9, sigma=1.0, seed=32), I.fd2d(40, 23, sigma=1.0, seed=33)]
    As, cis, vs, bs = [], [], [], []
    off, sys_ptr = 0, [0]
    for k, p in enumerate(probs):
        Ao, (rp, ci, v) = _assemble_both(N, p)
        As.append(Ao)
        cis.append(_np(ci) + off)
        vs.append(_np(v))
        bs.append(I.rhs(Ao.n, 60 + k))
        off += Ao.n
        sys_ptr.append(off)
    nnz_off = np.cumsum([0] + [a.nnz for a in As])
    rp_cat = np.concatenate([a.row_ptr[:-1] + nnz_off[k] for k, a in enumerate(As)] + [[nnz_off[-1]]])
    P = N.analyse(_gpu(rp_cat, torch.int32), _gpu(np.concatenate(cis), torch.int32), sys_ptr)
    v_cat = _gpu(np.concatenate(vs))
    b_cat = _gpu(np.concatenate(bs))
    Lg, _ = N.ic0_factor(P, v_cat)
    P.set_trsv(N.TRSV_LEVELSYNC)
    xb, sb = N.pcg_solve(P, v_cat, b_cat, N.PREC_LLT32, Lg, rtol=1e-8)
    P.set_trsv(N.TRSV_LEVELFLAG)
    xf, sf = N.pcg_solve(P, v_cat, b_cat, N.PREC_LLT32, Lg, rtol=1e-8)
    assert torch.equal(xb, xf)
    xs = _np(xf)
    for k, Ao in enumerate(As):
        _, ito, _, _ = O.pcg(Ao, bs[k], O.PREC_LLT, O.ic0(Ao)[0], rtol=1e-8)
        assert sf[k]["status"] == 0 and sf[k]["iters"] == sb[k]["iters"]
        assert abs(sf[k]["iters"] - ito) <= max(1, int(np.ceil(0.05 * ito)))
        seg = xs[sys_ptr[k]:sys_ptr[k + 1]]
        assert np.linalg.norm(bs[k] - O.spmv(Ao, seg)) / np.linalg.norm(bs[k]) <= 2e-8


@pytest.mark.parametrize("name", ["poisson2d_32", "fd2d_var", "fd3d_var", "fem34"])
def test_sgs_factor_and_pcg_parity(N, name):
    # the factor from the oracle's A values: one correctly rounded square root
    # and division per entry on both sides, so bit-identical; PCG with it
    # within one iteration of the oracle's, in the FP64 and the FP32 apply
    Ao, (rp, ci, v) = _assemble_both(N, PROBLEMS[name])
    P = N.analyse(rp, ci)
    Lo = O.sgs(Ao)
    Lg = N.sgs_factor(P, _gpu(Ao.val))
    assert np.array_equal(_np(Lg), Lo.val)
    b = I.rhs(Ao.n, 12)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    xg, st = N.pcg_solve(P, _gpu(Ao.val), _gpu(b), N.PREC_LLT, Lg, rtol=1e-8)
    assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(_np(xg) - xo) / np.linalg.norm(xo) <= 1e-8
    x32, s32 = N.pcg_solve(P, _gpu(Ao.val), _gpu(b), N.PREC_LLT32, Lg, rtol=1e-8)
    assert s32[0]["status"] == 0 and abs(s32[0]["iters"] - ito) <= max(1, int(np.ceil(0.05 * ito)))
    assert np.linalg.norm(b - O.spmv(Ao, _np(x32))) / np.linalg.norm(b) <= 2e-8


def test_sgs_solve_host(N):
    # the host-buffer entry point with the SGS method matches the device path
    Ao, (rp, ci, v) = _assemble_both(N, PROBLEMS["fem34"])
    P = N.analyse(rp, ci)
    b = I.rhs(Ao.n, 13)
    xd, sd = N.pcg_solve(P, v, _gpu(b), N.PREC_LLT, N.sgs_factor(P, v), rtol=1e-8)
    xh, sh = N.solve_host(P, _np(v), b, method=N.METHOD_SGS, rtol=1e-8)
    assert sh[0]["iters"] == sd[0]["iters"]
    assert np.array_equal(np.asarray(xh), _np(xd))


TIME_STEP = {
    "heat_fem_arc": I.heat2d(40, seed=3),
    "heat_fem_arc_wrap": I.Problem(I.FEM, 2, 24, 24, 0, 1.0, 0.1, 7, 2e-3, 80, 30),
    "heat_fem_all": I.Problem(I.FEM, 2, 30, 30, 0, 1.0, 0.1, 4, 1e-2),
    "stiff_fem_arc": I.Problem(I.FEM, 2, 26, 26, 0, 1.0, 0.1, 6, 0.0, 11, 30),
    "heat_fd3d": I.Problem(I.FD, 3, 9, 8, 7, 1.0, 0.1, 5, 0.05),
}


@pytest.mark.parametrize("name", list(TIME_STEP))
def test_time_step_assembly_parity(N, name):
    # M + tau K and Dirichlet arcs: pattern and numbering bit-exact, values
    # to the bar of the stiffness assembly
    prob = TIME_STEP[name]
    Ao, (rp, ci, v) = _assemble_both(N, prob)
    assert Ao.n == prob.n
    assert np.array_equal(_np(rp), Ao.row_ptr)
    assert np.array_equal(_np(ci), Ao.col_idx)
    assert _rel(_np(v), Ao.val) <= 1e-12


@pytest.mark.parametrize("name", list(TIME_STEP))
def test_time_step_pcg_parity(N, name):
    # IC(0) and symmetric Gauss-Seidel PCG on the time-step systems against
    # the oracle (the bars of the stiffness systems)
    prob = TIME_STEP[name]
    Ao, (rp, ci, v) = _assemble_both(N, prob)
    P = N.analyse(rp, ci)
    b = I.rhs(Ao.n, 14)
    for Lo, Lg in ((O.ic0(Ao)[0], N.ic0_factor(P, _gpu(Ao.val))[0]), (O.sgs(Ao), N.sgs_factor(P, _gpu(Ao.val)))):
        xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
        xg, st = N.pcg_solve(P, _gpu(Ao.val), _gpu(b), N.PREC_LLT, Lg, rtol=1e-8)
        assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= 1
        assert np.linalg.norm(_np(xg) - xo) / np.linalg.norm(xo) <= 1e-8


def test_time_step_rejects_bad_arcs(N):
    with pytest.raises(N.NpcgError):
        N.assemble_system(I.Problem(I.FD, 2, 8, 8, 0, 0.0, 0.1, 0, 0.1, 3, 4))
    with pytest.raises(N.NpcgError):
        N.assemble_system(I.Problem(I.FEM, 2, 8, 8, 0, 0.0, 0.1, 0, -1.0))


@pytest.mark.parametrize("mode", ["levelsync", "levelsplit"])
@pytest.mark.parametrize("prob", [I.heat2d(130, seed=0), I.heat2d(110, seed=2)])
def test_hybrid_window_far_dependencies(N, prob, mode):
    # free boundary points of these heat systems have no upper neighbours
    # and sit at backward level 0 while a reader comes thousands of
    # positions later (reach 11,332 and 8,507 > the 8,192-slot window): the
    # level-synchronous solve keeps the window and reads those dependencies
    # from its output; both directions against the oracle, and PCG
    Ao, (rp, ci, v) = _assemble_both(N, prob)
    P = N.analyse(rp, ci)
    _set_mode(N, P, mode)
    Lo, _ = O.ic0(Ao)
    N.factor_load(P, _gpu(Lo.val))
    r = np.random.default_rng(8).standard_normal(Ao.n)
    assert _rel(_np(N.sptrsv(P, _gpu(r))), O.trsv_lower(Lo, r)) <= 1e-12
    assert _rel(_np(N.sptrsv(P, _gpu(r), transpose=True)), O.trsv_upper(Lo, r)) <= 1e-12
    L32 = O.CSR(Lo.row_ptr, Lo.col_idx, Lo.val.astype(np.float32).astype(np.float64))
    r32 = r.astype(np.float32).astype(np.float64)
    _, y32 = N.sptrsv_timed(P, _gpu(r), transpose=True, reps=1, f32=True)
    assert _rel(_np(y32), O.trsv_upper(L32, r32)) <= 1e-4
    b = I.rhs(Ao.n, 15)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    for pc in (N.PREC_LLT, N.PREC_LLT32):
        xg, st = N.pcg_solve(P, _gpu(Ao.val), _gpu(b), pc, _gpu(Lo.val), rtol=1e-8)
        assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= max(1, int(np.ceil(0.05 * ito)))
        assert np.linalg.norm(b - O.spmv(Ao, _np(xg))) / np.linalg.norm(b) <= 2e-8


@pytest.mark.parametrize("kmax", [4, 30])
def test_spmv_and_pcg_row_mappings(N, kmax):
    # rows of at most 16 entries take the one-thread-per-row SpMV, longer
    # ones the eight-lanes-per-row mapping: both against the oracle, alone
    # and inside PCG
    Ao = _wide_spd(1600, 5, kmax)
    P = N.analyse(_gpu(Ao.row_ptr, torch.int32), _gpu(Ao.col_idx, torch.int32))
    longest = int(np.diff(Ao.row_ptr).max())
    assert P.max_row == longest and (longest <= 16) == (kmax == 4)
    x = np.random.default_rng(3).standard_normal(Ao.n)
    assert _rel(_np(N.spmv(P, _gpu(Ao.val), _gpu(x))), O.spmv(Ao, x)) <= 1e-13
    b = I.rhs(Ao.n, 16)
    Lo, _ = O.ic0(Ao)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    xg, st = N.pcg_solve(P, _gpu(Ao.val), _gpu(b), N.PREC_LLT, _gpu(Lo.val), rtol=1e-8)
    assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(_np(xg) - xo) / np.linalg.norm(xo) <= 1e-8


def _merge_or_skip(N, P):
    try:
        P.set_trsv(N.TRSV_LEVELMERGE)
    except N.NpcgError as e:
        if "not enabled" in str(e):
            pytest.skip("merged-level solves are not enabled in this build")
        raise


@pytest.mark.parametrize("name", ["poisson2d_32", "fem34", "fd3d_var"])
def test_merged_levels_parity(N, name):
    # groups of levels per step (substituted rows): both directions against
    # the oracle in FP64 and FP32, and PCG with IC(0) within one iteration
    Ao, (rp, ci, v) = _assemble_both(N, PROBLEMS[name])
    P = N.analyse(rp, ci)
    _merge_or_skip(N, P)
    assert P.trsv_mode == N.TRSV_LEVELMERGE
    Lo, _ = O.ic0(Ao)
    N.factor_load(P, _gpu(Lo.val))
    r = np.random.default_rng(5).standard_normal(Ao.n)
    assert _rel(_np(N.sptrsv(P, _gpu(r))), O.trsv_lower(Lo, r)) <= 1e-12
    assert _rel(_np(N.sptrsv(P, _gpu(r), transpose=True)), O.trsv_upper(Lo, r)) <= 1e-12
    L32 = O.CSR(Lo.row_ptr, Lo.col_idx, Lo.val.astype(np.float32).astype(np.float64))
    r32 = r.astype(np.float32).astype(np.float64)
    _, y32 = N.sptrsv_timed(P, _gpu(r), transpose=False, reps=1, f32=True)
    assert _rel(_np(y32), O.trsv_lower(L32, r32)) <= 1e-4
    b = I.rhs(Ao.n, 8)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    xg, st = N.pcg_solve(P, v, _gpu(b), N.PREC_LLT, _gpu(Lo.val), rtol=1e-8)
    assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(_np(xg) - xo) / np.linalg.norm(xo) <= 1e-8


def test_merged_levels_blocked_parity(N):
    # one system of 2^18 rows: the merged layouts in per-SM row blocks, with
    # dependencies on earlier blocks published and polled
    prob = I.fd3d(64, sigma=1.5, corr_len=0.1, seed=6)
    Ao, (rp, ci, v) = _assemble_both(N, prob)
    assert Ao.n == 1 << 18
    P = N.analyse(rp, ci)
    _merge_or_skip(N, P)
    assert P.trsv_mode == N.TRSV_LEVELMERGE
    Lo, _ = O.ic0(Ao)
    N.factor_load(P, _gpu(Lo.val))
    r = np.random.default_rng(6).standard_normal(Ao.n)
    assert _rel(_np(N.sptrsv(P, _gpu(r))), O.trsv_lower(Lo, r)) <= 1e-12
    assert _rel(_np(N.sptrsv(P, _gpu(r), transpose=True)), O.trsv_upper(Lo, r)) <= 1e-12
    L32 = O.CSR(Lo.row_ptr, Lo.col_idx, Lo.val.astype(np.float32).astype(np.float64))
    r32 = r.astype(np.float32).astype(np.float64)
    for tr, ref in ((False, O.trsv_lower(L32, r32)), (True, O.trsv_upper(L32, r32))):
        _, y32 = N.sptrsv_timed(P, _gpu(r), transpose=tr, reps=2, f32=True)
        assert _rel(_np(y32), ref) <= 1e-4
    b = I.rhs(Ao.n, 9)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    for prec in (N.PREC_LLT, N.PREC_LLT32):
        xg, st = N.pcg_solve(P, v, _gpu(b), prec, _gpu(Lo.val), rtol=1e-8)
        assert st[0]["status"] == 0
        if prec == N.PREC_LLT:
            assert abs(st[0]["iters"] - ito) <= 1
            assert np.linalg.norm(_np(xg) - xo) / np.linalg.norm(xo) <= 1e-8
        else:
            assert abs(st[0]["iters"] - ito) <= max(1, int(np.ceil(0.05 * ito)))
            assert np.linalg.norm(b - O.spmv(Ao, _np(xg))) / np.linalg.norm(b) <= 2e-8


def test_merged_levels_batched_pcg(N):
    probs = [I.fem2d(30, sigma=1.0, seed=41), I.heat2d(26, seed=42), I.fd3d(8, 7, 6, sigma=1.0, seed=43)]
    As, cis, vs, bs = [], [], [], []
    off, sys_ptr = 0, [0]
    for k, p in enumerate(probs):
        Ao, (rp, ci, v) = _assemble_both(N, p)
        As.append(Ao)
        cis.append(_np(ci) + off)
        vs.append(_np(v))
        bs.append(I.rhs(Ao.n, 80 + k))
        off += Ao.n
        sys_ptr.append(off)
    nnz_off = np.cumsum([0] + [a.nnz for a in As])
    rp_cat = np.concatenate([a.row_ptr[:-1] + nnz_off[k] for k, a in enumerate(As)] + [[nnz_off[-1]]])
    P = N.analyse(_gpu(rp_cat, torch.int32), _gpu(np.concatenate(cis), torch.int32), sys_ptr)
    _merge_or_skip(N, P)
    v_cat = _gpu(np.concatenate(vs))
    Lg, _ = N.ic0_factor(P, v_cat)
    x, st = N.pcg_solve(P, v_cat, _gpu(np.concatenate(bs)), N.PREC_LLT32, Lg, rtol=1e-8)
    xs = _np(x)
    for k, Ao in enumerate(As):
        _, ito, _, _ = O.pcg(Ao, bs[k], O.PREC_LLT, O.ic0(Ao)[0], rtol=1e-8)
        assert st[k]["status"] == 0 and abs(st[k]["iters"] - ito) <= max(1, int(np.ceil(0.05 * ito)))
        seg = xs[sys_ptr[k]:sys_ptr[k + 1]]
        assert np.linalg.norm(bs[k] - O.spmv(Ao, seg)) / np.linalg.norm(bs[k]) <= 2e-8
