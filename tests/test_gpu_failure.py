"""GPU failure paths through the C ABI, each made on the host (nothing
faults, traps or hangs the GPU):

* a bounded device wait that runs out: the sync-free triangular solve with
  its first slices never claimed, under a short wait limit, returns
  NPCG_ETIMEOUT and leaves the context usable;
* PCG breakdown (Algorithm 1: p^T A p <= 0, r^T z <= 0 or non-finite) on
  host-made inputs, with the oracle's status beside it;
* IC(0)'s shifted retry (Sec. 5.1 "Incomplete Cholesky", A + alpha diag(A))
  on Kershaw's matrix, alone and inside a batch, against the oracle.
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


def _csr_from_dense(D):
    rp, ci, v = [0], [], []
    for i in range(D.shape[0]):
        nz = np.nonzero(D[i])[0]
        ci += list(nz)
        v += list(D[i, nz])
        rp.append(len(ci))
    return O.CSR(rp, ci, v)


def _pattern(N, Ao, sys_ptr=None):
    return N.analyse(_gpu(Ao.row_ptr, torch.int32), _gpu(Ao.col_idx, torch.int32), sys_ptr)


KERSHAW = np.array([[3, -2, 0, 2], [-2, 3, -2, 0], [0, -2, 3, -2], [2, 0, -2, 3.0]])


@pytest.mark.parametrize("transpose", [False, True])
def test_wait_runs_out_and_context_stays_usable(N, transpose):
    Ao = O.assemble(I.fem2d(34, sigma=1.0, seed=5))
    P = _pattern(N, Ao)
    Lo, _ = O.ic0(Ao)
    N.factor_load(P, _gpu(Lo.val))
    r = np.random.default_rng(4).standard_normal(Ao.n)
    P.h.set_wait_limit(1 << 10)
    try:
        # slice 0 (the first 32 rows in level order) is never claimed: the
        # rows that depend on it give up after 1024 polls
        st = N.sptrsv_unclaimed(P, _gpu(r), skip=1, transpose=transpose)
        assert st == N.NPCG_ETIMEOUT
        # nothing waits when every slice is skipped
        nsl = (Ao.n + 31) // 32
        assert N.sptrsv_unclaimed(P, _gpu(r), skip=nsl, transpose=transpose) == N.NPCG_OK
        assert N.sptrsv_unclaimed(P, _gpu(r), skip=nsl + 1, transpose=transpose) == N.NPCG_EINVAL
    finally:
        P.h.set_wait_limit(0)
    # the same handle and pattern still solve correctly afterwards
    y = _np(N.sptrsv(P, _gpu(r), transpose=transpose))
    ref = O.trsv_upper(Lo, r) if transpose else O.trsv_lower(Lo, r)
    assert _rel(y, ref) <= 1e-12
    b = I.rhs(Ao.n, 3)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    xg, st = N.pcg_solve(P, _gpu(Ao.val), _gpu(b), N.PREC_LLT, _gpu(Lo.val), rtol=1e-8)
    assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= 1


def test_breakdown_negative_definite(N):
    # -A: p^T A p < 0 at the first step of plain CG and of Jacobi-PCG
    # (Jacobi: r^T z < 0 already), status EBREAKDOWN with no update, as in
    # the oracle
    Ao = O.assemble(I.fd2d(12, 9, sigma=1.0, seed=1))
    An = O.CSR(Ao.row_ptr, Ao.col_idx, -Ao.val)
    P = _pattern(N, An)
    b = I.rhs(An.n, 2)
    for prec_g, prec_o in ((N.PREC_NONE, O.PREC_NONE), (N.PREC_JACOBI, O.PREC_JACOBI)):
        _, ito, _, sto = O.pcg(An, b, prec_o, rtol=1e-8)
        _, st = N.pcg_solve(P, _gpu(An.val), _gpu(b), prec_g, None, rtol=1e-8)
        assert sto == 2 and ito == 0
        assert st[0]["status"] == N.NPCG_EBREAKDOWN and st[0]["iters"] == 0


def test_breakdown_non_finite(N):
    Ao = O.assemble(I.fem2d(20, sigma=1.0, seed=2))
    P = _pattern(N, Ao)
    b = I.rhs(Ao.n, 5)
    # a NaN in b: ||r_0|| is not finite
    bn = b.copy()
    bn[Ao.n // 2] = np.nan
    _, ito, _, sto = O.pcg(Ao, bn, O.PREC_NONE, rtol=1e-8)
    _, st = N.pcg_solve(P, _gpu(Ao.val), _gpu(bn), N.PREC_NONE, None, rtol=1e-8)
    assert sto == 2 and st[0]["status"] == N.NPCG_EBREAKDOWN and st[0]["iters"] == ito == 0
    # a factor with a zero pivot: the triangular solve divides by zero, so
    # r^T z is not finite before the first update (both sides)
    Lo, _ = O.ic0(Ao)
    Lz = Lo.val.copy()
    Lz[Lo.row_ptr[7] - 1] = 0.0                          # diagonal of row 6
    Lzc = O.CSR(Lo.row_ptr, Lo.col_idx, Lz)
    _, ito, _, sto = O.pcg(Ao, b, O.PREC_LLT, Lzc, rtol=1e-8)
    for prec in (N.PREC_LLT, N.PREC_LLT32):
        _, st = N.pcg_solve(P, _gpu(Ao.val), _gpu(b), prec, _gpu(Lz), rtol=1e-8)
        assert sto == 2 and st[0]["status"] == N.NPCG_EBREAKDOWN and st[0]["iters"] == ito == 0


def test_ic0_shift_kershaw(N):
    # Kershaw's SPD matrix breaks IC(0) down; the GPU takes the oracle's
    # shift alpha = 1e-3 * 2^t and its factor of A + alpha diag(A)
    Ao = _csr_from_dense(KERSHAW)
    P = _pattern(N, Ao)
    Lg, alpha = N.ic0_factor(P, _gpu(Ao.val))
    Lo, ao = O.ic0(Ao)
    assert ao > 0 and alpha[0] == ao
    assert _rel(_np(Lg), Lo.val) <= 1e-12
    b = np.array([1.0, -2.0, 0.5, 3.0])
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-10)
    xg, st = N.pcg_solve(P, _gpu(Ao.val), _gpu(b), N.PREC_LLT, Lg, rtol=1e-10)
    assert st[0]["status"] == 0 and abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(_np(xg) - xo) / np.linalg.norm(xo) <= 1e-8


def test_ic0_shift_per_system_in_a_batch(N):
    # only the member that breaks down is shifted; the others keep alpha = 0
    members = [O.assemble(I.fd2d(6, 5, sigma=1.0, seed=3)), _csr_from_dense(KERSHAW),
               O.assemble(I.fem2d(8, sigma=1.0, seed=4)), _csr_from_dense(KERSHAW)]
    off, nnz_off, sys_ptr, cis = 0, [0], [0], []
    for A in members:
        cis.append(A.col_idx + off)
        off += A.n
        sys_ptr.append(off)
        nnz_off.append(nnz_off[-1] + A.nnz)
    rp = np.concatenate([A.row_ptr[:-1] + nnz_off[k] for k, A in enumerate(members)] + [[nnz_off[-1]]])
    Acat = O.CSR(rp, np.concatenate(cis), np.concatenate([A.val for A in members]))
    P = _pattern(N, Acat, sys_ptr)
    Lg, alpha = N.ic0_factor(P, _gpu(Acat.val))
    Lg = _np(Lg)
    Lrp = _np(P.export()["L_row_ptr"])
    for k, A in enumerate(members):
        Lo, ao = O.ic0(A)
        assert alpha[k] == ao and ((ao > 0) == (k % 2 == 1))
        seg = Lg[Lrp[sys_ptr[k]]:Lrp[sys_ptr[k + 1]]]
        assert _rel(seg, Lo.val) <= 1e-12


# ------------------------------------------------- IC(0) fallback, stagnation
def test_fallback_to_ic0_after_breakdown(N):
    # a learned-style factor with a zero pivot breaks down before the first
    # update; the solve is handed to IC(0) from x_0 and matches the oracle's
    # IC(0)-PCG
    Ao = O.assemble(I.fem2d(24, sigma=1.0, seed=6))
    P = _pattern(N, Ao)
    b = I.rhs(Ao.n, 9)
    Lo, _ = O.ic0(Ao)
    Lz = Lo.val.copy()
    Lz[Lo.row_ptr[11] - 1] = 0.0
    x, st, status = N.pcg_solve_ex(P, _gpu(Ao.val), _gpu(b), N.PREC_LLT, _gpu(Lz), rtol=1e-8, fallback_ic0=True)
    xo, ito, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    assert status == N.NPCG_OK and st[0]["status"] == 0 and st[0]["fallback"] == 1
    assert st[0]["iters"] == st[0]["fallback_iters"] and abs(st[0]["iters"] - ito) <= 1
    assert np.linalg.norm(_np(x) - xo) / np.linalg.norm(xo) <= 1e-8
    # without the fallback the breakdown is reported
    _, st2, status2 = N.pcg_solve_ex(P, _gpu(Ao.val), _gpu(b), N.PREC_LLT, _gpu(Lz), rtol=1e-8)
    assert status2 == N.NPCG_EBREAKDOWN and st2[0]["fallback"] == 0


def test_fallback_to_ic0_after_max_iter(N):
    # a poor factor (diagonal only, L = D^1/2) runs out of max_iter; IC(0)
    # continues from that iterate with a fresh budget of max_iter updates,
    # which is enough for it (the budget sits between the two counts)
    Ao = O.assemble(I.fd3d(10, 9, 8, sigma=1.5, corr_len=0.2, seed=7))
    P = _pattern(N, Ao)
    b = I.rhs(Ao.n, 10)
    Lo, _ = O.ic0(Ao)
    Ld = np.zeros(Lo.nnz)
    Ld[Lo.row_ptr[1:] - 1] = np.sqrt(np.diag(Ao.dense()))
    _, it_d, _, _ = O.pcg(Ao, b, O.PREC_LLT, O.CSR(Lo.row_ptr, Lo.col_idx, Ld), rtol=1e-8)
    _, it_i, _, _ = O.pcg(Ao, b, O.PREC_LLT, Lo, rtol=1e-8)
    budget = (it_d + it_i) // 2
    assert it_i + 2 < budget < it_d - 2
    for prec in (N.PREC_LLT, N.PREC_LLT32):
        x, st, status = N.pcg_solve_ex(P, _gpu(Ao.val), _gpu(b), prec, _gpu(Ld), rtol=1e-8, max_iter=budget,
                                       fallback_ic0=True)
        assert status == N.NPCG_OK and st[0]["fallback"] == 1
        assert st[0]["iters"] == budget + st[0]["fallback_iters"] and 0 < st[0]["fallback_iters"] <= budget
        assert np.linalg.norm(b - O.spmv(Ao, _np(x))) / np.linalg.norm(b) <= 2e-8


def test_stagnation_window(N):
    # A = diag(1, 100), P = diag(100, 1), b = (1, 0.01): the first update
    # raises ||r|| from 1.00005 to 1.40007 (by hand: r_1 = (0.99, -0.99)), and
    # the second, P^-1 A having two eigenvalues, solves exactly.
    A = O.CSR([0, 1, 2], [0, 1], [1.0, 100.0])
    P = _pattern(N, A)
    b = np.array([1.0, 0.01])
    L = np.array([10.0, 1.0])
    _, it1, rel1, _ = O.pcg(A, b, O.PREC_LLT, O.CSR([0, 1, 2], [0, 1], L), rtol=0.0, max_iter=1)
    assert it1 == 1 and rel1 > 1.0
    # a window of one update: the rise stops the solve
    _, st, status = N.pcg_solve_ex(P, _gpu(A.val), _gpu(b), N.PREC_LLT, _gpu(L), rtol=1e-10, stall_iters=1)
    assert status == N.NPCG_ESTALL and st[0]["status"] == N.NPCG_ESTALL and st[0]["iters"] == 1
    # two: the next update converges
    x, st, status = N.pcg_solve_ex(P, _gpu(A.val), _gpu(b), N.PREC_LLT, _gpu(L), rtol=1e-10, stall_iters=2)
    assert status == N.NPCG_OK and st[0]["iters"] == 2
    assert np.allclose(_np(x), [1.0, 1e-4], rtol=1e-12)
    # one, with the fallback: IC(0) of a diagonal A is exact, one more update
    x, st, status = N.pcg_solve_ex(P, _gpu(A.val), _gpu(b), N.PREC_LLT, _gpu(L), rtol=1e-10, stall_iters=1,
                                   fallback_ic0=True)
    assert status == N.NPCG_OK and st[0]["fallback"] == 1 and st[0]["iters"] == 2 and st[0]["fallback_iters"] == 1
    assert np.allclose(_np(x), [1.0, 1e-4], rtol=1e-12)


# ------------------------------------------------------------ launch modes
@pytest.mark.parametrize("prec", ["PREC_LLT32", "PREC_JACOBI"])
def test_eager_iterations_identical_to_graph(N, prec):
    # the loop graph and one-launch-at-a-time iterations run the same
    # kernels in the same order: identical statistics and solution bits
    Ao = O.assemble(I.fem2d(40, sigma=1.0, seed=8))
    P = _pattern(N, Ao)
    b = I.rhs(Ao.n, 12)
    Lo, _ = O.ic0(Ao)
    L = _gpu(Lo.val) if prec == "PREC_LLT32" else None
    P.h.set_pcg_eager(False)
    x1, st1 = N.pcg_solve(P, _gpu(Ao.val), _gpu(b), getattr(N, prec), L, rtol=1e-8)
    x1 = _np(x1).copy()
    P.h.set_pcg_eager(True)
    try:
        x2, st2 = N.pcg_solve(P, _gpu(Ao.val), _gpu(b), getattr(N, prec), L, rtol=1e-8)
        x2 = _np(x2)
        # a maximum below the eager batch of 16 iterations stops on time too
        _, st3 = N.pcg_solve(P, _gpu(Ao.val), _gpu(b), getattr(N, prec), L, rtol=1e-8, max_iter=5)
    finally:
        P.h.set_pcg_eager(None)
    assert st1[0]["status"] == 0 and st2[0]["status"] == 0
    assert st1[0]["iters"] == st2[0]["iters"] and np.array_equal(x1, x2)
    assert st3[0]["status"] == N.NPCG_EMAXITER and st3[0]["iters"] == 5
