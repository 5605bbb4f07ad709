"""The allocation-free entry point npcg_pcg_solve_noalloc, for callers that
cannot allocate device memory (another arena or runtime owns it, or an
allocation's latency or failure is unacceptable in their loop).  Called
through the C ABI and checked against npcg_pcg_solve (the entry point that
allocates its workspace) on the same systems, twice in a row, since every
call shares the library's fixed device array.  Collected last so a run that
stops at the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_2305_16432_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MAX_N = 262144     # NPCG_NOALLOC_MAX_N in include/npcg.h


@pytest.fixture(scope="module")
def env():
    from paper_2305_16432_gb300 import build
    build.build()
    from paper_2305_16432_gb300 import npcg
    lib = npcg.lib()
    fn = lib.npcg_pcg_solve_noalloc
    fn.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                   C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.c_void_p]
    fn.restype = C.c_int
    return npcg, fn


def _noalloc(fn, rp, ci, v, b, precond, rtol, max_iter, x0=None):
    from paper_2305_16432_gb300.npcg import _Stats
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    st = _Stats()
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(C.c_void_p(stream), rp.numel() - 1, ci.numel(), C.c_void_p(rp.data_ptr()),
            C.c_void_p(ci.data_ptr()), C.c_void_p(v.data_ptr()), C.c_void_p(b.data_ptr()),
            C.c_void_p(x.data_ptr()), precond, rtol, max_iter, C.byref(st))
    return rc, x, st


@pytest.mark.parametrize("prob,precond", [(I.fem2d(34, sigma=1.0, seed=5), 1),
                                          (I.fd3d(9, 8, 7, sigma=1.5, corr_len=0.05, seed=4), 1),
                                          (I.poisson2d_32(), 0)])
def test_noalloc_matches_allocating_entry_point(env, prob, precond):
    N, fn = env
    rp, ci, v = N.assemble_system(prob)
    P = N.analyse(rp, ci)
    b = torch.as_tensor(I.rhs(P.n, 3), device="cuda")
    x_ref, st_ref = N.pcg_solve(P, v, b, precond, None, rtol=1e-8)
    for _ in range(2):                                    # two calls in a row
        rc, x, st = _noalloc(fn, rp, ci, v, b, precond, 1e-8, 10 * P.n)
        assert rc == 0 and st.status == 0
        assert abs(st.iters - st_ref[0]["iters"]) <= 1
        assert st.relres <= 1e-8
        # the same number of updates through the allocating path: same iterate
        xk, stk = N.pcg_solve(P, v, b, precond, None, rtol=0.0, max_iter=st.iters)
        d = (x - xk).norm() / xk.norm()
        assert float(d) <= 1e-8
    # the solution solves A x = b
    Ao = O.CSR(rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy())
    bn = b.cpu().numpy()
    assert np.linalg.norm(bn - O.spmv(Ao, x.cpu().numpy())) / np.linalg.norm(bn) <= 2e-8


def test_noalloc_limits_and_edge_cases(env):
    N, fn = env
    rp, ci, v = N.assemble_system(I.fd2d(9, 7))
    b = torch.zeros(63, dtype=torch.float64, device="cuda")
    rc, x, st = _noalloc(fn, rp, ci, v, b, 1, 1e-8, 100)
    assert rc == 0 and st.iters == 0                       # b = 0: nothing to do
    b = torch.as_tensor(I.rhs(63, 1), device="cuda")
    rc, x, st = _noalloc(fn, rp, ci, v, b, 0, 1e-14, 3)
    assert rc == N.NPCG_EMAXITER and st.iters == 3
    rc, x, st = _noalloc(fn, rp, ci, v, b, 2, 1e-8, 100)   # needs an analysed pattern
    assert rc == N.NPCG_EINVAL
    # a Jacobi system with a zero diagonal entry is an invalid input
    vz = v.clone()
    adiag = [k for k in range(rp[5].item(), rp[6].item()) if ci[k].item() == 5][0]
    vz[adiag] = 0.0
    rc, x, st = _noalloc(fn, rp, ci, vz, b, 1, 1e-8, 100)
    assert rc == N.NPCG_EINVAL
    # and the next call on the same array is unaffected
    rc, x, st = _noalloc(fn, rp, ci, v, b, 1, 1e-8, 100)
    assert rc == 0 and st.status == 0
    # sizes beyond the fixed array are rejected before any GPU work
    from paper_2305_16432_gb300.npcg import _Stats
    st = _Stats()
    rc = fn(None, MAX_N + 1, MAX_N + 1, C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()),
            C.c_void_p(v.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(b.data_ptr()), 1, 1e-8, 10,
            C.byref(st))
    assert rc == N.NPCG_EINVAL


def test_noalloc_largest_size_and_initial_guess(env):
    # n exactly at the limit (a 512 x 512 grid: every block of the array in
    # use, the last one full) and a nonzero initial guess (the A x_0 term of
    # the first pass), against the allocating entry point
    N, fn = env
    prob = I.fd2d(512, 512, sigma=1.0, seed=31)
    rp, ci, v = N.assemble_system(prob)
    assert rp.numel() - 1 == MAX_N
    P = N.analyse(rp, ci)
    b = torch.as_tensor(I.rhs(P.n, 32), device="cuda")
    x0 = torch.as_tensor(np.random.default_rng(33).standard_normal(P.n), device="cuda")
    for precond in (1, 0):
        x_ref, st_ref = N.pcg_solve(P, v, b, precond, None, rtol=1e-8, x0=x0)
        rc, x, st = _noalloc(fn, rp, ci, v, b, precond, 1e-8, 10 * P.n, x0=x0)
        assert rc == 0 and st.status == 0 and abs(st.iters - st_ref[0]["iters"]) <= max(1, st_ref[0]["iters"] // 100)
        xk, _ = N.pcg_solve(P, v, b, precond, None, rtol=0.0, max_iter=st.iters, x0=x0)
        assert float((x - xk).norm() / xk.norm()) <= 1e-6
