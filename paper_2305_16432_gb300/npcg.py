"""Thin Python binding of libnpcg (include/npcg.h): argument marshalling only.

Every function here forwards to the C-ABI function of the same name; all
arithmetic runs in the CUDA kernels of the library.  Arrays are torch CUDA
tensors (PyTorch supplies device memory and streams); the library has no
torch types in its interface.  If libnpcg.so is missing this module raises on
first use: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import sys
import threading

import numpy as np
import torch

from . import inputs as I

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnpcg.so")

(NPCG_OK, NPCG_EINVAL, NPCG_ENOMEM, NPCG_ECUDA, NPCG_ENOTSPD, NPCG_EBREAKDOWN, NPCG_EMAXITER, NPCG_ETIMEOUT,
 NPCG_ESTALL) = range(9)
FD, FEM = 0, 1
FP32, BF16 = 0, 1
DIAG_SOFTPLUS, DIAG_LDLT_DIAGA, DIAG_LDLT_ROWS = 0, 1, 2
LOSS_AB, LOSS_FROB = 0, 1
PREC_NONE, PREC_JACOBI, PREC_LLT, PREC_LLT32 = 0, 1, 2, 3
METHOD_GNN, METHOD_IC0, METHOD_JACOBI, METHOD_CG, METHOD_SGS = 0, 1, 2, 3, 4
TRSV_AUTO, TRSV_SYNCFREE, TRSV_LEVELSYNC, TRSV_LEVELFLAG, TRSV_LEVELSPLIT, TRSV_LEVELMERGE = 0, 1, 2, 3, 4, 5


class NpcgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status}: {msg}")
        self.status = status


class _Problem(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
                ("nz", C.c_int32), ("n_features", C.c_int32), ("sigma", C.c_double),
                ("omega", C.c_void_p), ("phase", C.c_void_p), ("jitter", C.c_void_p), ("tau", C.c_double),
                ("dir_start", C.c_int32), ("dir_len", C.c_int32)]


class _Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("nnz_L", C.c_int64), ("nsys", C.c_int32),
                ("nlev_fwd", C.c_int32), ("nlev_bwd", C.c_int32), ("trsv_mode", C.c_int32),
                ("tuned_ms_syncfree", C.c_float), ("tuned_ms_levelsync", C.c_float),
                ("tuned_ms_levelflag", C.c_float), ("tuned_ms_levelsplit", C.c_float), ("max_row", C.c_int32),
                ("tuned_ms_levelmerge", C.c_float), ("merge_levels", C.c_int32), ("block_units", C.c_int32)]


class _Cfg(C.Structure):
    _fields_ = [("n_mp", C.c_int32), ("l", C.c_int32), ("l_mp", C.c_int32), ("h", C.c_int32),
                ("diag_mode", C.c_int32), ("precision", C.c_int32), ("x0_head", C.c_int32), ("loss", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("relres", C.c_double), ("fallback", C.c_int32),
                ("fallback_iters", C.c_int32)]


class _Opts(C.Structure):
    _fields_ = [("stall_iters", C.c_int32), ("fallback_ic0", C.c_int32)]


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libnpcg.so is not built ({LIB_PATH}); run "
                                   "paper_2305_16432_gb300.build.build() first")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, dbl, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_float
            sig = {
                "npcg_create": [C.POINTER(vp), vp],
                "npcg_destroy": [vp],
                "npcg_assemble_count": [vp, C.POINTER(_Problem), C.POINTER(i64), C.POINTER(i64)],
                "npcg_assemble_system": [vp, C.POINTER(_Problem), vp, vp, vp],
                "npcg_analyse": [vp, i64, i64, vp, vp, i32, vp, C.POINTER(vp)],
                "npcg_pattern_free": [vp],
                "npcg_pattern_get_info": [vp, C.POINTER(_Info)],
                "npcg_pattern_set_trsv": [vp, i32],
                "npcg_pattern_export": [vp, vp, vp, vp, vp, vp, vp, vp],
                "npcg_gnn_nparams": [C.POINTER(_Cfg), C.POINTER(i64)],
                "npcg_gnn_factor": [vp, vp, vp, vp, C.POINTER(_Cfg), vp, vp],
                "npcg_gnn_factor_x0": [vp, vp, vp, vp, C.POINTER(_Cfg), vp, vp, vp],
                "npcg_ic0_factor": [vp, vp, vp, vp, vp],
                "npcg_sgs_factor": [vp, vp, vp, vp],
                "npcg_pcg_solve": [vp, vp, vp, vp, vp, i32, vp, dbl, i32, vp],
                "npcg_pcg_solve_batched": [vp, vp, vp, vp, vp, i32, vp, dbl, i32, vp],
                "npcg_pcg_solve_ex": [vp, vp, vp, vp, vp, i32, vp, dbl, i32, C.POINTER(_Opts), vp],
                "npcg_spmv": [vp, vp, vp, vp, vp],
                "npcg_factor_load": [vp, vp, vp],
                "npcg_sptrsv": [vp, vp, i32, vp, vp],
                "npcg_sptrsv_timed": [vp, vp, i32, i32, vp, vp, i32, C.POINTER(dbl)],
                "npcg_sptrsv_unclaimed": [vp, vp, i32, i32, vp, vp],
                "npcg_set_wait_limit": [vp, i64],
                "npcg_set_pcg_eager": [vp, i32],
                "npcg_loss_and_grad": [vp, vp, vp, i32, vp, vp, C.POINTER(_Cfg), vp, C.POINTER(dbl), vp],
                "npcg_adam_step": [vp, i64, vp, vp, vp, vp, i32, f32, f32, f32, f32],
                "npcg_solve_host": [vp, vp, i32, C.POINTER(_Cfg), vp, vp, vp, vp, dbl, i32, i32, vp],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.npcg_last_error.argtypes = [vp]
            L.npcg_last_error.restype = C.c_char_p
            L.npcg_status_string.argtypes = [C.c_int]
            L.npcg_status_string.restype = C.c_char_p
            _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


class Handle:
    """npcg_create on the current device and torch's current stream."""

    def __init__(self, stream: torch.cuda.Stream | None = None):
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        st = lib().npcg_create(C.byref(h), C.c_void_p(self.stream.cuda_stream))
        if st != NPCG_OK:
            raise NpcgError(st, "npcg_create failed")
        self.h = h

    def check(self, st):
        if st != NPCG_OK:
            msg = lib().npcg_last_error(self.h).decode()
            raise NpcgError(lib().npcg_status_string(st).decode(), msg)

    def set_wait_limit(self, polls: int):
        """npcg_set_wait_limit: polls before a device wait gives up (<= 0: default)."""
        self.check(lib().npcg_set_wait_limit(self.h, C.c_int64(int(polls))))

    def set_pcg_eager(self, eager):
        """npcg_set_pcg_eager: True launches PCG iterations one by one, False
        through the loop graph, None restores the default (one by one for a
        row-block solve's triangular-solve preconditioners, else the graph)."""
        self.check(lib().npcg_set_pcg_eager(self.h, -1 if eager is None else (1 if eager else 0)))

    def close(self):
        if getattr(self, "h", None):
            lib().npcg_destroy(self.h)
            self.h = None

    def __del__(self):
        # at interpreter exit the CUDA runtime may already be gone: leave the
        # memory to the process teardown
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


_default = {}


def handle() -> Handle:
    """Handle cached per (device, current stream)."""
    key = (torch.cuda.current_device(), torch.cuda.current_stream().cuda_stream)
    if key not in _default:
        _default[key] = Handle()
    return _default[key]


# ------------------------------------------------------------------ assembly
def assemble_system(problem: I.Problem, omega=None, phase=None, jitter=None, h: Handle | None = None):
    """A of a synthetic diffusion problem, assembled on the GPU.
    Returns (row_ptr int32, col_idx int32, val float64) CUDA tensors."""
    h = h or handle()
    if omega is None:
        omega, phase = I.grf_features(problem)
    if problem.kind == I.FEM and jitter is None:
        jitter = I.fem_jitter(problem)
    dev = torch.device("cuda", h.device)
    om = torch.as_tensor(np.ascontiguousarray(omega).reshape(-1), dtype=torch.float64, device=dev)
    ph = torch.as_tensor(np.ascontiguousarray(phase), dtype=torch.float64, device=dev)
    jt = torch.as_tensor(np.ascontiguousarray(jitter), dtype=torch.int32, device=dev) if jitter is not None else None
    pr = _Problem(problem.kind, problem.dim, problem.nx, problem.ny, problem.nz, len(ph),
                  float(problem.sigma), om.data_ptr(), ph.data_ptr(), jt.data_ptr() if jt is not None else None,
                  float(problem.tau), int(problem.dir_start), int(problem.dir_len))
    n, nnz = C.c_int64(), C.c_int64()
    h.check(lib().npcg_assemble_count(h.h, C.byref(pr), C.byref(n), C.byref(nnz)))
    rp = torch.empty(n.value + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(nnz.value, dtype=torch.int32, device=dev)
    v = torch.empty(nnz.value, dtype=torch.float64, device=dev)
    h.check(lib().npcg_assemble_system(h.h, C.byref(pr), _ptr(rp), _ptr(ci), _ptr(v)))
    return rp, ci, v


# ------------------------------------------------------------------ pattern
class Pattern:
    """npcg_analyse result; freed with npcg_pattern_free."""

    def __init__(self, h: Handle, row_ptr, col_idx, sys_ptr=None):
        row_ptr = _dev(row_ptr, torch.int32, "row_ptr")
        col_idx = _dev(col_idx, torch.int32, "col_idx")
        self.h = h
        n = row_ptr.numel() - 1
        nsys = 1 if sys_ptr is None else len(sys_ptr) - 1
        sp = None
        if sys_ptr is not None:
            self._sys = np.ascontiguousarray(sys_ptr, dtype=np.int64)
            sp = self._sys.ctypes.data_as(C.c_void_p)
        p = C.c_void_p()
        h.check(lib().npcg_analyse(h.h, n, col_idx.numel(), _ptr(row_ptr), _ptr(col_idx), nsys, sp, C.byref(p)))
        self.p = p
        info = _Info()
        lib().npcg_pattern_get_info(p, C.byref(info))
        self.n, self.nnz, self.nnz_L = info.n, info.nnz, info.nnz_L
        self.nsys, self.nlev_fwd, self.nlev_bwd = info.nsys, info.nlev_fwd, info.nlev_bwd
        self.trsv_mode = info.trsv_mode
        self.max_row = info.max_row
        self.tuned_ms = {"syncfree": info.tuned_ms_syncfree, "levelsync": info.tuned_ms_levelsync,
                         "levelflag": info.tuned_ms_levelflag, "levelsplit": info.tuned_ms_levelsplit,
                         "levelmerge": info.tuned_ms_levelmerge}
        self.merge_levels = info.merge_levels
        self.block_units = info.block_units
        self.sys_ptr = np.asarray(sys_ptr if sys_ptr is not None else [0, n], dtype=np.int64)

    def set_trsv(self, mode):
        """Force a triangular-solve design (TRSV_SYNCFREE / TRSV_LEVELSYNC /
        TRSV_LEVELFLAG / TRSV_LEVELSPLIT / TRSV_LEVELMERGE) or restore the
        tuned one (TRSV_AUTO)."""
        self.h.check(lib().npcg_pattern_set_trsv(self.p, int(mode)))
        info = _Info()
        lib().npcg_pattern_get_info(self.p, C.byref(info))
        self.trsv_mode = info.trsv_mode
        self.merge_levels = info.merge_levels

    def export(self):
        dev = torch.device("cuda", self.h.device)
        out = dict(L_row_ptr=torch.empty(self.n + 1, dtype=torch.int32, device=dev),
                   L_col_idx=torch.empty(self.nnz_L, dtype=torch.int32, device=dev),
                   lev_fwd=torch.empty(self.n, dtype=torch.int32, device=dev),
                   lev_bwd=torch.empty(self.n, dtype=torch.int32, device=dev),
                   perm_fwd=torch.empty(self.n, dtype=torch.int32, device=dev),
                   perm_bwd=torch.empty(self.n, dtype=torch.int32, device=dev))
        self.h.check(lib().npcg_pattern_export(self.h.h, self.p, *[_ptr(out[k]) for k in
                     ("L_row_ptr", "L_col_idx", "lev_fwd", "lev_bwd", "perm_fwd", "perm_bwd")]))
        torch.cuda.synchronize()
        return out

    def close(self):
        if getattr(self, "p", None):
            lib().npcg_pattern_free(self.p)
            self.p = None

    def __del__(self):
        # at interpreter exit the CUDA runtime may already be gone: leave the
        # memory to the process teardown
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def analyse(row_ptr, col_idx, sys_ptr=None, h: Handle | None = None) -> Pattern:
    return Pattern(h or handle(), row_ptr, col_idx, sys_ptr)


# ------------------------------------------------------------------ factors
def _cfg(cfg: I.GnnConfig, precision=FP32):
    return _Cfg(cfg.n_mp, cfg.l, cfg.l_mp, cfg.h, cfg.diag_mode, precision, int(getattr(cfg, "x0_head", 0)),
                int(getattr(cfg, "loss", 0)))


def gnn_nparams(cfg: I.GnnConfig) -> int:
    out = C.c_int64()
    c = _cfg(cfg)
    st = lib().npcg_gnn_nparams(C.byref(c), C.byref(out))
    if st != NPCG_OK:
        raise NpcgError(st, "bad config")
    return out.value


def gnn_factor(P: Pattern, A_val, b, cfg: I.GnnConfig, weights, precision=FP32, out=None):
    """L on tril(A) from the graph network (FP64 values [nnz_L])."""
    A_val = _dev(A_val, torch.float64, "A_val")
    b = _dev(b, torch.float64, "b")
    weights = _dev(weights, torch.float32, "weights")
    L = out if out is not None else torch.empty(P.nnz_L, dtype=torch.float64, device=A_val.device)
    c = _cfg(cfg, precision)
    P.h.check(lib().npcg_gnn_factor(P.h.h, P.p, _ptr(A_val), _ptr(b), C.byref(c), _ptr(weights), _ptr(L)))
    return L


def gnn_factor_x0(P: Pattern, A_val, b, cfg: I.GnnConfig, weights, precision=FP32):
    """(L, x0): the factor and the initial-guess head's x0 [n] from one pass
    (cfg.x0_head must be 1)."""
    A_val = _dev(A_val, torch.float64, "A_val")
    b = _dev(b, torch.float64, "b")
    weights = _dev(weights, torch.float32, "weights")
    L = torch.empty(P.nnz_L, dtype=torch.float64, device=A_val.device)
    x0 = torch.empty(P.n, dtype=torch.float64, device=A_val.device)
    c = _cfg(cfg, precision)
    P.h.check(lib().npcg_gnn_factor_x0(P.h.h, P.p, _ptr(A_val), _ptr(b), C.byref(c), _ptr(weights), _ptr(L),
                                       _ptr(x0)))
    return L, x0


def ic0_factor(P: Pattern, A_val, out=None):
    A_val = _dev(A_val, torch.float64, "A_val")
    L = out if out is not None else torch.empty(P.nnz_L, dtype=torch.float64, device=A_val.device)
    alpha = np.zeros(P.nsys, np.float64)
    P.h.check(lib().npcg_ic0_factor(P.h.h, P.p, _ptr(A_val), _ptr(L), alpha.ctypes.data_as(C.c_void_p)))
    return L, alpha


def sgs_factor(P: Pattern, A_val, out=None):
    """Symmetric Gauss-Seidel as P = L L^T: L = (D + L_A) D^{-1/2} on tril(A)."""
    A_val = _dev(A_val, torch.float64, "A_val")
    L = out if out is not None else torch.empty(P.nnz_L, dtype=torch.float64, device=A_val.device)
    P.h.check(lib().npcg_sgs_factor(P.h.h, P.p, _ptr(A_val), _ptr(L)))
    return L


# ------------------------------------------------------------------ solve
def _stats_list(arr):
    return [dict(iters=s.iters, status=s.status, relres=s.relres, fallback=s.fallback,
                 fallback_iters=s.fallback_iters) for s in arr]


def pcg_solve(P: Pattern, A_val, b, precond=PREC_LLT, L_val=None, rtol=1e-6, max_iter=None, x0=None,
              raise_on_fail=False):
    """Algorithm 1 on the GPU.  Returns (x, stats) with stats a list of dicts."""
    A_val = _dev(A_val, torch.float64, "A_val")
    b = _dev(b, torch.float64, "b")
    x = torch.zeros_like(b) if x0 is None else _dev(x0, torch.float64, "x0").clone()
    if L_val is not None:
        L_val = _dev(L_val, torch.float64, "L_val")
    if max_iter is None:
        max_iter = int(min(10 * P.n, 2**31 - 1))
    stats = (_Stats * P.nsys)()
    fn = lib().npcg_pcg_solve if P.nsys == 1 else lib().npcg_pcg_solve_batched
    st = fn(P.h.h, P.p, _ptr(A_val), _ptr(b), _ptr(x), precond, _ptr(L_val), float(rtol), int(max_iter),
            C.cast(stats, C.c_void_p))
    if st != NPCG_OK and (raise_on_fail or st not in (NPCG_EMAXITER, NPCG_EBREAKDOWN)):
        P.h.check(st)
    return x, _stats_list(stats)


def pcg_solve_ex(P: Pattern, A_val, b, precond=PREC_LLT, L_val=None, rtol=1e-6, max_iter=None, x0=None,
                 stall_iters=0, fallback_ic0=False):
    """npcg_pcg_solve_ex: PCG with a stagnation window and the IC(0) fallback.
    Returns (x, stats, status)."""
    A_val = _dev(A_val, torch.float64, "A_val")
    b = _dev(b, torch.float64, "b")
    x = torch.zeros_like(b) if x0 is None else _dev(x0, torch.float64, "x0").clone()
    if L_val is not None:
        L_val = _dev(L_val, torch.float64, "L_val")
    if max_iter is None:
        max_iter = int(min(10 * P.n, 2**31 - 1))
    stats = (_Stats * P.nsys)()
    opts = _Opts(int(stall_iters), 1 if fallback_ic0 else 0)
    st = lib().npcg_pcg_solve_ex(P.h.h, P.p, _ptr(A_val), _ptr(b), _ptr(x), precond, _ptr(L_val), float(rtol),
                                 int(max_iter), C.byref(opts), C.cast(stats, C.c_void_p))
    if st not in (NPCG_OK, NPCG_EMAXITER, NPCG_EBREAKDOWN, NPCG_ESTALL):
        P.h.check(st)
    return x, _stats_list(stats), st


def spmv(P: Pattern, A_val, x, out=None):
    A_val = _dev(A_val, torch.float64, "A_val")
    x = _dev(x, torch.float64, "x")
    y = out if out is not None else torch.empty_like(x)
    P.h.check(lib().npcg_spmv(P.h.h, P.p, _ptr(A_val), _ptr(x), _ptr(y)))
    return y


def factor_load(P: Pattern, L_val):
    L_val = _dev(L_val, torch.float64, "L_val")
    P.h.check(lib().npcg_factor_load(P.h.h, P.p, _ptr(L_val)))


def sptrsv(P: Pattern, r, transpose=False, out=None):
    """With the loaded factor: L y = r (transpose False) or L^T y = r."""
    r = _dev(r, torch.float64, "r")
    y = out if out is not None else torch.empty_like(r)
    P.h.check(lib().npcg_sptrsv(P.h.h, P.p, 1 if transpose else 0, _ptr(r), _ptr(y)))
    return y


def sptrsv_unclaimed(P: Pattern, r, skip, transpose=False, out=None):
    """npcg_sptrsv_unclaimed (failure-path tests): the sync-free solve with its
    first `skip` slices never claimed.  Returns the status code (no raise)."""
    r = _dev(r, torch.float64, "r")
    y = out if out is not None else torch.empty_like(r)
    return lib().npcg_sptrsv_unclaimed(P.h.h, P.p, 1 if transpose else 0, int(skip), _ptr(r), _ptr(y))


def sptrsv_timed(P: Pattern, r, transpose=False, reps=20, out=None, f32=False):
    """Mean duration (ms) of the triangular-solve kernel over reps launches
    (f32: FP32 factor and arithmetic, as in PREC_LLT32)."""
    r = _dev(r, torch.float64, "r")
    y = out if out is not None else torch.empty_like(r)
    ms = C.c_double()
    P.h.check(lib().npcg_sptrsv_timed(P.h.h, P.p, 1 if transpose else 0, 1 if f32 else 0, _ptr(r), _ptr(y),
                                      int(reps), C.byref(ms)))
    return ms.value, y


# ------------------------------------------------------------------ training
def loss_and_grad(P: Pattern, A_val, X, B, cfg: I.GnnConfig, weights, precision=FP32, grad=None):
    """Loss Eq. (loss_Ab) and d loss / d weights (FP32)."""
    A_val = _dev(A_val, torch.float64, "A_val")
    X = _dev(X, torch.float64, "X")
    B = _dev(B, torch.float64, "B")
    weights = _dev(weights, torch.float32, "weights")
    npairs = X.shape[0] if X.dim() == 2 else 1
    g = grad if grad is not None else torch.empty_like(weights)
    loss = C.c_double()
    c = _cfg(cfg, precision)
    P.h.check(lib().npcg_loss_and_grad(P.h.h, P.p, _ptr(A_val), npairs, _ptr(X), _ptr(B), C.byref(c),
                                       _ptr(weights), C.byref(loss), _ptr(g)))
    return loss.value, g


def adam_step(w, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, h: Handle | None = None):
    h = h or handle()
    for name, t_ in (("w", w), ("g", g), ("m", m), ("v", v)):
        _dev(t_, torch.float32, name)
    h.check(lib().npcg_adam_step(h.h, w.numel(), _ptr(w), _ptr(g), _ptr(m), _ptr(v), int(t), lr, beta1,
                                 beta2, eps))


def solve_host(P: Pattern, A_val_host: np.ndarray, b_host: np.ndarray, method=METHOD_GNN,
               cfg: I.GnnConfig | None = None, weights=None, precision=FP32, rtol=1e-6, max_iter=None,
               x_host: np.ndarray | None = None, f32_apply=False):
    """End to end from host buffers: copy in, build the preconditioner, PCG, copy x out."""
    x = x_host if x_host is not None else np.empty(P.n, np.float64)
    c = _cfg(cfg, precision) if cfg is not None else None
    stats = (_Stats * P.nsys)()
    if max_iter is None:
        max_iter = int(min(10 * P.n, 2**31 - 1))
    st = lib().npcg_solve_host(P.h.h, P.p, method, C.byref(c) if c is not None else None,
                               _ptr(weights) if weights is not None else None,
                               A_val_host.ctypes.data_as(C.c_void_p), b_host.ctypes.data_as(C.c_void_p),
                               x.ctypes.data_as(C.c_void_p), float(rtol), int(max_iter),
                               1 if f32_apply else 0, C.cast(stats, C.c_void_p))
    if st not in (NPCG_OK, NPCG_EMAXITER, NPCG_EBREAKDOWN):
        P.h.check(st)
    return x, _stats_list(stats)


class LlTLoss(torch.autograd.Function):
    """Loss Eq. (loss_Ab), mean over pairs of ||L L^T x_p - b_p||^2 with
    L = f_theta(A, b_p), as a differentiable function of the flat FP32 weights.

    forward runs the network and the loss on the GPU and keeps the gradient
    that the same call computed with the hand-written adjoint (Sec. 4.3:
    the loss, its derivative in L, then the decoder, message-passing layers
    and encoders in reverse, with per-tile recomputation); backward only
    scales it by the incoming gradient.  A and the (x, b) pairs are data.
    """

    @staticmethod
    def forward(ctx, weights, P, A_val, X, B, cfg, precision=FP32):
        loss, g = loss_and_grad(P, A_val, X, B, cfg, weights.detach(), precision=precision)
        ctx.save_for_backward(g)
        return torch.tensor(loss, dtype=torch.float64, device=weights.device)

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        return (g * gout.to(g.dtype)), None, None, None, None, None, None


def llt_loss(weights, P: Pattern, A_val, X, B, cfg: I.GnnConfig, precision=FP32):
    """Differentiable loss: ``llt_loss(w, ...).backward()`` fills ``w.grad``."""
    return LlTLoss.apply(weights, P, A_val, X, B, cfg, precision)
