"""ctypes binding of libbt (include/bt.h).

Argument marshalling only: every function here forwards to the C entry point
of the same name; all arithmetic runs in the library's CUDA kernels.  Device
arrays are torch CUDA float64 tensors (contiguous); work is queued on the
current torch stream unless a stream is given.

The library is loaded on first use.  If libbt.so is missing this raises;
there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbt.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "bt.h")

BT_OK, BT_ERR_ARG, BT_ERR_PARAM, BT_ERR_NOT_SPD, BT_ERR_NO_CONVERGENCE = 0, 1, 2, 3, 4
BT_ERR_BREAKDOWN, BT_ERR_NONFINITE, BT_ERR_TIMEOUT, BT_ERR_CUDA, BT_ERR_ALLOC, BT_ERR_STATE = 5, 6, 7, 8, 9, 10
BT_FP64, BT_MIXED = 0, 1

PRESETS = {"optimal": None, "polycoeff": "last7"}


class bt_params(C.Structure):
    _fields_ = [
        ("a", C.c_double),
        ("m", C.c_int),
        ("alpha", C.POINTER(C.c_double)),
        ("precision", C.c_int),
        ("tol_inner", C.c_double),
        ("max_outer", C.c_int),
        ("use_x0", C.c_int),
        ("cycle_budget", C.c_longlong),
        ("stream", C.c_void_p),
        ("ctas_per_sm", C.c_int),
        ("group_ctas", C.c_int),
        ("stage_kb", C.c_int),
        ("h_matrix_free", C.c_int),
        ("mrhs_engine", C.c_int),
        ("mixed_strict_fp64", C.c_int),
    ]


_lib = None


def lib() -> C.CDLL:
    """Load libbt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is the only compute path)")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip, llp = C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_longlong)
    H = C.c_void_p
    sig = {
        "bt_params_init": (None, [C.POINTER(bt_params)]),
        "bt_setup": (C.c_int, [C.c_int, C.c_int, dp, dp, C.POINTER(bt_params), C.POINTER(H)]),
        "bt_refactor": (C.c_int, [H, dp, dp]),
        "bt_setup_status": (C.c_int, [H]),
        "bt_pcg_solve_async": (C.c_int, [H, dp, dp, C.c_double, C.c_int, vp, vp]),
        "bt_apply_precond": (C.c_int, [H, dp, dp]),
        "bt_spmv": (C.c_int, [H, dp, dp]),
        "bt_spmv_f32": (C.c_int, [H, dp, dp]),
        "bt_pcg_solve": (C.c_int, [H, dp, dp, C.c_double, C.c_int, ip]),
        "bt_solve_info": (C.c_int, [H, C.c_int, ip, C.POINTER(C.c_double)]),
        "bt_setup_batched": (C.c_int, [C.c_int, ip, ip, llp, llp, dp, dp, C.POINTER(bt_params), C.POINTER(H)]),
        "bt_pcg_solve_batched": (C.c_int, [H, dp, dp, llp, C.c_double, C.c_int, ip, ip]),
        "bt_pcg_solve_batched_async": (C.c_int, [H, dp, dp, C.c_double, C.c_int, vp, vp]),
        "bt_graph_capture_batched": (C.c_int, [H, dp, dp, C.c_double, C.c_int, vp, vp]),
        "bt_graph_capture_refactor_solve": (C.c_int, [H, dp, dp, dp, dp, C.c_double, C.c_int, vp, vp]),
        "bt_graph_launch": (C.c_int, [H]),
        "bt_adjoint_blocks": (C.c_int, [H, dp, dp, dp, dp]),
        "bt_pcg_solve_noalloc": (C.c_int, [C.c_int, C.c_int, dp, dp, dp, dp, C.c_double, C.c_int,
                                           C.POINTER(bt_params), ip]),
        "bt_pcg_solve_multi": (C.c_int, [H, dp, dp, C.c_int, C.c_double, C.c_int, ip, ip]),
        "bt_multi_info": (C.c_int, [H, C.c_int, ip, C.POINTER(C.c_double)]),
        "bt_last_error": (C.c_int, [H, ip, ip, C.POINTER(C.c_double)]),
        "bt_params_check": (C.c_int, [C.POINTER(bt_params)]),
        "bt_estimate_rho": (C.c_int, [H, C.c_int, C.POINTER(C.c_double)]),
        "bt_autotune": (C.c_int, [H, dp, dp, C.c_double, C.c_int, C.c_int, ip, ip]),
        "bt_set_history": (C.c_int, [H, dp, C.c_int]),
        "bt_ritz_rho": (C.c_int, [H, dp, C.c_int, C.POINTER(C.c_double)]),
        "bt_alpha_chebyshev": (C.c_int, [C.c_int, C.c_double, C.POINTER(C.c_double)]),
        "bt_lqr_schur": (C.c_int, [C.c_int, ip, ip, ip, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, vp, ip, ip]),
        "bt_lqr_recover": (C.c_int, [C.c_int, ip, ip, ip, dp, dp, dp, dp, dp, dp, dp, dp, dp, vp]),
        "bt_lqr_refactor": (C.c_int, [H, ip, dp, dp, dp, dp, dp, dp, dp, dp, ip, ip]),
        "bt_lqr_recover_factored": (C.c_int, [H, ip, dp, dp, dp, dp, dp, dp, dp]),
        "bt_device_bytes": (C.c_longlong, [H]),
        "bt_destroy": (None, [H]),
        "bt_status_string": (C.c_char_p, [C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_functions() -> list:
    """Names of every function bt.h declares (used by the export test)."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bt_[a-z0-9_]+)\s*\(", txt)))


class BTError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().bt_status_string(status).decode()
        super().__init__(f"{where}: status {status} ({msg})")


def status_string(s: int) -> str:
    return lib().bt_status_string(s).decode()


def _ptr(t) -> C.c_void_p:
    if t is None:
        return C.c_void_p(0)
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda, "device arrays must be CUDA tensors"
    assert t.is_contiguous(), "device arrays must be contiguous"
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def polycoeff_alpha(m: int, last: float = 7.0) -> list:
    """alpha_{m-1} = 7, others 1 (the setting of the paper's experiments, Sec. 5)."""
    return [1.0] * m if m == 1 else [1.0] * (m - 1) + [last]


def make_params(m: int = 2, alpha: Optional[Sequence[float]] = None, precision: int = BT_FP64,
                tol_inner: float = 0.0, max_outer: int = 0, use_x0: bool = False, cycle_budget: int = 0,
                stream=None, ctas_per_sm: int = 0, group_ctas: int = 0, stage_kb: int = 0,
                a: float = 1.0, h_matrix_free: bool = False, mrhs_engine: int = 0,
                mixed_strict_fp64: bool = False):
    """Build a bt_params; returns (params, keepalive)."""
    p = bt_params()
    lib().bt_params_init(C.byref(p))
    p.a = a
    p.m = m
    keep = None
    if alpha is not None:
        keep = (C.c_double * len(alpha))(*[float(v) for v in alpha])
        p.alpha = C.cast(keep, C.POINTER(C.c_double))
    p.precision = precision
    p.tol_inner = tol_inner
    p.max_outer = max_outer
    p.use_x0 = 1 if use_x0 else 0
    p.cycle_budget = cycle_budget
    p.stream = _stream_ptr(stream)
    p.ctas_per_sm = ctas_per_sm
    p.group_ctas = group_ctas
    p.stage_kb = stage_kb
    p.h_matrix_free = 1 if h_matrix_free else 0
    p.mrhs_engine = mrhs_engine
    p.mixed_strict_fp64 = 1 if mixed_strict_fp64 else 0
    return p, keep


# ---------------------------------------------------------------------------
# Entry points with the C names.
# ---------------------------------------------------------------------------
def bt_setup(N: int, n: int, D, O, params: bt_params):
    h = C.c_void_p()
    st = lib().bt_setup(N, n, _ptr(D), _ptr(O) if O is not None and O.numel() else C.c_void_p(0),
                        C.byref(params), C.byref(h))
    return st, h


def bt_setup_batched(Ns, ns, d_off, o_off, D, O, params: bt_params):
    B = len(Ns)
    Na = (C.c_int * B)(*[int(v) for v in Ns])
    na = (C.c_int * B)(*[int(v) for v in ns])
    da = (C.c_longlong * B)(*[int(v) for v in d_off])
    oa = (C.c_longlong * B)(*[int(v) for v in o_off])
    h = C.c_void_p()
    st = lib().bt_setup_batched(B, Na, na, da, oa, _ptr(D), _ptr(O) if O is not None and O.numel() else C.c_void_p(0),
                                C.byref(params), C.byref(h))
    return st, h


def bt_refactor(h, D, O) -> int:
    return lib().bt_refactor(h, _ptr(D), _ptr(O) if O is not None and O.numel() else C.c_void_p(0))


def bt_setup_status(h) -> int:
    return lib().bt_setup_status(h)


def bt_pcg_solve_async(h, b, x, tol: float, maxit: int, d_iters=None, d_status=None) -> int:
    return lib().bt_pcg_solve_async(h, _ptr(b), _ptr(x), float(tol), int(maxit), _ptr(d_iters), _ptr(d_status))


def bt_apply_precond(h, r, z) -> int:
    return lib().bt_apply_precond(h, _ptr(r), _ptr(z))


def bt_spmv(h, x, y) -> int:
    return lib().bt_spmv(h, _ptr(x), _ptr(y))


def bt_spmv_f32(h, x, y) -> int:
    return lib().bt_spmv_f32(h, _ptr(x), _ptr(y))


def bt_pcg_solve(h, b, x, tol: float, maxit: int):
    it = C.c_int(0)
    st = lib().bt_pcg_solve(h, _ptr(b), _ptr(x), float(tol), int(maxit), C.byref(it))
    return st, it.value


def bt_solve_info(h, k: int = 0):
    o = C.c_int(0)
    r = C.c_double(0.0)
    st = lib().bt_solve_info(h, k, C.byref(o), C.byref(r))
    return st, o.value, r.value


def bt_pcg_solve_batched(h, b, x, B: int, tol: float, maxit: int, vec_off=None):
    it = (C.c_int * B)()
    ss = (C.c_int * B)()
    vo = None if vec_off is None else (C.c_longlong * B)(*[int(v) for v in vec_off])
    st = lib().bt_pcg_solve_batched(h, _ptr(b), _ptr(x), vo, float(tol), int(maxit), it, ss)
    return st, np.array(it[:], dtype=np.int64), np.array(ss[:], dtype=np.int64)


def bt_pcg_solve_batched_async(h, b, x, tol: float, maxit: int, d_iters=None, d_status=None) -> int:
    return lib().bt_pcg_solve_batched_async(h, _ptr(b), _ptr(x), float(tol), int(maxit), _ptr(d_iters),
                                            _ptr(d_status))


def bt_graph_capture_batched(h, b, x, tol: float, maxit: int, d_iters=None, d_status=None) -> int:
    return lib().bt_graph_capture_batched(h, _ptr(b), _ptr(x), float(tol), int(maxit), _ptr(d_iters),
                                          _ptr(d_status))


def bt_graph_capture_refactor_solve(h, D, O, b, x, tol: float, maxit: int, d_iters=None, d_status=None) -> int:
    return lib().bt_graph_capture_refactor_solve(h, _ptr(D), _ptr(O), _ptr(b), _ptr(x), float(tol), int(maxit),
                                                 _ptr(d_iters), _ptr(d_status))


def bt_graph_launch(h) -> int:
    return lib().bt_graph_launch(h)


def bt_adjoint_blocks(h, x, g, gD, gO) -> int:
    return lib().bt_adjoint_blocks(h, _ptr(x), _ptr(g), _ptr(gD), _ptr(gO))


def bt_pcg_solve_noalloc(N: int, n: int, D, O, b, x, tol: float, maxit: int, params: bt_params):
    it = C.c_int(0)
    st = lib().bt_pcg_solve_noalloc(N, n, _ptr(D), _ptr(O) if O is not None and O.numel() else C.c_void_p(0),
                                    _ptr(b), _ptr(x), float(tol), int(maxit), C.byref(params), C.byref(it))
    return st, it.value


def bt_pcg_solve_multi(h, B, X, nrhs: int, tol: float, maxit: int):
    it = (C.c_int * nrhs)()
    ss = (C.c_int * nrhs)()
    st = lib().bt_pcg_solve_multi(h, _ptr(B), _ptr(X), int(nrhs), float(tol), int(maxit), it, ss)
    return st, np.array(it[:], dtype=np.int64), np.array(ss[:], dtype=np.int64)


def bt_autotune(h, b, x, tol: float, maxit: int, trials: int = 2):
    """Returns (status, stage_kb, group_ctas)."""
    kb, g = C.c_int(0), C.c_int(0)
    st = lib().bt_autotune(h, _ptr(b), _ptr(x), float(tol), int(maxit), int(trials), C.byref(kb), C.byref(g))
    return st, kb.value, g.value


def bt_set_history(h, hist, length: int) -> int:
    return lib().bt_set_history(h, _ptr(hist) if hist is not None else C.c_void_p(0), int(length))


def bt_ritz_rho(h, b, iters: int, count: int):
    """Returns (status, rho per instance)."""
    r = (C.c_double * max(1, count))()
    st = lib().bt_ritz_rho(h, _ptr(b), int(iters), r)
    return st, list(r[:count])


def bt_estimate_rho(h, iters: int, count: int):
    """Returns (status, rho per instance)."""
    r = (C.c_double * max(1, count))()
    st = lib().bt_estimate_rho(h, int(iters), r)
    return st, list(r[:count])


def bt_alpha_chebyshev(m: int, rho: float):
    """Returns (status, alpha list)."""
    a = (C.c_double * max(1, m))()
    st = lib().bt_alpha_chebyshev(int(m), float(rho), a)
    return st, list(a[:m])


def _iarr(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def _optr(t):
    return _ptr(t) if t is not None and t.numel() else C.c_void_p(0)


def bt_lqr_schur(N, n, m, A, Bm, Q, R, q, r, c, D, O, gamma, stream=None):
    """Returns (status, bad_instance, bad_row)."""
    (Na, Np), (na, nP), (ma, mP) = _iarr(N), _iarr(n), _iarr(m)
    bi, br = C.c_int(-1), C.c_int(-1)
    st = lib().bt_lqr_schur(len(Na), Np, nP, mP, _optr(A), _optr(Bm), _ptr(Q), _optr(R), _ptr(q), _optr(r),
                            _ptr(c), _ptr(D), _optr(O), _ptr(gamma), _stream_ptr(stream), C.byref(bi), C.byref(br))
    return st, bi.value, br.value


def bt_lqr_refactor(h, m, A, Bm, Q, R, q, r, c, gamma):
    """Returns (status, bad_instance, bad_row)."""
    ma, mP = _iarr(m)
    bi, br = C.c_int(-1), C.c_int(-1)
    st = lib().bt_lqr_refactor(h, mP, _optr(A), _optr(Bm), _ptr(Q), _optr(R), _ptr(q), _optr(r), _ptr(c),
                               _ptr(gamma), C.byref(bi), C.byref(br))
    return st, bi.value, br.value


def bt_lqr_recover_factored(h, m, A, Bm, q, r, lam, x, u) -> int:
    ma, mP = _iarr(m)
    return lib().bt_lqr_recover_factored(h, mP, _optr(A), _optr(Bm), _ptr(q), _optr(r), _ptr(lam), _ptr(x),
                                         _optr(u))


def bt_lqr_recover(N, n, m, A, Bm, Q, R, q, r, lam, x, u, stream=None) -> int:
    (Na, Np), (na, nP), (ma, mP) = _iarr(N), _iarr(n), _iarr(m)
    return lib().bt_lqr_recover(len(Na), Np, nP, mP, _optr(A), _optr(Bm), _ptr(Q), _optr(R), _ptr(q), _optr(r),
                                _ptr(lam), _ptr(x), _optr(u), _stream_ptr(stream))


def bt_multi_info(h, j: int):
    o = C.c_int(0)
    r = C.c_double(0.0)
    st = lib().bt_multi_info(h, int(j), C.byref(o), C.byref(r))
    return st, o.value, r.value


def bt_last_error(h):
    i, b, v = C.c_int(0), C.c_int(0), C.c_double(0.0)
    st = lib().bt_last_error(h, C.byref(i), C.byref(b), C.byref(v))
    return st, i.value, b.value, v.value


def bt_device_bytes(h) -> int:
    return lib().bt_device_bytes(h)


def bt_destroy(h) -> None:
    lib().bt_destroy(h)


def bt_status_string(s: int) -> str:
    return status_string(s)
