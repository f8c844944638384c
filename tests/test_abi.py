"""The C-ABI library loads and exports every entry point include/bt.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import shutil

import pytest

from paper_2503_15269_gb300 import binding as bb


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(bb.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build libbt.so")
        from paper_2503_15269_gb300 import build
        build.build()
    return ctypes.CDLL(bb.LIB_PATH)


def test_header_declares_the_boundary():
    names = bb.header_functions()
    for required in ["bt_setup", "bt_apply_precond", "bt_spmv", "bt_pcg_solve", "bt_setup_batched",
                     "bt_pcg_solve_batched", "bt_last_error", "bt_destroy", "bt_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(built):
    missing = [n for n in bb.header_functions() if not hasattr(built, n)]
    assert not missing, missing


def test_status_strings_and_params_defaults(built):
    lib = bb.lib()
    for s in range(11):
        assert lib.bt_status_string(s)
    p = bb.bt_params()
    lib.bt_params_init(ctypes.byref(p))
    assert p.a == 1.0 and p.m == 2 and p.precision == bb.BT_FP64


def test_bad_arguments_rejected_without_a_gpu(built):
    """Argument checks run on the host before any CUDA call."""
    lib = bb.lib()
    p = bb.bt_params()
    lib.bt_params_init(ctypes.byref(p))
    h = ctypes.c_void_p()
    assert lib.bt_setup(0, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.byref(p), ctypes.byref(h)) == bb.BT_ERR_ARG
    assert lib.bt_setup(4, 65, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.byref(p), ctypes.byref(h)) == bb.BT_ERR_ARG
    p.a = -0.25  # outside the admissible set C_g = [0, 1] (Sec. 3.3)
    assert lib.bt_setup(4, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.byref(p), ctypes.byref(h)) == bb.BT_ERR_PARAM
    p.a = 0.5  # admissible, but the no-allocation entry implements a = 1 only
    it = ctypes.c_int()
    assert lib.bt_pcg_solve_noalloc(4, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                    ctypes.c_void_p(16), ctypes.c_double(1e-8), 10, ctypes.byref(p),
                                    ctypes.byref(it)) == bb.BT_ERR_PARAM
    p.a = 0.5  # polynomial coefficients other than ones only with (G_opt, H_opt)
    pc = (ctypes.c_double * 2)(1.0, 7.0)
    p.alpha = ctypes.cast(pc, ctypes.POINTER(ctypes.c_double))
    assert lib.bt_setup(4, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.byref(p), ctypes.byref(h)) == bb.BT_ERR_PARAM
    p.alpha = None
    p.a = 1.5
    assert lib.bt_setup(4, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.byref(p), ctypes.byref(h)) == bb.BT_ERR_PARAM
    p.a = 1.0
    p.m = 0
    assert lib.bt_setup(4, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.byref(p), ctypes.byref(h)) == bb.BT_ERR_PARAM
    p.m = 2
    bad = (ctypes.c_double * 2)(2.0, 7.0)
    p.alpha = ctypes.cast(bad, ctypes.POINTER(ctypes.c_double))
    assert lib.bt_setup(4, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.byref(p), ctypes.byref(h)) == bb.BT_ERR_PARAM
    neg = (ctypes.c_double * 2)(1.0, -1.0)
    p.alpha = ctypes.cast(neg, ctypes.POINTER(ctypes.c_double))
    assert lib.bt_setup(4, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.byref(p), ctypes.byref(h)) == bb.BT_ERR_PARAM
    assert lib.bt_pcg_solve(None, None, None, 1e-8, 10, None) == bb.BT_ERR_ARG
    assert lib.bt_autotune(None, None, None, 1e-8, 10, 1, None, None) == bb.BT_ERR_ARG
    # LQR formation: sizes are checked on the host before any CUDA call
    one = (ctypes.c_int * 1)(4)
    big = (ctypes.c_int * 1)(49)
    vp = ctypes.c_void_p(16)
    args = (vp,) * 10
    assert lib.bt_lqr_schur(1, one, big, one, *args, None, None, None) == bb.BT_ERR_ARG
    assert lib.bt_lqr_schur(0, one, one, one, *args, None, None, None) == bb.BT_ERR_ARG
    assert lib.bt_lqr_recover(1, one, one, big, *((vp,) * 9), None) == bb.BT_ERR_ARG
    assert lib.bt_lqr_refactor(None, one, *((vp,) * 8), None, None) == bb.BT_ERR_ARG
    # knots beyond the first need the dynamics, inputs and input costs
    two = (ctypes.c_int * 1)(2)
    assert lib.bt_lqr_schur(1, two, one, one, None, None, vp, None, vp, None, vp, vp, vp, vp, None, None,
                            None) == bb.BT_ERR_ARG
    assert lib.bt_lqr_recover(1, two, one, one, None, None, vp, None, vp, None, vp, vp, vp, None) == bb.BT_ERR_ARG
