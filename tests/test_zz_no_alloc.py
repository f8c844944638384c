"""bt_pcg_solve_noalloc: the solve for callers that cannot allocate device
memory (for example a real-time loop whose memory is fixed at start-up, where
cudaMalloc's device synchronisation and unbounded latency are not allowed).

It must give the same answer as the allocating path (bt_setup +
bt_pcg_solve) through the C ABI, on two calls in a row -- the second call
reuses the static scratch array the first one left behind, so it also checks
that each call clears what must start at zero -- and the oracle's answer.
This file is collected last, so it runs after the rest of the suite; one test
repeats the two-call check in a child process of its own, where the first
call meets the array as the module loaded it."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import dev, host, rel

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


def allocating_solve(inst, params, tol, maxit):
    st, h = bb.bt_setup(inst.N, inst.n, dev(inst.D), dev(inst.O), params)
    assert st == bb.BT_OK, bb.status_string(st)
    try:
        x = dev(np.zeros(inst.N * inst.n))
        st, it = bb.bt_pcg_solve(h, dev(inst.b.reshape(-1)), x, tol, maxit)
    finally:
        bb.bt_destroy(h)
    return st, it, host(x)


def noalloc_solve(inst, params, tol, maxit, x_init=None, b=None):
    x = dev(np.zeros(inst.N * inst.n) if x_init is None else x_init)
    bv = inst.b.reshape(-1) if b is None else b
    st, it = bb.bt_pcg_solve_noalloc(inst.N, inst.n, dev(inst.D), dev(inst.O), dev(bv), x, tol, maxit, params)
    return st, it, host(x)


def two_calls(precision, tol):
    """Two no-allocation solves of different shapes in a row, each against the
    allocating path (same status, iterations within 1, x within 1e-10) and
    against the oracle's direct solve (within cond(S) * tol, cond ~ 1e3)."""
    params, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=precision)
    first = wl.config1()                 # N = 128, n = 12
    second = wl.small_llt(7, 37, 9)      # different shape: odd N, odd n
    for inst in (first, second):
        # the allocating path on the persistent kernel at the shape the
        # no-allocation entry takes (one CTA up to N = 32, else N / 4)
        g = 1 if inst.N <= 32 else inst.N // 4
        p_alloc, keep_a = bb.make_params(m=2, alpha=[1.0, 7.0], precision=precision, group_ctas=g)
        st_a, it_a, x_a = allocating_solve(inst, p_alloc, tol, 2000)
        st_b, it_b, x_b = noalloc_solve(inst, params, tol, 2000, x_init=np.full(inst.N * inst.n, 3.0))
        assert st_a == bb.BT_OK and st_b == bb.BT_OK
        assert abs(it_a - it_b) <= 1
        assert rel(x_b, x_a) <= 1e-10
        xr = orc.direct_solve(inst.D, inst.O, inst.b).reshape(-1)
        assert rel(x_b, xr) <= 1e-6, rel(x_b, xr)


@pytest.mark.parametrize("precision,tol", [(bb.BT_FP64, 1e-10), (bb.BT_MIXED, 1e-10)])
def test_noalloc_matches_allocating_path_two_calls(precision, tol):
    two_calls(precision, tol)


def test_noalloc_clean_call_after_nonfinite_input():
    """A call whose b holds a NaN (status BT_ERR_NONFINITE) leaves non-finite
    values in the shared array; the next, smaller call must not see them."""
    params, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED)
    big = wl.config1()
    b = big.b.reshape(-1).copy()
    b[17] = np.nan
    st, it, _ = noalloc_solve(big, params, 1e-10, 2000, b=b)
    assert st == bb.BT_ERR_NONFINITE
    small = wl.small_llt(8, 21, 7)
    st_a, it_a, x_a = allocating_solve(small, params, 1e-10, 2000)
    st_b, it_b, x_b = noalloc_solve(small, params, 1e-10, 2000)
    assert st_a == bb.BT_OK and st_b == bb.BT_OK
    assert abs(it_a - it_b) <= 1 and rel(x_b, x_a) <= 1e-10


def test_noalloc_two_calls_in_a_fresh_process():
    code = ("import sys; sys.path[:0] = [%r, %r]; import test_zz_no_alloc as t; "
            "from paper_2503_15269_gb300 import binding as bb; bb.lib(); "
            "t.two_calls(bb.BT_MIXED, 1e-10); t.two_calls(bb.BT_FP64, 1e-10); print('fresh ok')"
            % (ROOT, os.path.join(ROOT, "tests")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0 and "fresh ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]


def test_noalloc_rejects_sizes_beyond_the_scratch():
    params, keep = bb.make_params(m=2, precision=bb.BT_FP64)
    N, n = 2048, 48  # float64 blocks alone exceed BT_NOALLOC_SCRATCH_BYTES
    D = dev(np.zeros(1))
    st, it = bb.bt_pcg_solve_noalloc(N, n, D, D, D, D, 1e-8, 10, params)
    assert st == bb.BT_ERR_ARG
