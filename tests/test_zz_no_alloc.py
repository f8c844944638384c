"""bt_pcg_solve_noalloc: the solve for callers that cannot allocate device
memory (for example a real-time loop whose memory is fixed at start-up, where
cudaMalloc's device synchronisation and unbounded latency are not allowed).

It must give the same answer as the allocating path (bt_setup +
bt_pcg_solve) through the C ABI, on two calls in a row -- the second call
reuses the static scratch array the first one left behind, so it also checks
that each call clears what must start at zero.  Runs on its own in a fresh
process and after the rest of the suite (this file is collected last)."""
import numpy as np
import pytest

from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import dev, host, rel

pytestmark = pytest.mark.gpu


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


def noalloc_solve(inst, params, tol, maxit, x_init=None):
    x = dev(np.zeros(inst.N * inst.n) if x_init is None else x_init)
    st, it = bb.bt_pcg_solve_noalloc(inst.N, inst.n, dev(inst.D), dev(inst.O), dev(inst.b.reshape(-1)), x,
                                     tol, maxit, params)
    return st, it, host(x)


@pytest.mark.parametrize("precision,tol", [(bb.BT_FP64, 1e-10), (bb.BT_MIXED, 1e-10)])
def test_noalloc_matches_allocating_path_two_calls(precision, tol):
    params, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=precision)
    first = wl.config1()                 # N = 128, n = 12
    second = wl.small_llt(7, 37, 9)      # different shape: odd N, odd n
    for inst in (first, second):
        st_a, it_a, x_a = allocating_solve(inst, params, tol, 2000)
        st_b, it_b, x_b = noalloc_solve(inst, params, tol, 2000, x_init=np.full(inst.N * inst.n, 3.0))
        assert st_a == bb.BT_OK and st_b == bb.BT_OK
        assert abs(it_a - it_b) <= 1
        assert rel(x_b, x_a) <= 1e-10


def test_noalloc_rejects_sizes_beyond_the_scratch():
    params, keep = bb.make_params(m=2, precision=bb.BT_FP64)
    N, n = 2048, 48  # float64 blocks alone exceed BT_NOALLOC_SCRATCH_BYTES
    D = dev(np.zeros(1))
    st, it = bb.bt_pcg_solve_noalloc(N, n, D, D, D, D, 1e-8, 10, params)
    assert st == bb.BT_ERR_ARG
