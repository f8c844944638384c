"""The shared-memory engine for small single instances, float64 and mixed
(one CTA, or a cluster of 2, 4 or 8 CTAs sharing the block rows, every block
resident):
against the oracle's PCG (iterations within 1, solution within 1e-10),
against the persistent kernel, status paths, history recording,
eligibility and the autotuner's choice between the two mappings."""
import numpy as np
import pytest
import torch

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import Single, dev, host, rel

pytestmark = pytest.mark.gpu

SMALL, PERSISTENT = -1, 1  # group_ctas: shared-memory engine (one CTA), persistent kernel on one CTA


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


def test_config0_small_engine_matches_oracle():
    inst = wl.config0()  # LL^T N = 16, n = 6, float64 to 1e-10
    alpha = [1.0, 7.0]
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, alpha, 1e-10, 500)
    with Single(inst, m=2, alpha=alpha, group_ctas=SMALL) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-10, 500)
    assert st == bb.BT_OK
    assert abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10


@pytest.mark.parametrize("N,n", [(1, 3), (2, 1), (3, 6), (7, 8), (16, 6), (40, 4), (16, 12)])
@pytest.mark.parametrize("m,alpha", [(1, [1.0]), (2, [1.0, 7.0]), (3, [1.0, 1.0, 1.0])])
def test_small_engine_matches_oracle_and_persistent(N, n, m, alpha):
    inst = wl.small_llt(90, N, n)
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, alpha, 1e-11, 2000)
    out = {}
    for g in (SMALL, PERSISTENT):
        with Single(inst, m=m, alpha=alpha, group_ctas=g) as s:
            s.ok()
            st, it, x = s.solve(inst.b, 1e-11, 2000)
            assert st == bb.BT_OK
            out[g] = (it, x)
    it, x = out[SMALL]
    assert abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10
    assert abs(it - out[PERSISTENT][0]) <= 1
    assert rel(x, out[PERSISTENT][1]) <= 1e-10


def test_config1_float64_on_a_cluster_matches_oracle():
    """LQR N = 128, n = 12 (1.1 MB of float64 blocks): the engine on a cluster
    of 8 CTAs (16 block rows each), as the automatic choice picks it."""
    inst = wl.config1()
    alpha = [1.0, 7.0]
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, alpha, 1e-10, 2000)
    for g in (-8, 0):
        with Single(inst, m=2, alpha=alpha, group_ctas=g) as s:
            s.ok()
            st, it, x = s.solve(inst.b, 1e-10, 2000)
        assert st == bb.BT_OK
        assert abs(it - ref.iters) <= 1
        assert rel(x, ref.x) <= 1e-10


# ragged row splits (N not a multiple of C; two rows in some CTAs), every H
# sweep reading two halo rows from a neighbour
@pytest.mark.parametrize("N,n,C", [(4, 6, 2), (9, 5, 4), (17, 8, 8), (16, 6, 8), (50, 12, 4), (33, 16, 8)])
@pytest.mark.parametrize("m,alpha", [(1, [1.0]), (2, [1.0, 7.0]), (3, [1.0, 2.0, 3.0])])
def test_cluster_engine_matches_oracle_and_persistent(N, n, C, m, alpha):
    inst = wl.small_llt(95, N, n)
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, alpha, 1e-11, 2000)
    out = {}
    for g in (-C, PERSISTENT):
        with Single(inst, m=m, alpha=alpha, group_ctas=g) as s:
            s.ok()
            st, it, x = s.solve(inst.b, 1e-11, 2000)
            assert st == bb.BT_OK
            out[g] = (it, x)
    it, x = out[-C]
    assert abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10
    assert rel(x, out[PERSISTENT][1]) <= 1e-10


def test_cluster_engine_status_paths_and_initial_guess():
    inst = wl.small_llt(96, 24, 6)
    xr = orc.direct_solve(inst.D, inst.O, inst.b)
    with Single(inst, m=2, alpha=[1.0, 7.0], group_ctas=-4, use_x0=True) as s:
        s.ok()
        st, it, x = s.solve(np.zeros_like(inst.b), 1e-10, 100, x0=np.zeros_like(inst.b))
        assert st == bb.BT_OK and it == 0 and np.all(x == 0)
        st, it, x = s.solve(inst.b, 1e-14, 3, x0=np.zeros_like(inst.b))
        assert st == bb.BT_ERR_NO_CONVERGENCE and it == 3
        b = inst.b.copy()
        b[20, 2] = np.inf
        st, it, x = s.solve(b, 1e-10, 100, x0=np.zeros_like(inst.b))
        assert st == bb.BT_ERR_NONFINITE
        x0 = xr + 1e-3 * np.random.default_rng(5).standard_normal(xr.shape)
        st, it, x = s.solve(inst.b, 1e-12, 300, x0=x0)
        assert st == bb.BT_OK
        ref = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-12, 300, x0=x0)
        assert abs(it - ref.iters) <= 1 and rel(x, xr) <= 1e-9


def test_cluster_engine_rejects_too_few_rows_per_cta():
    inst = wl.small_llt(97, 10, 4)  # 8 CTAs would hold one row each
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], group_ctas=-8)
    st, h = bb.bt_setup(inst.N, inst.n, dev(inst.D), dev(inst.O), p)
    assert st == bb.BT_ERR_ARG
    if h:
        bb.bt_destroy(h)


def test_small_engine_status_paths():
    inst = wl.small_llt(91, 12, 5)
    with Single(inst, m=2, alpha=[1.0, 7.0], group_ctas=SMALL) as s:
        s.ok()
        # zero right-hand side: x = 0, no iterations
        st, it, x = s.solve(np.zeros_like(inst.b), 1e-10, 100)
        assert st == bb.BT_OK and it == 0 and np.all(x == 0)
        # iteration limit
        st, it, x = s.solve(inst.b, 1e-14, 2)
        assert st == bb.BT_ERR_NO_CONVERGENCE and it == 2
        # non-finite input
        b = inst.b.copy()
        b[3, 1] = np.nan
        st, it, x = s.solve(b, 1e-10, 100)
        assert st == bb.BT_ERR_NONFINITE
        # a clean solve afterwards
        st, it, x = s.solve(inst.b, 1e-10, 200)
        assert st == bb.BT_OK
        assert rel(x, orc.direct_solve(inst.D, inst.O, inst.b)) <= 1e-8


def test_small_engine_initial_guess():
    inst = wl.small_llt(92, 10, 6)
    xr = orc.direct_solve(inst.D, inst.O, inst.b)
    x0 = xr + 1e-3 * np.random.default_rng(2).standard_normal(xr.shape)
    with Single(inst, m=2, alpha=[1.0, 7.0], group_ctas=SMALL, use_x0=True) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-12, 200, x0=x0)
    assert st == bb.BT_OK
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-12, 200, x0=x0)
    assert abs(it - ref.iters) <= 1
    assert rel(x, xr) <= 1e-9


def test_small_engine_history_matches_persistent():
    inst = wl.small_llt(93, 16, 6)
    hists = {}
    for g in (SMALL, -4, PERSISTENT):
        hist = torch.zeros(64 * 3, dtype=torch.float64, device="cuda")
        with Single(inst, m=2, alpha=[1.0, 7.0], group_ctas=g) as s:
            s.ok()
            assert bb.bt_set_history(s.h, hist, 64) == bb.BT_OK
            st, it, x = s.solve(inst.b, 1e-10, 64)
            assert st == bb.BT_OK
        hists[g] = (it, host(hist).reshape(64, 3))
    it = min(h[0] for h in hists.values())
    for g in (SMALL, -4):
        a, b = hists[g][1][:it], hists[PERSISTENT][1][:it]
        assert np.allclose(a, b, rtol=1e-8, atol=1e-14), g


def test_small_engine_rejected_where_it_does_not_fit():
    inst = wl.small_llt(94, 200, 16)  # 7 float64 block arrays of 200 x 16 x 16: 2.9 MB
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], group_ctas=SMALL)
    st, h = bb.bt_setup(inst.N, inst.n, dev(inst.D), dev(inst.O), p)
    assert st == bb.BT_ERR_ARG
    if h:
        bb.bt_destroy(h)


def test_autotune_chooses_between_the_mappings():
    inst = wl.config0()
    with Single(inst, m=2, alpha=[1.0, 7.0]) as s:
        s.ok()
        x = dev(np.zeros(inst.N * inst.n))
        st, kb, g = bb.bt_autotune(s.h, dev(inst.b.reshape(-1)), x, 1e-10, 500, 3)
        assert st == bb.BT_OK and (g in (-1, -2, -4, -8) or g >= 1)
        ref = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-10, 500)
        assert rel(host(x).reshape(inst.N, inst.n), ref.x) <= 1e-10
        st, it, x2 = s.solve(inst.b, 1e-10, 500)
        assert st == bb.BT_OK and abs(it - ref.iters) <= 1


@pytest.mark.parametrize("g", [0, -8])
def test_config1_mixed_on_the_shared_memory_engine(g):
    """LQR N = 128, n = 12, float32 PCG inside float64 refinement on the
    shared-memory engine (the automatic choice takes the smallest cluster that
    holds the float32 and float64 blocks): the true residual to tol and the
    solution within cond * tol of the oracle's direct solve, as the
    persistent kernel's mixed path."""
    inst = wl.config1()
    xr = orc.direct_solve(inst.D, inst.O, inst.b)
    out = {}
    for gg in (g, 32):
        with Single(inst, m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, group_ctas=gg) as s:
            s.ok()
            st, it, x = s.solve(inst.b, 1e-10, 2000)
            info = s.info()
        assert st == bb.BT_OK
        res = np.linalg.norm(orc.spmv(inst.D, inst.O, x) - inst.b) / np.linalg.norm(inst.b)
        assert res <= 1e-10 and info[2] <= 1e-10
        assert rel(x, xr) <= 1e-7
        out[gg] = (it, info[1])
    # the same refinement structure as the persistent kernel (outer steps)
    assert out[g][1] == out[32][1] and abs(out[g][0] - out[32][0]) <= 4


@pytest.mark.parametrize("N,n,g", [(16, 6, -1), (9, 12, -1), (40, 8, -2), (17, 16, -8)])
def test_mixed_small_engine_matches_direct_solve(N, n, g):
    inst = wl.small_llt(98, N, n)
    with Single(inst, m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, group_ctas=g) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-12, 3000)
        assert st == bb.BT_OK
        # zero right-hand side and the outer-step limit
        st0, it0, x0 = s.solve(np.zeros_like(inst.b), 1e-12, 100)
        assert st0 == bb.BT_OK and it0 == 0 and np.all(x0 == 0)
    assert rel(x, orc.direct_solve(inst.D, inst.O, inst.b)) <= 1e-8


def test_mixed_small_engine_outer_limit_and_nonfinite():
    inst = wl.small_llt(99, 12, 6)
    with Single(inst, m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, group_ctas=-1, max_outer=1) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-14, 3000)
        assert st == bb.BT_ERR_NO_CONVERGENCE and s.info()[1] == 1
        b = inst.b.copy()
        b[2, 3] = np.nan
        st, it, x = s.solve(b, 1e-10, 100)
        assert st == bb.BT_ERR_NONFINITE
