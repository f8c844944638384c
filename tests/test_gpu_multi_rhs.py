"""Many right-hand sides (64 columns sharing each block sweep) against the
oracle: per-column direct solves on small cases, and the 2048 x 48 workload
through every column's true residual plus sampled direct solves."""
import functools

import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import cond_estimate, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


def solve_multi(inst, nrhs, tol, maxit=20000, m=2, alpha=(1.0, 7.0), engine=0):
    p, keep = bb.make_params(m=m, alpha=list(alpha), precision=bb.BT_MIXED, mrhs_engine=engine)
    st, h = bb.bt_setup(inst.N, inst.n, dev(inst.D), dev(inst.O), p)
    assert st == bb.BT_OK
    try:
        B = inst.b.reshape(inst.N * inst.n, nrhs)
        X = dev(np.zeros(B.size))
        st, its, sts = bb.bt_pcg_solve_multi(h, dev(B.reshape(-1)), X, nrhs, tol, maxit)
        infos = [bb.bt_multi_info(h, j) for j in range(nrhs)]
    finally:
        bb.bt_destroy(h)
    return st, its, sts, host(X).reshape(inst.N, inst.n, nrhs), infos


SIMT, TC = 1, 2  # mrhs_engine: float32 SIMT tiles, tensor cores (3xTF32)


# SIMT, n <= 48: the k range of each product split over two thread halves (n =
# 4: one half empty; n = 44: an odd number of row groups); n = 52, 64: one pass

@pytest.mark.parametrize("N,n,nrhs", [(1, 4, 3), (2, 4, 64), (7, 8, 5), (33, 12, 64), (20, 16, 17), (9, 44, 64),
                                      (5, 52, 7), (6, 64, 64)])
def test_multi_rhs_matches_direct_solves(N, n, nrhs):
    inst = wl.small_llt(60, N, n, nrhs=nrhs)
    st, its, sts, X, infos = solve_multi(inst, nrhs, 1e-12, engine=SIMT)
    assert st == bb.BT_OK and (sts == 0).all()
    xr = orc.direct_solve(inst.D, inst.O, inst.b)
    for j in range(nrhs):
        err = np.linalg.norm(X[:, :, j] - xr[:, :, j]) / np.linalg.norm(xr[:, :, j])
        assert err <= 1e-8, (j, err)
        assert infos[j][2] <= 1e-12


# tensor-core engine (n a multiple of 8, n <= 48): one CTA (N = 1, 2: no
# neighbours), rows split over many CTAs with halo columns on both sides (N
# small against the 152 CTAs: CTAs of one row), ragged column counts
@pytest.mark.parametrize("N,n,nrhs", [(1, 8, 3), (2, 8, 64), (3, 16, 64), (7, 8, 5), (40, 24, 64), (17, 40, 33),
                                      (9, 48, 64), (300, 16, 64), (5, 32, 1)])
def test_multi_rhs_tensor_cores_match_direct_solves(N, n, nrhs):
    inst = wl.small_llt(70, N, n, nrhs=nrhs)
    st, its, sts, X, infos = solve_multi(inst, nrhs, 1e-12, engine=TC)
    assert st == bb.BT_OK and (sts == 0).all()
    xr = orc.direct_solve(inst.D, inst.O, inst.b)
    for j in range(nrhs):
        err = np.linalg.norm(X[:, :, j] - xr[:, :, j]) / np.linalg.norm(xr[:, :, j])
        assert err <= 1e-8, (j, err)
        assert infos[j][2] <= 1e-12


def test_multi_rhs_columns_match_single_solves():
    inst = wl.small_ocp(61, 40, 12)
    rng = np.random.default_rng(1)
    nrhs = 6
    b = rng.standard_normal((inst.N, inst.n, nrhs))
    multi = wl.Instance(D=inst.D, O=inst.O, b=b)
    st, its, sts, X, _ = solve_multi(multi, nrhs, 1e-8)
    assert st == bb.BT_OK
    for j in range(nrhs):
        res = np.linalg.norm(orc.spmv(inst.D, inst.O, X[:, :, j]) - b[:, :, j]) / np.linalg.norm(b[:, :, j])
        assert res <= 1e-8
    # a zero column converges at once
    b[:, :, 2] = 0.0
    st, its, sts, X, _ = solve_multi(wl.Instance(D=inst.D, O=inst.O, b=b), nrhs, 1e-8)
    assert st == bb.BT_OK and its[2] == 0 and np.all(X[:, :, 2] == 0)


@functools.lru_cache(maxsize=1)
def config3_cond():
    inst = wl.config3()
    return cond_estimate(inst.D, inst.O, inst.b[:, :, 0])


def test_config3_many_rhs_full_size():
    """LL^T, N = 2048, n = 48, 64 right-hand sides at the benchmark's
    tol = 1e-8: every column's float64 true residual <= 1e-8, and sampled
    columns against direct solves within cond(S) * tol."""
    inst = wl.config3()
    st, its, sts, X, infos = solve_multi(inst, 64, 1e-8)
    assert st == bb.BT_OK and (sts == 0).all()
    R = orc.spmv(inst.D, inst.O, X) - inst.b
    for j in range(64):
        res = np.linalg.norm(R[:, :, j]) / np.linalg.norm(inst.b[:, :, j])
        assert res <= 1e-8, (j, res)
    cond = config3_cond()
    xr = orc.direct_solve(inst.D, inst.O, inst.b[:, :, :2])
    for j in range(2):
        err = np.linalg.norm(X[:, :, j] - xr[:, :, j]) / np.linalg.norm(xr[:, :, j])
        assert err <= cond * 1e-8, (j, err, cond)


def test_config3_many_rhs_full_size_error_1e8():
    """The same system solved to tol = min(1e-8, 1e-8 / cond(S)) (cond from
    the oracle's Lanczos estimate, about 6.6e4), so that the mixed path's
    solution error is bounded by 1e-8: four sampled columns (first, last and
    two inside) against the oracle's direct solve at <= 1e-8, every column's
    true residual at <= tol."""
    inst = wl.config3()
    cond = config3_cond()
    tol = min(1e-8, 1e-8 / cond)
    st, its, sts, X, infos = solve_multi(inst, 64, tol)
    assert st == bb.BT_OK and (sts == 0).all(), (st, sts)
    R = orc.spmv(inst.D, inst.O, X) - inst.b
    for j in range(64):
        res = np.linalg.norm(R[:, :, j]) / np.linalg.norm(inst.b[:, :, j])
        assert res <= tol, (j, res, tol)
    cols = [0, 21, 42, 63]
    xr = orc.direct_solve(inst.D, inst.O, inst.b[:, :, cols])
    for c, j in enumerate(cols):
        err = np.linalg.norm(X[:, :, j] - xr[:, :, c]) / np.linalg.norm(xr[:, :, c])
        assert err <= 1e-8, (j, err, tol)


@pytest.mark.parametrize("m,alpha", [(1, (1.0,)), (3, (1.0, 1.0, 1.0)), (3, (1.0, 2.0, 3.0))])
@pytest.mark.parametrize("N,n,engine", [(13, 12, SIMT), (9, 48, SIMT), (4, 64, SIMT), (9, 48, TC), (31, 16, TC)])
def test_multi_rhs_polynomial_orders(m, alpha, N, n, engine):
    """m = 1 (z from the G sweep alone) and m = 3 (one H sweep summing into z
    from global memory, then the last one with r staged during the
    products), on both SIMT product layouts (n <= 48 split in k, n = 64 not)
    and on the tensor cores."""
    inst = wl.small_llt(63 + m, N, n, nrhs=9)
    st, its, sts, X, infos = solve_multi(inst, 9, 1e-12, m=m, alpha=alpha, engine=engine)
    assert st == bb.BT_OK and (sts == 0).all()
    xr = orc.direct_solve(inst.D, inst.O, inst.b)
    for j in range(9):
        err = np.linalg.norm(X[:, :, j] - xr[:, :, j]) / np.linalg.norm(xr[:, :, j])
        assert err <= 1e-8, (j, err)
        assert infos[j][2] <= 1e-12


def test_multi_rhs_engines_agree_and_tc_rejects_unsupported_n():
    """Both engines on one LQR system (n = 24): the same solutions to the
    tolerance, iteration counts within a few; the tensor-core engine asked for
    n = 12 (not a multiple of 8) returns BT_ERR_ARG."""
    inst = wl.small_ocp(62, 200, 24)
    rng = np.random.default_rng(3)
    b = rng.standard_normal((inst.N, inst.n, 64))
    multi = wl.Instance(D=inst.D, O=inst.O, b=b)
    res = {}
    for eng in (SIMT, TC):
        st, its, sts, X, _ = solve_multi(multi, 64, 1e-10, engine=eng)
        assert st == bb.BT_OK and (sts == 0).all()
        res[eng] = (its, X)
    assert np.abs(res[SIMT][0] - res[TC][0]).max() <= 3
    xr = orc.direct_solve(inst.D, inst.O, b)
    for eng in (SIMT, TC):
        err = np.linalg.norm(res[eng][1] - xr) / np.linalg.norm(xr)
        assert err <= 1e-8, (eng, err)
    small = wl.small_ocp(63, 10, 12)
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, mrhs_engine=TC)
    st, h = bb.bt_setup(small.N, small.n, dev(small.D), dev(small.O), p)
    assert st == bb.BT_OK
    try:
        B = dev(np.ones(small.N * small.n * 4))
        X = dev(np.zeros(small.N * small.n * 4))
        st, its, sts = bb.bt_pcg_solve_multi(h, B, X, 4, 1e-8, 100)
        assert st == bb.BT_ERR_ARG
    finally:
        bb.bt_destroy(h)
