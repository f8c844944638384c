"""GPU parity of the matrix-free H_opt (bt_params.h_matrix_free: H_opt = H_J^2
applied as two sweeps over D^-1 and O, no H blocks stored) against the
oracle, through the C ABI.  Same tolerances as the stored variant
(test_gpu_parity.py): the operator is the same, only the rounding order of
its products differs."""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import Single, dev, host, maxrel, rel

pytestmark = pytest.mark.gpu
SHAPES = [(1, 3), (2, 5), (3, 4), (7, 3), (16, 6), (33, 5), (40, 12), (30, 20), (25, 24), (64, 36), (9, 48)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


@pytest.mark.parametrize("N,n", SHAPES)
@pytest.mark.parametrize("m,alpha", [(2, [1.0, 7.0]), (3, [1.0, 0.5, 2.0])])
def test_apply_fp64(N, n, m, alpha):
    inst = wl.small_ocp(110, N, n)
    r = np.random.default_rng(N + n).standard_normal((N, n))
    ref = orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, alpha)
    with Single(inst, m=m, alpha=alpha, h_matrix_free=True) as s:
        s.ok()
        z = s.apply(r)
    assert maxrel(z, ref) <= 1e-12


@pytest.mark.parametrize("N,n", SHAPES)
def test_apply_mixed(N, n):
    inst = wl.small_ocp(111, N, n)
    r = np.random.default_rng(2 * N + n).standard_normal((N, n))
    ref = orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, [1.0, 7.0])
    with Single(inst, m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, h_matrix_free=True) as s:
        s.ok()
        z = s.apply(r)
    assert maxrel(z, ref) <= 2e-4


@pytest.mark.parametrize("m,alpha", [(2, [1.0, 7.0]), (3, None), (4, None)])
def test_solve_fp64_matches_oracle(m, alpha):
    inst = wl.config1()
    a = alpha if alpha is not None else [1.0] * m
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, a, 1e-10, 3000)
    with Single(inst, m=m, alpha=alpha, h_matrix_free=True) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-10, 3000)
    assert st == bb.BT_OK and abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10


@pytest.mark.parametrize("G", [2, 3, 5])
def test_group_ctas(G):
    inst = wl.small_ocp(112, 37, 6)
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-10, 2000)
    r = np.random.default_rng(G).standard_normal((37, 6))
    with Single(inst, m=2, alpha=[1.0, 7.0], group_ctas=G, h_matrix_free=True) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-10, 2000)
        z = s.apply(r)
    assert st == bb.BT_OK and abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10
    assert maxrel(z, orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, [1.0, 7.0])) <= 1e-12


def test_batched_mixed_like_stored_and_smaller():
    insts = wl.config2(indices=[0, 1, 2, 3, 100, 511, 777, 1023])
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    res = {}
    for mf in (False, True):
        p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, h_matrix_free=mf)
        st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dev(D), dev(O), p)
        assert st == bb.BT_OK
        x = dev(np.zeros(b.size))
        try:
            st, its, sts = bb.bt_pcg_solve_batched(h, dev(b), x, len(insts), 1e-8, 5000)
            nbytes = bb.bt_device_bytes(h)
        finally:
            bb.bt_destroy(h)
        assert st == bb.BT_OK and (sts == 0).all()
        xs = host(x)
        for k, inst in enumerate(insts):
            xk = xs[v_off[k]:v_off[k] + inst.N * inst.n].reshape(inst.N, inst.n)
            assert np.linalg.norm(orc.spmv(inst.D, inst.O, xk) - inst.b) <= 1e-8 * np.linalg.norm(inst.b)
        res[mf] = (its, nbytes)
    assert np.abs(res[True][0] - res[False][0]).max() <= 2
    assert res[True][1] < 0.8 * res[False][1]


def test_refused_combinations():
    inst = wl.small_ocp(113, 8, 12)
    s = Single(inst, m=2, a=0.5, h_matrix_free=True)
    try:
        assert s.st == bb.BT_ERR_PARAM
    finally:
        s.close()
    with Single(inst, m=2, precision=bb.BT_MIXED, h_matrix_free=True) as s:
        s.ok()
        B = dev(np.zeros(8 * 12 * 2))
        X = dev(np.zeros(8 * 12 * 2))
        assert bb.bt_pcg_solve_multi(s.h, B, X, 2, 1e-8, 100)[0] == bb.BT_ERR_PARAM
