"""The precision split of the mixed path: the default (float32 factor of each
D_i with a float64 refactor of the blocks whose pivots show cond(D_i) > 1e3,
float32 divisions of the inner CG step scalars) against the strict split
(every D_i factored in float64, step scalars divided in float64), each
against the oracle's direct solve."""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import Single, cond_estimate, dev, host, ill_conditioned, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


def batched(insts, tol, strict):
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, mixed_strict_fp64=strict)
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dev(D), dev(O), p)
    assert st == bb.BT_OK
    try:
        x = dev(np.zeros(b.size))
        st, its, sts = bb.bt_pcg_solve_batched(h, dev(b), x, len(insts), tol, 5000)
        assert st == bb.BT_OK and (sts == 0).all()
    finally:
        bb.bt_destroy(h)
    xs = host(x)
    return [xs[v_off[k]:v_off[k] + i.N * i.n].reshape(i.N, i.n) for k, i in enumerate(insts)], its


@pytest.mark.parametrize("strict", [False, True])
def test_mixed_precision_split_against_oracle(strict):
    """Both splits on bench-batch instances (n = 12, 24, 36): at tol 1e-8 every
    true residual <= 1e-8; at tol = 1e-8 / cond(S) every x within 1e-8 of the
    oracle's direct solve."""
    insts = wl.config2(indices=[0, 5, 17, 64, 300, 511, 777, 1023])
    xs, its = batched(insts, 1e-8, strict)
    for inst, x in zip(insts, xs):
        assert np.linalg.norm(orc.spmv(inst.D, inst.O, x) - inst.b) <= 1e-8 * np.linalg.norm(inst.b)
    cond = max(cond_estimate(i.D, i.O, i.b) for i in insts)
    xs, its = batched(insts, min(1e-8, 1e-8 / cond), strict)
    for inst, x in zip(insts, xs):
        assert rel(x, orc.direct_solve(inst.D, inst.O, inst.b)) <= 1e-8


@pytest.mark.parametrize("decades", [2, 3, 4])
def test_strict_split_apply_on_ill_conditioned_blocks(decades):
    """kappa(D_5) ~ 1e4 .. 1e8 (congruence that keeps S SPD): the strict
    split factors it in float64 like every block, and the float32 apply of
    M^-1 stays at float32 rounding of the float64 oracle's apply."""
    inst = ill_conditioned(wl.small_llt(71, 12, 8), 5, decades, 72)
    r = np.random.default_rng(73).standard_normal((inst.N, inst.n))
    ref = orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, [1.0])
    with Single(inst, m=1, precision=bb.BT_MIXED, mixed_strict_fp64=True) as s:
        s.ok()
        z = s.apply(r)
    assert rel(z, ref) <= 2e-5, rel(z, ref)


def test_noalloc_strict_split_matches_allocating_path():
    """The no-allocation entry against the allocating path on the same engine
    and shape (the persistent kernel on N / 4 CTAs; a single instance would
    otherwise go to the shared-memory engine, whose float32 sums run in
    another order)."""
    inst = wl.config1()
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, mixed_strict_fp64=True)
    pa, keep_a = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, mixed_strict_fp64=True,
                                group_ctas=inst.N // 4)
    st, h = bb.bt_setup(inst.N, inst.n, dev(inst.D), dev(inst.O), pa)
    assert st == bb.BT_OK
    try:
        xa = dev(np.zeros(inst.N * inst.n))
        st, ita = bb.bt_pcg_solve(h, dev(inst.b.reshape(-1)), xa, 1e-10, 2000)
        assert st == bb.BT_OK
    finally:
        bb.bt_destroy(h)
    xb = dev(np.zeros(inst.N * inst.n))
    st, itb = bb.bt_pcg_solve_noalloc(inst.N, inst.n, dev(inst.D), dev(inst.O), dev(inst.b.reshape(-1)), xb,
                                      1e-10, 2000, p)
    assert st == bb.BT_OK and abs(ita - itb) <= 1
    assert rel(host(xb), host(xa)) <= 1e-10
