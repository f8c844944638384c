"""GPU parity against the CPU oracle, through the C ABI.

Tolerances:
  * float64 blocks (apply, SpMV): max relative difference <= 1e-12 (a handful
    of n-term dot products in float64: n * u64 * cond(D_i) ~ 1e-13 here).
  * float32 blocks (mixed handle): <= 2e-4 (the same products in float32,
    u32 = 6e-8, with D_i^-1 formed in float32 from a float64 Cholesky factor;
    bound ~ n * cond(D_i) * u32 for the block condition numbers of these
    generators, measured far below it).
  * float64 PCG vs oracle PCG at the same tol: relative solution difference
    <= 1e-10 and iteration counts within 1.
  * mixed PCG vs the oracle's direct solve: relative error <= 1e-8 when run to
    a residual tolerance of 1e-8 / kappa-ish (1e-12 here).
"""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import Single, dev, host, ill_conditioned, maxrel, rel

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 5), (2, 3), (3, 2), (4, 1), (5, 7), (7, 3), (9, 6), (16, 6), (33, 5), (40, 12), (64, 36)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


@pytest.mark.parametrize("N,n", SHAPES)
@pytest.mark.parametrize("m,alpha", [(1, None), (2, [1.0, 7.0]), (3, [1.0, 0.5, 2.0])])
def test_apply_fp64_matches_oracle(N, n, m, alpha):
    inst = wl.small_ocp(50, N, n)
    r = np.random.default_rng(N * 100 + n).standard_normal((N, n))
    a = alpha if alpha is not None else [1.0] * m
    ref = orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, a)
    with Single(inst, m=m, alpha=alpha) as s:
        s.ok()
        z = s.apply(r)
    assert maxrel(z, ref) <= 1e-12


@pytest.mark.parametrize("N,n", SHAPES)
def test_spmv_fp64_matches_oracle(N, n):
    inst = wl.small_llt(51, N, n)
    x = np.random.default_rng(N + 7 * n).standard_normal((N, n))
    with Single(inst) as s:
        s.ok()
        y = s.spmv(x)
    assert maxrel(y, orc.spmv(inst.D, inst.O, x)) <= 1e-13


@pytest.mark.parametrize("N,n", SHAPES)
@pytest.mark.parametrize("m,alpha", [(1, None), (2, [1.0, 7.0])])
def test_apply_and_spmv_fp32_match_oracle(N, n, m, alpha):
    inst = wl.small_ocp(52, N, n)
    r = np.random.default_rng(3 * N + n).standard_normal((N, n))
    a = alpha if alpha is not None else [1.0] * m
    ref = orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, a)
    with Single(inst, m=m, alpha=alpha, precision=bb.BT_MIXED) as s:
        s.ok()
        z = s.apply(r)
        y = s.spmv(r, f32=True)
        y64 = s.spmv(r)
    assert maxrel(z, ref) <= 2e-4
    assert maxrel(y, orc.spmv(inst.D, inst.O, r)) <= 2e-4
    assert maxrel(y64, orc.spmv(inst.D, inst.O, r)) <= 1e-13


@pytest.mark.parametrize("alpha", [[1.0, 1.0], [1.0, 7.0]])
def test_config0_fp64_solve(alpha):
    inst = wl.config0()
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, alpha, 1e-10, 500)
    with Single(inst, m=2, alpha=alpha) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-10, 500)
    assert st == bb.BT_OK
    assert abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10


@pytest.mark.parametrize("G", [1, 2, 3, 5, 8])
def test_config1_fp64_solve_group_sizes(G):
    inst = wl.config1()
    alpha = [1.0, 7.0]
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, alpha, 1e-8, 1000)
    with Single(inst, m=2, alpha=alpha, group_ctas=G) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-8, 1000)
    assert st == bb.BT_OK
    assert abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10


@pytest.mark.parametrize("G", [1, 4])
@pytest.mark.parametrize("m,alpha", [(1, None), (2, [1.0, 7.0]), (3, [1.0, 1.0, 1.0])])
def test_config1_mixed_solve(G, m, alpha):
    inst = wl.config1()
    xref = orc.direct_solve(inst.D, inst.O, inst.b)
    with Single(inst, m=m, alpha=alpha, precision=bb.BT_MIXED, group_ctas=G) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-12, 5000)
        _, outer, res = s.info()
    assert st == bb.BT_OK
    assert res <= 1e-12
    assert rel(x, xref) <= 1e-8
    # and at the benchmark tolerance the true residual meets 1e-8
    with Single(inst, m=m, alpha=alpha, precision=bb.BT_MIXED, group_ctas=G) as s:
        st, it, x = s.solve(inst.b, 1e-8, 5000)
    assert st == bb.BT_OK
    assert np.linalg.norm(orc.spmv(inst.D, inst.O, x) - inst.b) <= 1e-8 * np.linalg.norm(inst.b)


@pytest.mark.parametrize("N,n,G", [(2, 3, 2), (3, 2, 3), (7, 3, 3), (33, 5, 6), (64, 36, 9)])
def test_multi_cta_fp64_matches_single(N, n, G):
    inst = wl.small_ocp(53, N, n)
    alpha = [1.0, 7.0]
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, alpha, 1e-10, 1000)
    with Single(inst, m=2, alpha=alpha, group_ctas=G) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-10, 1000)
        r = np.random.default_rng(1).standard_normal((N, n))
        z = s.apply(r)
        y = s.spmv(r)
    assert st == bb.BT_OK and abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10
    assert maxrel(z, orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, alpha)) <= 1e-12
    assert maxrel(y, orc.spmv(inst.D, inst.O, r)) <= 1e-13


def _batched(insts, m, alpha, precision, tol, maxit, **kw):
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    p, keep = bb.make_params(m=m, alpha=alpha, precision=precision, **kw)
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dev(D), dev(O if O.size else np.zeros(1)), p)
    assert st == bb.BT_OK, bb.status_string(st)
    x = dev(np.zeros(b.size))
    try:
        st, its, sts = bb.bt_pcg_solve_batched(h, dev(b), x, len(insts), tol, maxit)
        infos = [bb.bt_solve_info(h, k) for k in range(len(insts))]
    finally:
        bb.bt_destroy(h)
    xs = host(x)
    out = [xs[v_off[k]:v_off[k] + insts[k].N * insts[k].n].reshape(insts[k].N, insts[k].n) for k in range(len(insts))]
    return st, its, sts, out, infos


def test_batched_fp64_ragged_matches_oracle():
    rng = np.random.default_rng(9)
    insts = [wl.small_ocp(60 + k, int(rng.integers(1, 40)), int(rng.choice([1, 3, 6, 12]))) for k in range(24)]
    alpha = [1.0, 7.0]
    st, its, sts, xs, _ = _batched(insts, 2, alpha, bb.BT_FP64, 1e-10, 1000)
    assert st == bb.BT_OK and (sts == 0).all()
    for k, inst in enumerate(insts):
        ref = orc.pcg_opt(inst.D, inst.O, inst.b, alpha, 1e-10, 1000)
        assert abs(its[k] - ref.iters) <= 1, k
        assert rel(xs[k], ref.x) <= 1e-10, k


def test_batched_mixed_config2_sample():
    idx = [0, 1, 2, 3, 100, 511, 777, 1023]
    insts = wl.config2(indices=idx)
    st, its, sts, xs, infos = _batched(insts, 2, [1.0, 7.0], bb.BT_MIXED, 1e-8, 5000)
    assert st == bb.BT_OK and (sts == 0).all()
    for k, inst in enumerate(insts):
        res = np.linalg.norm(orc.spmv(inst.D, inst.O, xs[k]) - inst.b) / np.linalg.norm(inst.b)
        assert res <= 1e-8, (k, res)
        assert abs(infos[k][2] - res) <= 1e-9


def test_batched_mixed_accuracy_vs_direct():
    insts = wl.config2(indices=[5, 6, 7, 8])
    st, its, sts, xs, _ = _batched(insts, 2, [1.0, 7.0], bb.BT_MIXED, 1e-12, 5000)
    assert st == bb.BT_OK
    for k, inst in enumerate(insts):
        assert rel(xs[k], orc.direct_solve(inst.D, inst.O, inst.b)) <= 1e-8


# ---------------------------------------------------------------- statuses
def test_not_spd_reports_block():
    inst = wl.small_ocp(70, 10, 4)
    D = inst.D.copy()
    D[6] = -np.eye(4)
    bad = wl.Instance(D=D, O=inst.O, b=inst.b)
    s = Single(bad)
    try:
        assert s.st == bb.BT_ERR_NOT_SPD
        st, i, blk, val = bb.bt_last_error(s.h)
        assert (i, blk) == (0, 6) and val < 0
    finally:
        s.close()


def test_not_spd_reports_block_mixed():
    # the float32 factor refuses the block, the float64 refactor confirms it
    inst = wl.small_ocp(70, 10, 4)
    D = inst.D.copy()
    D[6] = -np.eye(4)
    bad = wl.Instance(D=D, O=inst.O, b=inst.b)
    s = Single(bad, precision=bb.BT_MIXED)
    try:
        assert s.st == bb.BT_ERR_NOT_SPD
        st, i, blk, val = bb.bt_last_error(s.h)
        assert (i, blk) == (0, 6) and val < 0
    finally:
        s.close()


def test_mixed_ill_conditioned_block_solve():
    # kappa(D_5) ~ 1e4, smallest pivot ratio ~ 8e-3: the float32 factor is
    # kept; refinement reaches the direct solve
    inst = ill_conditioned(wl.small_llt(71, 12, 8), 5, 2, 72)
    assert np.linalg.eigvalsh(orc.assemble(inst.D, inst.O)).min() > 0
    xref = orc.direct_solve(inst.D, inst.O, inst.b)
    with Single(inst, m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-12, 5000)
    assert st == bb.BT_OK
    assert rel(x, xref) <= 1e-8


@pytest.mark.parametrize("decades", [3, 4])
def test_mixed_ill_conditioned_block_apply(decades):
    # kappa(D_5) ~ 1e6 / 1e8, smallest pivot ratio ~ 8e-4 / 8e-6, below the
    # 1e-3 cut: the block goes to the float64 refactor.  A float32 Cholesky
    # would give D_5^-1 r with ~4e-4 / 0.2 relative error; the refactor keeps
    # it at float32 rounding.  (A float32 copy of such an S cannot carry its
    # smallest eigen-directions -- kappa(S) u32 > 1 -- so mixed refinement
    # is not expected to converge on it; only the apply is checked.)
    inst = ill_conditioned(wl.small_llt(71, 12, 8), 5, decades, 72)
    r = np.random.default_rng(73).standard_normal((inst.N, inst.n))
    ref = orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, [1.0])
    with Single(inst, m=1, precision=bb.BT_MIXED) as s:
        s.ok()
        z = s.apply(r)
    err = rel(z, ref)
    assert err <= 2e-5, err


def test_float32_copies_round_to_nearest_even():
    # D = diag(d), O = 0: the float32 SpMV with x = 1 returns exactly the
    # float32 copy of each d_i, which must be d_i rounded to nearest even
    # (values at, just above and just below float32 midpoints, and random)
    rng = np.random.default_rng(81)
    N, n = 40, 36
    f = rng.uniform(0.5, 4.0, N * n).astype(np.float32)
    ulp = np.spacing(f).astype(np.float64)
    d = f.astype(np.float64)
    d[0::5] += ulp[0::5] / 2
    d[1::5] -= ulp[1::5] / 2
    d[2::5] += ulp[2::5] * 0.5000001
    d[3::5] += ulp[3::5] * 0.4999999
    d[4::5] = rng.uniform(1e-3, 1e3, d[4::5].size)
    D = np.zeros((N, n, n))
    D[:, np.arange(n), np.arange(n)] = d.reshape(N, n)
    inst = wl.Instance(D=D, O=np.zeros((N - 1, n, n)), b=np.zeros((N, n)))
    with Single(inst, m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED) as s:
        s.ok()
        y = s.spmv(np.ones((N, n)), f32=True)
    assert np.array_equal(y.reshape(-1), d.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("bad", [1, 3])
def test_batched_mixed_not_spd_reports_instance_and_block(bad):
    # in a mixed batch, a non-SPD block of a later instance is refused by the
    # float32 factor, confirmed by the float64 refactor and reported with its
    # instance and block
    insts = [wl.small_ocp(90 + k, 10 + k, 4) for k in range(4)]
    D = insts[bad].D.copy()
    D[6] = -np.eye(4)
    insts[bad] = wl.Instance(D=D, O=insts[bad].O, b=insts[bad].b)
    Ns, ns, d_off, o_off, v_off, Dp, Op, b = wl.pack_batch(insts)
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED)
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dev(Dp), dev(Op), p)
    try:
        assert st == bb.BT_ERR_NOT_SPD
        st2, i, blk, val = bb.bt_last_error(h)
        assert (i, blk) == (bad, 6) and val < 0
    finally:
        if h:
            bb.bt_destroy(h)


def test_batched_mixed_matches_single_setups():
    # the same instances solved from one batched setup and from one
    # single-instance setup each: identical blocks and sweeps, identical iterates
    insts = wl.config2(indices=[3, 40, 41, 700, 701])
    st, its, sts, xs, _ = _batched(insts, 2, [1.0, 7.0], bb.BT_MIXED, 1e-10, 5000)
    assert st == bb.BT_OK and (sts == 0).all()
    for k, inst in enumerate(insts):
        with Single(inst, m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, group_ctas=1) as s1:
            s1.ok()
            st1, it1, x1 = s1.solve(inst.b, 1e-10, 5000)
        assert st1 == bb.BT_OK and it1 == its[k]
        assert np.array_equal(x1, xs[k])


def test_maxit_gives_no_convergence_and_last_iterate():
    inst = wl.config1()
    with Single(inst, m=2, alpha=[1.0, 7.0]) as s:
        st, it, x = s.solve(inst.b, 1e-14, 3)
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-14, 3)
    assert st == bb.BT_ERR_NO_CONVERGENCE and it == 3
    assert rel(x, ref.x) <= 1e-12


def test_nonfinite_rhs():
    inst = wl.config0()
    b = inst.b.copy()
    b[3, 2] = np.nan
    for prec in (bb.BT_FP64, bb.BT_MIXED):
        with Single(inst, precision=prec) as s:
            st, it, x = s.solve(b, 1e-10, 100)
        assert st == bb.BT_ERR_NONFINITE


def test_zero_rhs():
    inst = wl.config0()
    for prec in (bb.BT_FP64, bb.BT_MIXED):
        with Single(inst, precision=prec) as s:
            st, it, x = s.solve(np.zeros_like(inst.b), 1e-10, 100, x0=np.ones_like(inst.b))
        assert st == bb.BT_OK and it == 0 and np.all(x == 0)


def test_breakdown_on_indefinite_matrix():
    """D_i SPD (setup succeeds) but S indefinite: CG meets p.q <= 0."""
    n, N = 2, 6
    D = np.stack([np.eye(n)] * N)
    O = np.stack([3.0 * np.eye(n)] * (N - 1))
    b = np.ones((N, n))
    inst = wl.Instance(D=D, O=O, b=b)
    S = orc.assemble(D, O)
    assert np.linalg.eigvalsh(S).min() < 0
    ref = orc.pcg_opt(D, O, b, [1.0], 1e-10, 100)
    with Single(inst, m=1) as s:
        s.ok()
        st, it, x = s.solve(b, 1e-10, 100)
    assert ref.status == orc.BREAKDOWN
    assert st == bb.BT_ERR_BREAKDOWN


def test_timeout_from_tiny_cycle_budget_leaves_context_usable():
    inst = wl.config1()
    with Single(inst, m=2, alpha=[1.0, 7.0], cycle_budget=2000) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-12, 100000)
    assert st == bb.BT_ERR_TIMEOUT
    with Single(inst, m=2, alpha=[1.0, 7.0]) as s:
        st, it, x = s.solve(inst.b, 1e-8, 1000)
    assert st == bb.BT_OK


def test_warm_start():
    inst = wl.config1()
    xd = orc.direct_solve(inst.D, inst.O, inst.b)
    with Single(inst, m=2, alpha=[1.0, 7.0], use_x0=True) as s:
        st, it, x = s.solve(inst.b, 1e-10, 1000, x0=xd + 1e-9)
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-10, 1000, x0=xd + 1e-9)
    assert st == bb.BT_OK and abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10


def test_deterministic_bitwise():
    inst = wl.config1()
    outs = []
    for _ in range(2):
        with Single(inst, m=2, alpha=[1.0, 7.0], group_ctas=8) as s:
            outs.append(s.solve(inst.b, 1e-10, 1000)[2])
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("m,alpha", [(2, [1.0, 7.0]), (3, None)])
def test_batched_mixed_ragged_block_sizes(m, alpha):
    """Batched mixed solves over block sizes that take every sweep form:
    odd n (scalar staging, unpipelined), n % 4 == 0 at run-time sizes (8, 20:
    pipelined with generic products) and at compiled sizes (12, 24, 36, 48),
    horizons from 1 to 70 (one to several chunks, ragged tails).  Every
    instance meets the float64 true residual and matches the direct solve."""
    rng = np.random.default_rng(17)
    sizes = [1, 3, 5, 7, 8, 12, 20, 24, 36, 48]
    insts = [wl.small_ocp(130 + k, int(rng.integers(1, 71)), sizes[k % len(sizes)]) for k in range(30)]
    st, its, sts, xs, infos = _batched(insts, m, alpha, bb.BT_MIXED, 1e-10, 20000)
    assert st == bb.BT_OK and (sts == 0).all()
    for k, inst in enumerate(insts):
        res = np.linalg.norm(orc.spmv(inst.D, inst.O, xs[k]) - inst.b) / np.linalg.norm(inst.b)
        assert res <= 1e-10, (k, inst.N, inst.n, res)
        assert rel(xs[k], orc.direct_solve(inst.D, inst.O, inst.b)) <= 1e-8, k


def _ties(rng, shape, lo_exp, hi_exp):
    """float64 values exactly halfway between two neighbouring float32 values,
    or one float64 ulp either side of such a midpoint, over a spread of
    binades (the cases round-to-nearest-even decides)."""
    f = rng.uniform(1.0, 2.0, shape).astype(np.float32)
    nxt = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + nxt.astype(np.float64)) / 2
    nudge = rng.integers(-1, 2, shape)
    mid = np.where(nudge > 0, np.nextafter(mid, np.inf), np.where(nudge < 0, np.nextafter(mid, -np.inf), mid))
    sign = np.where(rng.random(shape) < 0.5, -1.0, 1.0)
    return sign * np.ldexp(mid, rng.integers(lo_exp, hi_exp, shape))


@pytest.mark.parametrize("N,n", [(3, 12), (4, 5), (2, 36)])
def test_fp32_block_copies_round_to_nearest_even(N, n):
    """The float32 copies of D_i and O_i that a mixed handle streams equal the
    IEEE round-to-nearest-even conversion of the caller's float64 blocks, bit
    for bit: S_32 e_j read back through the float32 SpMV is column j of S
    converted by numpy (a product with a unit vector adds only exact zeros)."""
    rng = np.random.default_rng(700 + n)
    D = np.zeros((N, n, n))
    for i in range(N):
        T = _ties(rng, (n, n), -40, -6)
        D[i] = np.tril(T, -1) + np.tril(T, -1).T + np.diag(np.abs(_ties(rng, n, 6, 7)))
    O = _ties(rng, (N - 1, n, n), -150, 8)  # reaches float32 subnormals
    inst = wl.Instance(D=D, O=O, b=np.zeros((N, n)))
    S = orc.assemble(D, O)
    with Single(inst, m=1, precision=bb.BT_MIXED) as s:
        s.ok()
        for j in range(N * n):
            e = np.zeros(N * n)
            e[j] = 1.0
            col = s.spmv(e.reshape(N, n), f32=True).reshape(-1)
            want = S[:, j].astype(np.float32).astype(np.float64)
            assert np.array_equal(col, want), j
