"""GPU parity of the general family member (a, b = 1 - 2a), through the C ABI.

The oracle side is `apply_family` (G_ab and H_ab from the block Jacobi matrix,
pinned densely against the multi-splitting definition of Sec. 3.1 in
test_oracle_closed_form.py) inside the oracle's textbook PCG.  Tolerances as
for the optimum (test_gpu_parity.py): float64 apply 1e-12, float32 apply 2e-4,
float64 PCG iterations within 1 and solutions within 1e-10, mixed solves to
the float64 residual tolerance.
"""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import Single, dev, host, maxrel, rel

pytestmark = pytest.mark.gpu

# block Jacobi, equal weights, stairs only, an interior point, next to the optimum
A_VALUES = [0.0, 1.0 / 3.0, 0.5, 0.8, 0.999]
# one and several chunks, ragged tails, the compile-time block sizes 12/24/36
# and run-time ones (5, 7, 20)
SHAPES = [(1, 3), (2, 5), (3, 4), (5, 7), (16, 6), (30, 20), (40, 12), (33, 24), (64, 36)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


def _family_pcg(inst, a, alpha, tol, maxit):
    return orc.pcg(inst.D, inst.O, inst.b, lambda r: orc.apply_family(inst.D, inst.O, r, a, alpha), tol, maxit)


@pytest.mark.parametrize("N,n", SHAPES)
@pytest.mark.parametrize("a", A_VALUES)
@pytest.mark.parametrize("m", [1, 2, 3])
def test_apply_fp64_family(N, n, a, m):
    inst = wl.small_ocp(80, N, n)
    r = np.random.default_rng(N * 31 + n).standard_normal((N, n))
    ref = orc.apply_family(inst.D, inst.O, r, a, [1.0] * m)
    with Single(inst, m=m, a=a) as s:
        s.ok()
        z = s.apply(r)
    assert maxrel(z, ref) <= 1e-12


@pytest.mark.parametrize("N,n", SHAPES)
@pytest.mark.parametrize("a", [0.0, 0.5, 0.8])
@pytest.mark.parametrize("m", [2, 4])
def test_apply_mixed_family(N, n, a, m):
    inst = wl.small_ocp(81, N, n)
    r = np.random.default_rng(N * 17 + n).standard_normal((N, n))
    ref = orc.apply_family(inst.D, inst.O, r, a, [1.0] * m)
    with Single(inst, m=m, a=a, precision=bb.BT_MIXED) as s:
        s.ok()
        z = s.apply(r)
    assert maxrel(z, ref) <= 2e-4


@pytest.mark.parametrize("a", A_VALUES)
@pytest.mark.parametrize("m", [1, 2, 3])
def test_solve_fp64_family_matches_oracle_pcg(a, m):
    inst = wl.small_ocp(82, 30, 20)
    alpha = [1.0] * m
    ref = _family_pcg(inst, a, alpha, 1e-10, 2000)
    assert ref.status == orc.OK
    with Single(inst, m=m, alpha=alpha, a=a) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-10, 2000)
    assert st == bb.BT_OK
    assert abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10


@pytest.mark.parametrize("G", [2, 3, 5])
@pytest.mark.parametrize("a", [0.0, 0.5])
def test_group_ctas_family(G, a):
    """Block-row ranges split over G CTAs: the two lower bands of H_ab cross
    each range start through the halo rows."""
    inst = wl.small_ocp(83, 37, 6)
    alpha = [1.0, 1.0]
    ref = _family_pcg(inst, a, alpha, 1e-10, 2000)
    r = np.random.default_rng(G).standard_normal((37, 6))
    with Single(inst, m=2, alpha=alpha, a=a, group_ctas=G) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-10, 2000)
        z = s.apply(r)
    assert st == bb.BT_OK and abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10
    assert maxrel(z, orc.apply_family(inst.D, inst.O, r, a, alpha)) <= 1e-12


@pytest.mark.parametrize("a", [0.0, 1.0 / 3.0, 0.5])
def test_solve_mixed_family(a):
    inst = wl.config1()
    xref = orc.direct_solve(inst.D, inst.O, inst.b)
    with Single(inst, m=2, a=a, precision=bb.BT_MIXED) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-12, 20000)
        _, outer, res = s.info()
    assert st == bb.BT_OK
    assert res <= 1e-12
    assert rel(x, xref) <= 1e-8


def test_batched_family_ragged_fp64():
    rng = np.random.default_rng(84)
    insts = [wl.small_ocp(90 + k, int(rng.integers(1, 40)), int(rng.choice([1, 3, 6, 12]))) for k in range(16)]
    a, alpha = 0.5, [1.0, 1.0, 1.0]
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    p, keep = bb.make_params(m=3, alpha=alpha, a=a)
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dev(D), dev(O if O.size else np.zeros(1)), p)
    assert st == bb.BT_OK, bb.status_string(st)
    x = dev(np.zeros(b.size))
    try:
        st, its, sts = bb.bt_pcg_solve_batched(h, dev(b), x, len(insts), 1e-10, 2000)
    finally:
        bb.bt_destroy(h)
    assert st == bb.BT_OK and (sts == 0).all()
    xs = host(x)
    for k, inst in enumerate(insts):
        ref = _family_pcg(inst, a, alpha, 1e-10, 2000)
        xk = xs[v_off[k]:v_off[k] + inst.N * inst.n].reshape(inst.N, inst.n)
        assert abs(its[k] - ref.iters) <= 1, k
        assert rel(xk, ref.x) <= 1e-10, k


def test_refactor_family_keeps_scaling():
    """bt_refactor re-runs the whole setup, the scaling by a included."""
    i1, i2 = wl.small_ocp(85, 12, 5), wl.small_ocp(86, 12, 5)
    r = np.random.default_rng(3).standard_normal((12, 5))
    with Single(i1, m=2, a=0.25) as s:
        s.ok()
        assert bb.bt_refactor(s.h, dev(i2.D), dev(i2.O)) == bb.BT_OK
        assert bb.bt_setup_status(s.h) == bb.BT_OK
        z = s.apply(r)
    assert maxrel(z, orc.apply_family(i2.D, i2.O, r, 0.25, [1.0, 1.0])) <= 1e-12


def test_general_a_limits():
    """H_ab needs 9 blocks of stage: n = 48 in float64 is refused at setup,
    the many-RHS engine implements a = 1 only."""
    inst = wl.small_ocp(87, 4, 48)
    s = Single(inst, m=2, a=0.5)
    try:
        assert s.st == bb.BT_ERR_ARG
    finally:
        s.close()
    inst = wl.small_ocp(88, 8, 12)
    with Single(inst, m=2, a=0.5, precision=bb.BT_MIXED) as s:
        s.ok()
        B = dev(np.zeros(8 * 12 * 2))
        X = dev(np.zeros(8 * 12 * 2))
        st = bb.bt_pcg_solve_multi(s.h, B, X, 2, 1e-8, 100)
        st = st[0] if isinstance(st, tuple) else st
        assert st == bb.BT_ERR_PARAM


def test_protocol_table_matches_oracle():
    """The numerical-results protocol on one matrix (N = 30, n = 20, unit-norm
    b, ||S x - b|| < 1e-6): float64 PCG iterations of every (setting, m) as
    the oracle's, and the orderings the section states hold on the GPU counts."""
    inst = wl.small_ocp(300, 30, 20)
    b = inst.b / np.linalg.norm(inst.b)
    gem = {}
    for name, a, pc in wl.PROTOCOL_SETTINGS:
        gem[name] = []
        for m in (1, 2, 3, 4):
            alpha = wl.protocol_alpha(m, pc)
            ref = orc.pcg(inst.D, inst.O, b, lambda v: orc.apply_family(inst.D, inst.O, v, a, alpha), 1e-6, 5000)
            with Single(inst, m=m, alpha=alpha, a=a) as s:
                s.ok()
                st, it, x = s.solve(b, 1e-6, 5000)
            assert st == bb.BT_OK and abs(it - ref.iters) <= 1, (name, m, it, ref.iters)
            assert np.linalg.norm(orc.spmv(inst.D, inst.O, x) - b) < 1e-6
            gem[name].append(it * orc.g_a(m, a))
    for k in range(4):
        assert gem["PolyCoeff"][k] <= min(g[k] for g in gem.values())
        assert (gem["optimal"][k] < gem["block Jacobi"][k]) == (k % 2 == 0)
    assert int(np.argmin(gem["PolyCoeff"])) == 1


@pytest.mark.parametrize("G", [2, 4])
def test_group_ctas_family_mixed(G):
    """Mixed precision over G CTAs: the float32 five-array H sweep across range
    starts (halo rows of both lower bands)."""
    inst = wl.small_ocp(89, 41, 12)
    xref = orc.direct_solve(inst.D, inst.O, inst.b)
    r = np.random.default_rng(G).standard_normal((41, 12))
    with Single(inst, m=3, a=0.5, precision=bb.BT_MIXED, group_ctas=G) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-12, 20000)
        z = s.apply(r)
    assert st == bb.BT_OK and rel(x, xref) <= 1e-8
    assert maxrel(z, orc.apply_family(inst.D, inst.O, r, 0.5, [1.0, 1.0, 1.0])) <= 2e-4
