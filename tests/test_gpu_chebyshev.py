"""GPU solves with the Chebyshev polynomial coefficients (bt_alpha_chebyshev,
alternating in sign for m >= 3) against the oracle's PCG with the same
coefficients, through the C ABI.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import Single, dev, host, maxrel, rel

pytestmark = pytest.mark.gpu
RHO = 0.985  # bounds rho(H_opt) on the LQR family (0.977-0.982 measured)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


@pytest.mark.parametrize("m", [2, 3, 4])
def test_fp64_solve_matches_oracle(m):
    inst = wl.small_ocp(400, 128, 12)
    st, a = bb.bt_alpha_chebyshev(m, RHO)
    assert st == bb.BT_OK
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, a, 1e-10, 3000)
    with Single(inst, m=m, alpha=a) as s:
        s.ok()
        st, it, x = s.solve(inst.b, 1e-10, 3000)
    assert st == bb.BT_OK and abs(it - ref.iters) <= 1
    assert rel(x, ref.x) <= 1e-10


@pytest.mark.parametrize("m", [3, 4])
@pytest.mark.parametrize("precision,tol", [(bb.BT_FP64, 1e-12), (bb.BT_MIXED, 2e-4)])
def test_apply_matches_oracle(m, precision, tol):
    inst = wl.small_ocp(401, 40, 36)
    st, a = bb.bt_alpha_chebyshev(m, RHO)
    r = np.random.default_rng(m).standard_normal((40, 36))
    with Single(inst, m=m, alpha=a, precision=precision) as s:
        s.ok()
        z = s.apply(r)
    assert maxrel(z, orc.apply_opt(orc.opt_blocks(inst.D, inst.O), r, a)) <= tol


def test_batched_mixed_fewer_iterations_than_polycoeff():
    insts = wl.config2(indices=[0, 1, 2, 3, 100, 511, 777, 1023])
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    out = {}
    for name, m, alpha in (("polycoeff", 2, [1.0, 7.0]), ("cheb3", 3, bb.bt_alpha_chebyshev(3, RHO)[1]),
                           ("cheb4", 4, bb.bt_alpha_chebyshev(4, RHO)[1])):
        p, keep = bb.make_params(m=m, alpha=alpha, precision=bb.BT_MIXED)
        st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dev(D), dev(O), p)
        assert st == bb.BT_OK
        x = dev(np.zeros(b.size))
        try:
            st, its, sts = bb.bt_pcg_solve_batched(h, dev(b), x, len(insts), 1e-8, 5000)
        finally:
            bb.bt_destroy(h)
        assert st == bb.BT_OK and (sts == 0).all()
        xs = host(x)
        for k, inst in enumerate(insts):
            xk = xs[v_off[k]:v_off[k] + inst.N * inst.n].reshape(inst.N, inst.n)
            assert np.linalg.norm(orc.spmv(inst.D, inst.O, xk) - inst.b) <= 1e-8 * np.linalg.norm(inst.b)
        out[name] = float(np.mean(its))
    assert out["cheb3"] < out["polycoeff"] and out["cheb4"] < out["cheb3"], out


@pytest.mark.parametrize("precision,tol", [(bb.BT_FP64, 1e-9), (bb.BT_MIXED, 1e-5)])
def test_estimate_rho_matches_oracle(precision, tol):
    """bt_estimate_rho per instance of a batched handle against the oracle's
    power iteration with the same start vector and step count."""
    insts = [wl.small_ocp(600 + k, N, n) for k, (N, n) in enumerate([(16, 6), (30, 20), (33, 12)])]
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=precision)
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dev(D), dev(O), p)
    assert st == bb.BT_OK
    try:
        st, rho = bb.bt_estimate_rho(h, 100, len(insts))
    finally:
        bb.bt_destroy(h)
    assert st == bb.BT_OK
    for k, inst in enumerate(insts):
        ref = orc.power_rho(inst.D, inst.O, 100)
        assert abs(rho[k] - ref) <= tol * ref, (k, rho[k], ref)


def test_estimate_rho_refuses_general_member():
    inst = wl.small_ocp(610, 8, 6)
    with Single(inst, m=2, a=0.5) as s:
        s.ok()
        assert bb.bt_estimate_rho(s.h, 10, 1)[0] == bb.BT_ERR_PARAM


def test_estimate_rho_matrix_free_handle():
    """The matrix-free variant applies the same G_opt: the same estimate."""
    inst = wl.small_ocp(620, 24, 12)
    ref = orc.power_rho(inst.D, inst.O, 60)
    with Single(inst, m=2, alpha=[1.0, 7.0], h_matrix_free=True) as s:
        s.ok()
        st, rho = bb.bt_estimate_rho(s.h, 60, 1)
    assert st == bb.BT_OK and abs(rho[0] - ref) <= 1e-9 * ref


@pytest.mark.parametrize("precision,tol", [(bb.BT_FP64, 1e-8), (bb.BT_MIXED, 1e-4)])
def test_ritz_rho_matches_oracle(precision, tol):
    """bt_ritz_rho per instance of a batched handle against the oracle's
    Ritz estimate from the same right-hand side and iteration count."""
    insts = [wl.small_ocp(630 + k, N, n) for k, (N, n) in enumerate([(16, 6), (30, 20), (33, 12)])]
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=precision)
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dev(D), dev(O), p)
    assert st == bb.BT_OK
    try:
        st, rho = bb.bt_ritz_rho(h, dev(b), 40, len(insts))
    finally:
        bb.bt_destroy(h)
    assert st == bb.BT_OK
    for k, inst in enumerate(insts):
        ref = orc.ritz_rho(inst.D, inst.O, inst.b, 40)
        assert abs(rho[k] - ref) <= tol, (k, rho[k], ref)


def test_history_records_the_oracle_iterates():
    """bt_set_history: relative residuals and CG scalars of a float64 solve
    equal those of the oracle's PCG, iteration by iteration."""
    inst = wl.config1()
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-10, 2000)
    L = 64
    hist = dev(np.full(L * 3, -1.0))
    with Single(inst, m=2, alpha=[1.0, 7.0]) as s:
        s.ok()
        assert bb.bt_set_history(s.h, hist, L) == bb.BT_OK
        st, it, x = s.solve(inst.b, 1e-10, 2000)
    assert st == bb.BT_OK
    hh = host(hist).reshape(L, 3)
    K = min(it, L)
    nb = np.linalg.norm(inst.b)
    np.testing.assert_allclose(hh[:K, 0], np.array(ref.res_history[1:K + 1]) / nb, rtol=1e-8)
    np.testing.assert_allclose(hh[:K, 1], np.array(ref.alphas[:K]), rtol=1e-8)
    np.testing.assert_allclose(hh[:K - 1, 2], np.array(ref.betas[:K - 1]), rtol=1e-8)
    assert (hh[K:, 0] == -1.0).all()
