"""GPU parity of the LQR Schur-complement formation and the dual-to-primal
recovery (bt_lqr_schur, bt_lqr_recover) against the oracle, through the C ABI.

Tolerances: both are float64 products of explicit inverses of SPD blocks
(Q_k, R_k with condition numbers below ~30 here), so the blocks, gamma and
the recovered primal variables agree to a max relative difference of 1e-12.
The end-to-end pipeline (formation, batched PCG, recovery) is compared with
the QP solution of the bordered KKT system at the solve's tolerance.
"""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import dev, host, maxrel, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


def _pack(probs):
    cat = lambda xs, shape_tail: (np.concatenate([x.reshape(-1) for x in xs]) if sum(x.size for x in xs)
                                  else np.zeros(0))
    A = cat([p.A for p in probs], None)
    Bm = cat([p.Bm for p in probs], None)
    Q = cat([p.Q for p in probs], None)
    R = cat([p.R for p in probs], None)
    q = cat([p.q for p in probs], None)
    r = cat([p.r for p in probs], None)
    c = cat([p.c for p in probs], None)
    return A, Bm, Q, R, q, r, c


def _dev_or_empty(a):
    import torch
    return dev(a) if a.size else torch.zeros(0, dtype=torch.float64, device="cuda:0")


def _split(flat, sizes, shapes):
    out, o = [], 0
    for s, sh in zip(sizes, shapes):
        out.append(flat[o:o + s].reshape(sh))
        o += s
    return out


PROBS = [(1, 3, 2), (2, 1, 1), (5, 4, 6), (16, 6, 2), (17, 12, 4), (33, 24, 8), (40, 36, 12), (3, 48, 48)]


def _schur_gpu(probs):
    A, Bm, Q, R, q, r, c = _pack(probs)
    Ns = [p.N for p in probs]
    ns = [p.n for p in probs]
    ms = [p.m for p in probs]
    dD = dev(np.zeros(sum(p.N * p.n * p.n for p in probs)))
    dO = _dev_or_empty(np.zeros(sum((p.N - 1) * p.n * p.n for p in probs)))
    dg = dev(np.zeros(sum(p.N * p.n for p in probs)))
    st, bi, br = bb.bt_lqr_schur(Ns, ns, ms, _dev_or_empty(A), _dev_or_empty(Bm), dev(Q), _dev_or_empty(R), dev(q),
                                 _dev_or_empty(r), dev(c), dD, dO, dg)
    return st, bi, br, host(dD), host(dO), host(dg)


def test_schur_matches_oracle_ragged_batch():
    probs = [wl.small_lqr(10 + k, N, n, m) for k, (N, n, m) in enumerate(PROBS)]
    st, _, _, D, O, g = _schur_gpu(probs)
    assert st == bb.BT_OK, bb.status_string(st)
    Ds = _split(D, [p.N * p.n * p.n for p in probs], [(p.N, p.n, p.n) for p in probs])
    Os = _split(O, [(p.N - 1) * p.n * p.n for p in probs], [(p.N - 1, p.n, p.n) for p in probs])
    gs = _split(g, [p.N * p.n for p in probs], [(p.N, p.n) for p in probs])
    for k, p in enumerate(probs):
        Dr, Or, gr = orc.lqr_schur(p.A, p.Bm, p.Q, p.R, p.q, p.r, p.c)
        assert maxrel(Ds[k], Dr) <= 1e-12, k
        if p.N > 1:
            assert maxrel(Os[k], Or) <= 1e-12, k
        assert maxrel(gs[k], gr) <= 1e-12, k


def test_recover_matches_oracle_ragged_batch():
    probs = [wl.small_lqr(30 + k, N, n, m) for k, (N, n, m) in enumerate(PROBS)]
    A, Bm, Q, R, q, r, c = _pack(probs)
    lam = np.random.default_rng(5).standard_normal(sum(p.N * p.n for p in probs))
    dx = dev(np.zeros(lam.size))
    du = _dev_or_empty(np.zeros(sum((p.N - 1) * p.m for p in probs)))
    st = bb.bt_lqr_recover([p.N for p in probs], [p.n for p in probs], [p.m for p in probs], _dev_or_empty(A),
                           _dev_or_empty(Bm), dev(Q), _dev_or_empty(R), dev(q), _dev_or_empty(r), dev(lam), dx, du)
    assert st == bb.BT_OK, bb.status_string(st)
    xs = _split(host(dx), [p.N * p.n for p in probs], [(p.N, p.n) for p in probs])
    us = _split(host(du), [(p.N - 1) * p.m for p in probs], [(p.N - 1, p.m) for p in probs])
    ls = _split(lam, [p.N * p.n for p in probs], [(p.N, p.n) for p in probs])
    for k, p in enumerate(probs):
        xr, ur = orc.lqr_recover(p.A, p.Bm, p.Q, p.R, p.q, p.r, ls[k])
        assert maxrel(xs[k], xr) <= 1e-12, k
        if p.N > 1:
            assert maxrel(us[k], ur) <= 1e-12, k


@pytest.mark.parametrize("precision", [bb.BT_FP64, bb.BT_MIXED])
def test_pipeline_solves_the_qp(precision):
    """Formation -> batched PCG (a = 1, m = 2, alpha = (1, 7)) -> recovery gives
    the QP's solution (the bordered KKT system solved densely)."""
    shapes = [(12, 6, 2), (30, 12, 4), (45, 24, 8), (20, 36, 12)]
    probs = [wl.small_lqr(50 + k, N, n, m) for k, (N, n, m) in enumerate(shapes)]
    A, Bm, Q, R, q, r, c = _pack(probs)
    Ns, ns, ms = [p.N for p in probs], [p.n for p in probs], [p.m for p in probs]
    dD = dev(np.zeros(sum(p.N * p.n * p.n for p in probs)))
    dO = dev(np.zeros(sum((p.N - 1) * p.n * p.n for p in probs)))
    dg = dev(np.zeros(sum(p.N * p.n for p in probs)))
    dA, dB, dQ, dR, dq, dr, dc = (dev(v) for v in (A, Bm, Q, R, q, r, c))
    st, _, _ = bb.bt_lqr_schur(Ns, ns, ms, dA, dB, dQ, dR, dq, dr, dc, dD, dO, dg)
    assert st == bb.BT_OK
    d_off = np.concatenate([[0], np.cumsum([p.N * p.n * p.n for p in probs])[:-1]]).astype(np.int64)
    o_off = np.concatenate([[0], np.cumsum([(p.N - 1) * p.n * p.n for p in probs])[:-1]]).astype(np.int64)
    v_off = np.concatenate([[0], np.cumsum([p.N * p.n for p in probs])[:-1]]).astype(np.int64)
    par, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=precision)
    st, h = bb.bt_setup_batched(np.array(Ns, np.int32), np.array(ns, np.int32), d_off, o_off, dD, dO, par)
    assert st == bb.BT_OK
    dl = dev(np.zeros(dg.numel()))
    try:
        st, its, sts = bb.bt_pcg_solve_batched(h, dg, dl, len(probs), 1e-12, 5000)
    finally:
        bb.bt_destroy(h)
    assert st == bb.BT_OK and (sts == 0).all()
    dx = dev(np.zeros(dg.numel()))
    du = dev(np.zeros(sum((p.N - 1) * p.m for p in probs)))
    assert bb.bt_lqr_recover(Ns, ns, ms, dA, dB, dQ, dR, dq, dr, dl, dx, du) == bb.BT_OK
    xs = _split(host(dx), [p.N * p.n for p in probs], [(p.N, p.n) for p in probs])
    us = _split(host(du), [(p.N - 1) * p.m for p in probs], [(p.N - 1, p.m) for p in probs])
    for k, p in enumerate(probs):
        G, g, C, cv = orc.lqr_dense(p.A, p.Bm, p.Q, p.R, p.q, p.r, p.c)
        nz, nl = G.shape[0], C.shape[0]
        sol = np.linalg.solve(np.block([[G, C.T], [C, np.zeros((nl, nl))]]), np.concatenate([-g, cv]))
        z = sol[:nz]
        zg = np.concatenate([np.concatenate([xs[k][i], us[k][i]]) if i < p.N - 1 else xs[k][i] for i in range(p.N)])
        assert rel(zg, z) <= 1e-8, k


def test_non_spd_blocks_are_reported():
    probs = [wl.small_lqr(70, 6, 4, 2), wl.small_lqr(71, 9, 4, 2)]
    probs[1].Q[5] = -np.eye(4)
    st, bi, br, *_ = _schur_gpu(probs)
    assert st == bb.BT_ERR_NOT_SPD and (bi, br) == (1, 5)
    probs = [wl.small_lqr(72, 6, 4, 2)]
    probs[0].R[3] = np.diag([1.0, -2.0])
    st, bi, br, *_ = _schur_gpu(probs)
    assert st == bb.BT_ERR_NOT_SPD and (bi, br) == (0, 3)


def test_single_knot_problems_without_dynamics():
    """N = 1 everywhere: no A, B, R, r; D_0 = Q_0^-1, gamma_0 = -(c_0 + Q_0^-1 q_0)."""
    probs = [wl.small_lqr(80 + k, 1, n, 2) for k, n in enumerate([1, 4, 7])]
    st, bi, br, D, O, g = _schur_gpu(probs)
    assert st == bb.BT_OK
    Ds = _split(D, [p.n * p.n for p in probs], [(1, p.n, p.n) for p in probs])
    gs = _split(g, [p.n for p in probs], [(1, p.n) for p in probs])
    for k, p in enumerate(probs):
        Dr, Or, gr = orc.lqr_schur(p.A, p.Bm, p.Q, p.R, p.q, p.r, p.c)
        assert maxrel(Ds[k], Dr) <= 1e-12 and maxrel(gs[k], gr) <= 1e-12


def _offsets(probs):
    cum = lambda xs: np.concatenate([[0], np.cumsum(xs)[:-1]]).astype(np.int64)
    return (cum([p.N * p.n * p.n for p in probs]), cum([(p.N - 1) * p.n * p.n for p in probs]),
            cum([p.N * p.n for p in probs]))


FUSED = [(1, 5, 2), (12, 6, 2), (17, 12, 4), (33, 24, 8), (40, 36, 12), (3, 48, 48), (20, 36, 12), (9, 7, 3)]


def test_lqr_refactor_matches_the_oracle():
    """bt_lqr_refactor (formation straight into a mixed handle, D_k factored on
    chip, then E and H) against the oracle: gamma as bt_lqr_schur gives it; the
    handle's float64 S (through bt_spmv) to 1e-12; the preconditioner built from
    its float32 blocks (bt_apply_precond) within the float32 bound of the
    parity tests; and the solve of S lam = gamma against the oracle's direct
    solve at the mixed path's 1e-8."""
    probs = [wl.small_lqr(90 + k, N, n, m) for k, (N, n, m) in enumerate(FUSED)]
    A, Bm, Q, R, q, r, c = _pack(probs)
    Ns, ns, ms = [p.N for p in probs], [p.n for p in probs], [p.m for p in probs]
    dA, dB, dQ, dR, dq, dr, dc = (dev(v) for v in (A, Bm, Q, R, q, r, c))
    dD = dev(np.zeros(sum(p.N * p.n * p.n for p in probs)))
    dO = dev(np.zeros(sum((p.N - 1) * p.n * p.n for p in probs)))
    dg = dev(np.zeros(sum(p.N * p.n for p in probs)))
    st, _, _ = bb.bt_lqr_schur(Ns, ns, ms, dA, dB, dQ, dR, dq, dr, dc, dD, dO, dg)
    assert st == bb.BT_OK
    d_off, o_off, v_off = _offsets(probs)
    par, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED)
    # a handle set up from unrelated blocks: everything it solves with must
    # come from the fused call
    dz = dev(np.concatenate([np.tile(np.eye(p.n).reshape(-1), p.N) for p in probs]))
    st, h = bb.bt_setup_batched(np.array(Ns, np.int32), np.array(ns, np.int32), d_off, o_off, dz,
                                dev(np.zeros(max(1, dO.numel()))), par)
    assert st == bb.BT_OK
    try:
        dg2 = dev(np.zeros(dg.numel()))
        st, bi, br = bb.bt_lqr_refactor(h, ms, dA, dB, dQ, dR, dq, dr, dc, dg2)
        assert st == bb.BT_OK, bb.status_string(st)
        assert np.array_equal(host(dg2), host(dg))
        rng = np.random.default_rng(11)
        xv = rng.standard_normal(dg.numel())
        y64 = dev(np.zeros(xv.size))
        assert bb.bt_spmv(h, dev(xv), y64) == bb.BT_OK
        z = dev(np.zeros(xv.size))
        assert bb.bt_apply_precond(h, dev(xv), z) == bb.BT_OK
        dl = dev(np.zeros(dg.numel()))
        st, its, sts = bb.bt_pcg_solve_batched(h, dg2, dl, len(probs), 1e-12, 5000)
        assert st == bb.BT_OK and (sts == 0).all()
        # primal recovery from the factors the formation kept, against the
        # oracle and against the factorizing recovery
        dx = dev(np.zeros(dg.numel()))
        du = dev(np.zeros(sum((p.N - 1) * p.m for p in probs)))
        assert bb.bt_lqr_recover_factored(h, [mm + 1 for mm in ms], dA, dB, dq, dr, dl, dx, du) == bb.BT_ERR_STATE
        assert bb.bt_lqr_recover_factored(h, ms, dA, dB, dq, dr, dl, dx, du) == bb.BT_OK
        dx2, du2 = dev(np.zeros(dg.numel())), dev(np.zeros(du.numel()))
        assert bb.bt_lqr_recover(Ns, ns, ms, dA, dB, dQ, dR, dq, dr, dl, dx2, du2) == bb.BT_OK
    finally:
        bb.bt_destroy(h)
    assert maxrel(host(dx), host(dx2)) <= 1e-12 and maxrel(host(du), host(du2)) <= 1e-12
    xs = _split(host(dx), [p.N * p.n for p in probs], [(p.N, p.n) for p in probs])
    us = _split(host(du), [(p.N - 1) * p.m for p in probs], [(p.N - 1, p.m) for p in probs])
    lams = _split(host(dl), [p.N * p.n for p in probs], [(p.N, p.n) for p in probs])
    for k, p in enumerate(probs):
        xr, ur = orc.lqr_recover(p.A, p.Bm, p.Q, p.R, p.q, p.r, lams[k])
        assert maxrel(xs[k], xr) <= 1e-12, k
        if p.N > 1:
            assert maxrel(us[k], ur) <= 1e-12, k
    # the two-step path (bt_lqr_schur's D, O through bt_setup_batched) leaves the
    # same handle: the same solve, bit for bit
    st, h2 = bb.bt_setup_batched(np.array(Ns, np.int32), np.array(ns, np.int32), d_off, o_off, dD, dO, par)
    assert st == bb.BT_OK
    try:
        dl2 = dev(np.zeros(dg.numel()))
        st, its2, sts2 = bb.bt_pcg_solve_batched(h2, dg, dl2, len(probs), 1e-12, 5000)
        assert st == bb.BT_OK and (sts2 == 0).all()
    finally:
        bb.bt_destroy(h2)
    assert (its2 == its).all() and np.array_equal(host(dl2), host(dl))
    ys, zs, ls, xs, gs = (_split(host(t) if not isinstance(t, np.ndarray) else t, [p.N * p.n for p in probs],
                                 [(p.N, p.n) for p in probs]) for t in (y64, z, dl, xv, dg2))
    for k, p in enumerate(probs):
        Dr, Or, gr = orc.lqr_schur(p.A, p.Bm, p.Q, p.R, p.q, p.r, p.c)
        assert maxrel(gs[k], gr) <= 1e-12, k
        assert maxrel(ys[k], orc.spmv(Dr, Or, xs[k])) <= 1e-12, k
        assert maxrel(zs[k], orc.apply_opt(orc.opt_blocks(Dr, Or), xs[k], [1.0, 7.0])) <= 2e-4, k
        assert rel(ls[k], orc.direct_solve(Dr, Or, gr)) <= 1e-8, k


def test_lqr_refactor_rejects_other_handles_and_reports_non_spd():
    probs = [wl.small_lqr(95, 6, 4, 2), wl.small_lqr(96, 9, 4, 2)]
    A, Bm, Q, R, q, r, c = _pack(probs)
    Ns, ns, ms = [p.N for p in probs], [p.n for p in probs], [p.m for p in probs]
    d_off, o_off, _ = _offsets(probs)
    dz = dev(np.concatenate([np.tile(np.eye(p.n).reshape(-1), p.N) for p in probs]))
    dO = dev(np.zeros(sum((p.N - 1) * p.n * p.n for p in probs)))
    dg = dev(np.zeros(sum(p.N * p.n for p in probs)))
    for prec in (bb.BT_FP64, bb.BT_MIXED):
        par, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=prec)
        st, h = bb.bt_setup_batched(np.array(Ns, np.int32), np.array(ns, np.int32), d_off, o_off, dz, dO, par)
        assert st == bb.BT_OK
        try:
            dx = dev(np.zeros(dg.numel()))
            du = dev(np.zeros(sum((p.N - 1) * p.m for p in probs)))
            # no formation on this handle yet: no factors to recover from
            assert bb.bt_lqr_recover_factored(h, ms, dev(A), dev(Bm), dev(q), dev(r), dg, dx, du) == bb.BT_ERR_STATE
            Qbad = Q.copy()
            Qbad[(6 * 16) + 5 * 16:(6 * 16) + 6 * 16] = -np.eye(4).reshape(-1)  # Q_5 of problem 1
            st, bi, br = bb.bt_lqr_refactor(h, ms, dev(A), dev(Bm), dev(Qbad), dev(R), dev(q), dev(r), dev(c), dg)
            if prec == bb.BT_FP64:
                assert st == bb.BT_ERR_STATE
            else:
                assert st == bb.BT_ERR_NOT_SPD and (bi, br) == (1, 5)
        finally:
            bb.bt_destroy(h)
