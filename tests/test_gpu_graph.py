"""CUDA-graph capture of the batched solve (one persistent launch per
replay) and the asynchronous entry points, against the synchronous call."""
import numpy as np
import pytest
import torch

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


def test_graph_replay_matches_direct_solve():
    insts = wl.config2(indices=[3, 9, 40, 200, 600, 1000])
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    B = len(insts)
    stream = torch.cuda.Stream()
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, stream=stream)
    dD, dO, db = dev(D), dev(O), dev(b)
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dD, dO, p)
    assert st == bb.BT_OK
    try:
        x_ref = dev(np.zeros(b.size))
        st, it_ref, st_ref = bb.bt_pcg_solve_batched(h, db, x_ref, B, 1e-8, 5000)
        assert st == bb.BT_OK
        x = dev(np.zeros(b.size))
        d_it = torch.zeros(B, dtype=torch.int32, device="cuda")
        d_st = torch.full((B,), -1, dtype=torch.int32, device="cuda")
        assert bb.bt_graph_capture_batched(h, db, x, 1e-8, 5000, d_it, d_st) == bb.BT_OK
        for _ in range(2):
            x.zero_()
            assert bb.bt_graph_launch(h) == bb.BT_OK
            stream.synchronize()
            assert np.array_equal(host(x), host(x_ref))
            assert np.array_equal(host(d_it), it_ref.astype(np.int32))
            assert (host(d_st) == 0).all()
        xs = host(x)
        for k, inst in enumerate(insts):
            xk = xs[v_off[k]:v_off[k] + inst.N * inst.n].reshape(inst.N, inst.n)
            assert np.linalg.norm(orc.spmv(inst.D, inst.O, xk) - inst.b) <= 1e-8 * np.linalg.norm(inst.b)
    finally:
        bb.bt_destroy(h)


def test_refactor_and_async_single_solve():
    """bt_refactor with new values (same shapes) + bt_pcg_solve_async equals a
    fresh setup + solve."""
    a = wl.small_ocp(95, 40, 6)
    b2 = wl.small_ocp(96, 40, 6)
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_FP64)
    st, h = bb.bt_setup(a.N, a.n, dev(a.D), dev(a.O), p)
    assert st == bb.BT_OK
    try:
        assert bb.bt_refactor(h, dev(b2.D), dev(b2.O)) == bb.BT_OK
        assert bb.bt_setup_status(h) == bb.BT_OK
        x = dev(np.zeros(b2.b.size))
        d = torch.zeros(2, dtype=torch.int32, device="cuda")
        assert bb.bt_pcg_solve_async(h, dev(b2.b.reshape(-1)), x, 1e-10, 1000, d[:1], d[1:]) == bb.BT_OK
        torch.cuda.synchronize()
        ref = orc.pcg_opt(b2.D, b2.O, b2.b, [1.0, 7.0], 1e-10, 1000)
        assert int(host(d)[1]) == 0 and abs(int(host(d)[0]) - ref.iters) <= 1
        assert np.linalg.norm(host(x).reshape(b2.N, b2.n) - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
        # a non-SPD block surfaces through bt_setup_status after a refactor
        Dbad = b2.D.copy()
        Dbad[7] = -np.eye(6)
        assert bb.bt_refactor(h, dev(Dbad), dev(b2.O)) == bb.BT_OK
        assert bb.bt_setup_status(h) == bb.BT_ERR_NOT_SPD
        st, i, blk, val = bb.bt_last_error(h)
        assert blk == 7
    finally:
        bb.bt_destroy(h)


def test_graph_of_refactor_and_solve_follows_new_values():
    """bt_graph_capture_refactor_solve: one replay re-forms every block from
    the values D, O hold at replay time and solves; after overwriting the
    captured buffers with another batch of the same shapes, a replay equals
    bt_refactor + bt_pcg_solve_batched on the new values, bit for bit, and
    each instance satisfies the oracle's residual test."""
    idx_a = [5, 11, 48, 300, 700, 1001]
    insts_a = wl.config2(indices=idx_a)
    shapes = [(i.N, i.n) for i in insts_a]
    insts_b = [wl.small_ocp(120 + k, N, n) for k, (N, n) in enumerate(shapes)]
    Ns, ns, d_off, o_off, v_off, Da, Oa, ba = wl.pack_batch(insts_a)
    _, _, _, _, _, Db, Ob, bb_ = wl.pack_batch(insts_b)
    B = len(insts_a)
    stream = torch.cuda.Stream()
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, stream=stream)
    dD, dO, db = dev(Da), dev(Oa), dev(ba)
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dD, dO, p)
    assert st == bb.BT_OK
    try:
        x = dev(np.zeros(ba.size))
        d_it = torch.zeros(B, dtype=torch.int32, device="cuda")
        d_st = torch.full((B,), -1, dtype=torch.int32, device="cuda")
        assert bb.bt_graph_capture_refactor_solve(h, dD, dO, db, x, 1e-8, 5000, d_it, d_st) == bb.BT_OK
        results = []
        for D_, O_, b_ in ((Da, Oa, ba), (Db, Ob, bb_)):
            with torch.cuda.stream(stream):
                dD.copy_(dev(D_))
                dO.copy_(dev(O_))
                db.copy_(dev(b_))
                x.zero_()
            assert bb.bt_graph_launch(h) == bb.BT_OK
            stream.synchronize()
            assert bb.bt_setup_status(h) == bb.BT_OK
            assert (host(d_st) == 0).all()
            results.append((host(x).copy(), host(d_it).copy()))
        # the same steps through the direct calls
        for (D_, O_, b_, insts), (xg, itg) in zip(((Da, Oa, ba, insts_a), (Db, Ob, bb_, insts_b)), results):
            dD.copy_(dev(D_))
            dO.copy_(dev(O_))
            torch.cuda.synchronize()
            assert bb.bt_refactor(h, dD, dO) == bb.BT_OK
            x_ref = dev(np.zeros(b_.size))
            st, it_ref, st_ref = bb.bt_pcg_solve_batched(h, dev(b_), x_ref, B, 1e-8, 5000)
            assert st == bb.BT_OK
            assert np.array_equal(xg, host(x_ref))
            assert np.array_equal(itg, it_ref.astype(np.int32))
            for k, inst in enumerate(insts):
                xk = xg[v_off[k]:v_off[k] + inst.N * inst.n].reshape(inst.N, inst.n)
                assert np.linalg.norm(orc.spmv(inst.D, inst.O, xk) - inst.b) <= 1e-8 * np.linalg.norm(inst.b)
    finally:
        bb.bt_destroy(h)
