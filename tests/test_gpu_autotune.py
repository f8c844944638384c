"""bt_autotune: the launch shape chosen by timing the handle's own solves
stays correct (parity with the oracle after tuning), for a batched and a
single-instance handle, and a CUDA graph captured afterwards replays it."""
import numpy as np
import pytest

from oracle import bt_oracle as orc
from paper_2503_15269_gb300 import binding as bb
from paper_2503_15269_gb300 import workloads as wl

from _util import Single, dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2503_15269_gb300 import build
    build.build()
    bb.lib()


def test_batched_autotune_keeps_parity():
    import torch
    insts = wl.config2(indices=[0, 1, 2, 3, 100, 511, 777, 1023])
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    stream = torch.cuda.Stream()
    p, keep = bb.make_params(m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED, stream=stream)
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dev(D), dev(O), p)
    assert st == bb.BT_OK
    db, x = dev(b), dev(np.zeros(b.size))
    try:
        st, kb, g = bb.bt_autotune(h, db, x, 1e-8, 5000, 1)
        assert st == bb.BT_OK and kb in (64, 72, 80) and g == 1
        x2 = dev(np.zeros(b.size))
        st, its, sts = bb.bt_pcg_solve_batched(h, db, x2, len(insts), 1e-8, 5000)
        assert st == bb.BT_OK and (sts == 0).all()
        x3 = dev(np.zeros(b.size))
        assert bb.bt_graph_capture_batched(h, db, x3, 1e-8, 5000) == bb.BT_OK
        assert bb.bt_graph_launch(h) == bb.BT_OK
        stream.synchronize()
    finally:
        bb.bt_destroy(h)
    for xx in (x, x2, x3):
        xs = host(xx)
        for k, inst in enumerate(insts):
            xk = xs[v_off[k]:v_off[k] + inst.N * inst.n].reshape(inst.N, inst.n)
            assert np.linalg.norm(orc.spmv(inst.D, inst.O, xk) - inst.b) <= 1e-8 * np.linalg.norm(inst.b)


@pytest.mark.parametrize("precision", [bb.BT_FP64, bb.BT_MIXED])
def test_single_autotune_keeps_parity(precision):
    inst = wl.config1()
    ref = orc.pcg_opt(inst.D, inst.O, inst.b, [1.0, 7.0], 1e-10, 2000)
    with Single(inst, m=2, alpha=[1.0, 7.0], precision=precision) as s:
        s.ok()
        db, x = dev(inst.b.reshape(-1)), dev(np.zeros(inst.b.size))
        st, kb, g = bb.bt_autotune(s.h, db, x, 1e-10, 2000, 1)
        # the persistent kernel on 1 .. N/2 CTAs, or (float64) the shared-memory engine on a cluster
        shapes = {1, 128 // 16, 128 // 8, 128 // 4, 128 // 2, -1, -2, -4, -8}
        assert st == bb.BT_OK and g in shapes
        st, it, xs = s.solve(inst.b, 1e-10, 2000)
    assert st == bb.BT_OK
    if precision == bb.BT_FP64:
        assert abs(it - ref.iters) <= 1 and rel(xs, ref.x) <= 1e-10
    else:
        assert rel(xs, orc.direct_solve(inst.D, inst.O, inst.b)) <= 1e-8
    assert rel(host(x).reshape(inst.b.shape), ref.x) <= 1e-8


def test_tune_cache_records_and_reuses_the_shape(tmp_path, monkeypatch):
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("BT_TUNE_CACHE", str(cache))
    inst = wl.small_ocp(140, 96, 12)
    db = dev(inst.b.reshape(-1))
    shapes = []
    for _ in range(2):
        with Single(inst, m=2, alpha=[1.0, 7.0], precision=bb.BT_MIXED) as s:
            s.ok()
            x = dev(np.zeros(inst.b.size))
            st, kb, g = bb.bt_autotune(s.h, db, x, 1e-8, 5000, 1)
            assert st == bb.BT_OK
            shapes.append((kb, g))
            res = np.linalg.norm(orc.spmv(inst.D, inst.O, host(x).reshape(inst.b.shape)) - inst.b)
            assert res <= 1e-8 * np.linalg.norm(inst.b)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1 and '"key": "single-' in lines[0]   # timed once, reused once
    assert shapes[0] == shapes[1]
