#!/usr/bin/env python
"""Benchmark of the block-tridiagonal PCG library on one GB300 (or N, weak).

Workload (one step): 1024 LQR Schur-complement instances, horizon
N ~ U{32..512}, block size n in {12, 24, 36}, input size n/3 -- setup of every
instance's preconditioner blocks (Cholesky in float64, float32 blocks) and a
mixed-precision PCG solve of all of them to relative residual 1e-8, in one
persistent launch, with the optimal-parameter preconditioner at m = 2,
alpha = (1, 7).  Inputs are larger than L2 (several GB), so no flush is
needed between steps.

Prints one JSON line (rank 0).  See --help for the options.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/s at rel. residual 1e-8: mixed+batched vs plain FP64 PCG; HBM % of peak"
UNIT = "solves/s"
TOL = 1e-8
ALPHA = (1.0, 7.0)
M = 2
KERNEL_SRC = os.path.join(ROOT, "paper_2503_15269_gb300", "csrc", "bt_pcg_kernel.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "pcg_batched_ocp1024_traffic.json")


def _jsonable(o):
    if hasattr(o, "item"):
        return o.item()
    if hasattr(o, "tolist"):
        return o.tolist()
    return str(o)


def emit(line):
    print(json.dumps(line, default=_jsonable), flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=1024, help="instances per step (1024 = the published workload)")
    ap.add_argument("--profile", action="store_true", help="timed loop only (for ncu): no baselines, e2e or clocks")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 one-at-a-time comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-sample", type=int, default=48, help="instances in the oracle CPU sample")
    ap.add_argument("--maxit", type=int, default=20000,
                    help="many_rhs: iteration limit (with --profile a short capture may stop early)")
    ap.add_argument("--mrhs-engine", type=int, default=0, choices=[0, 1, 2],
                    help="many_rhs: 0 automatic (tensor cores for n = 48), 1 float32 SIMT, 2 tensor cores")
    ap.add_argument("--workload", choices=["ocp_batch", "many_rhs", "adjoint", "small", "family", "lqr", "alpha",
                                           "matrix_free", "precision"],
                    default="ocp_batch",
                    help="ocp_batch: the headline workload (default); many_rhs: one LL^T system, N=2048, "
                         "n=48, 64 right-hand sides; adjoint: 256 LQR instances, N=256, n=24, forward + adjoint; "
                         "small: single instances LL^T N=16 n=6 (float64, tol 1e-10) and LQR N=128 n=12")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_job(args):
    """One instance of the sample: the oracle's PCG (timed: the CPU baseline)
    and, untimed, its direct solve (the reference for the GPU's error)."""
    idx, tol, want_x = args
    from oracle import bt_oracle as orc
    from paper_2503_15269_gb300 import workloads as wl
    inst = wl.config2(indices=[idx])[0]
    t0 = time.perf_counter()
    res = orc.pcg_opt(inst.D, inst.O, inst.b, list(ALPHA), tol, 5000)
    dt = time.perf_counter() - t0
    xd = orc.direct_solve(inst.D, inst.O, inst.b).reshape(-1) if want_x else None
    return idx, dt, res.iters, res.status, (res.x.reshape(-1) if want_x else None), xd


def sample_indices(batch: int, count: int):
    step = max(1, batch // count)
    return list(range(0, batch, step))[:count]


def run_oracle(indices, procs, want_x=False):
    """The oracle over a sample of instances in `procs` spawned processes;
    wall time of the timed PCG leg (with want_x the workers also return the
    PCG and direct-solve x of each instance, computed after the timed leg)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_job, [(indices[0], TOL, False)])  # warm the workers (imports)
        t0 = time.perf_counter()
        out = pool.map(_oracle_job, [(i, TOL, False) for i in indices], chunksize=1)
        wall = time.perf_counter() - t0
        if want_x:
            xs = pool.map(_oracle_job, [(i, TOL, True) for i in indices], chunksize=1)
            out = [(o[0], o[1], o[2], o[3], x[4], x[5]) for o, x in zip(out, xs)]
    return wall, out


def err_vs_oracle(x_gpu, v_off, Ns, ns, out):
    """Largest relative error, over the sampled instances, of the GPU's x
    against the oracle's direct solve (float64 block Cholesky) and against the
    oracle's PCG x at the same tolerance."""
    import numpy as np
    e_dir, e_pcg = 0.0, 0.0
    for o in out:
        k = o[0]
        xk = x_gpu[v_off[k]:v_off[k] + int(Ns[k]) * int(ns[k])]
        e_dir = max(e_dir, float(np.linalg.norm(xk - o[5]) / np.linalg.norm(o[5])))
        e_pcg = max(e_pcg, float(np.linalg.norm(xk - o[4]) / np.linalg.norm(o[4])))
    return {"max_rel_err_vs_direct": e_dir, "max_rel_err_vs_oracle_pcg": e_pcg, "instances": len(out),
            "reference": "oracle direct solve (float64 block Cholesky) and oracle PCG at the same tol"}


def max_over_ranks(ms, dist, device):
    """The job's time: the slowest rank's (every rank calls it; at N = 1 it
    returns ms).  The only exchange between ranks: instances are independent,
    each rank solves its own batch (weak scaling, no data-path collective)."""
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, steps, ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return world * units_per_rank * steps / (ms / 1e3)


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def reference_arm(a):
    """The oracle (numpy float64, as it stands) timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    procs = min(cpu_cores(), 16)
    idx = sample_indices(a.batch, min(a.cpu_sample, 32))
    for _ in range(a.warmup):
        run_oracle(idx[:procs], procs)
    walls = []
    n_done = 0
    for _ in range(a.steps):
        wall, out = run_oracle(idx, procs)
        walls.append(wall)
        n_done += len(out)
    value = n_done / sum(walls)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(walls) / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded LQR Schur complements)",
        "config": {"workload": f"ocp batch of {a.batch}: N~U{{32..512}}, n in {{12,24,36}}, m=n/3; "
                               f"each step solves a sample of {len(idx)}",
                   "preconditioner": "a=1, m=2, alpha=(1,7)", "tol": TOL},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": f"{len(idx)} of {a.batch} instances per step (every {a.batch // len(idx)}th)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line)


# ---------------------------------------------------------------------------
# Algorithmic bytes of the persistent solve kernel
# ---------------------------------------------------------------------------
def alg_bytes(Ns, ns, iters, outers, m=M):
    """Bytes the method must move (blocks at their size, no padding), per
    instance:  each float32 inner iteration streams S (D, O), G (D^-1, E) and
    H (Hd, Hu, Hl) once plus 14 vector passes; each inner restart applies
    M^-1 once more (G, H) and each refinement step streams the float64 D, O
    plus 3 float64 vector passes."""
    tot = 0
    for N, n, it, o in zip(Ns, ns, iters, outers):
        n2 = n * n
        s_blocks = (2 * N - 1) * n2
        g_blocks = (2 * N - 1) * n2
        h_blocks = max(3 * N - 4, 0) * n2 * (m - 1)
        it_b = 4 * (s_blocks + g_blocks + h_blocks) + 14 * 4 * N * n
        prec_b = 4 * (g_blocks + h_blocks) + 4 * 4 * N * n
        a64_b = 8 * s_blocks + 3 * 8 * N * n
        tot += it * it_b + o * (prec_b + a64_b)
    return tot


def kernel_hash():
    h = hashlib.sha256()
    for f in (KERNEL_SRC, os.path.join(ROOT, "paper_2503_15269_gb300", "csrc", "bt_common.cuh")):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def stored_traffic(abytes):
    """DRAM bytes (read + write) of one solve launch, from an ncu capture of a
    smaller batch of the same workload: its measured DRAM bytes per
    algorithmic byte, times this launch's algorithmic bytes (traffic grows
    with the bytes the solves stream).  None once the kernel sources differ
    from the captured ones."""
    try:
        t = json.load(open(TRAFFIC_FILE))
    except Exception:
        return None
    if t.get("kernel_hash") != kernel_hash():
        return None
    ratio = t.get("dram_bytes_per_alg_byte")
    return None if ratio is None else int(ratio * abytes)


def measured_peak():
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        # raw samples go to a scratch file; the JSON line carries their summary
        self.path = os.path.join(tempfile.gettempdir(), f"bt_clocks_{os.getpid()}.csv")
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        try:
            self.f.close()
        except Exception:
            pass

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for j, nme in enumerate(names):
                if len(r) > 5 + j and "Active" in r[5 + j] and "Not" not in r[5 + j]:
                    reasons.add(nme)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def main():
    a = parse()
    if a.impl == "reference":
        reference_arm(a)
        return
    if a.workload != "ocp_batch":
        other_workload(a)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2503_15269_gb300 import binding as bb
    from paper_2503_15269_gb300 import build
    from paper_2503_15269_gb300 import workloads as wl
    build.build()
    bb.lib()

    insts = wl.config2(count=max(a.batch, 1)) if a.batch == 1024 else wl.config2(indices=list(range(a.batch)))
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    B = len(insts)
    del insts
    stream = torch.cuda.Stream(device=dev)
    hD = torch.from_numpy(D).pin_memory()
    hO = torch.from_numpy(O).pin_memory()
    hb = torch.from_numpy(b).pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    hst = torch.empty(2 * B, dtype=torch.int32).pin_memory()
    dD = hD.to(dev)
    dO = hO.to(dev)
    db = hb.to(dev)
    dx = torch.zeros_like(db)
    d_it = torch.zeros(2 * B, dtype=torch.int32, device=dev)

    p, keep = bb.make_params(m=M, alpha=ALPHA, precision=bb.BT_MIXED, stream=stream)
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dD, dO, p)
    assert st == bb.BT_OK, bb.status_string(st)

    def step():
        s1 = bb.bt_refactor(h, dD, dO)
        s2 = bb.bt_pcg_solve_batched_async(h, db, dx, TOL, 5000, d_it[:B], d_it[B:])
        assert s1 == bb.BT_OK and s2 == bb.BT_OK

    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for _ in range(a.warmup):
            step()
    torch.cuda.synchronize()
    # per-instance iteration counts (bitwise-deterministic, same in every step)
    st, iters, sts = bb.bt_pcg_solve_batched(h, db, dx, B, TOL, 5000)
    outers = [bb.bt_solve_info(h, k)[1] for k in range(B)]
    resid = [bb.bt_solve_info(h, k)[2] for k in range(B)]
    assert st == bb.BT_OK and (sts == 0).all(), (st, np.unique(sts))
    assert max(resid) <= TOL, max(resid)

    # ---- device-timed steps ----
    # The timed region replays one CUDA graph per step: the refactor kernels
    # and the persistent solve, captured once (bt_graph_capture_refactor_solve).
    # A second pass launches the same kernels directly with events between
    # them, for the per-kernel durations behind the roofline.
    assert bb.bt_graph_capture_refactor_solve(h, dD, dO, db, dx, TOL, 5000, d_it[:B], d_it[B:]) == bb.BT_OK
    with torch.cuda.stream(stream):
        for _ in range(2):
            assert bb.bt_graph_launch(h) == bb.BT_OK
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local) if not a.profile else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.__enter__()
    with torch.cuda.stream(stream):
        e0.record(stream)
        for k in range(a.steps):
            assert bb.bt_graph_launch(h) == bb.BT_OK
        e1.record(stream)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(a.steps):
            ev[k][0].record(stream)
            assert bb.bt_refactor(h, dD, dO) == bb.BT_OK
            ev[k][1].record(stream)
            assert bb.bt_pcg_solve_batched_async(h, db, dx, TOL, 5000, d_it[:B], d_it[B:]) == bb.BT_OK
            ev[k][2].record(stream)
    torch.cuda.synchronize()
    if clocks:
        clocks.__exit__()
    if dist:
        dist.barrier()
    assert (d_it[B:] == 0).all()
    x_gpu = dx.double().cpu().numpy().copy()
    ms = e0.elapsed_time(e1)
    ms_setup = sum(x[0].elapsed_time(x[1]) for x in ev) / a.steps
    ms_solve = sum(x[1].elapsed_time(x[2]) for x in ev) / a.steps
    ms = max_over_ranks(ms, dist, dev)
    value = job_value(world, B, a.steps, ms)

    if a.profile:
        if rank == 0:
            ab = int(alg_bytes([int(v) for v in Ns], [int(v) for v in ns], [int(v) for v in iters], outers))
            emit({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms / a.steps,
                  "ms_solve": ms_solve, "ms_setup": ms_setup, "alg_bytes_per_solve_launch": ab,
                  "kernel_hash": kernel_hash()})
        return

    # ---- end to end through host buffers ----
    # Every step uploads its inputs (D, O, b) from pinned host memory and
    # reads x and the statuses back, inside the timed region.  The uploads run
    # on a copy stream into the other of two device input sets, so the upload
    # of step k+1 overlaps the refactor + solve of step k (the handle's
    # compute stream waits on the upload's event; the copy stream waits until
    # the solve that last read a buffer set has finished).
    cstream = torch.cuda.Stream(device=dev)
    bufs = [(dD, dO, db, dx), (torch.empty_like(dD), torch.empty_like(dO), torch.empty_like(db),
                               torch.empty_like(dx))]
    hxs = [hx, torch.empty_like(hx).pin_memory()]
    hsts = [hst, torch.empty_like(hst).pin_memory()]
    d_its = [d_it, torch.zeros_like(d_it)]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    freed = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(k):
        j = k % 2
        with torch.cuda.stream(cstream):
            if k >= 2:
                cstream.wait_event(freed[j])
            D_, O_, b_, _ = bufs[j]
            D_.copy_(hD, non_blocking=True)
            O_.copy_(hO, non_blocking=True)
            b_.copy_(hb, non_blocking=True)
            copied[j].record(cstream)

    def compute(k):
        j = k % 2
        D_, O_, b_, x_ = bufs[j]
        with torch.cuda.stream(stream):
            stream.wait_event(copied[j])
            s1 = bb.bt_refactor(h, D_, O_)
            s2 = bb.bt_pcg_solve_batched_async(h, b_, x_, TOL, 5000, d_its[j][:B], d_its[j][B:])
            assert s1 == bb.BT_OK and s2 == bb.BT_OK
            freed[j].record(stream)
            hxs[j].copy_(x_, non_blocking=True)
            hsts[j].copy_(d_its[j], non_blocking=True)

    def e2e_steps(K):
        upload(0)
        for k in range(K):
            if k + 1 < K:
                upload(k + 1)
            compute(k)

    torch.cuda.synchronize()
    e2e_steps(2)  # warm: both buffer sets
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(cstream)
    e2e_steps(a.steps)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(f0.elapsed_time(f1), dist, dev)
    e2e_value = job_value(world, B, a.steps, ms_e2e)
    for j in range(min(2, a.steps)):
        assert (hsts[j][B:].numpy() == 0).all()
    h2d = hD.numel() * 8 + hO.numel() * 8 + hb.numel() * 8
    d2h = hx.numel() * 8 + hst.numel() * 4

    # ---- roofline of the persistent solve kernel ----
    abytes = int(alg_bytes([int(v) for v in Ns], [int(v) for v in ns], [int(v) for v in iters], outers))
    achieved = abytes / (ms_solve / 1e3) / 1e9
    peak, peak_kind = measured_peak()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": stored_traffic(abytes), "peak_source": peak_kind,
            "kernel": "bt_persistent_kernel<float, 0> (batched mixed solve)",
            "alg_bytes_per_launch": abytes, "ms_per_launch": ms_solve,
            "timing": "CUDA events around the solve launches of the direct-launch pass (same kernels as the "
                      "graph replays that give value)"}

    # ---- plain FP64 single-instance PCG, one instance at a time ----
    fp64 = None
    if rank == 0 and world == 1 and not a.no_fp64:
        fp64 = fp64_one_at_a_time(bb, torch, dev, stream, Ns, ns, d_off, o_off, v_off, dD, dO, db)

    cpu = None
    err = None
    if rank == 0 and world == 1 and not a.no_cpu:
        procs = min(cpu_cores(), 16)
        idx = sample_indices(B, min(a.cpu_sample, B))
        wall, out = run_oracle(idx, procs, want_x=True)
        err = err_vs_oracle(x_gpu, v_off, Ns, ns, out)
        cpu = {"value": len(out) / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"{len(idx)} of the {B} instances (every {max(1, B // len(idx))}th), "
                         f"numpy float64 oracle PCG incl. its setup, {procs} spawn processes",
               "wall_s": wall, "oracle_iters_mean": float(np.mean([o[2] for o in out])),
               "err_vs_oracle": err}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded LQR Schur complements)",
            "config": {"workload": f"ocp batch of {B}: N~U{{32..512}}, n in {{12,24,36}}, m=n/3, "
                                   "mixed precision, one persistent launch",
                       "preconditioner": "a=1, m=2, alpha=(1,7)", "tol": TOL,
                       "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}",
                       "graph": True},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            # per step: the float32 factor and the fused E/H kernel once per
            # block-size class present (n = 12, 24, 36, other), k_factor_retry
            # (refactor), and the persistent solve kernel
            "gpu_launches": (2 * len({n if n in (12, 24, 36) else 0 for n in ns}) + 2) * a.steps,
            "roofline": roof,
            "err_vs_oracle": err,
            "cpu_baseline": cpu,
            "clocks": clocks.summary() if clocks else None,
            "detail": {"ms_setup": ms_setup, "ms_solve": ms_solve, "iters_mean": float(np.mean(iters)),
                       "iters_max": int(np.max(iters)), "outer_mean": float(np.mean(outers)),
                       "max_true_rel_residual": float(max(resid)), "fp64_one_at_a_time": fp64,
                       "device_bytes": bb.bt_device_bytes(h)},
        }
        emit(line)
    bb.bt_destroy(h)
    if dist:
        dist.destroy_process_group()


def other_workload(a):
    """The other measured rows, one GPU, inputs resident in HBM, CUDA events on
    the launching stream, steps after warm-ups:
      many_rhs  bt_pcg_solve_multi on the LL^T system N = 2048, n = 48 with 64
                right-hand sides to 1e-8 (setup excluded; roofline of the
                many-RHS kernel from its algorithmic bytes);
      adjoint   bt_solve forward + backward (second solve + gradient blocks)
                on 256 LQR instances, N = 256, n = 24, mixed, tol 1e-8."""
    import numpy as np
    import torch
    from paper_2503_15269_gb300 import binding as bb
    from paper_2503_15269_gb300 import workloads as wl
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.workload == "many_rhs":
        inst = wl.config3()
        N, n, J = inst.N, inst.n, 64
        dD = torch.tensor(inst.D, device=dev)
        dO = torch.tensor(inst.O, device=dev)
        dB = torch.tensor(inst.b.reshape(N * n, J), device=dev)
        dX = torch.zeros_like(dB)

        def timed(engine):
            p, keep = bb.make_params(m=M, alpha=ALPHA, precision=bb.BT_MIXED, mrhs_engine=engine)
            st, h = bb.bt_setup(N, n, dD, dO, p)
            assert st == bb.BT_OK, bb.status_string(st)
            for _ in range(a.warmup):
                st, its, sts = bb.bt_pcg_solve_multi(h, dB, dX, J, TOL, a.maxit)
                assert st == bb.BT_OK and (sts == 0).all()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(a.steps):
                st, its, sts = bb.bt_pcg_solve_multi(h, dB, dX, J, TOL, a.maxit)
            e1.record()
            torch.cuda.synchronize()
            outers = [bb.bt_multi_info(h, j)[1] for j in range(J)]
            bb.bt_destroy(h)
            return e0.elapsed_time(e1) / a.steps, its, sts, outers

        if a.profile:  # one short call for a profiler capture: no checks, no baselines
            ms, its, sts, outers = timed(a.mrhs_engine)
            emit({"workload": "many_rhs", "profile": True, "ms": ms, "iters_max": int(np.max(its))})
            return
        clocks = Clocks(0)
        clocks.__enter__()
        ms_simt = timed(1)[0] if a.mrhs_engine == 0 else None
        ms, its, sts, outers = timed(a.mrhs_engine)
        clocks.__exit__()
        assert (sts == 0).all()
        # error against the float64 oracle: every column's true residual
        # (oracle SpMV) and four sampled columns against its direct solve
        from oracle import bt_oracle as orc
        Xh = dX.cpu().numpy().reshape(N, n, J)
        R = orc.spmv(inst.D, inst.O, Xh) - inst.b
        res_max = max(float(np.linalg.norm(R[:, :, j]) / np.linalg.norm(inst.b[:, :, j])) for j in range(J))
        cols = [0, 21, 42, 63]
        xr = orc.direct_solve(inst.D, inst.O, inst.b[:, :, cols])
        e_dir = max(float(np.linalg.norm(Xh[:, :, j] - xr[:, :, c]) / np.linalg.norm(xr[:, :, c]))
                    for c, j in enumerate(cols))
        err = {"max_rel_err_vs_direct": e_dir, "columns": cols, "max_true_rel_residual": res_max,
               "reference": "oracle direct solve (float64 block Cholesky); residuals by the oracle's SpMV"}
        # bytes: every shared sweep streams the blocks once for all 64 columns;
        # the sweeps of an outer step run until its slowest column converges
        n2 = n * n
        it_b = 4 * ((2 * N - 1) + (2 * N - 1) + (3 * N - 4) * (M - 1)) * n2 + 14 * 4 * N * n * J
        prec_b = 4 * ((2 * N - 1) + (3 * N - 4) * (M - 1)) * n2 + 4 * 4 * N * n * J
        a64_b = 8 * (2 * N - 1) * n2 + 3 * 8 * N * n * J
        it_max, o_max = int(np.max(its)), int(np.max(outers))
        abytes = it_max * it_b + o_max * (prec_b + a64_b)
        peak, kind = measured_peak()
        achieved = abytes / (ms / 1e3) / 1e9
        emit({"metric": "right-hand sides solved per second to rel. residual 1e-8 (64 per call)",
              "value": J / (ms / 1e3), "unit": "rhs/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
              "ms_per_step": ms, "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic (seeded LL^T)",
              "config": {"workload": "LL^T N=2048 n=48, 64 right-hand sides, mixed, a=1 m=2 alpha=(1,7)"},
              "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak, "traffic": None, "peak_source": kind,
                           "kernel": "bt_mrhs_kernel<true>" if a.mrhs_engine != 1 else "bt_mrhs_kernel<false>",
                           "alg_bytes_per_launch": abytes, "ms_per_launch": ms},
              "err_vs_oracle": err, "clocks": clocks.summary(),
              "detail": {"iters_max": it_max, "iters_mean": float(np.mean(its)), "outer_max": o_max,
                         "engine": {0: "tensor cores (3xTF32, tcgen05)", 1: "float32 SIMT",
                                    2: "tensor cores (3xTF32, tcgen05)"}[a.mrhs_engine],
                         "ms_float32_simt_engine": ms_simt}})
        return
    if a.workload == "family":
        family_protocol(a, bb, wl, torch, dev)
        return
    if a.workload == "lqr":
        lqr_pipeline(a, bb, wl, torch, dev)
        return
    if a.workload == "alpha":
        alpha_choices(a, bb, wl, torch, dev)
        return
    if a.workload == "matrix_free":
        matrix_free(a, bb, wl, torch, dev)
        return
    if a.workload == "precision":
        precision_split(a, bb, wl, torch, dev)
        return
    if a.workload == "small":
        # latency-bound single instances: microseconds per solve and per PCG
        # iteration (one persistent launch per solve, setup excluded)
        rows = []
        # group -1: the shared-memory engine, 1: the persistent kernel on one CTA, 0: automatic
        for name, inst, prec, tol, grp in (("LL^T N=16 n=6", wl.config0(), bb.BT_FP64, 1e-10, 0),
                                           ("LL^T N=16 n=6", wl.config0(), bb.BT_FP64, 1e-10, -8),
                                           ("LL^T N=16 n=6", wl.config0(), bb.BT_FP64, 1e-10, 1),
                                           ("LQR N=128 n=12", wl.config1(), bb.BT_FP64, 1e-8, 0),
                                           ("LQR N=128 n=12", wl.config1(), bb.BT_FP64, 1e-8, 32),
                                           ("LQR N=128 n=12", wl.config1(), bb.BT_MIXED, 1e-8, 0),
                                           ("LQR N=128 n=12", wl.config1(), bb.BT_MIXED, 1e-8, 32)):
            dD = torch.tensor(inst.D, device=dev)
            dO = torch.tensor(inst.O, device=dev)
            db = torch.tensor(inst.b.reshape(-1), device=dev)
            dx = torch.zeros_like(db)
            p, keep = bb.make_params(m=M, alpha=ALPHA, precision=prec, group_ctas=grp)
            st, h = bb.bt_setup(inst.N, inst.n, dD, dO, p)
            assert st == bb.BT_OK, bb.status_string(st)
            for _ in range(a.warmup):
                st, it = bb.bt_pcg_solve(h, db, dx, tol, 5000)
                assert st == bb.BT_OK
            torch.cuda.synchronize()
            e0.record()
            for _ in range(a.steps):
                bb.bt_pcg_solve_async(h, db, dx, tol, 5000)
            e1.record()
            torch.cuda.synchronize()
            us = 1e3 * e0.elapsed_time(e1) / a.steps
            bb.bt_destroy(h)
            # group_ctas 0 picks the shared-memory engine for instances whose blocks
            # fit one CTA (LL^T N = 16, n = 6) or a cluster (LQR N = 128, n = 12: 8
            # CTAs), the persistent kernel otherwise; -8 asks for a cluster of 8
            engine = {0: "automatic", -8: "shared-memory engine, cluster of 8",
                      1: "persistent kernel, 1 CTA", 32: "persistent kernel, 32 CTAs"}[grp]
            rows.append({"instance": name, "precision": "f64" if prec == bb.BT_FP64 else "f32+f64", "tol": tol,
                         "engine": engine, "us_per_solve": us, "iters": it, "us_per_iter": us / max(it, 1)})
        emit({"metric": "microseconds per single-instance solve (latency-bound rows)", "value": rows[0]["us_per_solve"],
              "unit": "us", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "higher_is_better": False,
              "data": "synthetic (seeded)", "config": {"workload": "single instances, one launch each (setup excluded)"},
              "rows": rows})
        return
    adjoint_workload(a, bb, wl, torch, dev)


def adjoint_workload(a, bb, wl, torch, dev):
    """Forward + adjoint on 256 LQR instances, N = 256, n = 24 (input 8),
    mixed, tol 1e-8.  value: through the public API (bt_solve, a
    torch.autograd.Function: setup, forward solve, backward solve, gradient
    blocks) per step.  roofline: a second pass through the C ABI on one
    handle (refactor, forward batched solve, adjoint solve with the same
    preconditioner, bt_adjoint_blocks), CUDA events around each launch; the
    solve kernel's algorithmic bytes (forward + adjoint solves, the per
    instance iteration and refinement counts) over its event time.  Error
    against the oracle on sampled instances: x and dL/db against its direct
    solve and adjoint."""
    import numpy as np
    from oracle import bt_oracle as orc
    from paper_2503_15269_gb300.autograd import bt_solve
    insts = wl.config4()
    Ns, ns, d_off, o_off, v_off, D_, O_, b_ = wl.pack_batch(insts)
    D = torch.tensor(D_, device=dev, requires_grad=True)
    O = torch.tensor(O_, device=dev, requires_grad=True)
    b = torch.tensor(b_, device=dev, requires_grad=True)
    w = torch.tensor(np.random.default_rng(5).standard_normal(b.numel()), device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step():
        D.grad = O.grad = b.grad = None
        x = bt_solve(D, O, b, Ns, ns, d_off, o_off, precision=bb.BT_MIXED, tol=TOL)
        (x * w).sum().backward()
        return x

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.__enter__()
    e0.record()
    for _ in range(a.steps):
        x = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    B = len(insts)
    xs, gb = x.detach().cpu().numpy(), b.grad.cpu().numpy()

    # ---- the same work through the C ABI on one handle, per-launch events ----
    stream = torch.cuda.Stream(device=dev)
    p, keep = bb.make_params(m=M, alpha=ALPHA, precision=bb.BT_MIXED, stream=stream)
    Dd, Od, bd = D.detach(), O.detach(), b.detach()
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, Dd, Od, p)
    assert st == bb.BT_OK, bb.status_string(st)
    xd, gd = torch.zeros_like(bd), torch.zeros_like(bd)
    gD, gO = torch.empty_like(Dd), torch.empty_like(Od)
    st, it_f, sts = bb.bt_pcg_solve_batched(h, bd, xd, B, TOL, 10000)
    assert st == bb.BT_OK and (sts == 0).all()
    out_f = [bb.bt_solve_info(h, k)[1] for k in range(B)]
    st, it_b, sts = bb.bt_pcg_solve_batched(h, w, gd, B, TOL, 10000)
    assert st == bb.BT_OK and (sts == 0).all()
    out_b = [bb.bt_solve_info(h, k)[1] for k in range(B)]
    d_it = torch.zeros(2 * B, dtype=torch.int32, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(a.steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(a.steps):
            ev[k][0].record(stream)
            assert bb.bt_refactor(h, Dd, Od) == bb.BT_OK
            ev[k][1].record(stream)
            assert bb.bt_pcg_solve_batched_async(h, bd, xd, TOL, 10000, d_it[:B], d_it[B:]) == bb.BT_OK
            ev[k][2].record(stream)
            assert bb.bt_pcg_solve_batched_async(h, w, gd, TOL, 10000, d_it[:B], d_it[B:]) == bb.BT_OK
            ev[k][3].record(stream)
            assert bb.bt_adjoint_blocks(h, xd, gd, gD, gO) == bb.BT_OK
            ev[k][4].record(stream)
    torch.cuda.synchronize()
    clocks.__exit__()
    bb.bt_destroy(h)
    t = [sum(e[i].elapsed_time(e[i + 1]) for e in ev) / a.steps for i in range(4)]
    ms_refactor, ms_fwd, ms_bwd, ms_adj = t
    abytes = alg_bytes(Ns, ns, it_f, out_f) + alg_bytes(Ns, ns, it_b, out_b)
    achieved = abytes / ((ms_fwd + ms_bwd) / 1e3) / 1e9
    peak, kind = measured_peak()
    adj_bytes = sum(8 * ((2 * int(N) - 1) * int(n) ** 2 + 2 * int(N) * int(n)) for N, n in zip(Ns, ns))
    # error against the oracle on sampled instances
    e_x, e_g = 0.0, 0.0
    wn = w.cpu().numpy()
    samples = (0, 77, 255)
    for k in samples:
        inst = insts[k]
        sl = slice(v_off[k], v_off[k] + inst.N * inst.n)
        xr = orc.direct_solve(inst.D, inst.O, inst.b)
        g, _, _ = orc.adjoint(inst.D, inst.O, xr, wn[sl].reshape(inst.N, inst.n))
        e_x = max(e_x, float(np.linalg.norm(xs[sl].reshape(inst.N, inst.n) - xr) / np.linalg.norm(xr)))
        e_g = max(e_g, float(np.linalg.norm(gb[sl].reshape(inst.N, inst.n) - g) / np.linalg.norm(g)))
    emit({"metric": "forward + adjoint solves per second (x = S^-1 b and dL/d(D, O, b)), rel. residual 1e-8",
          "value": B / (ms / 1e3), "unit": "instances/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
          "ms_per_step": ms, "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic (seeded LQR)",
          "config": {"workload": "256 LQR instances N=256 n=24 (input size 8), setup + forward + adjoint per step"},
          "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                       "traffic": None, "peak_source": kind,
                       "kernel": "bt_persistent_kernel<float, 0> (forward and adjoint batched solves)",
                       "alg_bytes_per_launch": abytes / 2, "ms_per_launch": (ms_fwd + ms_bwd) / 2},
          "err_vs_oracle": {"max_rel_err_x_vs_direct": e_x, "max_rel_err_grad_b_vs_oracle_adjoint": e_g,
                            "instances": list(samples),
                            "reference": "oracle direct solve and oracle adjoint (float64)"},
          "clocks": clocks.summary(),
          "detail": {"ms_refactor": ms_refactor, "ms_forward_solve": ms_fwd, "ms_adjoint_solve": ms_bwd,
                     "ms_adjoint_blocks": ms_adj, "adjoint_blocks_gbs": adj_bytes / (ms_adj / 1e3) / 1e9,
                     "iters_mean_forward": float(np.mean(it_f)), "iters_mean_adjoint": float(np.mean(it_b))}})


def family_protocol(a, bb, wl, torch, dev):
    """The experiment protocol of the numerical-results section on the GPU:
    five settings of the family (block Jacobi a = 0, equal a = 1/3, stairs
    only a = 1/2, optimal a = 1, PolyCoeff a = 1 with alpha_{m-1} = 7) at
    m = 1..4; per (setting, m) 100 LQR matrices N = 30, n = 20, each with 100
    unit-norm right-hand sides, solved by float64 PCG to ||S x - b|| < 1e-6 in
    one batched launch of 10^4 instances (setup untimed).  Per row: mean
    iterations, block gemvs n_itr * g_a(m) and solves/s; the roofline is the
    float64 arithmetic of the block products (0.25 flop per streamed byte
    exceeds the float64 rate / HBM bandwidth ratio of GB300)."""
    import numpy as np
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.protocol_batch()
    B, N, n = len(Ns), int(Ns[0]), int(ns[0])
    dD, dO, db = (torch.tensor(v, device=dev) for v in (D, O, b))
    dx = torch.zeros_like(db)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows, tot_ms, tot_solves, tot_flop, tot_bytes = [], 0.0, 0, 0.0, 0.0
    n2 = n * n
    for name, aa, pc in wl.PROTOCOL_SETTINGS:
        for m in (1, 2, 3, 4):
            alpha = wl.protocol_alpha(m, pc)
            p, keep = bb.make_params(m=m, alpha=alpha, a=aa)
            st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dD, dO, p)
            assert st == bb.BT_OK, bb.status_string(st)
            for _ in range(a.warmup):
                st, its, sts = bb.bt_pcg_solve_batched(h, db, dx, B, 1e-6, 5000)
                assert st == bb.BT_OK and (sts == 0).all(), (name, m, st)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(a.steps):
                bb.bt_pcg_solve_batched_async(h, db, dx, 1e-6, 5000)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / a.steps
            bb.bt_destroy(h)
            # blocks each iteration streams: S, G, and m-1 H applications
            # (3 arrays for H_opt, 5 for H_ab; a = 0 streams the zero a H_opt too)
            h_blocks = (3 * N - 4) if aa == 1.0 else (5 * N - 6)
            blocks = (2 * N - 1) + (2 * N - 1) + h_blocks * (m - 1)
            it_mean = float(np.mean(its))
            g = (2 * m + 2) if aa == 0.0 else ((3 * m + 3) if aa == 1.0 else (5 * m + 1))
            flop = 2.0 * n2 * blocks * float(np.sum(its))
            byts = 8.0 * n2 * blocks * float(np.sum(its))
            rows.append({"setting": name, "a": aa, "m": m, "alpha": alpha, "iters_mean": it_mean,
                         "gemv_mean": it_mean * g, "ms": ms, "solves_per_s": B / (ms / 1e3),
                         "fp64_tflops": flop / (ms / 1e3) / 1e12, "hbm_gbs": byts / (ms / 1e3) / 1e9})
            tot_ms += ms
            tot_solves += B
            tot_flop += flop
            tot_bytes += byts
    peak_tf = 1.25  # GB300 nominal float64 (non-tensor) rate, TFLOP/s
    hbm, kind = measured_peak()
    achieved = tot_flop / (tot_ms / 1e3) / 1e12
    emit({"metric": "protocol solves per second (float64 PCG to ||Sx-b|| < 1e-6, 5 settings x m=1..4)",
          "value": tot_solves / (tot_ms / 1e3), "unit": "solves/s", "n_gpus": 1, "steps": a.steps,
          "warmup": a.warmup, "ms_per_step": tot_ms, "higher_is_better": True, "dtype": "f64",
          "data": "synthetic (seeded LQR, unit-norm b)",
          "config": {"workload": f"{B} solves per (setting, m): 100 LQR matrices N={N} n={n} x 100 b"},
          "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                       "frac": achieved / peak_tf, "traffic": None, "peak_source": "nominal float64 rate",
                       "kernel": "bt_persistent_kernel (float64)",
                       "hbm_gbs": tot_bytes / (tot_ms / 1e3) / 1e9, "hbm_peak": hbm, "hbm_peak_source": kind},
          "rows": rows})


def matrix_free(a, bb, wl, torch, dev):
    """The bench batch (1024 LQR instances, mixed, m = 2, alpha = (1, 7),
    tol 1e-8), refactor + solve per step as in the headline, with H_opt
    stored (3 block arrays per application) and matrix-free (H_J twice from
    D^-1 and O: 4 block reads per application, no H storage); per row the
    step time, the handle's device bytes and the solve kernel's algorithmic
    HBM bandwidth (H counted at 4 arrays for the matrix-free row)."""
    import numpy as np
    insts = wl.config2()
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    dD, dO, db = (torch.tensor(v, device=dev) for v in (D, O, b))
    dx = torch.zeros_like(db)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    peak, kind = measured_peak()
    rows = []
    for mf in (False, True):
        p, keep = bb.make_params(m=M, alpha=ALPHA, precision=bb.BT_MIXED, h_matrix_free=mf)
        st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dD, dO, p)
        assert st == bb.BT_OK, bb.status_string(st)
        for _ in range(a.warmup):
            assert bb.bt_refactor(h, dD, dO) == bb.BT_OK
            st, its, sts = bb.bt_pcg_solve_batched(h, db, dx, len(insts), TOL, 5000)
            assert st == bb.BT_OK and (sts == 0).all()
        outers = [bb.bt_solve_info(h, k)[1] for k in range(len(insts))]
        t_set = t_sol = 0.0
        for _ in range(a.steps):
            torch.cuda.synchronize()
            ev[0].record()
            bb.bt_refactor(h, dD, dO)
            ev[1].record()
            bb.bt_pcg_solve_batched_async(h, db, dx, TOL, 5000)
            ev[2].record()
            torch.cuda.synchronize()
            t_set += ev[0].elapsed_time(ev[1])
            t_sol += ev[1].elapsed_time(ev[2])
        nbytes = bb.bt_device_bytes(h)
        bb.bt_destroy(h)
        ms_set, ms_sol = t_set / a.steps, t_sol / a.steps
        ab = alg_bytes(Ns, ns, its, outers)
        if mf:  # each H application reads D^-1 and O twice instead of Hd, Hu, Hl once
            n2 = np.asarray(ns, dtype=np.float64) ** 2
            N_ = np.asarray(Ns, dtype=np.float64)
            extra = 4.0 * ((4 * N_ - 2) - np.maximum(3 * N_ - 4, 0)) * n2 * (M - 1)
            ab += float(np.sum(np.asarray(its, dtype=np.float64) * extra + np.asarray(outers) * extra))
        gbs = ab / (ms_sol / 1e3) / 1e9
        rows.append({"h": "matrix-free" if mf else "stored", "ms_refactor": ms_set, "ms_solve": ms_sol,
                     "solves_per_s": len(insts) / ((ms_set + ms_sol) / 1e3), "device_bytes": nbytes,
                     "iters_mean": float(np.mean(its)), "hbm_gbs": gbs, "frac": gbs / peak})
    r = rows[1]
    emit({"metric": "solves/s at rel. residual 1e-8 with the matrix-free H_opt (refactor + solve per step)",
          "value": r["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
          "ms_per_step": r["ms_refactor"] + r["ms_solve"], "higher_is_better": True, "dtype": "f32+f64",
          "data": "synthetic (seeded LQR Schur complements)",
          "config": {"workload": "ocp batch of 1024, a=1 m=2 alpha=(1,7), H_opt matrix-free"},
          "roofline": {"bound": "hbm", "achieved": r["hbm_gbs"], "peak": peak, "unit": "GB/s", "frac": r["frac"],
                       "traffic": None, "peak_source": kind, "kernel": "bt_persistent_kernel<float, 2>"},
          "rows": rows})


def precision_split(a, bb, wl, torch, dev):
    """The headline step (refactor + batched mixed solve of the 1024 LQR
    instances to 1e-8) under the two precision splits of the mixed path:
    default (float32 factor of each D_i, float64 refactor of blocks with
    cond(D_i) > 1e3, float32 divisions of the inner step scalars) and strict
    (every D_i factored in float64, step scalars divided in float64).  Per row
    the refactor and solve times, iterations and the error against the
    oracle's direct solve on a sample of 48 instances."""
    import numpy as np
    from oracle import bt_oracle as orc
    insts = wl.config2()
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    dD, dO, db = (torch.tensor(v, device=dev) for v in (D, O, b))
    dx = torch.zeros_like(db)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    sample = sample_indices(len(insts), 48)
    xref = {k: orc.direct_solve(insts[k].D, insts[k].O, insts[k].b) for k in sample}
    peak, kind = measured_peak()
    rows = []
    for strict in (False, True):
        p, keep = bb.make_params(m=M, alpha=ALPHA, precision=bb.BT_MIXED, mixed_strict_fp64=strict)
        st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dD, dO, p)
        assert st == bb.BT_OK, bb.status_string(st)
        for _ in range(a.warmup):
            assert bb.bt_refactor(h, dD, dO) == bb.BT_OK
            st, its, sts = bb.bt_pcg_solve_batched(h, db, dx, len(insts), TOL, 5000)
            assert st == bb.BT_OK and (sts == 0).all()
        outers = [bb.bt_solve_info(h, k)[1] for k in range(len(insts))]
        resid = max(bb.bt_solve_info(h, k)[2] for k in range(len(insts)))
        t_set = t_sol = 0.0
        for _ in range(a.steps):
            torch.cuda.synchronize()
            ev[0].record()
            bb.bt_refactor(h, dD, dO)
            ev[1].record()
            bb.bt_pcg_solve_batched_async(h, db, dx, TOL, 5000)
            ev[2].record()
            torch.cuda.synchronize()
            t_set += ev[0].elapsed_time(ev[1])
            t_sol += ev[1].elapsed_time(ev[2])
        bb.bt_destroy(h)
        xs = dx.cpu().numpy()
        err = max(float(np.linalg.norm(xs[v_off[k]:v_off[k] + Ns[k] * ns[k]].reshape(Ns[k], ns[k]) - xref[k])
                        / np.linalg.norm(xref[k])) for k in sample)
        ms_set, ms_sol = t_set / a.steps, t_sol / a.steps
        gbs = alg_bytes(Ns, ns, its, outers) / (ms_sol / 1e3) / 1e9
        rows.append({"split": "strict float64 factor and step scalars" if strict else "default",
                     "ms_refactor": ms_set, "ms_solve": ms_sol,
                     "solves_per_s": len(insts) / ((ms_set + ms_sol) / 1e3), "iters_mean": float(np.mean(its)),
                     "outer_mean": float(np.mean(outers)), "max_true_rel_residual": resid,
                     "max_rel_err_vs_direct_sample48": err, "solve_hbm_frac": gbs / peak})
    r = rows[1]
    emit({"metric": "solves/s at rel. residual 1e-8 under the strict float64 split (refactor + solve per step)",
          "value": r["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
          "ms_per_step": r["ms_refactor"] + r["ms_solve"], "higher_is_better": True, "dtype": "f32+f64",
          "data": "synthetic (seeded LQR Schur complements)",
          "config": {"workload": "ocp batch of 1024, a=1 m=2 alpha=(1,7), default vs strict precision split"},
          "err_vs_oracle": {"default": rows[0]["max_rel_err_vs_direct_sample48"],
                            "strict": rows[1]["max_rel_err_vs_direct_sample48"],
                            "reference": "oracle direct solve, 48 sampled instances"},
          "rows": rows})


def alpha_choices(a, bb, wl, torch, dev):
    """The bench batch (1024 LQR instances, mixed, tol 1e-8, one persistent
    launch per step, refactor untimed) with the polynomial coefficients of the
    paper's PolyCoeff (m = 2, alpha = (1, 7)) and the Chebyshev choice
    (bt_alpha_chebyshev) for rho(H_opt) <= 0.985 at m = 2..5; per row the
    solve time, solves/s, mean iterations and the solve kernel's algorithmic
    HBM bandwidth."""
    import numpy as np
    insts = wl.config2()
    Ns, ns, d_off, o_off, v_off, D, O, b = wl.pack_batch(insts)
    dD, dO, db = (torch.tensor(v, device=dev) for v in (D, O, b))
    dx = torch.zeros_like(db)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    peak, kind = measured_peak()
    rows = []
    choices = [("PolyCoeff", 2, [1.0, 7.0])] + [(f"Chebyshev rho<=0.985", m, bb.bt_alpha_chebyshev(m, 0.985)[1])
                                                for m in (2, 3, 4, 5)]
    for name, m, alpha in choices:
        p, keep = bb.make_params(m=m, alpha=alpha, precision=bb.BT_MIXED)
        st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dD, dO, p)
        assert st == bb.BT_OK, bb.status_string(st)
        for _ in range(a.warmup):
            st, its, sts = bb.bt_pcg_solve_batched(h, db, dx, len(insts), TOL, 5000)
            assert st == bb.BT_OK and (sts == 0).all()
        outers = [bb.bt_solve_info(h, k)[1] for k in range(len(insts))]
        torch.cuda.synchronize()
        e0.record()
        for _ in range(a.steps):
            bb.bt_pcg_solve_batched_async(h, db, dx, TOL, 5000)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.steps
        bb.bt_destroy(h)
        ab = alg_bytes(Ns, ns, its, outers, m=m)
        gbs = ab / (ms / 1e3) / 1e9
        rows.append({"alpha": name, "m": m, "coefficients": [round(v, 4) for v in alpha], "ms_solve": ms,
                     "solves_per_s": len(insts) / (ms / 1e3), "iters_mean": float(np.mean(its)),
                     "hbm_gbs": gbs, "frac": gbs / peak})
    best = max(rows, key=lambda r: r["solves_per_s"])
    emit({"metric": "batched mixed solves/s at rel. residual 1e-8 by choice of polynomial coefficients",
          "value": best["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
          "ms_per_step": best["ms_solve"], "higher_is_better": True, "dtype": "f32+f64",
          "data": "synthetic (seeded LQR Schur complements)",
          "config": {"workload": "ocp batch of 1024 (solve only, refactor untimed)", "best": best["alpha"],
                     "best_m": best["m"]},
          "roofline": {"bound": "hbm", "achieved": best["hbm_gbs"], "peak": peak, "unit": "GB/s",
                       "frac": best["frac"], "traffic": None, "peak_source": kind,
                       "kernel": "bt_persistent_kernel<float, false>"},
          "rows": rows})


def lqr_pipeline(a, bb, wl, torch, dev):
    """LQR problems end to end on the device, for 1024 LQR problems with the
    shapes of the bench batch (N ~ U{32..512}, n in {12, 24, 36}, m = n/3;
    dense SPD Q, R), each stage timed with CUDA events, two ways:
      fused:    bt_lqr_refactor (the Schur complement formed straight into the
                mixed handle, D_k factored from there, then E and H), batched
                PCG to 1e-8 (a = 1, m = 2, alpha = (1, 7)), recovery from the
                factors of Q_k and R_k the formation kept
                (bt_lqr_recover_factored);
      two-step: bt_lqr_schur (D, O in the caller's layout), bt_refactor, the
                same solve and recovery.
    value is the fused pipeline.  The formation runs in double-float pairs on
    the float32 pipe; its roofline counts pair FMAs per block row --
    2n^3 + m^3/3 + (n m^2 + n^2 m)/2 for S, n^3/2 more for the fused factor
    of D_k -- against the float32 issue rate divided by the 12 float32
    instructions of one pair FMA."""
    import numpy as np
    shapes = wl.config2_shapes(1024)[:max(1, min(a.batch, 1024))]  # --batch: the first problems only
    probs = [wl.lqr_data(wl._rng(6, k), N, n, max(1, n // 3)) for k, (N, n) in enumerate(shapes)]
    cat = lambda f: np.concatenate([getattr(p, f).reshape(-1) for p in probs])
    dA, dB, dQ, dR, dq, dr, dc = (torch.tensor(cat(f), device=dev) for f in ("A", "Bm", "Q", "R", "q", "r", "c"))
    Ns = np.array([p.N for p in probs], np.int32)
    ns = np.array([p.n for p in probs], np.int32)
    ms = np.array([p.m for p in probs], np.int32)
    dD = torch.zeros(dQ.numel(), dtype=torch.float64, device=dev)
    dO = torch.zeros(dA.numel(), dtype=torch.float64, device=dev)
    dg = torch.zeros(dq.numel(), dtype=torch.float64, device=dev)
    dl, dx = torch.zeros_like(dg), torch.zeros_like(dg)
    du = torch.zeros(dr.numel(), dtype=torch.float64, device=dev)
    d_off = np.concatenate([[0], np.cumsum(Ns.astype(np.int64) * ns * ns)[:-1]]).astype(np.int64)
    o_off = np.concatenate([[0], np.cumsum((Ns.astype(np.int64) - 1) * ns * ns)[:-1]]).astype(np.int64)
    st, _, _ = bb.bt_lqr_schur(Ns, ns, ms, dA, dB, dQ, dR, dq, dr, dc, dD, dO, dg)
    assert st == bb.BT_OK, bb.status_string(st)
    p, keep = bb.make_params(m=M, alpha=ALPHA, precision=bb.BT_MIXED)
    st, h = bb.bt_setup_batched(Ns, ns, d_off, o_off, dD, dO, p)
    assert st == bb.BT_OK, bb.status_string(st)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    t2 = {"schur": 0.0, "refactor": 0.0, "solve": 0.0, "recover": 0.0}
    tf = {"lqr_refactor": 0.0, "solve": 0.0, "recover": 0.0}

    def step_two(timed):
        ev[0].record()
        st, _, _ = bb.bt_lqr_schur(Ns, ns, ms, dA, dB, dQ, dR, dq, dr, dc, dD, dO, dg)
        assert st == bb.BT_OK
        ev[1].record()
        assert bb.bt_refactor(h, dD, dO) == bb.BT_OK
        ev[2].record()
        assert bb.bt_pcg_solve_batched_async(h, dg, dl, TOL, 5000) == bb.BT_OK
        ev[3].record()
        assert bb.bt_lqr_recover(Ns, ns, ms, dA, dB, dQ, dR, dq, dr, dl, dx, du) == bb.BT_OK
        ev[4].record()
        torch.cuda.synchronize()
        if timed:
            for i, k in enumerate(t2):
                t2[k] += ev[i].elapsed_time(ev[i + 1])

    def step_fused(timed):
        ev[0].record()
        st, _, _ = bb.bt_lqr_refactor(h, ms, dA, dB, dQ, dR, dq, dr, dc, dg)
        assert st == bb.BT_OK
        ev[1].record()
        assert bb.bt_pcg_solve_batched_async(h, dg, dl, TOL, 5000) == bb.BT_OK
        ev[2].record()
        assert bb.bt_lqr_recover_factored(h, ms, dA, dB, dq, dr, dl, dx, du) == bb.BT_OK
        ev[3].record()
        torch.cuda.synchronize()
        if timed:
            for i, k in enumerate(tf):
                tf[k] += ev[i].elapsed_time(ev[i + 1])

    for _ in range(a.warmup):
        step_two(False)
    for _ in range(a.steps):
        step_two(True)
    st, its2, sts = bb.bt_pcg_solve_batched(h, dg, dl, len(probs), TOL, 5000)
    assert st == bb.BT_OK and (sts == 0).all()
    for _ in range(a.warmup):
        step_fused(False)
    for _ in range(a.steps):
        step_fused(True)
    st, its, sts = bb.bt_pcg_solve_batched(h, dg, dl, len(probs), TOL, 5000)
    assert st == bb.BT_OK and (sts == 0).all()
    # formation alone (bt_lqr_schur) for its roofline
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        bb.bt_lqr_schur(Ns, ns, ms, dA, dB, dQ, dR, dq, dr, dc, dD, dO, dg)
    e1.record()
    torch.cuda.synchronize()
    ms_schur = e0.elapsed_time(e1) / a.steps
    bb.bt_destroy(h)
    ms_two = {k: v / a.steps for k, v in t2.items()}
    ms_fused = {k: v / a.steps for k, v in tf.items()}
    tot = sum(ms_fused.values())
    ddfma = sum(int(N) * (2 * n ** 3 + m ** 3 / 3 + (n * m * m + n * n * m) / 2) for N, n, m in zip(Ns, ns, ms))
    achieved = 2 * ddfma / (ms_schur / 1e3) / 1e12
    props = torch.cuda.get_device_properties(dev)
    # float32 lanes per SM (4 x 32) x SMs x 2.07 GHz / 12 instructions per pair FMA x 2 flops
    peak_tf = props.multi_processor_count * 128 * 2.07e9 / 12 * 2 / 1e12
    emit({"metric": "LQR problems per second end to end on the device (formation fused with the refactor, "
                    "PCG to 1e-8, recovery)",
          "value": len(probs) / (tot / 1e3), "unit": "problems/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
          "ms_per_step": tot, "higher_is_better": True, "dtype": "f32-pair formation and recovery + f32/f64 solve",
          "data": "synthetic (seeded LQR, dense SPD Q and R)",
          "config": {"workload": f"{len(probs)} LQR problems, N~U{{32..512}}, n in {{12,24,36}}, m=n/3"},
          "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s (float64-equivalent)",
                       "frac": achieved / peak_tf, "traffic": None,
                       "peak_source": "float32 issue rate / 12 instructions per pair FMA (SMs x 128 lanes x 2.07 GHz)",
                       "kernel": "k_lqr_schur (bt_lqr_schur alone)", "ms_per_launch": ms_schur,
                       "flop_per_launch": 2 * ddfma},
          "detail": {"ms_fused": ms_fused, "ms_two_step": ms_two,
                     "formation_plus_refactor_ms": ms_fused["lqr_refactor"],
                     "two_step_formation_plus_refactor_ms": ms_two["schur"] + ms_two["refactor"],
                     "two_step_problems_per_s": len(probs) / (sum(ms_two.values()) / 1e3),
                     "iters_mean": float(np.mean(its)), "iters_mean_two_step": float(np.mean(its2))}})


def fp64_one_at_a_time(bb, torch, dev, stream, Ns, ns, d_off, o_off, v_off, dD, dO, db):
    """The same instances solved by the plain float64 PCG, one persistent
    launch per instance (setup refactor + solve), back to back on one stream."""
    B = len(Ns)
    hs = []
    p, keep = bb.make_params(m=M, alpha=ALPHA, precision=bb.BT_FP64, stream=stream)
    views = []
    for k in range(B):
        N, n = int(Ns[k]), int(ns[k])
        Dk = dD[d_off[k]:d_off[k] + N * n * n]
        Ok = dO[o_off[k]:o_off[k] + max(N - 1, 1) * n * n] if N > 1 else dO[:n * n]
        bk = db[v_off[k]:v_off[k] + N * n]
        xk = torch.zeros_like(bk)
        st, h = bb.bt_setup(N, n, Dk, Ok, p)
        assert st == bb.BT_OK
        hs.append(h)
        views.append((Dk, Ok, bk, xk))
    dits = torch.zeros(2 * B, dtype=torch.int32, device=dev)

    def run():
        for k in range(B):
            Dk, Ok, bk, xk = views[k]
            assert bb.bt_refactor(hs[k], Dk, Ok) == bb.BT_OK
            assert bb.bt_pcg_solve_async(hs[k], bk, xk, TOL, 5000, dits[k:k + 1], dits[B + k:B + k + 1]) == bb.BT_OK

    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        run()
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        g0.record(stream)
        run()
        g1.record(stream)
    torch.cuda.synchronize()
    ms = g0.elapsed_time(g1)
    its = dits[:B].cpu().numpy()
    sts = dits[B:].cpu().numpy()
    for h in hs:
        bb.bt_destroy(h)
    return {"value": B / (ms / 1e3), "unit": UNIT, "ms": ms, "iters_mean": float(its.mean()),
            "all_ok": bool((sts == 0).all())}


if __name__ == "__main__":
    main()
