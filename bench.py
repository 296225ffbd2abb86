#!/usr/bin/env python3
"""Headline benchmark: exact triangle counting on R-MAT scale 22.

One step = one pass of the whole method over the graph: build the oriented
CSR and its partition (tc_build_oriented_csr) and count the total and every
per-vertex count (tc_count), inputs resident in HBM.  The metric is input
undirected edges per second.

Workload (default): R-MAT scale 22, edge factor 16, (a, b, c, d) =
(0.57, 0.19, 0.19, 0.05), seeded relabelling, symmetrised, de-duplicated,
self-loops dropped (about 4.19M vertices, 64.2M undirected edges), int64
row_ptr + int32 col.  The input CSR (547 MB) and the oriented CSR exceed the
129 MB L2, so no explicit L2 flush is done between steps.

Other workloads (``--workload``): grid4096, er1024, ba_batch4096 (one batched
pass vs one launch per graph), serve (Poisson request stream through
tc_submit/tc_poll, p50/p99 latency).

``--impl reference`` times the CPU oracle (the paper's sequential forward
algorithm, written here as plain C) on the host cores, on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024


# ----------------------------------------------------------------------------- helpers
def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_graph(name, seed, rmat_scale=22):
    from paper_1804_06926_gb300 import gen
    if name == "rmat22":
        return gen.rmat(rmat_scale, 16, seed=seed), f"R-MAT s{rmat_scale} ef16 (0.57,0.19,0.19,0.05)"
    if name == "grid4096":
        return gen.grid(4096, 4096, seed=seed), "grid 4096x4096 + diag p=0.3 + 1% long-range"
    if name == "er1024":
        return gen.er(1024, 8192, seed=seed), "Erdos-Renyi G(1024, 8192)"
    raise KeyError(name)


def oriented_out_degrees(g):
    """d+(x) from the rank order (d, id); bookkeeping for the byte model."""
    deg = np.diff(g.row_ptr).astype(np.int64)
    u = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    v = g.col.astype(np.int64)
    keep = (deg[u] < deg[v]) | ((deg[u] == deg[v]) & (u < v))
    return np.bincount(u[keep], minlength=g.n).astype(np.int64), deg


def class_bytes(g, dplus, small_max=8, warp_max=128):
    """Split the per-edge list bytes 4*(d+(u)+d+(v)) over the kernels that own
    each oriented edge (the partition of tc_build_oriented_csr): thread-per-edge
    merge, warp tables, CTA tables, and edges that cannot close a triangle."""
    deg = np.diff(g.row_ptr).astype(np.int64)
    u = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    v = g.col.astype(np.int64)
    keep = (deg[u] < deg[v]) | ((deg[u] == deg[v]) & (u < v))
    u, v = u[keep], v[keep]
    a, b = dplus[u], dplus[v]
    skip = (a <= 1) | (b == 0)
    small = ~skip & (np.maximum(a, b) <= small_max)
    piv = ~skip & ~small
    p = np.where(a >= b, u, v)
    cta = piv & (dplus[p] > warp_max)
    warp = piv & ~cta
    w = 4 * (a + b)
    mn = 4 * np.minimum(a, b)
    return {"small": int(w[small].sum()), "warp": int(w[warp].sum()), "cta": int(w[cta].sum()),
            "skip": int(w[skip].sum()), "cta_edges": int(cta.sum()),
            "cta_shorter_list": int(mn[cta].sum()), "warp_shorter_list": int(mn[warp].sum())}


def algorithmic_bytes(g, per_vertex=True):
    """Bytes the per-edge intersection must read by definition (both sorted
    lists of every oriented edge) plus compulsory structure and output traffic:
    4*sum_{(u,v) in E+}(d+(u)+d+(v)) + 4|E+| + 8(n+1) + 8n[per-vertex] + 8.
    sum_{E+}(d+(u)+d+(v)) = sum_x d+(x) * d(x) (x is the source of d+(x) edges
    and the target of d(x)-d+(x) edges, each contributing d+(x))."""
    dplus, deg = oriented_out_degrees(g)
    s = int((dplus * deg).sum())
    m = g.m
    b = 4 * s + 4 * m + 8 * (g.n + 1) + (8 * g.n if per_vertex else 0) + 8
    return b, s, dplus, deg


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.rows = []
        self.proc = None
        self.uuid = device_uuid

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        time.sleep(0.25)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for nm, val in zip(names, r[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def device_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


COUNT_SOURCES = ("paper_1804_06926_gb300/csrc/tc_count.cu", "paper_1804_06926_gb300/csrc/tc_internal.cuh")

# Every traced phase of a build + count step belongs to one of the two parts:
# the build (a-1..a-4: degree, rank sort, orientation, row partition, work
# partition) and the count (a-5, a-6: output init, the intersection kernels).
# "fused" is the one-call kernel, which does both and is timed on its own.
BUILD_PHASES = ("degree", "validate", "rank", "orient_count", "orient_scan", "orient_scatter", "row_sort",
                "pivot_count", "pivot_scan", "pivot_scatter", "items", "edge_sort")
COUNT_PHASES = ("count_init", "count_small", "count_warp", "count_cta", "count_merge")


def code_digest(paths=COUNT_SOURCES):
    """First 16 hex digits of sha256 over the code of the count kernels' sources
    with // comments, trailing blanks and empty lines removed (a comment edit
    leaves it unchanged, any code edit changes it)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for p in paths:
        for line in open(os.path.join(ROOT, p), encoding="utf-8"):
            code = re.sub(r"//.*", "", line).rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag):
    """DRAM bytes per launch of the timed kernel from the committed ncu summary,
    if that summary was taken on the current code of the count kernels."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.ncu.txt")
    try:
        sha = code_digest()
        kv = {}
        for line in open(path):
            if ":" in line:
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_sha256_16") != sha:
            return None
        return float(kv["dram_bytes_per_launch_fullsize"])
    except Exception:
        return None


# ----------------------------------------------------------------------------- CPU oracle
CPU_SAMPLE_WORK = 4e9  # merge steps in the oracle's row sample (about 10 s on one core)


def oracle_sample(g, target_work=CPU_SAMPLE_WORK):
    """Orient the full graph with the oracle and choose its row sample: every
    `stride`-th source row, stride set so that the sample holds about
    target_work merge steps.  Returns (rpp, colp, t_orient, w_row, stride)."""
    import oracle
    t0 = time.perf_counter()
    rpp, colp = oracle.orient(g.n, g.row_ptr, g.col)
    t_orient = time.perf_counter() - t0
    dplus = np.diff(rpp)
    # merge work of row u: sum_{v in N+(u)} (d+(u) + d+(v))
    src = np.repeat(np.arange(g.n, dtype=np.int64), dplus)
    w_edge = dplus[src] + dplus[colp.astype(np.int64)]
    w_row = np.bincount(src, weights=w_edge, minlength=g.n)
    W = float(w_row.sum())
    stride = max(1, int(W / target_work)) if W > 0 else 1
    return rpp, colp, t_orient, w_row, stride


def oracle_rate(g, target_work=CPU_SAMPLE_WORK, label="", all_cores=None):
    """Time the CPU oracle on a bounded sample: orientation of the full graph,
    then the forward count over every k-th source row; extrapolate to the whole
    graph by merge work.  Returns (edges/s, description, seconds)."""
    import oracle
    rpp, colp, t_orient, w_row, stride = oracle_sample(g, target_work)
    W = float(w_row.sum())
    w_sample = float(w_row[::stride].sum())
    t1 = time.perf_counter()
    oracle.count_rows(g.n, rpp, colp, 0, g.n, stride)
    t_sample = time.perf_counter() - t1
    frac = w_sample / W if W else 1.0
    t_full = t_orient + (t_sample / frac if frac > 0 else 0.0)
    desc = (f"{label}oracle orientation of the full graph ({t_orient:.2f} s) + forward count over every "
            f"{stride}th source row ({100 * frac:.1f}% of the merge work, {t_sample:.2f} s), "
            f"extrapolated by merge work to {t_full:.1f} s for the whole graph; 1 thread")
    if all_cores is not None:
        if t_sample >= 1.0:
            all_cores.update(oracle_rate_all_cores(g, rpp, colp, stride, frac, t_orient))
        else:  # worker start-up would dominate a sample this small
            all_cores.update({"value": None, "sample": f"not split: the 1-thread sample took {t_sample:.2f} s"})
    return g.m / t_full, desc, t_orient + t_sample


def reference_arm(g, desc, args, world):
    """The reference arm: the oracle on one host core, step by step.  Step j
    orients the whole graph and counts one shard of the row sample that
    cpu_baseline uses (rows j*stride, j*stride + K*stride, ...); the K timed
    steps together cover exactly that sample, so the two CPU figures measure
    the same rows.  value = edges / (median orientation time + sample time
    extrapolated by merge work)."""
    import oracle
    K, Wu = max(1, args.steps), max(0, args.warmup)
    rpp, colp, _, w_row, stride = oracle_sample(g)
    Wtot = float(w_row.sum())
    t_or, t_cnt, frac = [], 0.0, 0.0
    for i in range(Wu + K):
        j = i % K
        t0 = time.perf_counter()
        oracle.orient(g.n, g.row_ptr, g.col)
        t1 = time.perf_counter()
        oracle.count_rows(g.n, rpp, colp, j * stride, g.n, stride * K)
        t2 = time.perf_counter()
        if i >= Wu:
            t_or.append(t1 - t0)
            t_cnt += t2 - t1
            frac += float(w_row[j * stride::stride * K].sum()) / Wtot if Wtot else 1.0 / K
    t_full = statistics.median(t_or) + (t_cnt / frac if frac > 0 else 0.0)
    v = g.m / t_full
    sample = (f"oracle on 1 host core; each step orients the full graph and counts 1/{K} of the "
              f"every-{stride}th-row sample of cpu_baseline ({100 * frac:.1f}% of the merge work over the "
              f"{K} timed steps, {t_cnt:.2f} s), extrapolated by merge work to {t_full:.1f} s per graph")
    return {"impl": "reference", "metric": "edges/s (undirected input edges, build + count per step)",
            "value": v, "unit": "edges/s", "n_gpus": world, "steps": K, "warmup": Wu,
            "ms_per_step": t_full * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32 ids / int64 counts", "data": "synthetic",
            "config": {"workload": desc, "n": g.n, "m_undirected": g.m},
            "cpu_baseline": {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _oracle_rows(args):
    """Pool worker: the oracle's forward count over rows start, start+step, ..."""
    import oracle
    path, n, start, step = args
    d = np.load(path)
    return oracle.count_rows(n, d["rpp"], d["colp"], start, n, step)


def _noop(_):
    return 0


def oracle_rate_all_cores(g, rpp, colp, stride, frac, t_orient):
    """The same sample as oracle_rate, its rows split over every host core
    (spawn-started worker processes, each running the oracle unchanged on an
    interleaved share); the orientation stays one call of the oracle on one
    core."""
    import multiprocessing as mp
    import tempfile
    procs = max(1, os.cpu_count() or 1)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "ocsr.npz")
        np.savez(path, rpp=rpp, colp=colp)
        with mp.get_context("spawn").Pool(procs) as pool:
            pool.map(_noop, range(procs))
            t1 = time.perf_counter()
            pool.map(_oracle_rows, [(path, g.n, j * stride, stride * procs) for j in range(procs)])
            t_par = time.perf_counter() - t1
    t_full = t_orient + (t_par / frac if frac > 0 else 0.0)
    return {"value": g.m / t_full, "unit": "edges/s", "cores": procs, "kind": "oracle",
            "sample": f"the same rows as the 1-thread sample over {procs} worker processes ({t_par:.2f} s), "
                      f"orientation on one core ({t_orient:.2f} s), extrapolated to {t_full:.1f} s"}


# ----------------------------------------------------------------------------- GPU arm
def run_rmat_like(args, torch, binding, dev, rank, world):
    name = args.workload
    shard = args.multi == "shard" and world > 1
    # replicas: every rank counts its own graph (seed = rank); shard: all ranks
    # count one graph (seed 0), each its part of the work, then one all-reduce
    g, desc = workload_graph(name, seed=0 if shard else rank, rmat_scale=args.rmat_scale)
    log(f"[rank {rank}] {desc}: n={g.n} m={g.m}")
    B_alg, S, dplus, deg = algorithmic_bytes(g, per_vertex=True)
    ctx = binding.Context(dev.index)
    stream = torch.cuda.current_stream()
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    total = torch.zeros(1, dtype=torch.int64, device=dev)
    pv = torch.zeros(g.n, dtype=torch.int64, device=dev)

    def step():
        o = ctx.build(g.n, rp, col, stream=stream)
        if shard:
            ctx.count_shard(o, rank, world, total, pv, stream=stream)
            torch.distributed.all_reduce(total)
            torch.distributed.all_reduce(pv)
        else:
            ctx.count(o, total, pv, stream=stream)
        o.release(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    T_gpu = int(total.item())
    pv_sum = int(pv.sum().item())
    assert pv_sum == 3 * T_gpu, "per-vertex counts do not sum to 3T"

    sampler = ClockSampler(device_uuid(torch, dev))
    sampler.start()
    ctx.read_trace()  # reset
    ctx.set_trace(True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms_total = e0.elapsed_time(e1)
    ctx.set_trace(False)
    tr = ctx.read_trace()
    clocks = sampler.stop()
    ms = ms_total / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())

    ph = {k: v / args.steps for k, v in tr["phase_ms"].items()}
    count_ms = sum(ph[k] for k in COUNT_PHASES)
    build_ms = sum(ph[k] for k in BUILD_PHASES)

    # end to end through the public API: pinned host CSR in, host results out
    h_rp = torch.from_numpy(g.row_ptr).pin_memory()
    h_col = torch.from_numpy(g.col).pin_memory()
    h_tot = torch.zeros(1, dtype=torch.int64).pin_memory()
    h_pv = torch.zeros(g.n, dtype=torch.int64).pin_memory()

    def e2e_step():
        o = ctx.build(g.n, h_rp, h_col, stream=stream)
        ctx.count(o, h_tot, h_pv, stream=stream)  # host outputs: copies back and synchronises
        o.release(stream)

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 3)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    assert int(h_tot[0]) == T_gpu
    h2d = 8 * (g.n + 1) + 4 * g.nnz
    d2h = 8 + 8 * g.n

    # small graphs are launch-bound: the same step replayed as one CUDA graph
    # (tc_batch_plan over a batch of this one graph), counts checked
    replay = None
    if g.m <= 1_000_000 and not shard:
        vo = torch.tensor([0, g.n], dtype=torch.int64, device=dev)
        eo = torch.tensor([0, g.nnz], dtype=torch.int64, device=dev)
        rtot = torch.zeros(1, dtype=torch.int64, device=dev)
        rpv = torch.zeros(g.n, dtype=torch.int64, device=dev)
        plan = ctx.batch_plan(vo, eo, rp, col, rtot, rpv, stream=stream)
        for _ in range(args.warmup):
            plan.launch(stream)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            plan.launch(stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        rms = ev0.elapsed_time(ev1) / args.steps
        assert int(rtot.item()) == T_gpu and torch.equal(rpv, pv)
        plan.close()
        replay = {"ms_per_step": rms, "edges_per_s": g.m / (rms * 1e-3), "how": "tc_batch_plan of this one graph, replayed"}

    # the one-call path (tc_count_graph): a graph that fits one CTA's shared
    # memory is oriented, compacted and counted by one fused kernel launch
    one_call = None
    if g.n <= 8192 and not shard:
        ftot = torch.zeros(1, dtype=torch.int64, device=dev)
        fpv = torch.zeros(g.n, dtype=torch.int64, device=dev)
        for _ in range(args.warmup):
            ctx.count_graph(g.n, rp, col, ftot, fpv, stream=stream)
        torch.cuda.synchronize()
        ctx.read_trace()
        ctx.set_trace(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            ctx.count_graph(g.n, rp, col, ftot, fpv, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ctx.set_trace(False)
        fl = ctx.read_trace()["launches"] / args.steps
        fms = ev0.elapsed_time(ev1) / args.steps
        assert int(ftot.item()) == T_gpu and torch.equal(fpv, pv)
        one_call = {"ms_per_step": fms, "edges_per_s": g.m / (fms * 1e-3), "launches_per_step": fl,
                    "how": "tc_count_graph: degree, (degree, id) order, orientation, compaction, "
                           "intersection and reduction in one call; one fused kernel launch when the graph "
                           "fits one CTA's shared memory (every CTA orients it, each counts its share of "
                           "the edges), else build + count"}

    peak, peak_kind = peaks()
    cfg = ctx.get_config()
    cb = class_bytes(g, dplus, cfg["small_max"], cfg["warp_max"])
    # the dominant kernel: the CTA-table intersection.  Its algorithmic bytes are
    # the bytes its formulation must stream: the shorter list of every oriented
    # edge it owns (the longer list is the shared-memory table, loaded once per
    # work item).  The both-lists figure of the merge definition is reported
    # beside it as "logical": most of those bytes never leave shared memory.
    cta_ms = ph["count_cta"]
    achieved = cb["cta_shorter_list"] / (cta_ms * 1e-3) / 1e9 if cta_ms > 0 else None
    # the committed capture is of the full-size workload only
    traffic = profiled_traffic(f"k_count_cta_{name}") if (name != "rmat22" or args.rmat_scale == 22) else None
    # whole count (all three kernels): the shorter list of every pivot edge,
    # both lists of every thread-merged edge, structure and outputs
    B_probe = (cb["cta_shorter_list"] + cb["warp_shorter_list"] + cb["small"] + 4 * g.m + 8 * (g.n + 1) + 8 * g.n + 8)
    units = g.m * (1 if shard else world)
    res = {
        "metric": "edges/s (undirected input edges, build + count per step)",
        "value": units / (ms * 1e-3),
        "unit": "edges/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None,
        "dtype": "int32 ids / int64 counts",
        "data": "synthetic (seeded generator; the paper's SNAP/DIMACS graphs are not available)",
        "config": {"workload": desc, "n": g.n, "m_undirected": g.m, "per_vertex": True,
                   "l2": "no flush: input CSR %.0f MB > 129 MB L2" % ((8 * (g.n + 1) + 4 * g.nnz) / 1e6),
                   "seed": 0 if shard else rank,
                   "parallelism": ("sharded count + all-reduce of (T, t)" if shard else
                                   "replicas only (one graph per GPU)") if world > 1 else "1 GPU"},
        "triangles": T_gpu,
        "phases_ms": {k: round(v, 4) for k, v in ph.items() if v > 0},
        "build_ms": build_ms,
        "count_ms": count_ms,
        "roofline": {"bound": "hbm", "kernel": "k_count_cta", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                     "traffic": traffic, "algorithmic_bytes_per_launch": cb["cta_shorter_list"],
                     "bytes_model": "4 * sum of min(d+(u), d+(v)) over the oriented edges of the kernel's class",
                     "kernel_ms": cta_ms, "kernel_share_of_step": cta_ms / ms if ms else None,
                     "traffic_frac": (traffic / (cta_ms * 1e-3) / 1e9 / peak) if (traffic and cta_ms > 0) else None,
                     # both lists per edge (the merge definition): logical bytes, served mostly
                     # from shared memory and L2, so this ratio is not a bandwidth fraction
                     "logical_bytes_per_launch": cb["cta"],
                     "logical_frac": (cb["cta"] / (cta_ms * 1e-3) / 1e9 / peak) if cta_ms > 0 else None},
        "count_roofline": {"bytes": B_probe, "count_ms": count_ms,
                           "achieved_gbs": B_probe / (count_ms * 1e-3) / 1e9 if count_ms > 0 else None,
                           "frac": (B_probe / (count_ms * 1e-3) / 1e9 / peak) if count_ms > 0 else None,
                           "logical_bytes": B_alg, "sum_dplus_u_plus_dplus_v": S,
                           "logical_frac": (B_alg / (count_ms * 1e-3) / 1e9 / peak) if count_ms > 0 else None,
                           "class_bytes": cb},
        "e2e": {"value": units / e2e_s, "unit": "edges/s", "ms_per_step": e2e_s * 1e3,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(tr["launches"]),
        "clocks": clocks,
    }
    if replay:
        res["graph_replay"] = replay
    if one_call:
        res["one_call"] = one_call
    return res, g


def run_batch(args, torch, binding, dev, rank, world):
    """4096 Barabasi-Albert graphs: one batched pass (CUDA-graph plan) against
    one build + count per graph, identical counts."""
    from paper_1804_06926_gb300 import gen
    G = args.batch_graphs
    b = gen.ba_batch(G, 100, 20000, 2, 16, seed0=rank * G)
    m_tot = int(b.edge_off[-1] // 2)
    log(f"[rank {rank}] BA batch: G={G} n={int(b.vtx_off[-1])} m={m_tot}")
    vo, eo, rp, col = (torch.from_numpy(x).to(dev) for x in (b.vtx_off, b.edge_off, b.row_ptr, b.col))
    # strategy, thresholds and tile sizes for this size class, measured on the device
    from paper_1804_06926_gb300 import autotune
    tuned = autotune.tune_batch(vo, eo, rp, col, per_vertex=True, reps=1, device=dev.index,
                                tuner=autotune.Autotuner(device_name=torch.cuda.get_device_name(dev)))
    ctx = binding.Context(dev.index, **tuned.best)
    totals = torch.zeros(G, dtype=torch.int64, device=dev)
    pv = torch.zeros(int(b.vtx_off[-1]), dtype=torch.int64, device=dev)
    plan = ctx.batch_plan(vo, eo, rp, col, totals, pv)
    for _ in range(args.warmup):
        plan.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(device_uuid(torch, dev))
    sampler.start()
    e0.record()
    for _ in range(args.steps):
        plan.launch()
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms_batch = e0.elapsed_time(e1) / args.steps
    T_batch = totals.cpu().numpy().copy()
    # one launch sequence per graph
    graphs = [b.graph(i) for i in range(G)]
    dev_graphs = [(gg.n, torch.from_numpy(gg.row_ptr).to(dev), torch.from_numpy(gg.col).to(dev)) for gg in graphs]
    tot1 = torch.zeros(G, dtype=torch.int64, device=dev)
    pvs = [torch.zeros(gg.n, dtype=torch.int64, device=dev) for gg in graphs]

    def per_graph():
        for i, (n, r, c) in enumerate(dev_graphs):
            o = ctx.build(n, r, c)
            ctx.count(o, tot1[i:i + 1], pvs[i])
            o.release(None)

    per_graph()
    torch.cuda.synchronize()
    reps = max(1, args.steps // 10)
    e0.record()
    for _ in range(reps):
        per_graph()
    e1.record()
    torch.cuda.synchronize()
    ms_single = e0.elapsed_time(e1) / reps
    assert np.array_equal(tot1.cpu().numpy(), T_batch), "batched counts differ from per-graph counts"
    res = {
        "metric": "graphs/s and edges/s (4096 BA graphs per batch, build + count)",
        "value": m_tot / (ms_batch * 1e-3), "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32 ids / int64 counts", "data": "synthetic",
        "config": {"workload": f"BA batch G={G}, n~U[100,20000], k~U[2,16]", "m_undirected": m_tot,
                   "l2": "no flush: batch CSR %.0f MB > 129 MB L2" % ((b.row_ptr.nbytes + b.col.nbytes) / 1e6)},
        "graphs_per_s": G / (ms_batch * 1e-3),
        "one_launch_per_graph": {"ms": ms_single, "edges_per_s": m_tot / (ms_single * 1e-3),
                                 "graphs_per_s": G / (ms_single * 1e-3)},
        "batch_speedup": ms_single / ms_batch,
        "autotuned_config": tuned.best,
        "autotune_ms": tuned.times_ms,
        "triangles_total": int(T_batch.sum()),
        "clocks": clocks,
    }
    return res, None


def run_serve(args, torch, binding, dev, rank, world):
    """Poisson request stream mixing R-MAT scales 10..20 and BA graphs, through
    tc_submit / tc_poll with a 40 GB budget; latency percentiles and edges/s."""
    from paper_1804_06926_gb300 import gen
    rng = np.random.default_rng(args.seed)
    pool = []
    for i in range(args.serve_pool):
        if rng.random() < 0.5:
            pool.append(gen.rmat(int(rng.integers(10, 21)), 16, seed=int(rng.integers(1 << 30))))
        else:
            pool.append(gen.ba(int(rng.integers(100, 20001)), int(rng.integers(2, 17)), seed=int(rng.integers(1 << 30))))
    srv = binding.Server(device=dev.index, slots=args.slots, hbm_budget_bytes=40 << 30)
    # closed-loop capacity first, then an open-loop Poisson stream at ~0.7x of it
    t0 = time.perf_counter()
    tks = [srv.submit(g.n, g.row_ptr, g.col) for g in pool]
    for t in tks:
        srv.wait(t, 600000)
        srv.release(t)
    cap_rps = len(pool) / (time.perf_counter() - t0)
    rate = args.serve_rate or 0.7 * cap_rps
    nreq = args.serve_requests
    arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq))
    picks = rng.integers(0, len(pool), nreq)
    lat, edges = [], 0
    tickets = []
    start = time.perf_counter()
    for i in range(nreq):
        now = time.perf_counter() - start
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        g = pool[picks[i]]
        key = int(picks[i]) + 1 if args.serve_cache else 0
        tickets.append((srv.submit(g.n, g.row_ptr, g.col, key=key), g.m))
    for t, m in tickets:
        r = srv.wait(t, 600000)
        assert r["status"] == 0
        lat.append(r["latency_ms"])
        edges += m
        srv.release(t)
    wall = time.perf_counter() - start
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    # saturated throughput with all slots against one slot, no resident graphs:
    # the gain of overlapping requests on the device
    def run_all(sv, ids, clients=8):
        # `clients` submitting threads (the ABI call releases the GIL), as many
        # callers of one server would; each waits for its own tickets
        from concurrent.futures import ThreadPoolExecutor

        def client(part):
            tks = [(sv.submit(pool[i].n, pool[i].row_ptr, pool[i].col), pool[i].m) for i in part]
            e = 0
            for tk, m in tks:
                r = sv.wait(tk, 600000)
                assert r["status"] == 0
                e += m
                sv.release(tk)
            return e

        t0 = time.perf_counter()
        with ThreadPoolExecutor(clients) as ex:
            e = sum(ex.map(client, [ids[c::clients] for c in range(clients)]))
        return e, time.perf_counter() - t0

    def saturated_ids(ids, slots, fuse):
        # one untimed pass fills the server's pinned staging pool, the second is timed
        sv = binding.Server(device=dev.index, slots=slots, hbm_budget_bytes=40 << 30, batch_graphs=fuse)
        run_all(sv, ids)
        b0 = sv.stats()["batches"]
        e, wall_s = run_all(sv, ids)
        nb = sv.stats()["batches"] - b0
        sv.close()
        return e / wall_s, len(ids) / wall_s, nb

    def saturated(slots, k, fuse=0):
        return saturated_ids([int(picks[i]) for i in range(k)], slots, fuse)[:2]
    nsat = min(nreq, args.serve_seq_requests)
    sat_many = saturated(args.slots, nsat)
    sat_one = saturated(1, nsat, fuse=1)  # one request at a time: one slot, no fused batches
    # the same comparison on the small requests alone (BA graphs and R-MAT s10-s14), where
    # one request does not fill the GPU and overlapping requests is what serving adds
    small_ids = [i for i, g in enumerate(pool) if g.m <= 400000]
    picks_small = rng.choice(small_ids, nsat) if small_ids else picks[:nsat]

    def saturated_small(slots, fuse=0):
        return saturated_ids([int(i) for i in picks_small], slots, fuse)
    small_many = saturated_small(args.slots)
    small_slots = saturated_small(args.slots, fuse=1)  # slots overlap, no fused batches
    small_one = saturated_small(1, fuse=1)
    res = {
        "metric": "served count requests: edges/s, p50/p99 latency", "value": edges / wall, "unit": "edges/s",
        "n_gpus": world, "steps": nreq, "warmup": len(pool), "ms_per_step": wall * 1e3 / nreq,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32 ids / int64 counts",
        "data": "synthetic", "config": {"workload": f"{nreq} Poisson requests at {rate:.1f}/s over a pool of "
                                                    f"{len(pool)} graphs (R-MAT s10-20 / BA), 40 GB budget, "
                                                    f"{args.slots} slots, cache={'on' if args.serve_cache else 'off'}"},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "closed_loop_capacity_rps": cap_rps, "server_stats": st,
        "saturated": {"requests": nsat, "clients": 8, "slots": args.slots, "edges_per_s": sat_many[0], "requests_per_s": sat_many[1],
                      "one_slot_edges_per_s": sat_one[0], "one_slot_requests_per_s": sat_one[1],
                      "gain": sat_many[0] / sat_one[0]},
        "saturated_small": {"requests": nsat, "graphs": "pool members with m <= 400000", "clients": 8,
                            "slots": args.slots, "requests_per_s": small_many[1], "edges_per_s": small_many[0],
                            "one_slot_requests_per_s": small_one[1], "one_slot_edges_per_s": small_one[0],
                            "slots_without_fusing_requests_per_s": small_slots[1],
                            "fused_batches": small_many[2],
                            "gain": small_many[1] / small_one[1]},
    }
    return res, None


def serve_saturated(binding, dev, graphs, ids, slots, fuse, clients=8):
    """Every request of `ids` submitted by `clients` threads (the ABI call
    releases the GIL) to a server with `slots` slots; one untimed pass fills
    the pinned staging pool, the second is timed.  Returns (edges/s,
    requests/s, fused batches, totals by request position)."""
    from concurrent.futures import ThreadPoolExecutor
    sv = binding.Server(device=dev.index, slots=slots, hbm_budget_bytes=40 << 30, batch_graphs=fuse)

    def one_pass():
        def client(part):
            tks = [(k, sv.submit(graphs[i].n, graphs[i].row_ptr, graphs[i].col), graphs[i].m) for k, i in part]
            out = []
            for k, tk, m in tks:
                r = sv.wait(tk, 600000)
                assert r["status"] == 0
                out.append((k, r["total"], m))
                sv.release(tk)
            return out

        pos = list(enumerate(ids))
        t0 = time.perf_counter()
        with ThreadPoolExecutor(clients) as ex:
            res = [x for part in ex.map(client, [pos[c::clients] for c in range(clients)]) for x in part]
        return res, time.perf_counter() - t0

    one_pass()
    b0 = sv.stats()["batches"]
    res, wall = one_pass()
    nb = sv.stats()["batches"] - b0
    sv.close()
    totals = [t for _, t, _ in sorted(res)]
    edges = sum(m for _, _, m in res)
    return edges / wall, len(ids) / wall, nb, totals


def run_secondary(args, torch, binding, dev):
    """Batch and serving evidence beside the headline line: the 4096-graph BA
    batch in one CUDA-graph pass against one build + count per graph (counts
    asserted equal), and a saturated serving comparison (many slots with fused
    small requests against one slot, one request at a time; totals asserted
    equal)."""
    from paper_1804_06926_gb300 import gen
    sub = argparse.Namespace(**vars(args))
    sub.steps, sub.warmup = 5, 2
    rb, _ = run_batch(sub, torch, binding, dev, 0, 1)
    out = {"ba_batch4096": {k: rb[k] for k in ("value", "unit", "ms_per_step", "graphs_per_s", "one_launch_per_graph",
                                               "batch_speedup", "autotuned_config", "triangles_total")}}
    out["ba_batch4096"]["counts_equal_per_graph_launches"] = True
    rng = np.random.default_rng(args.seed + 7)
    graphs = []
    for _ in range(32):
        if rng.random() < 0.5:
            graphs.append(gen.rmat(int(rng.integers(10, 17)), 16, seed=int(rng.integers(1 << 30))))
        else:
            graphs.append(gen.ba(int(rng.integers(100, 20001)), int(rng.integers(2, 17)), seed=int(rng.integers(1 << 30))))
    ids = [int(i) for i in rng.integers(0, len(graphs), 300)]
    many = serve_saturated(binding, dev, graphs, ids, args.slots, 0)
    one = serve_saturated(binding, dev, graphs, ids, 1, 1)
    assert many[3] == one[3], "served totals differ between the mixed and the one-at-a-time server"
    # latency: an open-loop Poisson stream at 0.7x the saturated request rate
    rate = 0.7 * many[1]
    nreq = 1000
    arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq))
    picks = rng.integers(0, len(graphs), nreq)
    srv = binding.Server(device=dev.index, slots=args.slots, hbm_budget_bytes=40 << 30)
    tickets, lat = [], []
    start = time.perf_counter()
    for i in range(nreq):
        now = time.perf_counter() - start
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        g = graphs[int(picks[i])]
        tickets.append(srv.submit(g.n, g.row_ptr, g.col, key=int(picks[i]) + 1))
    for tk in tickets:
        r = srv.wait(tk, 600000)
        assert r["status"] == 0
        lat.append(r["latency_ms"])
        srv.release(tk)
    srv.close()
    out["serving_saturated"] = {
        "requests": len(ids), "clients": 8, "pool": "32 graphs: R-MAT s10-16 ef16 and BA n~U[100,20000], k~U[2,16]",
        "slots": args.slots, "edges_per_s": many[0], "requests_per_s": many[1], "fused_batches": many[2],
        "one_slot_edges_per_s": one[0], "one_slot_requests_per_s": one[1], "gain": many[0] / one[0],
        "totals_equal_alone_and_mixed": True}
    lat = np.array(lat)
    out["serving_poisson"] = {"requests": nreq, "rate_per_s": rate, "slots": args.slots, "resident_cache": True,
                              "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}
    return out


# ----------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat22", choices=["rmat22", "grid4096", "er1024", "ba_batch4096", "serve"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--secondary", type=int, default=1,
                    help="rmat22 at 1 GPU: also measure the BA batch and saturated serving (secondary object)")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rate", type=float, default=0.0)
    ap.add_argument("--serve-cache", type=int, default=1)
    ap.add_argument("--serve-seq-requests", type=int, default=500)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--multi", default="replica", choices=["replica", "shard"],
                    help="N>1: independent replicas (weak scaling) or one graph sharded over the GPUs (strong)")
    ap.add_argument("--rmat-scale", type=int, default=22, help="R-MAT scale of the rmat22 workload (small cases for profiling)")
    args = ap.parse_args()
    world, rank, local = dist_env()

    if args.impl == "reference":
        if rank != 0:
            return 0
        g, desc = workload_graph(args.workload if args.workload in ("rmat22", "grid4096", "er1024") else "rmat22", 0,
                                 args.rmat_scale)
        print(json.dumps(reference_arm(g, desc, args, world)), flush=True)
        return 0

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1804_06926_gb300 import _build, binding
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    binding.load(build_if_missing=False)

    if args.workload == "ba_batch4096":
        res, g = run_batch(args, torch, binding, dev, rank, world)
    elif args.workload == "serve":
        res, g = run_serve(args, torch, binding, dev, rank, world)
    else:
        res, g = run_rmat_like(args, torch, binding, dev, rank, world)

    if rank == 0 and world == 1 and args.workload == "rmat22" and args.secondary:
        res["secondary"] = run_secondary(args, torch, binding, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and g is not None:
        allc = {}
        v, d, _ = oracle_rate(g, all_cores=allc)
        res["cpu_baseline"] = {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": d,
                               "all_cores": allc}
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
