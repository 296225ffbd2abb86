"""Autotuner for the partition thresholds and kernel shapes (tc_config).

The paper leaves the small/large threshold of its dynamic grouping open
(Sec. 4.2.2: "carefully choosing a threshold value").  Here the choice is
measured: for a size class of input, every candidate configuration runs the
whole path (build + count, per-vertex counts included) on the device, timed
with CUDA events on the launching stream, and the fastest is cached per
(GPU, size class) in a JSON file.  No candidate changes a result, only the
speed; the tuner checks that every candidate returns the same total.

Knobs: the probe strategy (hash/bitmap/direct tables or binary search), the
thread-per-edge and warp-table thresholds (small_max, warp_max), threads per
row of the thread-merge class (small_lanes), the CTA table capacity
(table_cap), partners per work item (chunk), threads per CTA (cta_threads),
the bitmap/direct span limits, the degree-ratio switch that sends balanced
edges to the warp merge path (merge_ratio, merge_max; the paper's choice
between its two intersection strategies, Sec. 4.2.2), and the staging of
partner lists by the copy engine (stage).

The search has two stages: every candidate below (one knob changed from the
default, or a pair that only makes sense together) is measured; then, from
the fastest, the other candidates that beat the default are merged in one at
a time, greedily, each kept only if the merged configuration is faster.
"""
from __future__ import annotations

import json
import math
import os
import threading
from dataclasses import dataclass, field

# Candidate configurations (fields of tc_config; absent = library default).
CANDIDATES = [
    {},
    {"chunk": 2048},
    {"warp_max": 32},
    {"warp_max": 128, "chunk": 2048},
    {"small_max": 4},
    {"small_max": 16},
    {"small_max": 32},
    {"cta_threads": 512},
    {"table_cap": 2048, "chunk": 2048},
    {"direct_span": -1},
    {"probe": 2},
    {"merge_ratio": 150, "merge_max": 128},
    {"merge_ratio": 300, "merge_max": 512},
    {"stage": 1},
    {"small_lanes": 2},
    {"small_lanes": 4},
]


def size_class(n: int, nnz: int, graphs: int = 1) -> str:
    """Inputs within a factor of two in vertices and entries share a class."""
    lg = lambda x: int(math.log2(max(int(x), 1)))
    return f"n{lg(n)}_e{lg(nnz)}_g{lg(graphs)}"


def default_cache_path() -> str:
    base = os.environ.get("TC_AUTOTUNE_CACHE")
    if base:
        return base
    root = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(root, "tc_autotune.json")


@dataclass
class TuneResult:
    key: str
    best: dict
    times_ms: list = field(default_factory=list)  # (config, ms) per candidate


class Autotuner:
    """Chooses tc_config per (device name, size class); results persist in JSON."""

    def __init__(self, cache_path: str | None = None, device_name: str | None = None):
        self.path = cache_path or default_cache_path()
        self.device_name = device_name or "unknown-device"
        self._lock = threading.Lock()
        self._cache = self._read()

    def _read(self) -> dict:
        try:
            with open(self.path) as f:
                data = json.load(f)
            return data if isinstance(data, dict) else {}
        except (OSError, ValueError):
            return {}

    def _write(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = f"{self.path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(self._cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def key(self, cls: str) -> str:
        return f"{self.device_name}|{cls}"

    def lookup(self, cls: str) -> dict | None:
        with self._lock:
            e = self._cache.get(self.key(cls))
            return dict(e["best"]) if e else None

    def record(self, cls: str, best: dict, times) -> None:
        with self._lock:
            self._cache[self.key(cls)] = {"best": best, "times_ms": times}
            self._write()

    def tune(self, cls: str, run, candidates=None, reps: int = 3, force: bool = False,
             combine: bool = True) -> TuneResult:
        """run(config) -> (milliseconds, total); the fastest config wins.

        With combine, the candidates that beat the default ({} when it is
        among them, else the first) are merged into the fastest one greedily
        (disjoint knobs only), each merge kept if it is faster.  Cached
        classes are not re-measured unless force=True."""
        if not force:
            hit = self.lookup(cls)
            if hit is not None:
                return TuneResult(self.key(cls), hit, [])
        cands = candidates if candidates is not None else CANDIDATES
        times = []
        ref = []

        def measure(cfg):
            ms, total = min((run(cfg) for _ in range(max(1, reps))), key=lambda x: x[0])
            if not ref:
                ref.append(total)
            elif total != ref[0]:
                raise RuntimeError(f"candidate {cfg} changed the count: {total} != {ref[0]}")
            times.append([dict(cfg), ms])
            return ms

        measured = [(measure(cfg), dict(cfg)) for cfg in cands]
        best_ms, best = min(measured, key=lambda x: x[0]) if measured else (math.inf, None)
        if combine and measured:
            base_ms = next((ms for ms, cfg in measured if not cfg), measured[0][0])
            better = sorted((x for x in measured if x[0] < base_ms and x[1] and x[1] != best), key=lambda x: x[0])
            for _, cfg in better:
                if set(cfg) & set(best):
                    continue
                merged = {**best, **cfg}
                ms = measure(merged)
                if ms < best_ms:
                    best, best_ms = merged, ms
        self.record(cls, best, times)
        return TuneResult(self.key(cls), best, times)


# ----------------------------------------------------------------------------- device drivers
def _device_name(torch, dev) -> str:
    try:
        return torch.cuda.get_device_name(dev).replace("|", "_")
    except Exception:
        return "cuda"


def tune_graph(n, row_ptr, col, per_vertex=True, tuner: Autotuner | None = None, candidates=None,
               reps=2, force=False, device=0) -> TuneResult:
    """Tune one graph already resident on the device (torch tensors)."""
    import torch

    from . import binding
    dev = torch.device("cuda", device)
    tuner = tuner or Autotuner(device_name=_device_name(torch, dev))
    total = torch.zeros(1, dtype=torch.int64, device=dev)
    pv = torch.zeros(n, dtype=torch.int64, device=dev) if per_vertex else None
    stream = torch.cuda.current_stream(dev)

    def run(cfg):
        ctx = binding.Context(device, **cfg)
        try:
            o = ctx.build(n, row_ptr, col, stream=stream)  # warm-up: attributes, pool
            ctx.count(o, total, pv, stream=stream)
            o.release(stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            o = ctx.build(n, row_ptr, col, stream=stream)
            ctx.count(o, total, pv, stream=stream)
            o.release(stream)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1), int(total.item())
        finally:
            ctx.close()

    return tuner.tune(size_class(n, int(col.shape[0])), run, candidates, reps, force)


def tune_batch(vtx_off, edge_off, row_ptr, col, per_vertex=True, tuner: Autotuner | None = None,
               candidates=None, reps=2, force=False, device=0) -> TuneResult:
    """Tune a batch of graphs (device tensors in the tc_batch layout)."""
    import torch

    from . import binding
    dev = torch.device("cuda", device)
    tuner = tuner or Autotuner(device_name=_device_name(torch, dev))
    G = int(vtx_off.shape[0] - 1)
    nsum = int(row_ptr.shape[0] - 1)
    totals = torch.zeros(G, dtype=torch.int64, device=dev)
    pv = torch.zeros(nsum, dtype=torch.int64, device=dev) if per_vertex else None
    stream = torch.cuda.current_stream(dev)

    def run(cfg):
        ctx = binding.Context(device, **cfg)
        try:
            ctx.count_batch(vtx_off, edge_off, row_ptr, col, totals, pv, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.count_batch(vtx_off, edge_off, row_ptr, col, totals, pv, stream=stream)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1), int(totals.sum().item())
        finally:
            ctx.close()

    return tuner.tune(size_class(nsum, int(col.shape[0]), G), run, candidates, reps, force)
