"""Batched filtering of mixed-length pairs: one persistent launch, captured in
a CUDA graph, with a tiling picked by an autotuner.

The library does all the work (gk_filter_batched: classify, scan, scatter,
persistent filter).  This module owns the device buffers (workspace,
outputs), captures the call into a CUDA graph for replay, and searches the
tiling space on a sample of the workload, timing each candidate with CUDA
events.  The autotuner's table is JSON keyed by GPU name and workload
signature.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from . import gk

DEFAULT_TILING = (1, 256, 4, 8)
WPT_CHOICES = (1, 2, 3, 4, 6, 8)
TILE_CHOICES = (64, 256, 1024, 4096)
GRID_CHOICES = ((1, 8), (2, 8), (3, 8), (4, 8), (8, 4), (4, 4), (16, 2))
TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiling_table.json")


def tiling(t) -> gk.Tiling:
    return t if isinstance(t, gk.Tiling) else gk.Tiling(*t)


class BatchedFilter:
    """Runs gk_filter_batched over fixed device buffers.  ``run`` enqueues it;
    ``capture`` records one call into a CUDA graph that ``replay`` launches."""

    def __init__(self, ref: gk.Reference, reads: torch.Tensor, stride_words: int, n_reads: int,
                 read_len: torch.Tensor, read_nflag: torch.Tensor | None, pair_read: torch.Tensor,
                 pair_off: torch.Tensor, pair_e, tiling_=DEFAULT_TILING, count_mode=gk.GK_COUNT_RUNS4,
                 flags=0, err_count: torch.Tensor | None = None):
        self.ref, self.reads, self.sw, self.n_reads = ref, reads, stride_words, n_reads
        self.read_len, self.nflag = read_len, read_nflag
        self.pair_read, self.pair_off, self.pair_e = pair_read, pair_off, pair_e
        self.tiling = tiling(tiling_)
        self.count_mode, self.flags, self.err = count_mode, flags, err_count
        n = pair_read.numel()
        dev = pair_read.device
        self.workspace = torch.empty(max(256, gk.gk_filter_batched_workspace(n)), dtype=torch.uint8, device=dev)
        self.accept = torch.empty(n, dtype=torch.uint8, device=dev)
        self.edits = torch.empty(n, dtype=torch.int16, device=dev)
        self.graph = None

    def run(self, stream=None):
        gk.gk_filter_batched(self.ref, self.reads, self.sw, self.n_reads, self.read_len, self.nflag,
                             self.pair_read, self.pair_off, self.pair_e, self.tiling, self.workspace,
                             self.count_mode, self.flags, self.accept, self.edits, self.err, stream)
        return self.accept, self.edits

    def capture(self):
        """Record one call into a CUDA graph (warm-up call first, on a side
        stream, as graph capture requires)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(s)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self.graph

    def replay(self):
        self.graph.replay()
        return self.accept, self.edits


def signature(read_len: np.ndarray, pair_read: np.ndarray, pair_e) -> str:
    """Workload signature of the tiling table: words-per-read range and the
    threshold range."""
    m = read_len[pair_read]
    W = (m.astype(np.int64) + 31) // 32
    e = np.asarray(pair_e) if not np.isscalar(pair_e) else np.array([pair_e])
    return f"W{int(W.min())}-{int(W.max())}_e{int(e.min())}-{int(e.max())}"


def _time(bf: BatchedFilter, reps: int) -> float:
    bf.run()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        bf.run()
    e.record()
    e.synchronize()
    return s.elapsed_time(e) / reps


def autotune(ref, reads, stride_words, n_reads, read_len, read_nflag, pair_read, pair_off, pair_e,
             reps: int = 3, budget_s: float = 60.0, log=None):
    """Coordinate search over the tiling on the given (sample) pairs: words
    per lane first, then tile size, then grid shape; every candidate timed with
    CUDA events, invalid ones (a block that does not fit) skipped.  The
    default tiling is always measured; the budget stops the search after it.
    Returns (best tiling tuple, {candidate: ms})."""
    t0 = time.perf_counter()
    results = {}

    def measure(t, first=False):
        if t in results:
            return results[t]
        if not first and time.perf_counter() - t0 > budget_s:
            return float("inf")
        try:
            bf = BatchedFilter(ref, reads, stride_words, n_reads, read_len, read_nflag, pair_read, pair_off,
                               pair_e, t)
            ms = _time(bf, reps)
        except gk.GKError:
            ms = float("inf")
        results[t] = ms
        if log:
            log(f"tiling {t}: {ms:.3f} ms")
        return ms

    best = DEFAULT_TILING
    measure(best, first=True)
    for wpt in WPT_CHOICES:
        cand = (wpt,) + best[1:]
        if measure(cand) < results[best]:
            best = cand
    for tile in TILE_CHOICES:
        cand = (best[0], tile) + best[2:]
        if measure(cand) < results[best]:
            best = cand
    for bpsm, wpb in GRID_CHOICES:
        cand = best[:2] + (bpsm, wpb)
        if measure(cand) < results[best]:
            best = cand
    return best, results


def load_table(path: str = TABLE_PATH) -> dict:
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


def save_table(entry_key: str, best, results: dict, path: str = TABLE_PATH):
    table = load_table(path)
    table[entry_key] = {"tiling": list(best),
                        "measured_ms": {",".join(map(str, k)): v for k, v in results.items()
                                        if v != float("inf")}}
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def table_key(sig: str) -> str:
    return f"{torch.cuda.get_device_name()}|{sig}"


def lookup(sig: str, path: str = TABLE_PATH):
    ent = load_table(path).get(table_key(sig))
    return tuple(ent["tiling"]) if ent else None
