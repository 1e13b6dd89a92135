#!/usr/bin/env python
"""Throughput benchmark of the GateKeeper-GPU filter on GB300.

Metric: filtered (read, candidate) pairs per second, x10^9 (Gpairs/s), the
paper's filtering throughput (Sec. 4.3, Table 2) measured on seeded
synthetic stand-ins for its 30M-pair mrFAST sets.

Default workload (configuration 2): 20M pairs of 100 bp reads against a
100 Mbp synthetic genome (5M reads x 4 candidates; 1 true origin with 0-2%
edits, 3 random offsets).  One step is one pass of the whole hot path over
that batch: the device encode of the reads (Sec. 3.3) and the filter at every
threshold e = 0..10 (11 launches, Sec. 2.1/3.4), so a step filters 220M pairs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N (under torchrun) every rank filters its own 20M-pair shard on
its own GPU with no collective (weak scaling; the paper's multi-GPU mode
splits equal batches, Sec. 3.1).  --impl reference times the CPU oracle on
the host cores instead, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Integer-pipe peak of the filter's instruction mix (logic + funnel shift),
# derived from unit counts and clocks: SMs x integer lanes issued per clock
# per SM x maximum SM clock.  The per-SM rate is the one gk_probe_alu measures
# on this GPU (recorded in the design notes); the bench also re-measures it
# live and reports both.
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
ALU_LANES_PER_SM_CLK = 64.0
ALU_PEAK_TOPS = SM_COUNT * ALU_LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12

E_SWEEP = list(range(0, 11))
L2_BYTES = 129 * 1024 * 1024


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the 20M-pair workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline")
    ap.add_argument("--es", default="0-10", help="thresholds of the sweep, e.g. 0-10 or 2,10")
    ap.add_argument("--probe-all", action="store_true", help="run every integer probe kind")
    ap.add_argument("--config", default="c2", choices=["c2", "c3", "c4", "c5"],
                    help="c2: the default line; c3: 150/250 bp with N; c4: batched mixed lengths")
    ap.add_argument("--tune-seconds", type=float, default=8.0, help="autotuner budget (config 4)")
    ap.add_argument("--no-extra", action="store_true", help="config 2 only (no config 3/4/5 keys)")
    ap.add_argument("--level-seconds", type=float, default=10.0, help="arrival time per serving load level")
    ap.add_argument("--round-pairs", type=int, default=32_000_000, help="pairs per serving round, at most")
    ap.add_argument("--serve-streams", type=int, default=3, help="streams of the serving executor")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---- algorithmic work per pair (fixed once; never tuned) -------------------

def ops_per_pair(m: int, e: int) -> int:
    """Integer ops of the word formulation: W words; the Hamming mask costs 9
    per word (2 XOR + OR + amendment 6), each of the 2e shifted masks 11 per
    word (2 funnel shifts + 2 XOR + OR + amendment 6), the count 4 per word."""
    W = -(-m // 32)
    ek = min(e, max(m - 1, 0))
    return W * (9 + 22 * ek + 4)


def sliced_ops_per_pair(m: int, e: int) -> float:
    """Integer ops of the bit-sliced formulation (32 pairs per word): per base
    position, 4 per mask (2 for the difference, 1 AND of the dilation into
    the running vector, 1 OR carried for the next dilation) for the 2K+1
    masks, 2 for the erosion and 4 for the count, shared by 32 pairs."""
    K = min(e, max(m - 1, 0))
    return m * (8 * K + 10) / 32


def sliced_bytes_per_pair(m: int) -> float:
    """Bytes a sliced filter launch moves per pair: the read and window planes
    (2 bits per base each, m/2), the status words (8 per 32 pairs) and the
    accept byte + 16-bit count."""
    return m / 2 + 8 / 32 + 3


# Shift-count ranges the library's sweep kernels filter in one launch each
# (gk_filter_sliced_sweep); a threshold outside them is a single launch.
SWEEP_RANGES = ((0, 5), (6, 10))


def sweep_launches(es, m: int):
    """The launches gk_filter_sliced_sweep makes for the consecutive
    thresholds es at read length m: [(e_first, e_last, klo, khi)], the
    kernel of compiled shift counts klo..khi writing e_first..e_last (klo ==
    khi: a single-threshold kernel)."""
    out = []
    e, top = es[0], es[-1]
    while e <= top:
        last, klo, khi = e, min(e, m - 1), min(e, m - 1)
        if e <= m - 1:
            for lo, hi in SWEEP_RANGES:
                if lo <= e <= hi and min(hi, top, m - 1) > e:
                    last, klo, khi = min(hi, top, m - 1), lo, hi
        out.append((e, last, klo, khi))
        e = last + 1
    return out


def sweep_ops_per_pair(m: int, klo: int, khi: int) -> float:
    """Integer ops per pair of one sweep launch over shift counts klo..khi
    (bit-sliced, 32 pairs per word): per base position 4 per mask for the
    2*khi+1 masks (the running AND of count K is the one of K-1 with two
    more masks, so every mask is computed once), and per shift count 2 for
    the erosion and 4 for the count; klo == khi is sliced_ops_per_pair."""
    return m * (4 * (2 * khi + 1) + 6 * (khi - klo + 1)) / 32


def sweep_bytes_per_pair(m: int, n_written: int, result_byte: bool = False) -> float:
    """Bytes one sweep launch moves per pair: the planes once (m/2), the
    status words (8 per 32 pairs), and the results of each threshold it
    writes (accept + 16-bit count, or one result byte)."""
    return m / 2 + 8 / 32 + (1 if result_byte else 3) * n_written


def pp_sweep_ops_per_pair(m: int, e_lo: int, e_hi: int) -> float:
    """Integer ops per pair of one per-pair sweep launch (gk_filter_sweep),
    word formulation: the Hamming mask and the 2K masks of the largest shift
    count K = min(e_hi, m-1) once (the survey's 9 + 22K per word), and the
    count (4 per word) for each of the thresholds."""
    W = -(-m // 32)
    K = min(e_hi, max(m - 1, 0))
    return W * (9 + 22 * K + 4 * (e_hi - e_lo + 1))


def pp_sweep_bytes_per_pair(m: int, c: float, n_thresholds: int, result_byte: bool = False) -> float:
    """Algorithmic bytes per pair of one per-pair sweep launch: the pair's
    inputs once (bytes_per_pair without its results) and the results of each
    threshold (accept + 16-bit count, or one result byte)."""
    return bytes_per_pair(m, c, False) - 3 + (1 if result_byte else 3) * n_thresholds


def bytes_per_pair(m: int, c: float, per_pair_e: bool) -> float:
    """Algorithmic bytes: offset 4, read id 4/c, packed read + N flag
    (m/4 + 1)/c, reference window m/4 (2 bits/base) + its N bits m/8,
    e (if per pair) 1, accept + edits 3."""
    return 4 + 4 / c + (m / 4 + 1) / c + m / 4 + m / 8 + (1 if per_pair_e else 0) + 3


# ---- clocks during the timed region ----------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        self.uuid = uuid
        self.path = os.path.join(tempfile.gettempdir(), f"gk_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        sm = [r[0] for r in rows]
        top = max(sm)
        loaded = [s for s in sm if s >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": rows[0][1], "reasons": reasons,
                "samples": len(rows)}


# ---- workload ----------------------------------------------------------------

def shard_seed(rank: int) -> int:
    """Seed of rank `rank`'s shard: every rank filters its own independent
    workload of the same size (weak scaling, no data-path collective)."""
    from paper_2103_14978_gb300 import synth
    return synth.SEED_BASE + 1 + 1000 * rank


def reduce_max(x: float, world: int, device) -> float:
    """The slowest rank's figure: all-reduce MAX over the ranks (nccl on the
    GPUs, gloo in the CPU tests); the value itself at world size 1."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(pairs_per_step: int, world: int, steps: int, max_ms: float) -> float:
    """Whole-job Gpairs/s: the pairs every rank filtered in `steps` steps over
    the slowest rank's time."""
    return pairs_per_step * world * steps / (max_ms * 1e-3) / 1e9


def make_workload(scale: float, rank: int):
    from paper_2103_14978_gb300 import synth
    return synth.config2(scale=scale, seed=shard_seed(rank))


def kernel_source_hash(kind: str = "per_pair") -> str:
    """Hash of a filter kernel's sources (kernel body, instantiation units,
    shared declarations): a recorded traffic figure is only reported while
    these are unchanged.  kind: "per_pair" (filter.cuh, filter_w*.cu) or
    "sliced" (sliced.cuh, sliced_kernels.cuh, sliced_m*.cu)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2103_14978_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if kind == "sliced":
            take = name in ("sliced.cuh", "sliced_kernels.cuh", "gk_internal.cuh") or (
                name.startswith("sliced_m") and name.endswith(".cu"))
        else:
            take = name == "filter.cuh" or name == "gk_internal.cuh" or (
                name.startswith("filter_w") and name.endswith(".cu"))
        if take:
            h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, kind: str = "per_pair"):
    """DRAM bytes per filter launch from the committed ncu summary, if it was
    taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "filter_traffic.json" if kind == "per_pair" else "sliced_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != kernel_source_hash(kind):
        return None
    return rec.get("per_launch", {}).get(workload)


# ---- CPU oracle (baseline and reference arm) ------------------------------

def oracle_sample(w, n: int, seed: int = 7):
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.n_pairs, size=min(n, w.n_pairs), replace=False))
    return idx


def time_oracle(w, idx, es):
    from oracle import oracle as O
    pr, po = w.pair_read[idx], w.pair_off[idx]
    t0 = time.perf_counter()
    threads = 0
    for e in es:
        _, _, threads = O.filter_batch(w.reads, w.read_start, w.read_len, w.ref, pr, po, e)
    return time.perf_counter() - t0, threads


def calibrated_sample(w, target_s: float):
    probe = oracle_sample(w, 20_000, seed=11)
    t, _ = time_oracle(w, probe, E_SWEEP)
    n = int(probe.size * max(0.05, target_s / max(t, 1e-3)))
    return max(1000, min(n, w.n_pairs))


def cpu_baseline(w, target_s: float):
    n = calibrated_sample(w, target_s)
    idx = oracle_sample(w, n)
    t, threads = time_oracle(w, idx, E_SWEEP)
    return {"value": idx.size * len(E_SWEEP) / t / 1e9, "unit": "Gpairs/s", "cores": threads,
            "kind": "oracle",
            "sample": f"{idx.size} seeded-random pairs of the 20M-pair 100 bp workload x e=0..10 "
                      f"({idx.size * len(E_SWEEP)} filtrations, {t:.1f} s)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = make_workload(args.scale, 0)
    n = calibrated_sample(w, 4.0)
    times = []
    threads = 0
    for step in range(args.warmup + args.steps):
        idx = oracle_sample(w, n, seed=100 + step)
        t, threads = time_oracle(w, idx, E_SWEEP)
        if step >= args.warmup:
            times.append(t)
    per_step = n * len(E_SWEEP)
    value = per_step * len(times) / sum(times) / 1e9
    line = {
        "metric": "filtered pairs/s (x10^9), 100 bp, e sweep 0..10", "value": value, "unit": "Gpairs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic", "impl": "reference",
        "config": {"workload": "config 2: 100 bp, 5M reads x 4 candidates, 100 Mbp genome, e=0..10",
                   "sample_pairs_per_step": n, "pairs_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": "Gpairs/s", "cores": threads, "kind": "oracle",
                         "sample": f"{n} seeded-random pairs per step x e=0..10"},
        "e2e": {"value": value, "unit": "Gpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- the GPU arm ---------------------------------------------------------------

def probe_alu(torch, gk, stream, every=False):
    """Measured integer issue rate of the filter's mix (ops/s)."""
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads, iters = sms * 8, 256, 4096
    out = {}
    kinds = [(0, "lop3"), (1, "shf"), (2, "mix")]
    if every:
        kinds += [(3, "imad"), (4, "lop3+imad"), (5, "iadd"), (6, "lop3+iadd"), (7, "shf+imad"),
                  (8, "addc"), (9, "lop3+addc"), (10, "wide"), (11, "lop3+wide"), (12, "lop3x3+wide"),
                  (13, "mulhi+lop3"), (14, "funnel_fma+lop3")]
    for kind, name in kinds:
        gk.gk_probe_alu(kind, 64, blocks, threads, sink, stream)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        gk.gk_probe_alu(kind, iters, blocks, threads, sink, stream)
        e.record(stream)
        e.synchronize()
        ms = s.elapsed_time(e)
        out[name] = blocks * threads * iters * 64 / (ms * 1e-3)
    return out


def run_mine(args):
    import torch
    import torch.distributed as dist

    from paper_2103_14978_gb300 import build, device_data as dd, gk

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    gk.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    stream = torch.cuda.Stream()

    w = make_workload(args.scale, rank)
    m = 100
    c = w.n_pairs / w.n_reads
    ref = gk.gk_load_reference(w.ref)
    # Inputs resident in HBM: ASCII reads (encoded every step), pairs.
    asc = torch.from_numpy(w.reads).to(dev)
    sw = gk.words_for(m)
    packed = torch.empty(w.n_reads * sw * 2, dtype=torch.int32, device=dev)
    nflag = torch.empty(w.n_reads, dtype=torch.uint8, device=dev)
    pairs = dd.upload_pairs(w.pair_read, w.pair_off, None, dev)
    accept = torch.empty(w.n_pairs, dtype=torch.uint8, device=dev)
    edits = torch.empty(w.n_pairs, dtype=torch.int16, device=dev)
    torch.cuda.synchronize()

    sliced_ok = all(gk.sliced_supported(m, e) for e in E_SWEEP)
    sbuf = torch.empty(gk.gk_sliced_bytes(w.n_pairs, m), dtype=torch.uint8, device=dev) if sliced_ok else None

    def encode():
        gk.gk_encode(asc, w.n_reads, w.stride, fixed_len=m, stride_words=sw, packed=packed, nflag=nflag,
                     stream=stream)

    def step_pp(ev=None):
        """Per-pair kernels: device encode, then one gk_filter per threshold."""
        encode()
        for i, e in enumerate(E_SWEEP):
            if ev is not None:
                ev[i][0].record(stream)
            gk.gk_filter(ref, packed, sw, w.n_reads, nflag, m, pairs.pair_read, pairs.pair_off, e,
                         accept=accept, edits=edits, stream=stream)
            if ev is not None:
                ev[i][1].record(stream)

    def step_sl(ev=None):
        """Bit-sliced, one launch per threshold: device encode, the batch
        sliced once (ev[0]), then one gk_filter_sliced per threshold."""
        encode()
        if ev is not None:
            ev[0][0].record(stream)
        gk.gk_slice(ref, packed, sw, w.n_reads, nflag, m, pairs.pair_read, pairs.pair_off, out=sbuf,
                    stream=stream)
        if ev is not None:
            ev[0][1].record(stream)
        for i, e in enumerate(E_SWEEP):
            if ev is not None:
                ev[i + 1][0].record(stream)
            gk.gk_filter_sliced(sbuf, w.n_pairs, m, e, accept=accept, edits=edits, stream=stream)
            if ev is not None:
                ev[i + 1][1].record(stream)

    contiguous = E_SWEEP == list(range(E_SWEEP[0], E_SWEEP[-1] + 1))
    launches = sweep_launches(E_SWEEP, m) if contiguous else []
    n_th = len(E_SWEEP)
    if sliced_ok and contiguous:
        sw_acc = torch.empty(n_th * w.n_pairs, dtype=torch.uint8, device=dev)
        sw_ed = torch.empty(n_th * w.n_pairs, dtype=torch.int16, device=dev)

    sweep_ok = contiguous and all(min(e, m - 1) <= gk.GK_SWEEP_MAX_SHIFT for e in E_SWEEP)
    if sweep_ok:
        ps_acc = torch.empty(n_th * w.n_pairs, dtype=torch.uint8, device=dev)
        ps_ed = torch.empty(n_th * w.n_pairs, dtype=torch.int16, device=dev)

    def step_ps(ev=None):
        """Per-pair sweep: device encode (ev[0]), then one gk_filter_sweep
        (ev[1]): every threshold's results, threshold-major, each pair's
        masks built once up to the largest threshold."""
        if ev is not None:
            ev[0][0].record(stream)
        encode()
        if ev is not None:
            ev[0][1].record(stream)
            ev[1][0].record(stream)
        gk.gk_filter_sweep(ref, packed, sw, w.n_reads, nflag, m, pairs.pair_read, pairs.pair_off, E_SWEEP[0],
                           E_SWEEP[-1], accept=ps_acc, edits=ps_ed, out_stride=w.n_pairs, stream=stream)
        if ev is not None:
            ev[1][1].record(stream)

    def step_sw(ev=None):
        """Bit-sliced sweep: device encode (ev[0]), the batch sliced once
        (ev[1]), then one gk_filter_sliced_sweep per launch range (ev[2..]):
        every threshold's results, threshold-major."""
        if ev is not None:
            ev[0][0].record(stream)
        encode()
        if ev is not None:
            ev[0][1].record(stream)
            ev[1][0].record(stream)
        gk.gk_slice(ref, packed, sw, w.n_reads, nflag, m, pairs.pair_read, pairs.pair_off, out=sbuf,
                    stream=stream)
        if ev is not None:
            ev[1][1].record(stream)
        for i, (lo, hi, _, _) in enumerate(launches):
            if ev is not None:
                ev[2 + i][0].record(stream)
            o = (lo - E_SWEEP[0]) * w.n_pairs
            gk.gk_filter_sliced_sweep(sbuf, w.n_pairs, m, lo, hi, accept=sw_acc[o:], edits=sw_ed[o:],
                                      out_stride=w.n_pairs, stream=stream)
            if ev is not None:
                ev[2 + i][1].record(stream)

    def timed(fn, steps, n_seg, clocks=None):
        """W untimed steps, then `steps` steps between two events on the
        launching stream, a barrier and a synchronize on both sides.  Returns
        the total ms (slowest rank), each segment's mean ms (events around
        the launches) and the clock record."""
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
                for _ in range(n_seg)] for _ in range(steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if clocks is not None:
            clocks.start()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0.record(stream)
        for k in range(steps):
            fn(evs[k])
        t1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clk = clocks.stop() if clocks is not None else None
        total = reduce_max(t0.elapsed_time(t1), world, dev)
        seg = [statistics.mean(evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(steps)) for i in range(n_seg)]
        return total, seg, clk

    uuid = None
    try:
        uuid = "GPU-" + str(props.uuid)
    except Exception:
        pass
    pairs_per_step = w.n_pairs * len(E_SWEEP)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_basis = f"{SM_COUNT} SMs x {ALU_LANES_PER_SM_CLK:.0f} int lanes/clk x {SM_MAX_MHZ:.0f} MHz"

    def per_pair_roofline(per_e_ms):
        """Word formulation: algorithmic ops per launch summed over the sweep,
        over the summed CUDA-event durations of those launches."""
        ops = sum(w.n_pairs * ops_per_pair(m, e) for e in E_SWEEP)
        tops = ops / (sum(per_e_ms) * 1e-3) / 1e12
        bpp = bytes_per_pair(m, c, False)
        gbs = w.n_pairs * bpp * len(E_SWEEP) / (sum(per_e_ms) * 1e-3) / 1e9
        # Per threshold: the launch against the slower of its bytes at the
        # HBM peak and its word-formulation ops at the integer peak.
        per_e = {}
        for e, ms in zip(E_SWEEP, per_e_ms):
            ceil = min(hbm_peak * 1e9 / bpp, ALU_PEAK_TOPS * 1e12 / ops_per_pair(m, e))
            rate = w.n_pairs / (ms * 1e-3)
            per_e[str(e)] = {"gpairs_s": rate / 1e9, "roofline_gpairs_s": ceil / 1e9, "frac": rate / ceil}
        return {"bound": "alu", "achieved": tops, "peak": ALU_PEAK_TOPS, "unit": "Tops/s",
                "frac": tops / ALU_PEAK_TOPS, "traffic": recorded_traffic("c2-100bp-e0..10"),
                "kernel": ("filter_pair2_kernel<W, 4, K> (e 0-2, two pairs per thread, shift count fixed at "
                           "compile time) | filter_pair2_kernel<W, 2> (e 3-10)"),
                "ops_basis": "W*(9 + 22e + 4) per pair (word formulation)", "peak_basis": peak_basis,
                "bytes_side": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak,
                               "bytes_per_pair": bpp},
                "per_e_of_roofline": per_e}

    def sliced_roofline(per_e_ms, slice_ms):
        """Bit-sliced formulation: its algorithmic ops and bytes per launch,
        summed over the sweep, over the summed launch durations; 'combined'
        holds the roofline time (each launch at the slower of its ops at the
        integer peak and its bytes at the HBM peak) against the measured one."""
        ops = sum(w.n_pairs * sliced_ops_per_pair(m, e) for e in E_SWEEP)
        bts = w.n_pairs * sliced_bytes_per_pair(m) * len(E_SWEEP)
        t = sum(per_e_ms)
        tops = ops / (t * 1e-3) / 1e12
        gbs = bts / (t * 1e-3) / 1e9
        roof_ms = 1e3 * sum(max(w.n_pairs * sliced_ops_per_pair(m, e) / (ALU_PEAK_TOPS * 1e12),
                                w.n_pairs * sliced_bytes_per_pair(m) / (hbm_peak * 1e9)) for e in E_SWEEP)
        return {"bound": "alu", "achieved": tops, "peak": ALU_PEAK_TOPS, "unit": "Tops/s",
                "frac": tops / ALU_PEAK_TOPS, "traffic": recorded_traffic("c2-100bp-e0..10", kind="sliced"),
                "kernel": f"sliced_filter_kernel<K, K, {m}> (K = e = {E_SWEEP[0]}..{E_SWEEP[-1]})",
                "ops_basis": "m*(8K + 10)/32 per pair (bit-sliced formulation)", "peak_basis": peak_basis,
                "bytes_side": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak,
                               "bytes_per_pair": sliced_bytes_per_pair(m)},
                "combined": {"roofline_ms": roof_ms, "measured_ms": t, "frac": roof_ms / t},
                "slice_ms": slice_ms}

    def sweep_roofline(range_ms, encode_ms, slice_ms):
        """The sweep launches: their algorithmic ops (sweep_ops_per_pair) and
        bytes (sweep_bytes_per_pair) over their summed CUDA-event durations;
        'combined' holds the roofline time (each launch at the slower of its
        ops at the integer peak and its bytes at the HBM peak) against the
        measured one; 'survey_basis' the same time against the per-filtration
        counts of the word formulation (each threshold a separate pass)."""
        t = sum(range_ms)
        ops = sum(w.n_pairs * sweep_ops_per_pair(m, klo, khi) for _, _, klo, khi in launches)
        bts = sum(w.n_pairs * sweep_bytes_per_pair(m, hi - lo + 1) for lo, hi, _, _ in launches)
        tops = ops / (t * 1e-3) / 1e12
        gbs = bts / (t * 1e-3) / 1e9
        roof_ms = 1e3 * sum(max(w.n_pairs * sweep_ops_per_pair(m, klo, khi) / (ALU_PEAK_TOPS * 1e12),
                                w.n_pairs * sweep_bytes_per_pair(m, hi - lo + 1) / (hbm_peak * 1e9))
                            for lo, hi, klo, khi in launches)
        survey_b = w.n_pairs * bytes_per_pair(m, c, False) * n_th
        survey_ops = sum(w.n_pairs * ops_per_pair(m, e) for e in E_SWEEP)
        names = [f"sliced_filter_kernel<{klo}, {khi}, {m}>" for _, _, klo, khi in launches]
        return {"bound": "alu", "achieved": tops, "peak": ALU_PEAK_TOPS, "unit": "Tops/s",
                "frac": tops / ALU_PEAK_TOPS, "traffic": recorded_traffic("c2-100bp-sweep", kind="sliced"),
                "kernel": " + ".join(names) + " (one launch per shift-count range)",
                "ops_basis": "m*(4(2*khi+1) + 6(khi-klo+1))/32 per pair and launch (bit-sliced sweep: each mask "
                             "once per launch, erosion + count per threshold)",
                "peak_basis": peak_basis,
                "per_launch_ms": {f"{lo}-{hi}": x for (lo, hi, _, _), x in zip(launches, range_ms)},
                "bytes_side": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak,
                               "bytes_per_pair": bts / w.n_pairs,
                               "basis": "planes once per launch (m/2 + 0.25 B) + accept and count per threshold"},
                "combined": {"roofline_ms": roof_ms, "measured_ms": t, "frac": roof_ms / t},
                "survey_basis": {
                    "bytes_per_filtration": bytes_per_pair(m, c, False),
                    "hbm_frac": survey_b / (t * 1e-3) / 1e9 / hbm_peak,
                    "word_ops_x_alu_peak": survey_ops / (t * 1e-3) / 1e12 / ALU_PEAK_TOPS,
                    "note": "per-filtration counts (every threshold reading its inputs and building its masks "
                            "anew); the sweep shares both across the thresholds, so these exceed 1"},
                "encode_ms": encode_ms, "slice_ms": slice_ms,
                "step": step_roofline(roof_ms, encode_ms + slice_ms + t, slice_pass=True)}

    W_m = -(-m // 32)
    enc_bytes = w.n_reads * (m + 8 * W_m + 1)  # ASCII rows in, planes + N flag out

    def step_roofline(kernels_roof_ms, measured_ms, slice_pass=False):
        """The whole step against its roofline time: the filter launches'
        roofline plus the encoder's bytes (and the slice pass's: the pair's
        inputs read, the planes written) at the HBM peak."""
        extra = enc_bytes
        if slice_pass:
            extra += w.n_pairs * (bytes_per_pair(m, c, False) - 3 + sliced_bytes_per_pair(m) - 3)
        roof = kernels_roof_ms + 1e3 * extra / (hbm_peak * 1e9)
        return {"roofline_ms": roof, "measured_ms": measured_ms, "frac": roof / measured_ms,
                "basis": "filter launches at the slower of their ops (ALU peak) and bytes (HBM peak), plus "
                         "the encoder's bytes" + (" and the slice pass's bytes" if slice_pass else "") +
                         " at the HBM peak"}

    def pp_sweep_roofline(sweep_ms, encode_ms):
        """The per-pair sweep launch: its algorithmic ops (pp_sweep_ops_per_pair)
        and bytes (pp_sweep_bytes_per_pair) over its CUDA-event duration;
        'survey_basis' the same time against the per-filtration counts (each
        threshold a separate pass over its inputs and masks)."""
        ops = w.n_pairs * pp_sweep_ops_per_pair(m, E_SWEEP[0], E_SWEEP[-1])
        bts = w.n_pairs * pp_sweep_bytes_per_pair(m, c, n_th)
        tops = ops / (sweep_ms * 1e-3) / 1e12
        gbs = bts / (sweep_ms * 1e-3) / 1e9
        survey_b = w.n_pairs * bytes_per_pair(m, c, False) * n_th
        survey_ops = sum(w.n_pairs * ops_per_pair(m, e) for e in E_SWEEP)
        W = -(-m // 32)
        kern = f"filter_pair2_kernel<{W}, 3>" if W <= 4 else f"filter_kernel<{W}, 3, false>"
        return {"bound": "alu", "achieved": tops, "peak": ALU_PEAK_TOPS, "unit": "Tops/s",
                "frac": tops / ALU_PEAK_TOPS, "traffic": recorded_traffic("c2-100bp-sweep", kind="per_pair"),
                "kernel": kern + " (gk_filter_sweep, one launch for every threshold)",
                "ops_basis": "W*(9 + 22*K + 4*n_thresholds) per pair, K = min(e_hi, m-1): the word formulation's "
                             "masks once up to the largest threshold, the count per threshold",
                "peak_basis": peak_basis, "launch_ms": sweep_ms,
                "bytes_side": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak,
                               "bytes_per_pair": bts / w.n_pairs,
                               "basis": "the pair's inputs once (offset, read id, read, window, N bits) + "
                                        "accept and count per threshold"},
                "survey_basis": {
                    "bytes_per_filtration": bytes_per_pair(m, c, False),
                    "hbm_frac": survey_b / (sweep_ms * 1e-3) / 1e9 / hbm_peak,
                    "word_ops_x_alu_peak": survey_ops / (sweep_ms * 1e-3) / 1e12 / ALU_PEAK_TOPS,
                    "note": "per-filtration counts (every threshold reading its inputs and building its masks "
                            "anew); the sweep shares both across the thresholds, so these exceed 1"},
                "encode_ms": encode_ms,
                "step": step_roofline(1e3 * max(ops / (ALU_PEAK_TOPS * 1e12), bts / (hbm_peak * 1e9)),
                                      encode_ms + sweep_ms)}

    probe = probe_alu(torch, gk, stream, args.probe_all)
    clocks = ClockSampler(uuid)
    per_threshold = None
    per_pair = None
    sliced_sweep = None
    side_steps = max(3, min(args.steps, 20))
    if sweep_ok:
        total_ms, seg, clk = timed(step_ps, args.steps, 2, clocks)
        roofline = pp_sweep_roofline(seg[1], seg[0])
        per_e_ms = None
        step_desc = (f"device encode + one gk_filter_sweep launch over e = {E_SWEEP[0]}..{E_SWEEP[-1]}: each "
                     f"pair's masks are built once up to the largest threshold and every threshold's count is "
                     f"taken from the running AND on the way")
        launches_per_step = 2
    if sliced_ok and contiguous:
        if sweep_ok:
            sw_total, sw_seg, _ = timed(step_sw, side_steps, 2 + len(launches))
            sliced_sweep = {
                "gpairs_s": whole_job_rate(pairs_per_step, world, side_steps, sw_total),
                "ms_per_step": sw_total / side_steps, "steps": side_steps,
                "step": (f"device encode + slice once + {len(launches)} gk_filter_sliced_sweep launches "
                         f"({', '.join(f'e {lo}..{hi}' for lo, hi, _, _ in launches)})"),
                "roofline": sweep_roofline(sw_seg[2:], sw_seg[0], sw_seg[1])}
        else:
            total_ms, seg, clk = timed(step_sw, args.steps, 2 + len(launches), clocks)
            roofline = sweep_roofline(seg[2:], seg[0], seg[1])
            per_e_ms = None
            step_desc = (f"device encode + slice once + {len(launches)} gk_filter_sliced_sweep launches "
                         f"({', '.join(f'e {lo}..{hi}' for lo, hi, _, _ in launches)}): the masks of threshold e "
                         f"are shared with every larger threshold of its launch, the planes read once per launch")
            launches_per_step = 2 + len(launches)
        sl_total, sl_seg, _ = timed(step_sl, side_steps, n_th + 1)
        per_threshold = {"gpairs_s": whole_job_rate(pairs_per_step, world, side_steps, sl_total),
                         "ms_per_step": sl_total / side_steps, "steps": side_steps,
                         "step": "device encode + slice once + one gk_filter_sliced per threshold",
                         "per_e_gpairs_s": {str(e): w.n_pairs / (t * 1e-3) / 1e9 for e, t in zip(E_SWEEP, sl_seg[1:])},
                         "roofline": sliced_roofline(sl_seg[1:], sl_seg[0])}
        per_threshold["roofline"]["survey_basis"] = {
            "bytes_per_filtration": bytes_per_pair(m, c, False),
            "hbm_frac": w.n_pairs * bytes_per_pair(m, c, False) * n_th / (sum(sl_seg[1:]) * 1e-3) / 1e9 / hbm_peak}
    elif sliced_ok and not sweep_ok:
        total_ms, seg, clk = timed(step_sl, args.steps, n_th + 1, clocks)
        per_e_ms = seg[1:]
        roofline = sliced_roofline(per_e_ms, seg[0])
        step_desc = "device encode + slice once + one sliced filter launch per threshold"
        launches_per_step = 2 + n_th
    elif not sweep_ok:
        total_ms, seg, clk = timed(step_pp, args.steps, n_th, clocks)
        per_e_ms = seg
        roofline = per_pair_roofline(per_e_ms)
        step_desc = "device encode + one filter launch per threshold"
        launches_per_step = 1 + n_th
    if sliced_ok or sweep_ok:
        pp_steps = max(3, min(args.steps, 20))
        pp_total, pp_seg, _ = timed(step_pp, pp_steps, n_th)
        per_pair = {"gpairs_s": whole_job_rate(pairs_per_step, world, pp_steps, pp_total),
                    "ms_per_step": pp_total / pp_steps, "steps": pp_steps,
                    "step": "device encode + one gk_filter (per-pair kernels) per threshold",
                    "per_e_gpairs_s": {str(e): w.n_pairs / (t * 1e-3) / 1e9 for e, t in zip(E_SWEEP, pp_seg)},
                    "roofline": per_pair_roofline(pp_seg)}
    elapsed_ms = total_ms
    value = whole_job_rate(pairs_per_step, world, args.steps, elapsed_ms)
    roofline["probe_measured_tops"] = {k: v / 1e12 for k, v in probe.items()}

    # the paper's device-encoded mode at one threshold (Table 2's e = 2 and 5):
    # ASCII reads encoded inside the filter kernel (gk_filter_ascii) against
    # the encoder pass followed by gk_filter
    device_encoded = {}
    for e in (0, 2, 5):
        def sep(e=e):
            gk.gk_encode(asc, w.n_reads, w.stride, fixed_len=m, stride_words=sw, packed=packed, nflag=nflag,
                         stream=stream)
            gk.gk_filter(ref, packed, sw, w.n_reads, nflag, m, pairs.pair_read, pairs.pair_off, e, accept=accept,
                         edits=edits, stream=stream)

        def fused(e=e):
            gk.gk_filter_ascii(ref, asc, w.stride, w.n_reads, m, pairs.pair_read, pairs.pair_off, e, accept=accept,
                               edits=edits, stream=stream)

        for f in (sep, fused, sep, fused):
            f()
        device_encoded[f"e{e}"] = {
            "fused_gpairs_s": w.n_pairs / (time_events(torch, fused, 20, stream) * 1e-3) / 1e9,
            "encode_then_filter_gpairs_s": w.n_pairs / (time_events(torch, sep, 20, stream) * 1e-3) / 1e9}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, gk, dd, w, ref, m, sw, stream, args, world)
        split = run_e2e(torch, gk, dd, w, ref, m, sw, stream, args, world, result_byte=False)
        e2e["split_results"] = {k: split[k] for k in ("value", "d2h_bytes_per_step", "ms_per_step",
                                                     "windows_ms_per_step", "results")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds)

    in_mib = (asc.numel() + 8 * w.n_pairs) / 2**20
    extra = {}
    if world == 1 and not args.no_extra:
        # The other configurations, each on its own inputs (the 20M-pair
        # config 2 buffers are released first).
        del asc, packed, nflag, pairs, accept, edits, sbuf
        if sliced_ok and contiguous:
            del sw_acc, sw_ed
        if sweep_ok:
            del ps_acc, ps_ed
        ref.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        # A configuration that fails records its error in the line instead of
        # taking the other measurements down with it.
        for name, fn in (("c3", lambda: measure_c3(args, hbm_peak)), ("c4", lambda: {"c4": measure_c4(args)}),
                         ("c5", lambda: {"c5": measure_c5(args)})):
            try:
                extra.update(fn())
            except Exception as exc:  # noqa: BLE001
                extra[name + "_error"] = f"{type(exc).__name__}: {exc}"
                print(f"bench: {name} failed: {exc!r}", file=sys.stderr, flush=True)
        extra["extra_configs_wall_s"] = time.perf_counter() - t0

    if rank != 0:
        return
    line = {
        "metric": "filtered pairs/s (x10^9), 100 bp, e sweep 0..10",
        "value": value, "unit": "Gpairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "config 2: 100 bp, 5M reads x 4 candidates, 100 Mbp genome, e=0..10",
                   "pairs": w.n_pairs, "pairs_per_step": pairs_per_step, "read_len": m,
                   "e_sweep": [E_SWEEP[0], E_SWEEP[-1]], "step": step_desc,
                   "l2": f"inputs {in_mib:.0f} MiB per step > L2 "
                         f"(the 25 MiB packed genome stays L2-resident by design)",
                   "parallelism": f"replicas x{world}"},
        "per_e_gpairs_s": (None if per_e_ms is None else
                           {str(e): w.n_pairs / (t * 1e-3) / 1e9 for e, t in zip(E_SWEEP, per_e_ms)}),
        "roofline": roofline,
        "gpu_launches": args.steps * launches_per_step,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "sliced_sweep_step": sliced_sweep,
        "per_threshold_sliced_step": per_threshold,
        "per_pair_step": per_pair,
        "device_encoded_one_threshold": device_encoded,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


E2E_WINDOWS = 3
E2E_MIN_STEPS = 100
E2E_MIN_SECONDS = 1.0


def run_e2e(torch, gk, dd, w, ref, m, sw, stream, args, world, result_byte=True):
    """Same metric through the streamed pipeline of the public API (gk_pipe_*)
    from pinned host buffers: every step copies the ASCII reads and the pairs
    in, encodes them on the device, filters at e = 0..10 and copies every
    result out (one result byte per pair and threshold with
    GK_FLAG_RESULT_BYTE, else accept bytes and 16-bit counts).  Three steps
    are in flight, so one step's copies overlap another's filtering; the
    timed region runs from the first submit to the last step's results in
    host memory (wall clock, slowest rank).  The window is a few hundred ms,
    so it is taken E2E_WINDOWS times back to back and the median reported,
    every window listed beside it."""
    dev = torch.device("cuda", torch.cuda.current_device())
    h_asc = torch.from_numpy(w.reads).pin_memory()
    # The candidates of a read sit side by side: they travel as one start per
    # read (GK_PIPE_READ_STARTS) instead of a read id per pair.
    starts = bool(np.all(np.diff(w.pair_read.astype(np.int64)) >= 0))
    link = np.searchsorted(w.pair_read, np.arange(w.n_reads)).astype(np.uint32) if starts else w.pair_read
    h_pr = dd.as_i32(link).pin_memory()
    h_po = dd.as_i32(w.pair_off).pin_memory()
    n = w.n_pairs
    slots = 3
    outs = [(torch.empty(len(E_SWEEP) * n, dtype=torch.uint8).pin_memory(),
             None if result_byte else torch.empty(len(E_SWEEP) * n, dtype=torch.int16).pin_memory())
            for _ in range(slots)]
    pipe = gk.Pipe(ref, w.n_reads, w.stride, m, n, E_SWEEP, n_slots=slots,
                   flags=(gk.GK_FLAG_RESULT_BYTE if result_byte else 0) | (gk.GK_PIPE_READ_STARTS if starts else 0))

    def run(k_steps):
        tickets = []
        for k in range(k_steps):
            if k >= slots:  # the step's host result buffers are free again
                pipe.wait(tickets[k - slots])
            acc, ed = outs[k % slots]
            tickets.append(pipe.submit(h_asc, w.n_reads, h_pr, h_po, acc, ed))
        pipe.wait(tickets[-1])

    run(2 * slots)  # every slot's buffers used once before the timed region
    # Windows of at least E2E_MIN_STEPS steps and E2E_MIN_SECONDS each, sized
    # from one short untimed run, so that one stall of the shared host link
    # cannot move the median.
    t_est = time.perf_counter()
    run(2 * slots)
    est_ms = (time.perf_counter() - t_est) * 1e3 / (2 * slots)
    steps = max(E2E_MIN_STEPS, int(E2E_MIN_SECONDS * 1e3 / max(est_ms, 1e-3)) + 1)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([steps], dtype=torch.int64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        steps = int(t.item())
    windows = []
    for _ in range(E2E_WINDOWS):
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        t0 = time.perf_counter()
        run(steps)
        wall_ms = (time.perf_counter() - t0) * 1e3
        windows.append(reduce_max(wall_ms, world, dev))
    ms = statistics.median(windows)
    pipe.close()
    h2d = h_asc.numel() + 4 * n + 4 * h_pr.numel()
    d2h = len(E_SWEEP) * n * (1 if result_byte else 3)
    fmt = ("one result byte per pair and threshold (count capped at 253 or a sentinel; accept = byte <= e "
           "or undefined)" if result_byte else "accept byte + 16-bit count per pair and threshold")
    return {"value": whole_job_rate(n * len(E_SWEEP), world, steps, ms), "unit": "Gpairs/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps, "ms_per_step": ms / steps,
            "windows_ms_per_step": [x / steps for x in windows],
            "timing": f"median of {E2E_WINDOWS} back-to-back windows of {steps} steps (at least {E2E_MIN_STEPS} "
                      f"steps and {E2E_MIN_SECONDS:g} s each), each the slowest rank's wall clock (the host link "
                      f"is shared with the machine's other GPUs)",
            "path": "pinned host ASCII reads + pairs -> gk_pipe (copy-in, device encode + one gk_filter_sweep "
                    "over the thresholds, copy-out on three streams, 3 steps in flight) -> results in pinned "
                    "host memory",
            "pairs_in": ("offset per pair + one start per read (GK_PIPE_READ_STARTS)" if starts
                         else "offset + read id per pair"),
            "results": fmt}


def parse_es(spec: str):
    out = []
    for part in spec.split(","):
        if "-" in part:
            a, b = part.split("-")
            out += list(range(int(a), int(b) + 1))
        else:
            out.append(int(part))
    return out


def time_events(torch, fn, steps, stream):
    """Mean ms of fn() over `steps` calls, CUDA events on `stream`."""
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record(stream)
    for _ in range(steps):
        fn()
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e) / steps


def measure_c3(args, hbm_peak: float) -> dict:
    """Config 3: 10M pairs at 150 bp (e 0..15) and 250 bp (e 0..25), 8-64
    candidates per read, N at 0.1% of genome and read positions.  Three forms
    over the same pairs: the per-pair sweep (one gk_filter_sweep over every
    threshold; the queue skips undefined pairs), the sliced batch (gk_slice
    once, gk_filter_sliced_sweep over the thresholds its shift counts cover,
    gk_filter_sweep above) and the per-pair kernels once per threshold
    (gk_filter); the line's value is the fastest, all reported."""
    import torch

    from paper_2103_14978_gb300 import build, device_data as dd, gk, synth

    build.build()
    stream = torch.cuda.Stream()
    steps, warm = max(3, min(args.steps, 10)), max(1, min(args.warmup, 3))
    out = {}
    for m, e_hi in ((150, 15), (250, 25)):
        w = synth.config3(m, scale=args.scale)
        c = w.n_pairs / w.n_reads
        es = list(range(0, e_hi + 1))
        ref = gk.gk_load_reference(w.ref)
        reads = dd.upload_reads(w.reads, w.read_len, w.stride, stream=stream)
        pairs = dd.upload_pairs(w.pair_read, w.pair_off, None)
        n = w.n_pairs
        acc = torch.empty(n, dtype=torch.uint8, device="cuda")
        ed = torch.empty(n, dtype=torch.int16, device="cuda")

        def timeit(f):
            for _ in range(warm):
                f()
            return time_events(torch, f, steps, stream)

        per_e = {}
        for e in es:
            per_e[e] = timeit(lambda e=e: gk.gk_filter(ref, reads.packed, reads.stride_words, reads.n_reads,
                                                       reads.nflag, m, pairs.pair_read, pairs.pair_off, e,
                                                       accept=acc, edits=ed, stream=stream))
        torch.cuda.synchronize()
        undefined = int((dd.edits_u16(ed) == gk.GK_EDITS_UNDEFINED).sum())
        filtered = n - undefined
        pp_ms = sum(per_e.values())
        pp_ops = sum(filtered * ops_per_pair(m, e) for e in es)
        per_pair = {"gpairs_s": n * len(es) / (pp_ms * 1e-3) / 1e9, "ms": pp_ms,
                    "per_e_gpairs_s": {str(e): n / (t * 1e-3) / 1e9 for e, t in per_e.items()},
                    "alu_frac": pp_ops / (pp_ms * 1e-3) / 1e12 / ALU_PEAK_TOPS,
                    "alu_basis": "W(13 + 22e) per filtered (non-N) pair, word formulation",
                    "survey_bytes_frac": n * bytes_per_pair(m, c, False) * len(es) / (pp_ms * 1e-3) / 1e9 / hbm_peak}
        # per-pair sweep: one launch for every threshold
        psa = torch.empty(len(es) * n, dtype=torch.uint8, device="cuda")
        pse = torch.empty(len(es) * n, dtype=torch.int16, device="cuda")
        ps_ms = timeit(lambda: gk.gk_filter_sweep(ref, reads.packed, reads.stride_words, reads.n_reads, reads.nflag,
                                                  m, pairs.pair_read, pairs.pair_off, es[0], es[-1], accept=psa,
                                                  edits=pse, out_stride=n, stream=stream))
        ps_ops = filtered * pp_sweep_ops_per_pair(m, es[0], es[-1])
        pp_sweep = {"gpairs_s": n * len(es) / (ps_ms * 1e-3) / 1e9, "ms": ps_ms,
                    "form": f"one gk_filter_sweep over e {es[0]}..{es[-1]}",
                    "alu_frac": ps_ops / (ps_ms * 1e-3) / 1e12 / ALU_PEAK_TOPS,
                    "alu_basis": "W(9 + 22K + 4 n_thresholds) per filtered (non-N) pair, K = min(e_hi, m-1)",
                    "bytes_frac": n * pp_sweep_bytes_per_pair(m, c, len(es)) / (ps_ms * 1e-3) / 1e9 / hbm_peak,
                    "survey_bytes_frac": n * bytes_per_pair(m, c, False) * len(es) / (ps_ms * 1e-3) / 1e9 / hbm_peak}
        del psa, pse
        # sliced: slice once, sweep the covered thresholds, the per-pair sweep above
        cover = [e for e in es if gk.sliced_supported(m, e)]
        rest = [e for e in es if e not in cover]
        sbuf = torch.empty(gk.gk_sliced_bytes(n, m), dtype=torch.uint8, device="cuda")
        sacc = torch.empty(len(cover) * n, dtype=torch.uint8, device="cuda")
        sed = torch.empty(len(cover) * n, dtype=torch.int16, device="cuda")
        slice_ms = timeit(lambda: gk.gk_slice(ref, reads.packed, reads.stride_words, reads.n_reads, reads.nflag, m,
                                              pairs.pair_read, pairs.pair_off, out=sbuf, stream=stream))
        launches = sweep_launches(cover, m)
        launch_ms = []
        for lo, hi, _, _ in launches:
            o = (lo - cover[0]) * n
            launch_ms.append(timeit(lambda lo=lo, hi=hi, o=o: gk.gk_filter_sliced_sweep(
                sbuf, n, m, lo, hi, accept=sacc[o:], edits=sed[o:], out_stride=n, stream=stream)))
        rest_ms = 0.0
        if rest:
            ra = torch.empty(len(rest) * n, dtype=torch.uint8, device="cuda")
            rd = torch.empty(len(rest) * n, dtype=torch.int16, device="cuda")
            rest_ms = timeit(lambda: gk.gk_filter_sweep(ref, reads.packed, reads.stride_words, reads.n_reads,
                                                        reads.nflag, m, pairs.pair_read, pairs.pair_off, rest[0],
                                                        rest[-1], accept=ra, edits=rd, out_stride=n, stream=stream))
            del ra, rd
        sl_ms = slice_ms + sum(launch_ms) + rest_ms
        sl_ops = sum(n * sweep_ops_per_pair(m, klo, khi) for _, _, klo, khi in launches)
        sliced = {"gpairs_s": n * len(es) / (sl_ms * 1e-3) / 1e9, "ms": sl_ms, "slice_ms": slice_ms,
                  "form": f"slice once + gk_filter_sliced_sweep for e {cover[0]}..{cover[-1]}"
                          + (f" + gk_filter_sweep for e {rest[0]}..{rest[-1]}" if rest else ""),
                  "per_launch_ms": {f"{lo}-{hi}": t for (lo, hi, _, _), t in zip(launches, launch_ms)},
                  "sweep_alu_frac": sl_ops / (sum(launch_ms) * 1e-3) / 1e12 / ALU_PEAK_TOPS,
                  "alu_basis": "sweep_ops_per_pair over every pair (the sliced kernels filter N pairs too)",
                  "survey_bytes_frac": n * bytes_per_pair(m, c, False) * len(es) / (sl_ms * 1e-3) / 1e9 / hbm_peak}
        forms = {"per_pair_sweep": pp_sweep, "sliced": sliced, "per_pair": per_pair}
        best = max(forms, key=lambda k: forms[k]["gpairs_s"])
        out[f"c3_{m}bp"] = {
            "value": forms[best]["gpairs_s"], "unit": "Gpairs/s", "form": best,
            "pairs": n, "e_sweep": [0, e_hi], "candidates_per_read": c, "undefined_frac": undefined / n,
            "survey_bytes_frac": forms[best]["survey_bytes_frac"], **forms,
            "per_e_gpairs_s": per_pair["per_e_gpairs_s"]}
        ref.close()
        del reads, pairs, acc, ed, sbuf, sacc, sed
        torch.cuda.empty_cache()
    return out


def measure_c4(args) -> dict:
    """Config 4: 50M pairs, lengths U{50..300}, per-pair e = ceil(rate m),
    shuffled: one graph-captured gk_filter_batched (classify, scan, scatter,
    persistent filter) with the autotuner's tiling, against the plain filter
    launched once per read length over the same pairs."""
    import torch

    from paper_2103_14978_gb300 import batch, build, device_data as dd, gk, synth

    build.build()
    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    w = synth.config4(scale=args.scale)
    t_gen = time.perf_counter() - t_gen
    ref = gk.gk_load_reference(w.ref)
    reads = dd.upload_reads(w.reads, w.read_len, w.stride)
    read_len = dd.as_i16(w.read_len).cuda()
    pairs = dd.upload_pairs(w.pair_read, w.pair_off, w.pair_e)
    sig = batch.signature(w.read_len, w.pair_read, w.pair_e)
    results = {}
    if args.tune_seconds > 0:  # autotune on a seeded sample of the pairs
        rng = np.random.default_rng(3)
        samp = np.sort(rng.choice(w.n_pairs, min(w.n_pairs, 4_000_000), replace=False))
        sp = dd.upload_pairs(w.pair_read[samp], w.pair_off[samp], w.pair_e[samp])
        best, results = batch.autotune(ref, reads.packed, reads.stride_words, reads.n_reads, read_len,
                                       reads.nflag, sp.pair_read, sp.pair_off, sp.pair_e, reps=2,
                                       budget_s=args.tune_seconds)
        del sp
    else:
        best = batch.lookup(sig) or batch.DEFAULT_TILING
    bf = batch.BatchedFilter(ref, reads.packed, reads.stride_words, reads.n_reads, read_len, reads.nflag,
                             pairs.pair_read, pairs.pair_off, pairs.pair_e, best)
    bf.capture()
    steps = max(3, min(args.steps, 10))
    for _ in range(max(1, args.warmup)):
        bf.replay()
    batched_ms = time_events(torch, bf.replay, steps, stream)
    m_pair = w.read_len[w.pair_read]
    order = np.argsort(m_pair, kind="stable")
    ms_sorted = m_pair[order]
    bounds = np.flatnonzero(np.diff(ms_sorted)) + 1
    starts = np.concatenate([[0], bounds])
    ends = np.concatenate([bounds, [w.n_pairs]])
    gp = dd.upload_pairs(w.pair_read[order], w.pair_off[order], w.pair_e[order])
    acc = torch.empty(w.n_pairs, dtype=torch.uint8, device="cuda")
    ed = torch.empty(w.n_pairs, dtype=torch.int16, device="cuda")

    def plain():
        for a, b in zip(starts, ends):
            gk.gk_filter(ref, reads.packed, reads.stride_words, reads.n_reads, reads.nflag, int(ms_sorted[a]),
                         gp.pair_read[a:b], gp.pair_off[a:b], gp.pair_e[a:b], accept=acc[a:b], edits=ed[a:b],
                         stream=stream)

    for _ in range(max(1, args.warmup)):
        plain()
    plain_ms = time_events(torch, plain, steps, stream)
    torch.cuda.synchronize()
    inv = torch.from_numpy(np.argsort(order))
    same = bool(torch.equal(acc.cpu()[inv], bf.accept.cpu()) and torch.equal(ed.cpu()[inv], bf.edits.cpu()))
    Wp = (m_pair.astype(np.int64) + 31) // 32
    ek = np.minimum(w.pair_e.astype(np.int64), m_pair.astype(np.int64) - 1)
    ops = float(np.sum(Wp * (13 + 22 * ek)))
    ref.close()
    return {
        "value": w.n_pairs / (batched_ms * 1e-3) / 1e9, "unit": "Gpairs/s", "ms": batched_ms, "steps": steps,
        "pairs": w.n_pairs, "form": "one CUDA-graph replay of gk_filter_batched (classify, scan, scatter, "
                                    "persistent filter)",
        "tiling": {"words_per_thread": best[0], "tile_pairs": best[1], "blocks_per_sm": best[2],
                   "warps_per_block": best[3], "source": "autotuned on a 4M-pair sample" if results else "table"},
        "autotune_candidates_ms": {",".join(map(str, k)): v for k, v in results.items()},
        "plain_per_length": {"value": w.n_pairs / (plain_ms * 1e-3) / 1e9, "ms": plain_ms,
                             "launches": int(len(starts)), "identical_results": same},
        "alu_frac": ops / (batched_ms * 1e-3) / 1e12 / ALU_PEAK_TOPS,
        "alu_basis": "W(13 + 22 min(e, m-1)) per pair, word formulation, over the whole graph",
        "generation_s": t_gen}


def measure_c5(args) -> dict:
    """Config 5: serving.  The 100 Mbp genome stays resident; requests of
    log-uniform 1k-1M pairs, m in {100, 150, 250}, one e = ceil(rate m) per
    request, arrive as a Poisson stream.  First the server's own saturated
    throughput (arrivals far above it), then offered loads of 0.5 / 0.8 /
    0.95 of that, each with `level_seconds` of arrivals; latency and rates
    over the requests that arrive after the first second."""
    import torch

    from paper_2103_14978_gb300 import build, gk, serve, synth

    build.build()
    ref = synth.reference()
    gkref = gk.gk_load_reference(ref)
    lengths, rates = (100, 150, 250), (0.02, 0.05, 0.10)
    # Requests arrive back to back in per-length pinned buffers (sequential
    # cuts, rows at each length's own stride); the server has one lane per
    # stride.
    pool = serve.RequestPool(ref, lengths=lengths, reads_per_len=260_000, stride_words=None, sequential=True,
                             pair_format="starts", compact_reads=True)
    lanes = tuple(sorted({pool.by_len[m]["sw"] for m in lengths}))
    stream = torch.cuda.current_stream()
    per_combo = {}  # the plain filter on the mix, every (m, e) equally likely
    for m in lengths:
        p = pool.by_len[m]
        n = p["pair_read"][1].shape[0]
        packed, nflag = p["packed"][0].cuda(), p["nflag"][0].cuda()
        pr, po = p["pair_read"][0].cuda(), p["pair_off"][0].cuda()
        acc = torch.empty(n, dtype=torch.uint8, device="cuda")
        ed = torch.empty(n, dtype=torch.int16, device="cuda")
        for rate in rates:
            e = int(np.ceil(round(rate * m, 9)))
            f = lambda: gk.gk_filter(gkref, packed, p["sw"], p["lens"][1].shape[0], nflag, m, pr, po, e,  # noqa
                                     accept=acc, edits=ed)
            f()
            per_combo[f"{m}bp_e{e}"] = n / (time_events(torch, f, 5, stream) * 1e-3)
    plain = 1.0 / np.mean([1.0 / v for v in per_combo.values()])
    lo, hi = 1_000, 1_000_000
    mean_size = (hi - lo) / np.log(hi / lo)
    # Candidates as one start per read (expanded on the device), results as
    # one byte per pair, three streams: the host link carries about 17 bytes
    # per pair in and 1 out, and a round's copies run while the previous
    # round filters.
    cfg = serve.ServeConfig(mem_cap_bytes=16 << 30, max_round_pairs=args.round_pairs, copy_results=False, lanes=lanes,
                            pair_format="starts", result_bytes=True, n_streams=args.serve_streams)
    ex = serve.GpuExecutor(gkref, cfg)
    skip = 1.0

    def level(rate_pairs_s, seconds, seed, stop=False):
        plan = serve.poisson_plan_for(seconds, rate_pairs_s / mean_size, seed)
        reqs = [pool.request(q["id"], q["m"], q["e"], q["n_pairs"], q["start"], q["arrival"]) for q in plan]
        srv = serve.Server(ex, cfg)
        t0 = time.perf_counter()
        srv.run(reqs, stop_at=seconds if stop else None)
        summ = serve.steady_state_summary(reqs, min(skip, seconds / 2), seconds)
        summ.update({"rounds": srv.rounds_launched, "mean_requests_per_round": float(np.mean(srv.coalesced)),
                     "wall_s": time.perf_counter() - t0, "max_inflight_rounds": srv.max_inflight_seen})
        return summ

    level(0.5 * plain, 1.0, 2103_14978 + 50)  # warm the rings and the pinned pool
    sat = level(1.5 * plain, max(3.0, args.level_seconds / 3), 2103_14978 + 51, stop=True)
    capacity = sat["served_gpairs_s"] * 1e9
    levels = {}
    for load in (0.5, 0.8, 0.95):
        levels[str(load)] = level(load * capacity, args.level_seconds, 2103_14978 + 5 + int(load * 100))
        levels[str(load)]["load"] = load
    # per read: packed row + start (one length per request; N flags only for
    # requests with an N read, none in this pool's reads)
    h2d_pp = float(np.mean([(8 * pool.by_len[m]["sw"] + 4) / pool.cands + 4 for m in lengths]))
    ok = all(abs(v["served_gpairs_s"] / v["offered_gpairs_s"] - 1) < 0.05 for v in levels.values())
    mono = levels["0.5"]["p99_ms"] <= levels["0.8"]["p99_ms"] <= levels["0.95"]["p99_ms"]
    gkref.close()
    return {"unit": "Gpairs/s", "server_saturated_gpairs_s": sat["served_gpairs_s"],
            "saturation_run": sat, "plain_filter_capacity_gpairs_s": plain / 1e9,
            "plain_per_combo_gpairs_s": {k: v / 1e9 for k, v in per_combo.items()},
            "levels": levels, "served_matches_offered": ok, "p99_rises_with_load": mono,
            "method": f"Poisson arrivals for {args.level_seconds:g} s per level at 0.5/0.8/0.95 of the server's "
                      f"saturated throughput (measured first: arrivals at 1.5x the plain filter's capacity, "
                      f"completions counted until the arrivals stop); "
                      f"latency = arrival -> results on the host, over requests arriving after {skip:g} s",
            "lanes": [{"row_words": sw, "read_slots": nr, "pair_slots": npr} for sw, nr, npr in ex.lanes],
            "copies_per_round_last": ex.copies_last_round,
            "streams": cfg.n_streams,
            "host_link_bytes_per_pair": {"in": h2d_pp, "out": 1.0,
                                         "basis": "per read: packed row (8 x row words) + start 4, per pair: "
                                                  "offset 4; one length per request and no N flags for requests "
                                                  "without N (written on the device); 4 candidates per read, "
                                                  "lengths 100/150/250 equally likely"},
            "inputs": "requests received back to back into per-length pinned buffers (rows at each length's "
                      "own stride); a round's copies merge per lane and array; candidates as one start per read "
                      "(gk_expand_pairs), results as one byte per pair (GK_FLAG_RESULT_BYTE)"}


def run_config(args, which: str):
    """One of the other configurations as its own JSON line."""
    import torch  # noqa: F401

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    if which == "c3":
        out = measure_c3(args, float(peaks.get("hbm_gbs", 6800.0)))
    elif which == "c4":
        out = {"c4": measure_c4(args)}
    else:
        out = {"c5": measure_c5(args)}
    print(json.dumps({"metric": f"filtered pairs/s (x10^9), {which}", "n_gpus": 1, "dtype": "u32",
                      "data": "synthetic", **out}), flush=True)


def main():
    global E_SWEEP
    args = parse_args()
    E_SWEEP = parse_es(args.es)
    if args.impl == "reference":
        run_reference(args)
    elif args.config in ("c3", "c4", "c5"):
        run_config(args, args.config)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
