"""Continuous-batching server for the filter: the encoded genome stays
resident, requests (reads + candidate pairs + one threshold) are admitted as
device memory frees up, coalesced into shared launches, and their work
overlaps on two streams.

Memory admission.  At start the server sizes two device rings from the free
device memory (or a cap): read slots (ASCII row, packed planes, length, N
flag) and pair slots (read id, offset, threshold, accept, edits).  A request
is admitted when both rings have room for it, in arrival order; its slots are
released when its launch has completed.  A request larger than the rings is
rejected.

Requests arrive host-encoded (2-bit planes written by gk_encode's host path,
the paper's host-encoded mode, Sec. 3.3): a 100 bp read moves as 32 bytes
instead of 100.  A request's candidates come as one read id per pair, or
(pair_format "starts") as each read's first-candidate index, CSR style: one
32-bit value per read instead of one per pair, expanded on the device by
gk_expand_pairs.  With result_bytes the results return as one byte per pair
(GK_FLAG_RESULT_BYTE) instead of an accept byte and a 16-bit count.

Rounds.  Whenever a stream is free, every admitted request not yet launched
(up to `max_round_pairs` pairs) forms one round: one gk_copy_many call moves
all their inputs host to device (one copy per array per request), one
gk_rebase_pairs moves each request's read ids to its slots and writes its
threshold into its pairs, one gk_filter_batched filters every pair (any mix
of read lengths and thresholds), and one gk_copy_many copies the results back
to pinned host memory.  Two events per round give the device-side and
host-side completion times.

The filter work is entirely in libgk; this module is the scheduler.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

GK_MAX_WORDS = 16


@dataclasses.dataclass
class Request:
    """One request: ``packed`` uint32 reads as gk_encode writes them
    (n_reads x stride_words x 2, the stride of one of the server's lanes),
    ``nflag`` uint8 and ``lens`` uint16 per read, ``pair_off`` uint32 genome
    offsets, one threshold ``e``, and the pairs' reads as either
    ``pair_read`` uint32 read ids (id - ``read_base`` indexes these reads) or
    ``read_start`` uint32 per read (pairs read_start[k] - start_base ..
    read_start[k+1] - start_base - 1 are read k's; the last read's run ends
    at the last pair).  For asynchronous copies the arrays should live in
    pinned host memory.  ``arrival`` is the time (s, from the start of
    ``run``) the request arrives.  Results: ``accept`` and ``edits``, or with
    a result-byte server the result bytes in ``accept`` and ``edits`` None."""

    id: int
    packed: np.ndarray
    nflag: np.ndarray | None
    lens: np.ndarray | None
    pair_read: np.ndarray | None
    pair_off: np.ndarray
    e: int
    arrival: float = 0.0
    max_len: int = -1  # longest read, if known (else computed from lens)
    status: str = "queued"  # queued, admitted, running, done, rejected, cancelled, failed
    error: str = ""
    read_slot: int = -1
    pair_slot: int = -1
    t_admit: float = float("nan")
    t_dispatch: float = float("nan")
    t_device_done: float = float("nan")
    t_done: float = float("nan")
    accept: np.ndarray | None = None
    edits: np.ndarray | None = None
    ascii: np.ndarray | None = None  # the reads' ASCII rows, kept only for checking
    read_base: int = 0  # pair_read - read_base indexes these reads (ids of a larger numbering)
    lane: int = -1
    read_start: np.ndarray | None = None  # CSR form of the pairs' reads (instead of pair_read)
    start_base: int = 0                   # read_start - start_base counts from this request's first pair
    read_len: int = 0                     # with read_start: one length for every read (lens None)

    def __post_init__(self):
        # Sizes and host addresses are read once here: the scheduler handles
        # tens of thousands of requests a second.  n_reads, n_pairs and
        # stride_words (packed words per read row) are plain attributes;
        # host_ptrs[3] is the pair-to-read array of either form.
        if (self.pair_read is None) == (self.read_start is None):
            raise ValueError("a request gives exactly one of pair_read and read_start")
        if self.lens is None or self.nflag is None:
            # One length for all reads and / or no N in any: the device writes
            # the per-read values (starts form only).
            if self.read_start is None or (self.lens is None and self.read_len <= 0):
                raise ValueError("lens / nflag may be left out only with read_start (and read_len for lens)")
        if self.lens is None and self.max_len < 0:
            self.max_len = int(self.read_len)
        self.n_reads = int(self.lens.shape[0] if self.lens is not None else self.read_start.shape[0])
        if self.nflag is not None and self.nflag.shape[0] != self.n_reads:
            raise ValueError("nflag needs one value per read")
        self.n_pairs = int(self.pair_off.shape[0])
        if self.pair_read is not None and self.pair_read.shape[0] != self.n_pairs:
            raise ValueError("pair_read and pair_off differ in length")
        if self.read_start is not None and self.read_start.shape[0] != self.n_reads:
            raise ValueError("read_start needs one value per read")
        self.pair_format = "ids" if self.pair_read is not None else "starts"
        self.stride_words = int(self.packed.size // (2 * self.n_reads)) if self.n_reads else 0
        link = self.pair_read if self.pair_read is not None else self.read_start
        self.host_ptrs = tuple(int(x.__array_interface__["data"][0]) if x is not None else 0
                               for x in (self.packed, self.nflag, self.lens, link, self.pair_off))
        # the per-segment word gk_expand_pairs takes: a shared length, no N
        self.read_info = (int(self.read_len) & 0xFFFF if self.lens is None else 0) | (
            0x10000 if self.nflag is None else 0)

    def cancel(self) -> bool:
        """Cancel a request that has not been admitted yet."""
        if self.status == "queued":
            self.status = "cancelled"
            return True
        return False


def encode_request(rid: int, reads_ascii: np.ndarray, lens: np.ndarray, pair_read: np.ndarray,
                   pair_off: np.ndarray, e: int, stride_words: int = 8, arrival: float = 0.0) -> Request:
    """Build a request from ASCII reads (n_reads x row bytes) with the
    library's host encoder."""
    import torch

    from . import gk

    n = int(lens.shape[0])
    rows = np.ascontiguousarray(reads_ascii, np.uint8).reshape(n, -1)
    packed, nflag = gk.gk_encode(torch.from_numpy(rows.reshape(-1)), n, rows.shape[1],
                                 lens=torch.from_numpy(np.ascontiguousarray(lens, np.uint16).view(np.int16)),
                                 stride_words=stride_words)
    return Request(rid, packed.numpy().view(np.uint32), nflag.numpy(), np.ascontiguousarray(lens, np.uint16),
                   np.ascontiguousarray(pair_read, np.uint32), np.ascontiguousarray(pair_off, np.uint32), int(e),
                   arrival=arrival, max_len=int(lens.max(initial=0)))


class FifoRing:
    """Contiguous slot ranges handed out and released in FIFO order from a
    circular buffer of `size` slots (an allocation never wraps; the tail gap
    it skips is free again once the older allocations are released)."""

    def __init__(self, size: int):
        self.size = int(size)
        self.live = collections.deque()  # (start, n) in allocation order
        self.head = 0

    def free_slots(self) -> int:
        return self.size - sum(n for _, n in self.live)

    def alloc(self, n: int):
        n = int(n)
        if n <= 0 or n > self.size:
            raise ValueError(f"allocation of {n} slots in a ring of {self.size}")
        if not self.live:
            self.head = 0
            start = 0
        else:
            tail = self.live[0][0]
            if self.head > tail:
                if self.head + n <= self.size:
                    start = self.head
                elif n <= tail:
                    start = 0
                else:
                    return None
            elif self.head < tail:
                if self.head + n <= tail:
                    start = self.head
                else:
                    return None
            else:  # head == tail with live allocations: full
                return None
        self.live.append((start, n))
        self.head = start + n
        return start

    def undo_last(self):
        start, _ = self.live.pop()
        self.head = start if self.live else 0

    def release_oldest(self):
        self.live.popleft()
        if not self.live:
            self.head = 0


@dataclasses.dataclass
class ServeConfig:
    stride_words: int = 8             # packed words per read (reads up to 32 x this), one lane
    lanes: tuple | None = None        # several lanes: their row strides (words per read); a request
                                      # goes to the lane of its own row stride
    max_read_len: int = 256
    pairs_per_read: float = 4.0       # expected candidates per read, to split the memory budget
    mem_fraction: float = 0.25        # share of the free device memory the rings may take
    mem_cap_bytes: int | None = None  # hard cap on the rings' memory (simulated small device)
    max_round_pairs: int = 4_000_000
    n_streams: int = 2
    tiling: tuple = (1, 256, 3, 8)
    round_timeout_s: float = 30.0     # host watchdog on a launched round
    copy_results: bool = True         # copy each request's results out of the result ring
    gather_inputs: bool = False       # move a round's inputs with one gk_gather kernel instead of
                                      # one copy-engine transfer per array and request
    gather_entries: int = 1 << 17     # gather table capacity per stream (64 KiB entries)
    pair_format: str = "ids"          # requests' pair-to-read form: "ids" or "starts" (CSR)
    result_bytes: bool = False        # results as one byte per pair (thresholds <= 252)


@dataclasses.dataclass
class Round:
    requests: list
    slot: int
    handle: object = None
    t_dispatch: float = 0.0


class Server:
    """Scheduler over an executor (GpuExecutor on a GPU, a fake in host-logic
    tests)."""

    def __init__(self, executor, config: ServeConfig):
        self.ex = executor
        self.cfg = config
        # One (stride, read ring, pair ring) per lane of the executor; an
        # executor without lanes is one lane of the configured stride.
        lanes = getattr(executor, "lanes", None) or [(config.stride_words, executor.n_read_slots,
                                                     executor.n_pair_slots)]
        self.lane_stride = [int(st) for st, _, _ in lanes]
        self.read_rings = [FifoRing(nr) for _, nr, _ in lanes]
        self.pair_rings = [FifoRing(npr) for _, _, npr in lanes]
        self.read_ring, self.pair_ring = self.read_rings[0], self.pair_rings[0]
        self.rounds_launched = 0
        self.max_inflight_seen = 0
        self.coalesced = []  # requests per round

    def lane_of(self, r: Request) -> int:
        sw = r.stride_words if r.n_reads else self.lane_stride[0]
        return self.lane_stride.index(sw) if sw in self.lane_stride else -1

    def fits_at_all(self, r: Request) -> bool:
        lane = self.lane_of(r)
        if lane < 0:
            return False
        return (r.n_reads <= self.read_rings[lane].size and r.n_pairs <= self.pair_rings[lane].size
                and r.n_pairs <= self.cfg.max_round_pairs
                and (r.max_len if r.max_len >= 0 else int(r.lens.max(initial=0))) <= min(
                    self.cfg.max_read_len, 32 * self.lane_stride[lane])
                and 0 <= r.e <= (252 if self.cfg.result_bytes else 255)
                and getattr(r, "pair_format", "ids") == self.cfg.pair_format)

    def _admit(self, r: Request, now: float) -> bool:
        lane = self.lane_of(r)
        rs = self.read_rings[lane].alloc(max(r.n_reads, 1))
        if rs is None:
            return False
        ps = self.pair_rings[lane].alloc(max(r.n_pairs, 1))
        if ps is None:
            self.read_rings[lane].undo_last()
            return False
        r.lane, r.read_slot, r.pair_slot, r.status, r.t_admit = lane, rs, ps, "admitted", now
        return True

    def run(self, requests: list, clock=time.perf_counter, idle_sleep: float = 20e-6,
            stop_at: float | None = None) -> list:
        """Serve `requests` (sorted by arrival) to completion; returns them with
        status, timings and (if configured) results.  With `stop_at` (s from
        the start) nothing new is launched after that time: the rounds in
        flight complete, and requests not launched by then keep their status
        ("queued" or "admitted")."""
        t0 = clock()
        self.ex.start(t0)
        pending = collections.deque(sorted(requests, key=lambda q: q.arrival))
        admitted = collections.deque()
        inflight = collections.deque()
        free_slots = collections.deque(range(self.cfg.n_streams))
        while pending or admitted or inflight:
            now = clock() - t0
            if stop_at is not None and now > stop_at:
                if not inflight:
                    break
                pending.clear()
                admitted.clear()
            while inflight and self.ex.done(inflight[0].handle):
                self._complete(inflight.popleft(), clock() - t0, free_slots)
            if inflight and now - inflight[0].t_dispatch > self.cfg.round_timeout_s:
                rnd = inflight[0]
                for r in rnd.requests:
                    r.status, r.error = "failed", "round did not complete before the watchdog limit"
                raise TimeoutError(f"round of {len(rnd.requests)} requests exceeded "
                                   f"{self.cfg.round_timeout_s} s; the server stopped")
            while pending and pending[0].arrival <= now:
                r = pending[0]
                if r.status == "cancelled":
                    pending.popleft()
                    continue
                if not self.fits_at_all(r):
                    r.status, r.error = "rejected", "request larger than the server's rings or limits"
                    pending.popleft()
                    continue
                if not self._admit(r, now):
                    break  # wait for memory: FIFO, no overtaking
                admitted.append(pending.popleft())
            if admitted and free_slots:
                batch, total = [], 0
                while admitted and total + admitted[0].n_pairs <= self.cfg.max_round_pairs:
                    total += admitted[0].n_pairs
                    batch.append(admitted.popleft())
                slot = free_slots.popleft()
                rnd = Round(batch, slot, t_dispatch=clock() - t0)
                for r in batch:
                    r.status, r.t_dispatch = "running", rnd.t_dispatch
                rnd.handle = self.ex.launch(batch, slot)
                inflight.append(rnd)
                self.rounds_launched += 1
                self.coalesced.append(len(batch))
                self.max_inflight_seen = max(self.max_inflight_seen, len(inflight))
                continue
            if not (pending and pending[0].arrival <= now):
                time.sleep(idle_sleep)
        return requests

    def _complete(self, rnd: Round, now: float, free_slots):
        dev_t = self.ex.device_done_time(rnd.handle)
        for r in rnd.requests:
            r.t_done = now
            r.t_device_done = dev_t
            if self.cfg.copy_results:
                r.accept, r.edits = self.ex.results(r)
            r.status = "done"
            self.read_rings[r.lane].release_oldest()
            self.pair_rings[r.lane].release_oldest()
        free_slots.append(rnd.slot)


def steady_state_summary(requests: list, skip_s: float, window_end_s: float) -> dict:
    """Rates and latency over the window [skip_s, window_end_s) of a run:
    offered = pairs of the requests arriving in the window per second;
    served = pairs of the requests completing in the window per second (all
    of them, whenever they arrived); latency (arrival -> results on the
    host, and -> results on the device) percentiles over the requests that
    arrived in the window, every one of which must have completed."""
    span = window_end_s - skip_s
    arrived = [r for r in requests if skip_s <= r.arrival < window_end_s]
    done_in = [r for r in requests if r.status == "done" and skip_s <= r.t_done < window_end_s]
    fin = [r for r in arrived if r.status == "done"]
    out = {"window_s": [skip_s, window_end_s], "requests_in_window": len(arrived),
           "completed_of_window": len(fin),
           "offered_gpairs_s": sum(r.n_pairs for r in arrived) / span / 1e9,
           "served_gpairs_s": sum(r.n_pairs for r in done_in) / span / 1e9}
    if fin:
        host = np.array([r.t_done - r.arrival for r in fin]) * 1e3
        dev = np.array([r.t_device_done - r.arrival for r in fin]) * 1e3
        out.update({"p50_ms": float(np.percentile(host, 50)), "p99_ms": float(np.percentile(host, 99)),
                    "max_ms": float(host.max()), "device_p50_ms": float(np.percentile(dev, 50)),
                    "device_p99_ms": float(np.percentile(dev, 99))})
    return out


def latency_summary(requests: list) -> dict:
    done = [r for r in requests if r.status == "done"]
    if not done:
        return {"done": 0}
    host = np.array([r.t_done - r.arrival for r in done]) * 1e3
    dev = np.array([r.t_device_done - r.arrival for r in done]) * 1e3
    pairs = sum(r.n_pairs for r in done)
    span = max(r.t_done for r in done) - min(r.arrival for r in done)
    return {"done": len(done), "pairs": pairs, "gpairs_s": pairs / span / 1e9 if span > 0 else None,
            "p50_ms": float(np.percentile(host, 50)), "p99_ms": float(np.percentile(host, 99)),
            "max_ms": float(host.max()), "device_p50_ms": float(np.percentile(dev, 50)),
            "device_p99_ms": float(np.percentile(dev, 99))}


def merge_ranges(dst: np.ndarray, src: np.ndarray, nb: np.ndarray):
    """merge_copies on int64 arrays, vectorized: every run of entries whose
    destination and source both continue the previous entry becomes one."""
    keep = nb > 0
    dst, src, nb = dst[keep], src[keep], nb[keep]
    if dst.shape[0] == 0:
        return dst, src, nb
    brk = np.ones(dst.shape[0], bool)
    brk[1:] = (dst[1:] != dst[:-1] + nb[:-1]) | (src[1:] != src[:-1] + nb[:-1])
    starts = np.flatnonzero(brk)
    return dst[starts], src[starts], np.add.reduceat(nb, starts)


def merge_copies(dst: list, src: list, nb: list):
    """Copies (dst, src, bytes) with every run of back-to-back entries
    (destination and source both continuing the previous entry) merged into
    one; empty entries dropped.  Returns three uint64 arrays."""
    md, ms, mn = [], [], []
    for d, s_, n in zip(dst, src, nb):
        if n == 0:
            continue
        if mn and md[-1] + mn[-1] == d and ms[-1] + mn[-1] == s_:
            mn[-1] += n
        else:
            md.append(d)
            ms.append(s_)
            mn.append(n)
    return np.array(md, np.uint64), np.array(ms, np.uint64), np.array(mn, np.uint64)


class GpuExecutor:
    """Device rings, per-stream workspaces and the library calls of a round.

    With ``config.lanes`` the device memory holds one lane per row stride:
    read rings at that stride (a 100 bp read moves 32 bytes, not the widest
    lane's row) and pair rings, sized by an equal share of the budget.  A
    round's requests are grouped by lane; per lane and array the copies of
    consecutive requests whose host and ring ranges continue each other are
    merged, so that requests received back to back into a pinned buffer move
    in a few large transfers."""

    def __init__(self, ref, config: ServeConfig, device=None):
        import torch

        from . import gk

        self.torch, self.gk, self.cfg, self.ref = torch, gk, config, ref
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.dev = dev
        strides = tuple(config.lanes) if config.lanes else (config.stride_words,)
        if max(strides) * 32 < config.max_read_len and not config.lanes:
            raise ValueError("stride_words too small for max_read_len")
        free, _ = torch.cuda.mem_get_info(dev)
        budget = int(free * config.mem_fraction)
        if config.mem_cap_bytes is not None:
            budget = min(budget, int(config.mem_cap_bytes))
        ws_bytes = max(256, gk.gk_filter_batched_workspace(config.max_round_pairs))
        rest = budget - config.n_streams * ws_bytes
        share = rest // len(strides)
        e = lambda n, dt: torch.empty(n, dtype=dt, device=dev)  # noqa: E731
        self.lane_bufs = []
        self.lanes = []
        starts, rbytes = config.pair_format == "starts", config.result_bytes
        if config.pair_format not in ("ids", "starts"):
            raise ValueError("pair_format must be 'ids' or 'starts'")
        for sw in strides:
            per_read = 8 * sw + 3 + (4 if starts else 0)
            per_pair = 10 if rbytes else 12
            unit = per_read + per_pair * config.pairs_per_read
            if share < unit * 16:
                raise MemoryError(f"device budget {budget} B too small for the rings")
            n_reads = int(share // unit)
            n_pairs = int(n_reads * config.pairs_per_read)
            self.lanes.append((sw, n_reads, n_pairs))
            self.lane_bufs.append(dict(
                sw=sw, packed=e(n_reads * sw * 2, torch.int32), lens=e(n_reads, torch.int16),
                nflag=e(n_reads, torch.uint8), pread=e(n_pairs, torch.int32), poff=e(n_pairs, torch.int32),
                rstart=e(n_reads, torch.int32) if starts else None,
                pe=e(n_pairs, torch.uint8), acc=e(n_pairs, torch.uint8),
                ed=None if rbytes else e(n_pairs, torch.int16),
                h_acc=torch.empty(n_pairs, dtype=torch.uint8, pin_memory=True),
                h_ed=None if rbytes else torch.empty(n_pairs, dtype=torch.int16, pin_memory=True)))
            lb = self.lane_bufs[-1]
            ptr = lambda t: t.data_ptr() if t is not None else 0  # noqa: E731
            lb["base"] = tuple(ptr(lb[x]) for x in ("packed", "nflag", "lens", "rstart" if starts else "pread",
                                                    "poff", "acc", "ed"))
            lb["h_base"] = (ptr(lb["h_acc"]), ptr(lb["h_ed"]))
        # the single-lane view the scheduler's tests and callers read
        self.sw = strides[0]
        self.n_read_slots, self.n_pair_slots = self.lanes[0][1], self.lanes[0][2]
        b0 = self.lane_bufs[0]
        self.packed, self.lens, self.nflag = b0["packed"], b0["lens"], b0["nflag"]
        self.pread, self.poff, self.pe, self.acc, self.ed = b0["pread"], b0["poff"], b0["pe"], b0["acc"], b0["ed"]
        self.h_acc, self.h_ed = b0["h_acc"], b0["h_ed"]
        self.ring_bytes = sum(nr * (8 * sw + 3 + (4 if starts else 0)) + npr * (10 if rbytes else 12)
                              for sw, nr, npr in self.lanes)
        self.streams = [torch.cuda.Stream(dev) for _ in range(config.n_streams)]
        self.ws = [e(ws_bytes, torch.uint8) for _ in range(config.n_streams)]
        self.max_req_per_round = max_req = 65536
        # per stream slot, host staging and device copies of the segment
        # tables: int64 pair ends | read-id deltas (ids) or read ends | read
        # slots (starts), uint32 start bases | read info (starts), uint8
        # thresholds
        self.h_seg = [torch.empty(3 * max_req, dtype=torch.int64, pin_memory=True) for _ in self.streams]
        self.h_segb = [torch.empty(2 * max_req, dtype=torch.int32, pin_memory=True) for _ in self.streams]
        self.h_sege = [torch.empty(max_req, dtype=torch.uint8, pin_memory=True) for _ in self.streams]
        self.d_seg = [e(3 * max_req, torch.int64) for _ in self.streams]
        self.d_segb = [e(2 * max_req, torch.int32) for _ in self.streams]
        self.d_sege = [e(max_req, torch.uint8) for _ in self.streams]
        # per stream slot: gk_gather tables (dst | src | bytes), pinned so the kernel reads them directly
        self.h_gather = [torch.empty(3 * config.gather_entries, dtype=torch.int64, pin_memory=True)
                         for _ in self.streams]
        self.tiling = gk.Tiling(*config.tiling)
        self.ev0 = None
        self.copies_last_round = 0

    def start(self, t0):
        self.ev0 = self.torch.cuda.Event(enable_timing=True)
        self.ev0.record(self.streams[0])
        self.t0 = t0

    def launch(self, batch, slot):
        torch, gk = self.torch, self.gk
        st = self.streams[slot]
        M = self.max_req_per_round
        if len(batch) > M:
            raise ValueError("too many requests in one round")
        hseg = self.h_seg[slot].numpy()
        hsegb = self.h_segb[slot].numpy().view(np.uint32)
        hsege = self.h_sege[slot].numpy()
        starts = self.cfg.pair_format == "starts"
        by_lane = collections.defaultdict(list)
        for r in batch:
            by_lane[max(r.lane, 0)].append(r)
        plans = []  # (lane, runs): pair runs contiguous in the lane's ring, each with its segments
        dst, src, nb = [], [], []
        k = 0
        for lane, reqs in sorted(by_lane.items()):
            b = self.lane_bufs[lane]
            sw8 = b["sw"] * 8
            n = len(reqs)
            rs = np.fromiter((r.read_slot for r in reqs), np.int64, n)
            ps = np.fromiter((r.pair_slot for r in reqs), np.int64, n)
            nr = np.fromiter((r.n_reads for r in reqs), np.int64, n)
            npr = np.fromiter((r.n_pairs for r in reqs), np.int64, n)
            ptr = np.array([r.host_ptrs for r in reqs], np.int64).reshape(n, 5)
            base = b["base"]
            link = (base[3] + 4 * rs, 4 * nr) if starts else (base[3] + 4 * ps, 4 * npr)
            has_nf = (ptr[:, 1] != 0).astype(np.int64)  # per-read arrays a request left out move nothing
            has_ln = (ptr[:, 2] != 0).astype(np.int64)
            for c, (dd, nn) in enumerate(((base[0] + rs * sw8, nr * sw8), (base[1] + rs, nr * has_nf),
                                          (base[2] + 2 * rs, 2 * nr * has_ln), link, (base[4] + 4 * ps, 4 * npr))):
                d, s_, z = merge_ranges(dd, ptr[:, c], nn)
                dst.append(d)
                src.append(s_)
                nb.append(z)
            # pair runs contiguous in the ring; per request the cumulative end
            # inside its run, the id shift and the threshold
            brk = np.ones(n, bool)
            brk[1:] = ps[1:] != ps[:-1] + npr[:-1]
            run_id = np.cumsum(brk) - 1
            csum = np.cumsum(npr)
            before = np.concatenate([[0], csum[:-1]])
            run0 = np.flatnonzero(brk)
            hseg[k:k + n] = csum - before[run0][run_id]
            if starts:
                rsum = np.cumsum(nr)
                rbefore = np.concatenate([[0], rsum[:-1]])
                hseg[M + k:M + k + n] = rsum - rbefore[run0][run_id]
                hseg[2 * M + k:2 * M + k + n] = rs
                hsegb[k:k + n] = np.fromiter((r.start_base & 0xFFFFFFFF for r in reqs), np.uint32, n)
                hsegb[M + k:M + k + n] = np.fromiter((r.read_info for r in reqs), np.uint32, n)
            else:
                hseg[M + k:M + k + n] = rs - np.fromiter((r.read_base for r in reqs), np.int64, n)
            hsege[k:k + n] = np.fromiter((r.e for r in reqs), np.uint8, n)
            ends = np.concatenate([run0[1:], [n]])
            run_pairs = np.add.reduceat(npr, run0)
            run_reads = np.add.reduceat(nr, run0)
            runs = [(int(ps[a]), int(cnt), k + int(a), int(e - a), int(rc))
                    for a, e, cnt, rc in zip(run0, ends, run_pairs, run_reads)]
            plans.append((lane, runs))
            k += n
        dseg, dsegb, dsege = self.d_seg[slot], self.d_segb[slot], self.d_sege[slot]
        seg_ptr = self.h_seg[slot].data_ptr()
        segb_ptr = self.h_segb[slot].data_ptr()
        dst.append(np.array([dseg.data_ptr(), dseg.data_ptr() + 8 * M, dseg.data_ptr() + 16 * M,
                             dsegb.data_ptr(), dsegb.data_ptr() + 4 * M, dsege.data_ptr()], np.int64))
        src.append(np.array([seg_ptr, seg_ptr + 8 * M, seg_ptr + 16 * M, segb_ptr, segb_ptr + 4 * M,
                             self.h_sege[slot].data_ptr()], np.int64))
        nb.append(np.array([8 * k, 8 * k, 8 * k if starts else 0, 4 * k if starts else 0,
                            4 * k if starts else 0, k], np.int64))
        dst, src, nb = (np.concatenate(x).astype(np.uint64) for x in (dst, src, nb))
        self.copies_last_round = int(dst.shape[0])
        self._copy_in(dst, src, nb, slot, st)
        out_d, out_s, out_n = [], [], []
        rbytes = self.cfg.result_bytes
        flags = gk.GK_FLAG_RESULT_BYTE if rbytes else 0
        for lane, runs in plans:
            b = self.lane_bufs[lane]
            nr = self.lanes[lane][1]
            for p0, np_, k0, ns, nrr in runs:
                if starts:
                    gk.gk_expand_pairs(b["pread"][p0:p0 + np_], b["pe"][p0:p0 + np_], b["rstart"],
                                       dseg[M + k0:M + k0 + ns], dseg[k0:k0 + ns], dseg[2 * M + k0:2 * M + k0 + ns],
                                       dsegb[k0:k0 + ns], dsege[k0:k0 + ns], n_reads=nrr,
                                       seg_read_info=dsegb[M + k0:M + k0 + ns], read_len=b["lens"],
                                       read_nflag=b["nflag"], stream=st)
                else:
                    gk.gk_rebase_pairs(b["pread"][p0:p0 + np_], dseg[k0:k0 + ns], dseg[M + k0:M + k0 + ns],
                                       pair_e=b["pe"][p0:p0 + np_], seg_e=dsege[k0:k0 + ns], stream=st)
                gk.gk_filter_batched(self.ref, b["packed"], b["sw"], nr, b["lens"], b["nflag"],
                                     b["pread"][p0:p0 + np_], b["poff"][p0:p0 + np_], b["pe"][p0:p0 + np_],
                                     self.tiling, self.ws[slot], flags=flags, accept=b["acc"][p0:p0 + np_],
                                     edits=None if rbytes else b["ed"][p0:p0 + np_], stream=st)
                out_d.append(b["h_base"][0] + p0)
                out_s.append(b["base"][5] + p0)
                out_n.append(np_)
                if not rbytes:
                    out_d.append(b["h_base"][1] + 2 * p0)
                    out_s.append(b["base"][6] + 2 * p0)
                    out_n.append(2 * np_)
        ev_dev = torch.cuda.Event(enable_timing=True)
        ev_dev.record(st)
        if out_n:
            d, s_, n = merge_ranges(np.array(out_d, np.int64), np.array(out_s, np.int64), np.array(out_n, np.int64))
            gk.gk_copy_many(d.astype(np.uint64), s_.astype(np.uint64), n.astype(np.uint64), gk.D2H, st)
        ev_host = torch.cuda.Event(enable_timing=False)
        ev_host.record(st)
        return (ev_dev, ev_host)

    def _copy_in(self, dst, src, nb, slot, st):
        """Host-to-device copies of a round: by default one copy-engine
        transfer per merged range; with `gather_inputs`, one gk_gather
        kernel reading the pinned request buffers (208 GB/s on this pattern
        against 135 GB/s for the copy engines on an idle GPU, but it needs
        SMs: behind the other stream's persistent filter it waits, and the
        server measured 4.06 against 4.52 Gpairs/s at 0.8 load)."""
        gk = self.gk
        if self.cfg.gather_inputs:
            cd, cs, cn = gk.gather_chunks(dst, src, nb)
            k = cd.shape[0]
            cap = self.cfg.gather_entries
            if k <= cap:
                tab = self.h_gather[slot]
                t = tab.numpy()
                t[:k] = cd.view(np.int64)
                t[cap:cap + k] = cs.view(np.int64)
                t[2 * cap:2 * cap + k] = cn.view(np.int64)
                gk.gk_gather(tab[:cap], tab[cap:2 * cap], tab[2 * cap:], k, st)
                return
        gk.gk_copy_many(dst, src, nb, gk.H2D, st)

    def done(self, handle) -> bool:
        return handle[1].query()

    def device_done_time(self, handle) -> float:
        return self.ev0.elapsed_time(handle[0]) * 1e-3

    def results(self, r: Request):
        """(accept, edits) of a completed request, or (result bytes, None)."""
        b = self.lane_bufs[max(r.lane, 0)]
        a = b["h_acc"].numpy()[r.pair_slot:r.pair_slot + r.n_pairs].copy()
        if b["h_ed"] is None:
            return a, None
        e = b["h_ed"].numpy()[r.pair_slot:r.pair_slot + r.n_pairs].view(np.uint16).copy()
        return a, e


class RequestPool:
    """Pinned host payloads that requests are cut from: per read length, reads
    sampled from the genome with their candidates (one true origin, the rest
    random), encoded once by the library's host encoder (as a client
    sending host-encoded reads would).

    stride_words: packed words per read row (None: ceil(m/32) per length,
    the rows of a server lane of that stride).  sequential: each length's
    requests are cut one after another from its pool (wrapping at the end),
    as requests received back to back into a pinned buffer would lie; their
    pair ids then number the pool's reads (read_base set accordingly) so that
    consecutive requests' arrays continue each other.  Otherwise a request
    starts at ``start_read`` and its ids count from its first read.
    pair_format: "ids" (a read id per pair) or "starts" (a start per read,
    the pool's own numbering with start_base set when sequential).
    compact_reads (starts form only): a request gives one read length
    instead of per-read lengths, and no N flags when none of its reads holds
    an N (as a client that knows its reads' length and content would)."""

    def __init__(self, ref_ascii: np.ndarray, lengths=(100, 150, 250), reads_per_len: int = 260_000,
                 cands: int = 4, stride_words: int | None = 8, seed: int = 2103_14978 + 4, pin: bool = True,
                 keep_ascii: bool = False, sequential: bool = False, pair_format: str = "ids",
                 compact_reads: bool = False):
        import torch

        from . import gk, synth

        if pair_format not in ("ids", "starts"):
            raise ValueError("pair_format must be 'ids' or 'starts'")
        if compact_reads and pair_format != "starts":
            raise ValueError("compact_reads needs pair_format 'starts'")
        self.cands, self.pin, self.sequential, self.pair_format = cands, pin, sequential, pair_format
        self.compact_reads = compact_reads
        self.sw = stride_words if stride_words is not None else 8
        self.by_len = {}
        self.cursor = {}
        for m in lengths:
            sw = stride_words if stride_words is not None else -(-m // 32)
            w = synth.pairs_workload(f"pool-{m}", seed=seed + m, ref=ref_ascii, n_pairs=reads_per_len * cands,
                                     m=m, cands=cands, e=0, read_edit_rate=0.02)
            packed, nflag = gk.gk_encode(torch.from_numpy(w.reads), w.n_reads, w.stride, fixed_len=m,
                                         stride_words=sw)
            self.by_len[m] = self._pin(pin, packed=packed.numpy().view(np.uint32), nflag=nflag.numpy(),
                                       lens=np.full(w.n_reads, m, np.uint16), pair_read=w.pair_read,
                                       pair_off=w.pair_off)
            self.by_len[m]["sw"] = sw
            # N reads before each read: whether a cut holds any is two lookups
            self.by_len[m]["n_before"] = np.concatenate([[0], np.cumsum(nflag.numpy() != 0)])
            self.cursor[m] = 0
            if keep_ascii:
                self.by_len[m]["ascii"] = (None, w.reads.reshape(w.n_reads, w.stride))
        # The pool's pairs are grouped by read, `cands` per read, so the ids of
        # any slice relative to its first read are k // cands: one array serves
        # every request.
        max_reads = max(p["lens"][1].shape[0] for p in self.by_len.values())
        max_pairs = cands * max_reads
        self.rel_ids = self._pin(pin, a=(np.arange(max_pairs, dtype=np.uint32) // cands))["a"]
        # Read k's first pair is cands * k, in the pool and in any cut (minus its base).
        self.rel_starts = self._pin(pin, a=(np.arange(max_reads, dtype=np.uint32) * cands))["a"]

    @staticmethod
    def _pin(pin, **arrays):
        out = {}
        for k, a in arrays.items():
            if pin:
                import torch

                t = torch.empty(a.shape, dtype=getattr(torch, {"uint8": "uint8", "uint16": "int16",
                                                                 "uint32": "int32"}[a.dtype.name]),
                                pin_memory=True)
                v = t.numpy().view(a.dtype)
                v[...] = a
                out[k] = (t, v)
            else:
                out[k] = (None, np.ascontiguousarray(a))
        return out

    def reset(self):
        """Restart every length's sequential cut at the pool's first read."""
        for m in self.cursor:
            self.cursor[m] = 0

    def request(self, rid: int, m: int, e: int, n_pairs: int, start_read: int, arrival: float) -> Request:
        """Cut a request of n_pairs pairs (rounded up to whole reads) of length m
        starting at pool read `start_read` (the next read of the length's
        pool when sequential)."""
        p = self.by_len[m]
        n_reads = -(-n_pairs // self.cands)
        total = p["lens"][1].shape[0]
        if self.sequential:
            r0 = self.cursor[m]
            if r0 + n_reads > total:
                r0 = 0
            self.cursor[m] = r0 + n_reads
        else:
            r0 = start_read % max(1, total - n_reads)
        r1 = r0 + n_reads
        n = n_reads * self.cands
        w2 = p["sw"] * 2
        ids = starts = None
        base = sbase = 0
        if self.pair_format == "starts":
            if self.sequential:  # the pool's numbering: consecutive requests' starts continue each other
                starts, sbase = self.rel_starts[1][r0:r1], r0 * self.cands
            else:
                starts = self.rel_starts[1][:n_reads]
        elif self.sequential:  # the pool's own ids: consecutive requests' id arrays continue each other
            ids, base = p["pair_read"][1][r0 * self.cands:r1 * self.cands], r0
        else:
            ids = self.rel_ids[1][:n]
        lens, nflag = p["lens"][1][r0:r1], p["nflag"][1][r0:r1]
        if self.compact_reads:
            lens = None
            if p["n_before"][r1] == p["n_before"][r0]:
                nflag = None
        return Request(id=rid, packed=p["packed"][1][r0 * w2:r1 * w2], nflag=nflag,
                       lens=lens, pair_read=ids,
                       pair_off=p["pair_off"][1][r0 * self.cands:r1 * self.cands], e=e, arrival=arrival,
                       max_len=m, ascii=p["ascii"][1][r0:r1] if "ascii" in p else None, read_base=base,
                       read_start=starts, start_base=sbase, read_len=m if self.compact_reads else 0)


def poisson_plan(n_requests: int, rate_per_s: float, seed: int, size_lo=1_000, size_hi=1_000_000,
                 lengths=(100, 150, 250), rates=(0.02, 0.05, 0.10)):
    """Arrival times (Poisson) and request shapes of the serving
    configuration: log-uniform sizes, a read length and one
    e = ceil(rate x m) per request."""
    rng = np.random.default_rng([seed, n_requests, 7])
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(rng.uniform(np.log(size_lo), np.log(size_hi), n_requests)).astype(np.int64)
    ms = np.asarray(lengths)[rng.integers(0, len(lengths), n_requests)]
    rs = np.asarray(rates)[rng.integers(0, len(rates), n_requests)]
    es = np.ceil(np.round(rs * ms, 9)).astype(np.int64)
    starts = rng.integers(0, 1 << 30, n_requests)
    return [dict(id=i, arrival=float(arrivals[i]), n_pairs=int(sizes[i]), m=int(ms[i]), e=int(es[i]),
                 start=int(starts[i])) for i in range(n_requests)]


def poisson_plan_for(seconds: float, rate_per_s: float, seed: int, **kw):
    """poisson_plan with arrivals during `seconds` seconds (the requests
    arriving before then)."""
    n = int(rate_per_s * seconds * 1.1) + 64
    while True:
        plan = poisson_plan(n, rate_per_s, seed, **kw)
        if plan[-1]["arrival"] >= seconds:
            return [q for q in plan if q["arrival"] < seconds]
        n *= 2
