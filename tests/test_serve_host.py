"""Host logic of the serving loop, on the CPU: the FIFO ring allocator, memory
admission, coalescing, rejection, cancellation and the watchdog, driven by a
fake executor on a simulated clock whose results come from the oracle."""
import random

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_14978_gb300 import serve, synth


def test_fifo_ring_never_overlaps():
    rng = random.Random(4)
    for size in (1, 7, 64, 1000):
        ring = serve.FifoRing(size)
        live = []
        for _ in range(3000):
            if live and (rng.random() < 0.45 or not ring.free_slots()):
                ring.release_oldest()
                live.pop(0)
                continue
            n = rng.randint(1, max(1, size // 3))
            start = ring.alloc(n)
            if start is None:
                assert ring.free_slots() < size  # refusals only when something is live
                continue
            assert 0 <= start and start + n <= size
            for s, k in live:
                assert start + n <= s or s + k <= start, "overlap"
            live.append((start, n))
        with pytest.raises(ValueError):
            ring.alloc(size + 1)


def test_fifo_ring_wraps_and_frees():
    ring = serve.FifoRing(10)
    assert ring.alloc(6) == 0
    assert ring.alloc(3) == 6
    assert ring.alloc(2) is None          # 1 slot at the end, 0 at the start
    ring.release_oldest()                 # frees 0..5
    assert ring.alloc(2) == 0             # skips the one-slot gap at the end
    assert ring.alloc(5) is None          # 2..5 free: only 4 slots before the tail at 6
    assert ring.alloc(4) == 2
    ring.undo_last()
    assert ring.alloc(4) == 2


def ids_of(r):
    """Pair -> read index within the request, from read ids or per-read starts."""
    if r.pair_read is not None:
        return (r.pair_read.astype(np.int64) - r.read_base).astype(np.uint32)
    rel = r.read_start.astype(np.int64) - r.start_base
    ends = np.append(rel[1:], r.n_pairs)
    return np.repeat(np.arange(r.n_reads, dtype=np.uint32), ends - rel)


class FakeExecutor:
    """Completes a round `delay` simulated seconds after its launch; results
    from the oracle on the request's own reads and the genome."""

    def __init__(self, genome, n_read_slots, n_pair_slots, delay=0.005, never=False, lanes=None):
        self.genome = genome
        self.n_read_slots, self.n_pair_slots = n_read_slots, n_pair_slots
        if lanes:
            self.lanes = lanes
        self.delay, self.never = delay, never
        self.now = 0.0
        self.out = {}
        self.launches = []

    def start(self, t0):
        self.t0 = t0

    def launch(self, batch, slot):
        self.launches.append([r.id for r in batch])
        for r in batch:
            rows = np.ascontiguousarray(r.ascii).reshape(-1)
            starts = np.arange(r.n_reads, dtype=np.uint64) * np.uint64(r.ascii.shape[1])
            lens = r.lens if r.lens is not None else np.full(r.n_reads, r.read_len, np.uint16)
            a, e, _ = O.filter_batch(rows, starts, lens, self.genome, ids_of(r), r.pair_off, r.e)
            self.out[r.id] = (a, e)
        return self.now + self.delay

    def done(self, handle):
        return not self.never and self.now >= handle

    def device_done_time(self, handle):
        return handle

    def results(self, r):
        return self.out[r.id]


class SimClock:
    def __init__(self, ex, step=1e-4):
        self.ex, self.t, self.step = ex, 0.0, step

    def __call__(self):
        self.t += self.step
        self.ex.now = self.t
        return self.t


@pytest.fixture(scope="module")
def pool():
    ref = synth.reference(300_000, 17, 0.05, 0.0)
    return ref, serve.RequestPool(ref, lengths=(60, 100), reads_per_len=3000, stride_words=4, pin=False,
                                  keep_ascii=True)


def make_requests(pool_, n, seed, size_hi=4000, spread=0.01):
    _, p = pool_
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        m = int(rng.choice([60, 100]))
        reqs.append(p.request(i, m, int(rng.integers(0, 8)), int(rng.integers(1, size_hi)),
                              int(rng.integers(0, 1 << 20)), float(rng.uniform(0, spread))))
    return reqs


def serve_with(pool_, reqs, n_read_slots=100_000, n_pair_slots=400_000, **cfg):
    ref, _ = pool_
    ex = FakeExecutor(ref, n_read_slots, n_pair_slots, never=cfg.pop("never", False))
    conf = serve.ServeConfig(stride_words=4, max_read_len=128, **cfg)
    srv = serve.Server(ex, conf)
    srv.run(reqs, clock=SimClock(ex), idle_sleep=0)
    return srv, ex


def test_every_request_served_and_identical_alone_and_in_the_mix(pool):
    reqs = make_requests(pool, 40, 1)
    srv, ex = serve_with(pool, reqs)
    assert all(r.status == "done" for r in reqs)
    assert max(len(b) for b in ex.launches) > 1          # coalesced rounds
    assert srv.max_inflight_seen <= 2
    for r in reqs:
        alone = make_requests(pool, 40, 1)[r.id]
        serve_with(pool, [alone])
        assert np.array_equal(alone.accept, r.accept) and np.array_equal(alone.edits, r.edits)
        assert r.t_done >= r.t_device_done >= r.arrival


def test_memory_admission_waits_and_rejects(pool):
    reqs = make_requests(pool, 30, 2, size_hi=3000)
    big = pool[1].request(99, 100, 3, 5000, 0, 0.0)  # 1250 reads > ring of 800 slots
    srv, ex = serve_with(pool, reqs + [big], n_read_slots=800, n_pair_slots=3200)
    assert big.status == "rejected"
    assert all(r.status == "done" for r in reqs)
    # rings never held more than their size: every launch fits
    for ids in ex.launches:
        assert sum(reqs[i].n_pairs for i in ids) <= 3200


def test_cancelled_requests_are_skipped(pool):
    reqs = make_requests(pool, 10, 4, spread=1.0)
    reqs[3].cancel()
    reqs[7].cancel()
    serve_with(pool, reqs)
    assert reqs[3].status == reqs[7].status == "cancelled"
    assert sum(r.status == "done" for r in reqs) == 8


def test_watchdog_stops_a_round_that_never_completes(pool):
    reqs = make_requests(pool, 3, 5)
    with pytest.raises(TimeoutError):
        serve_with(pool, reqs, never=True, round_timeout_s=0.05)
    assert any(r.status == "failed" for r in reqs)


def test_gather_chunks_split_copies_into_bounded_entries():
    from paper_2103_14978_gb300 import gk

    rng = np.random.default_rng(5)
    nb = np.concatenate([[0, 1, 65535, 65536, 65537, 3 * 65536], rng.integers(0, 400_000, 50)]).astype(np.uint64)
    dst = (np.arange(nb.shape[0], dtype=np.uint64) << np.uint64(32)) + np.uint64(7)
    src = (np.arange(nb.shape[0], dtype=np.uint64) << np.uint64(33)) + np.uint64(3)
    cd, cs, cn = gk.gather_chunks(dst, src, nb)
    assert (cn > 0).all() and (cn <= gk.GK_GATHER_MAX_BYTES).all()
    assert int(cn.sum()) == int(nb.sum())
    # entries tile every copy contiguously, in order
    i = 0
    for d, s, z in zip(dst, src, nb):
        covered = 0
        while covered < z:
            assert cd[i] == d + np.uint64(covered) and cs[i] == s + np.uint64(covered)
            covered += int(cn[i])
            i += 1
        assert covered == z
    assert i == cd.shape[0]


def test_stop_time_drains_inflight_and_leaves_the_rest(pool):
    """With stop_at, rounds launched before the stop complete and nothing is
    launched after it."""
    reqs = make_requests(pool, 60, 6, spread=0.2)
    ref, _ = pool
    ex = FakeExecutor(ref, 100_000, 400_000, delay=0.01)
    srv = serve.Server(ex, serve.ServeConfig(stride_words=4, max_read_len=128, max_round_pairs=6000))
    srv.run(reqs, clock=SimClock(ex), idle_sleep=0, stop_at=0.1)
    done = [r for r in reqs if r.status == "done"]
    assert done and len(done) < len(reqs)
    assert all(r.t_dispatch <= 0.1 + 1e-3 for r in done)
    assert all(r.status in ("queued", "admitted") for r in reqs if r.status != "done")


def test_steady_state_summary_counts_the_window():
    def req(n, arrival, t_done, status="done"):
        r = serve.Request(0, np.zeros(0, np.uint32), np.zeros(0, np.uint8), np.zeros(0, np.uint16),
                          np.zeros(n, np.uint32), np.zeros(n, np.uint32), 0, arrival=arrival)
        r.status, r.t_done, r.t_device_done = status, t_done, t_done - 0.001
        return r

    reqs = [req(1000, 0.5, 1.2),   # arrived before the window, completed in it: served only
            req(2000, 1.5, 1.6),   # in the window both ways, 100 ms
            req(3000, 2.5, 2.8),   # 300 ms
            req(4000, 2.9, 3.5)]   # arrived in the window, completed after it: offered only
    s = serve.steady_state_summary(reqs, 1.0, 3.0)
    assert s["requests_in_window"] == 3 and s["completed_of_window"] == 3
    assert abs(s["offered_gpairs_s"] - 9000 / 2.0 / 1e9) < 1e-15
    assert abs(s["served_gpairs_s"] - 6000 / 2.0 / 1e9) < 1e-15
    assert abs(s["max_ms"] - 600.0) < 1e-6 and 100.0 <= s["p50_ms"] <= 300.0


def test_poisson_plan_for_covers_the_duration():
    plan = serve.poisson_plan_for(2.0, 500.0, 9)
    arr = np.array([q["arrival"] for q in plan])
    assert arr.max() < 2.0 and arr.max() > 1.9 and (np.diff(arr) >= 0).all()
    assert 800 < len(plan) < 1200  # about 500 per second


def test_merge_copies_joins_back_to_back_ranges():
    d, s_, n = serve.merge_copies([100, 110, 200, 210, 300, 400], [1000, 1010, 5000, 5011, 7000, 0],
                                  [10, 20, 10, 5, 0, 7])
    # 100+110 continue on both sides; 210 does not continue 5000 on the source side; the empty copy drops
    assert d.tolist() == [100, 200, 210, 400] and s_.tolist() == [1000, 5000, 5011, 0]
    assert n.tolist() == [30, 10, 5, 7]


def test_merge_ranges_equals_merge_copies():
    rng = np.random.default_rng(12)
    for _ in range(50):
        n = int(rng.integers(0, 40))
        nb = rng.integers(0, 5, n) * 8
        dst = np.cumsum(np.concatenate([[1000], nb[:-1] + rng.integers(0, 2, max(n - 1, 0)) * 8]))[:n]
        src = np.cumsum(np.concatenate([[9000], nb[:-1] + rng.integers(0, 2, max(n - 1, 0)) * 16]))[:n]
        a = serve.merge_copies(list(dst), list(src), list(nb))
        b = serve.merge_ranges(dst.astype(np.int64), src.astype(np.int64), nb.astype(np.int64))
        assert all(np.array_equal(x.astype(np.int64), y) for x, y in zip(a, b))


def test_lanes_admit_by_row_stride_and_sequential_cuts_continue():
    """Requests go to the lane of their own row stride (60 bp: 2 words, 100
    bp: 4), results equal the oracle; a sequential pool's consecutive
    requests of one length continue each other in host memory."""
    ref = synth.reference(300_000, 19, 0.05, 0.0)
    pool = serve.RequestPool(ref, lengths=(60, 100), reads_per_len=3000, stride_words=None, pin=False,
                             keep_ascii=True, sequential=True)
    rng = np.random.default_rng(9)
    reqs = [pool.request(i, int(rng.choice([60, 100])), int(rng.integers(0, 8)), int(rng.integers(4, 3000)), 0,
                         float(rng.uniform(0, 0.01))) for i in range(40)]
    by_m = {}
    for r in reqs:
        by_m.setdefault(r.max_len, []).append(r)
    for m, rs in by_m.items():
        assert all(r.stride_words == -(-m // 32) for r in rs)
        for a, b in zip(rs, rs[1:]):
            if b.read_base == a.read_base + a.n_reads:  # no wrap between them
                assert b.packed.ctypes.data == a.packed.ctypes.data + a.packed.nbytes
                assert b.pair_read.ctypes.data == a.pair_read.ctypes.data + a.pair_read.nbytes
    ex = FakeExecutor(ref, 0, 0, lanes=[(2, 20_000, 80_000), (4, 20_000, 80_000)])
    srv = serve.Server(ex, serve.ServeConfig(stride_words=4, max_read_len=128))
    srv.run(reqs, clock=SimClock(ex), idle_sleep=0)
    assert all(r.status == "done" for r in reqs)
    assert {r.lane for r in by_m[60]} == {0} and {r.lane for r in by_m[100]} == {1}
    for r in reqs[::5]:
        rows = np.ascontiguousarray(r.ascii).reshape(-1)
        starts = np.arange(r.n_reads, dtype=np.uint64) * np.uint64(r.ascii.shape[1])
        ids = (r.pair_read.astype(np.int64) - r.read_base).astype(np.uint32)
        a, e, _ = O.filter_batch(rows, starts, r.lens, ref, ids, r.pair_off, r.e)
        assert np.array_equal(a, r.accept) and np.array_equal(e, r.edits)


def test_read_starts_requests_validate_continue_and_serve():
    """A request names its pairs' reads by ids or by per-read starts, not
    both; a sequential pool's start arrays continue each other with the
    start base of their first pair; a server in the starts format serves
    them (results equal the oracle) and turns away requests of the other
    format."""
    ref = synth.reference(300_000, 21, 0.05, 0.0)
    pool = serve.RequestPool(ref, lengths=(100,), reads_per_len=3000, stride_words=4, pin=False,
                             keep_ascii=True, sequential=True, pair_format="starts")
    a = pool.request(0, 100, 3, 400, 0, 0.0)
    b = pool.request(1, 100, 5, 1000, 0, 0.001)
    assert a.pair_read is None and a.start_base == 0 and a.read_start[0] == 0
    assert b.start_base == a.n_pairs and b.read_start[0] == a.n_pairs
    assert b.read_start.ctypes.data == a.read_start.ctypes.data + a.read_start.nbytes
    with pytest.raises(ValueError):
        serve.Request(9, a.packed, a.nflag, a.lens, None, a.pair_off, 3)
    with pytest.raises(ValueError):
        serve.Request(9, a.packed, a.nflag, a.lens, np.zeros(a.n_pairs, np.uint32), a.pair_off, 3,
                      read_start=a.read_start)
    ids_pool = serve.RequestPool(ref, lengths=(100,), reads_per_len=3000, stride_words=4, pin=False,
                                 keep_ascii=True)
    other = ids_pool.request(2, 100, 4, 500, 0, 0.002)
    ex = FakeExecutor(ref, 100_000, 400_000)
    srv = serve.Server(ex, serve.ServeConfig(stride_words=4, max_read_len=128, pair_format="starts"))
    srv.run([a, b, other], clock=SimClock(ex), idle_sleep=0)
    assert a.status == b.status == "done" and other.status == "rejected"
    for r in (a, b):
        rows = np.ascontiguousarray(r.ascii).reshape(-1)
        starts = np.arange(r.n_reads, dtype=np.uint64) * np.uint64(r.ascii.shape[1])
        want = O.filter_batch(rows, starts, r.lens, ref, (np.arange(r.n_pairs) // 4).astype(np.uint32),
                              r.pair_off, r.e)
        assert np.array_equal(want[0], r.accept) and np.array_equal(want[1], r.edits)


def test_compact_read_descriptions():
    """A starts-form request may give one read length instead of per-read
    lengths and leave out the N flags when no read holds an N: the pool
    does so per cut (flags kept where a read has an N), the per-segment word
    for the device says which, and ids-form requests must give both."""
    ref = synth.reference(300_000, 23, 0.05, 0.002)
    pool = serve.RequestPool(ref, lengths=(100,), reads_per_len=3000, stride_words=4, pin=False,
                             keep_ascii=True, sequential=True, pair_format="starts", compact_reads=True)
    reqs = [pool.request(i, 100, 2, 40, 0, 0.0) for i in range(60)]
    assert all(r.lens is None and r.read_len == 100 and r.max_len == 100 for r in reqs)
    with_n = [r for r in reqs if r.nflag is not None]
    without = [r for r in reqs if r.nflag is None]
    assert with_n and without
    for r in with_n:
        assert r.nflag.any() and r.read_info == 100
    for r in without:
        assert not pool.by_len[100]["nflag"][1][r.start_base // 4:r.start_base // 4 + r.n_reads].any()
        assert r.read_info == 100 | 0x10000
    a = reqs[0]
    with pytest.raises(ValueError):
        serve.Request(9, a.packed, None, None, np.zeros(a.n_pairs, np.uint32), a.pair_off, 3, read_len=100)
    with pytest.raises(ValueError):
        serve.Request(9, a.packed, None, None, None, a.pair_off, 3, read_start=a.read_start)
    with pytest.raises(ValueError):
        serve.RequestPool(ref, lengths=(100,), reads_per_len=100, pin=False, compact_reads=True)
    ex = FakeExecutor(ref, 100_000, 400_000)
    srv = serve.Server(ex, serve.ServeConfig(stride_words=4, max_read_len=128, pair_format="starts"))
    srv.run(reqs, clock=SimClock(ex), idle_sleep=0)
    assert all(r.status == "done" for r in reqs)
