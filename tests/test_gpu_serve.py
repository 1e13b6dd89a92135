"""The serving loop on the GPU: every request's results are the same served
alone and in the coalesced mix (tolerance 0), and equal the oracle; memory
admission under a small device budget."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2103_14978_gb300 import gk, serve, synth
from tests.gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    require_gpu()
    ref = synth.reference(20_000_000, 51, 0.05, 0.001)
    gkref = gk.gk_load_reference(ref)
    pool = serve.RequestPool(ref, lengths=(100, 150, 250), reads_per_len=60_000, keep_ascii=True)
    return ref, gkref, pool


def requests(pool, n, rate, seed, size_hi=200_000, lengths=(100, 150, 250)):
    plan = serve.poisson_plan(n, rate, seed, size_lo=1_000, size_hi=size_hi, lengths=lengths)
    return [pool.request(p["id"], p["m"], p["e"], p["n_pairs"], p["start"], p["arrival"]) for p in plan]


def ids_of(r):
    """The request's pair -> read index (0-based within the request), from
    either form: read ids, or per-read starts (CSR) written out one by one."""
    if r.pair_read is not None:
        return (r.pair_read.astype(np.int64) - r.read_base).astype(np.uint32)
    rel = r.read_start.astype(np.int64) - r.start_base
    ends = np.append(rel[1:], r.n_pairs)
    out = np.empty(r.n_pairs, np.uint32)
    for k in range(r.n_reads):
        out[rel[k]:ends[k]] = k
    return out


def lens_of(r):
    return r.lens.view(np.uint16) if r.lens is not None else np.full(r.n_reads, r.read_len, np.uint16)


def oracle_of(ref, r):
    rows = np.ascontiguousarray(r.ascii).reshape(-1)
    starts = np.arange(r.n_reads, dtype=np.uint64) * np.uint64(r.ascii.shape[1])
    a, e, _ = O.filter_batch(rows, starts, lens_of(r), ref, ids_of(r), r.pair_off, r.e)
    return a, e


def result_bytes_of(a, e):
    """The documented result byte of an oracle (accept, count) pair."""
    e = e.astype(np.int64)
    return np.where(e == 0xFFFF, gk.GK_RESULT_UNDEFINED,
                    np.where(e == 0xFFFE, gk.GK_RESULT_INVALID, np.minimum(e, gk.GK_RESULT_MAX_COUNT))).astype(np.uint8)


def test_read_starts_and_result_bytes_equal_the_oracle(setup):
    """Pairs sent as one start per read (expanded on the device), one read
    length per request and no N flags for requests without N (written on
    the device), results returned as one byte per pair, three streams,
    lanes per stride: every checked request's result bytes equal the
    oracle's counts in that format, and the mix equals the same requests
    served with read ids, per-read lengths and flags."""
    ref, gkref, _ = setup
    out = {}
    for fmt, rb in (("starts", True), ("ids", False)):
        pool = serve.RequestPool(ref, lengths=(100, 150, 250), reads_per_len=60_000, stride_words=None,
                                 keep_ascii=True, sequential=True, pair_format=fmt, compact_reads=fmt == "starts")
        cfg = serve.ServeConfig(mem_cap_bytes=3 << 30, max_round_pairs=2_000_000, lanes=(4, 5, 8), n_streams=3,
                                pair_format=fmt, result_bytes=rb)
        ex = serve.GpuExecutor(gkref, cfg)
        reqs = requests(pool, 300, 20_000.0, 65)
        srv = serve.Server(ex, cfg)
        srv.run(reqs)
        assert all(r.status == "done" for r in reqs)
        assert max(srv.coalesced) > 10
        out[fmt] = reqs
    assert all(r.lens is None for r in out["starts"])
    for r in sorted(out["starts"], key=lambda q: q.n_pairs)[:30] + out["starts"][::30]:
        assert r.edits is None
        a, e = oracle_of(ref, r)
        assert np.array_equal(result_bytes_of(a, e), r.accept), r.id
    for r, q in zip(out["starts"], out["ids"]):
        assert np.array_equal(r.accept, result_bytes_of(q.accept, q.edits)), r.id


def test_requests_without_n_flags_equal_the_oracle():
    """On a genome without N every compact request leaves out its N flags
    and its lengths; the device writes both: results equal the oracle."""
    require_gpu()
    ref = synth.reference(4_000_000, 53, 0.05, 0.0)
    gkref = gk.gk_load_reference(ref)
    pool = serve.RequestPool(ref, lengths=(100, 150), reads_per_len=20_000, stride_words=None, keep_ascii=True,
                             sequential=True, pair_format="starts", compact_reads=True)
    cfg = serve.ServeConfig(mem_cap_bytes=1 << 30, max_round_pairs=500_000, lanes=(4, 5), pair_format="starts")
    reqs = requests(pool, 120, 20_000.0, 66, size_hi=40_000, lengths=(100, 150))
    assert all(r.nflag is None and r.lens is None for r in reqs)
    srv = serve.Server(serve.GpuExecutor(gkref, cfg), cfg)
    srv.run(reqs)
    assert all(r.status == "done" for r in reqs)
    for r in reqs[::4]:
        a, e = oracle_of(ref, r)
        assert np.array_equal(a, r.accept) and np.array_equal(e, r.edits), r.id


def test_expand_pairs_writes_every_pair_once():
    """gk_expand_pairs: segments at scattered read rows with start bases,
    reads with 0..7 candidates, a malformed segment (starts decreasing and
    past its pairs): ids and thresholds equal the CSR definition, unclaimed
    pairs get 0xFFFFFFFF (no two reads claim one pair: the definition's
    ranges here never overlap)."""
    require_gpu()
    rng = np.random.default_rng(12)
    n_rows = 5000
    read_start = np.zeros(n_rows, np.uint32)
    seg_read_end, seg_pair_end, seg_slot, seg_base, seg_e = [], [], [], [], []
    want_id, want_e = [], []
    slot, r_tot, p_tot = 7, 0, 0
    for i in range(40):
        nr = int(rng.integers(0, 60))
        counts = rng.integers(0, 8, nr)
        base = int(rng.integers(0, 1 << 32))
        rel = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64) if nr else np.zeros(0, np.int64)
        npairs = int(counts.sum())
        ids = np.repeat(np.arange(slot, slot + nr), counts).astype(np.uint32)
        if i == 17:  # malformed: the first read starts at 2 (pairs 0, 1 unclaimed), the last past the end
            nr = max(nr, 4)
            counts = rng.integers(2, 8, nr)
            rel = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
            npairs = int(counts.sum())
            rel[0] = 2
            rel[-1] = npairs + 5
            ids = np.full(npairs, 0xFFFFFFFF, np.uint32)
            for k in range(nr):
                lo = min(rel[k], npairs)
                hi = min(rel[k + 1] if k + 1 < nr else npairs, npairs)
                ids[lo:hi] = slot + k
        read_start[slot:slot + nr] = (rel + base) & 0xFFFFFFFF
        e = int(rng.integers(0, 256))
        want_id.append(ids)
        want_e.append(np.full(npairs, e, np.uint8))
        r_tot += nr
        p_tot += npairs
        seg_read_end.append(r_tot)
        seg_pair_end.append(p_tot)
        seg_slot.append(slot)
        seg_base.append(base)
        seg_e.append(e)
        slot += nr + int(rng.integers(0, 5))
    want_id, want_e = np.concatenate(want_id), np.concatenate(want_e)
    d = lambda a, dt: torch.from_numpy(np.asarray(a).astype(dt)).cuda()  # noqa: E731
    pread = torch.zeros(p_tot, dtype=torch.int32, device="cuda")
    pe = torch.zeros(p_tot, dtype=torch.uint8, device="cuda")
    # per segment: a shared length (or 0: given per read) and / or "no N"
    info = np.array([(int(rng.integers(1, 300)) if i % 3 else 0) | (gk.GK_SEG_NO_N if i % 2 else 0)
                     for i in range(len(seg_e))], np.uint32)
    lens = torch.full((n_rows,), 7, dtype=torch.int16, device="cuda")
    nfl = torch.full((n_rows,), 9, dtype=torch.uint8, device="cuda")
    gk.gk_expand_pairs(pread, pe, d(read_start.view(np.int32), np.int32), d(seg_read_end, np.int64),
                       d(seg_pair_end, np.int64), d(seg_slot, np.int64),
                       d(np.array(seg_base, np.uint64).astype(np.uint32).view(np.int32), np.int32),
                       d(seg_e, np.uint8), n_reads=r_tot, seg_read_info=d(info.view(np.int32), np.int32),
                       read_len=lens, read_nflag=nfl)
    torch.cuda.synchronize()
    got = pread.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, want_id)
    claimed = want_id != 0xFFFFFFFF
    assert np.array_equal(pe.cpu().numpy()[claimed], want_e[claimed])
    want_len = np.full(n_rows, 7, np.int16)
    want_nf = np.full(n_rows, 9, np.uint8)
    r0 = 0
    for i, (re_, sl) in enumerate(zip(seg_read_end, seg_slot)):
        rows = slice(sl, sl + re_ - r0)
        if info[i] & 0xFFFF:
            want_len[rows] = info[i] & 0xFFFF
        if info[i] & gk.GK_SEG_NO_N:
            want_nf[rows] = 0
        r0 = re_
    assert np.array_equal(lens.cpu().numpy(), want_len) and np.array_equal(nfl.cpu().numpy(), want_nf)


def test_lanes_merged_copies_equal_the_oracle(setup):
    """Lanes per row stride (100 / 150 / 250 bp rows of 4 / 5 / 8 words),
    requests cut back to back from their pools so that a round's copies
    merge: every request equals the oracle, and rounds move in far fewer
    copies than requests."""
    ref, gkref, _ = setup
    pool = serve.RequestPool(ref, lengths=(100, 150, 250), reads_per_len=60_000, stride_words=None,
                             keep_ascii=True, sequential=True)
    cfg = serve.ServeConfig(mem_cap_bytes=3 << 30, max_round_pairs=2_000_000, lanes=(4, 5, 8))
    ex = serve.GpuExecutor(gkref, cfg)
    reqs = requests(pool, 300, 20_000.0, 64)
    srv = serve.Server(ex, cfg)
    srv.run(reqs)
    assert all(r.status == "done" for r in reqs)
    assert max(srv.coalesced) > 10 and ex.copies_last_round < 40
    for r in sorted(reqs, key=lambda q: q.n_pairs)[:40] + reqs[::25]:
        a, e = oracle_of(ref, r)
        assert np.array_equal(a, r.accept) and np.array_equal(e, r.edits), r.id


def test_same_result_alone_and_in_the_mix(setup):
    ref, gkref, pool = setup
    cfg = serve.ServeConfig(mem_cap_bytes=3 << 30, max_round_pairs=2_000_000)
    ex = serve.GpuExecutor(gkref, cfg)
    mix = requests(pool, 300, 20_000.0, 61)
    srv = serve.Server(ex, cfg)
    srv.run(mix)
    assert all(r.status == "done" for r in mix)
    assert max(srv.coalesced) > 1, "no round coalesced several requests"
    summ = serve.latency_summary(mix)
    assert summ["done"] == 300 and summ["p99_ms"] >= summ["p50_ms"] > 0
    again = requests(pool, 300, 20_000.0, 61)
    for r in again[::15]:
        r.arrival = 0.0
        serve.Server(ex, cfg).run([r])
        m = mix[r.id]
        assert np.array_equal(r.accept, m.accept) and np.array_equal(r.edits, m.edits), r.id
    for r in sorted(mix, key=lambda q: q.n_pairs)[:40]:
        a, e = oracle_of(ref, r)
        assert np.array_equal(a, r.accept) and np.array_equal(e, r.edits), r.id


def test_admission_under_a_small_memory_budget(setup):
    ref, gkref, pool = setup
    cfg = serve.ServeConfig(mem_cap_bytes=7 << 20, max_round_pairs=150_000)
    ex = serve.GpuExecutor(gkref, cfg)
    assert ex.n_pair_slots < 200_000
    reqs = requests(pool, 120, 50_000.0, 62, size_hi=300_000)
    srv = serve.Server(ex, cfg)
    srv.run(reqs)
    too_big = [r for r in reqs if r.n_pairs > min(ex.n_pair_slots, 150_000) or r.n_reads > ex.n_read_slots]
    assert too_big and all(r.status == "rejected" for r in too_big)
    served = [r for r in reqs if r.status == "done"]
    assert len(served) == len(reqs) - len(too_big)
    for r in served[::10]:
        a, e = oracle_of(ref, r)
        assert np.array_equal(a, r.accept) and np.array_equal(e, r.edits), r.id


def test_round_inputs_by_gather_kernel_or_copy_engines_agree(setup):
    """The same requests served with their inputs moved by one gk_gather
    kernel per round and by one copy-engine transfer per array give the same
    results (tolerance 0)."""
    ref, gkref, pool = setup
    out = []
    for gather in (True, False):
        cfg = serve.ServeConfig(mem_cap_bytes=2 << 30, max_round_pairs=1_000_000, gather_inputs=gather)
        reqs = requests(pool, 80, 40_000.0, 63)
        serve.Server(serve.GpuExecutor(gkref, cfg), cfg).run(reqs)
        assert all(r.status == "done" for r in reqs)
        out.append(reqs)
    for a, b in zip(*out):
        assert np.array_equal(a.accept, b.accept) and np.array_equal(a.edits, b.edits), a.id


def test_gather_kernel_copies_exactly():
    """gk_gather through the C ABI: entries of 0..65536 bytes at every
    relative alignment (16-, 4- and 1-byte paths), from pinned host memory
    and from device memory, bytes outside the entries untouched, entries
    above the maximum skipped."""
    require_gpu()
    rng = np.random.default_rng(8)
    n_bytes = 8 << 20
    host = torch.from_numpy(rng.integers(0, 256, n_bytes, dtype=np.uint8)).pin_memory()
    dev_src = host.cuda()
    for src_t in (host, dev_src):
        dst = torch.full((n_bytes,), 0xAB, dtype=torch.uint8, device="cuda")
        sizes = np.concatenate([[0, 1, 2, 3, 4, 15, 16, 17, 31, 33, 4095, 4096, 65535, 65536],
                                rng.integers(0, 65537, 60)]).astype(np.int64)
        want = np.full(n_bytes, 0xAB, np.uint8)
        hs = host.numpy()
        d_off, s_off, pos = [], [], 0
        for k, z in enumerate(sizes):
            so = int(rng.integers(0, n_bytes - 70_000))
            do = pos + int(rng.integers(0, 32))  # destinations never overlap
            pos = do + int(z) + 64
            assert pos < n_bytes
            d_off.append(do)
            s_off.append(so)
            want[do:do + z] = hs[so:so + z]
        # one entry above the maximum: skipped
        d_off.append(pos)
        s_off.append(0)
        sizes = np.append(sizes, 65537)
        tab = torch.empty(3 * len(sizes), dtype=torch.int64, pin_memory=True)
        t = tab.numpy()
        n = len(sizes)
        t[:n] = dst.data_ptr() + np.array(d_off, np.int64)
        t[n:2 * n] = src_t.data_ptr() + np.array(s_off, np.int64)
        t[2 * n:] = sizes
        gk.gk_gather(tab[:n], tab[n:2 * n], tab[2 * n:], n)
        torch.cuda.synchronize()
        assert np.array_equal(dst.cpu().numpy(), want)
