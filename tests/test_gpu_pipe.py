"""The streamed host pipeline (gk_pipe_*): batches of host reads and pairs,
several in flight, every threshold's results back in host memory, equal to
the oracle pair by pair."""
import numpy as np
import pytest
import torch

from paper_2103_14978_gb300 import gk, synth
from tests.gpu_helpers import accept_of_result_bytes, assert_same, oracle_run, require_gpu

pytestmark = pytest.mark.gpu

THRESHOLDS = (0, 2, 5, 10)


def batches_of(w: synth.Workload, read_cuts):
    """Split a workload whose pairs are grouped by read into batches of whole
    reads: (ascii, n_reads, pair_read rebased, pair_off, global pair index)."""
    out = []
    for r0, r1 in zip(read_cuts[:-1], read_cuts[1:]):
        idx = np.nonzero((w.pair_read >= r0) & (w.pair_read < r1))[0]
        asc = np.ascontiguousarray(w.reads.reshape(w.n_reads, w.stride)[r0:r1]).reshape(-1)
        out.append((asc, r1 - r0, (w.pair_read[idx] - r0).astype(np.uint32), w.pair_off[idx].copy(), idx))
    return out


def pinned(a: np.ndarray) -> torch.Tensor:
    t = torch.from_numpy(a.view(np.int32) if a.dtype == np.uint32 else a).pin_memory()
    return t


@pytest.mark.parametrize("n_slots,ths,flags", [(2, THRESHOLDS, 0), (3, THRESHOLDS, 0), (4, THRESHOLDS, 0),
                                               (3, (1, 12), 0), (3, (0, 1, 2, 5, 6, 7, 29, 30, 31, 40), 0),
                                               (3, THRESHOLDS, 4), (2, (1, 12), 4), (3, THRESHOLDS, 8),
                                               (2, (1, 12), 12)])
def test_pipe_batches_equal_the_oracle(n_slots, ths, flags):
    """Runs of consecutive thresholds take one gk_filter_sweep each (shift
    counts up to 30), thresholds above it gk_filter; with GK_PIPE_SLICED
    (flags 4) gk_slice + gk_filter_sliced_sweep where the sliced filter
    covers the set, gk_filter otherwise; with GK_PIPE_READ_STARTS (flags 8)
    the pairs' reads travel as one start per read."""
    require_gpu()
    THRESHOLDS = ths
    w = synth.config2(scale=0.001, ref_bases=2_000_000)
    ref = gk.gk_load_reference(w.ref)
    cuts = [0, 700, 700, 1900, 2600, 4100, w.n_reads]  # includes an empty batch
    bs = batches_of(w, cuts)
    max_reads = max(b[1] for b in bs)
    max_pairs = max(b[2].size for b in bs)
    want = {e: oracle_run(w, e) for e in THRESHOLDS}
    with gk.Pipe(ref, max_reads, w.stride, 100, max_pairs, THRESHOLDS, n_slots=n_slots, flags=flags) as pipe:
        jobs = []
        for asc, nr, pr, po, idx in bs:
            acc = torch.empty(len(THRESHOLDS) * pr.size, dtype=torch.uint8).pin_memory()
            ed = torch.empty(len(THRESHOLDS) * pr.size, dtype=torch.int16).pin_memory()
            link = pr
            if flags & gk.GK_PIPE_READ_STARTS:  # the batch's pairs are grouped by read
                assert np.all(np.diff(pr.astype(np.int64)) >= 0)
                link = np.searchsorted(pr, np.arange(nr)).astype(np.uint32)
            t = pipe.submit(pinned(asc), nr, pinned(link), pinned(po), acc, ed)
            jobs.append((t, acc, ed, idx))
        assert [j[0] for j in jobs] == list(range(len(bs)))
        pipe.wait(jobs[-1][0])  # the last ticket covers every earlier one
        for t, acc, ed, idx in jobs:
            n = idx.size
            a = acc.numpy().reshape(len(THRESHOLDS), n)
            d = ed.numpy().view(np.uint16).reshape(len(THRESHOLDS), n)
            for i, e in enumerate(THRESHOLDS):
                assert_same((a[i], d[i]), (want[e][0][idx], want[e][1][idx]), f"batch {t} e={e}")
    ref.close()


def test_pipe_reuses_slots_many_times_and_rejects_oversize():
    require_gpu()
    w = synth.config2(scale=0.0005, ref_bases=2_000_000)
    ref = gk.gk_load_reference(w.ref)
    bs = batches_of(w, list(range(0, w.n_reads + 1, 250)))
    want = oracle_run(w, 3)
    pipe = gk.Pipe(ref, 250, w.stride, 100, max(b[2].size for b in bs), (3,), n_slots=2)
    acc_all = np.zeros(w.n_pairs, np.uint8)
    ed_all = np.zeros(w.n_pairs, np.uint16)
    pending = []
    for asc, nr, pr, po, idx in bs:
        acc = torch.empty(pr.size, dtype=torch.uint8).pin_memory()
        ed = torch.empty(pr.size, dtype=torch.int16).pin_memory()
        pending.append((pipe.submit(pinned(asc), nr, pinned(pr), pinned(po), acc, ed), acc, ed, idx))
        if len(pending) == 3:  # consume in order, a few batches behind
            t, a, d, i = pending.pop(0)
            pipe.wait(t)
            acc_all[i], ed_all[i] = a.numpy(), d.numpy().view(np.uint16)
    for t, a, d, i in pending:
        pipe.wait(t)
        acc_all[i], ed_all[i] = a.numpy(), d.numpy().view(np.uint16)
    assert_same((acc_all, ed_all), want, "10 batches through 2 slots")
    big = np.zeros(251 * w.stride, np.uint8)
    with pytest.raises(gk.GKError) as ex:
        pipe.submit(big, 251, np.zeros(1, np.uint32), np.zeros(1, np.uint32), np.zeros(1, np.uint8),
                    np.zeros(1, np.uint16))
    assert ex.value.code == gk.GK_ERANGE
    with pytest.raises(gk.GKError):
        pipe.wait(10_000)
    pipe.close()
    ref.close()


def _result_bytes_of(acc, ed):
    """Expected GK_FLAG_RESULT_BYTE bytes from the split results."""
    ed = ed.astype(np.int64)
    out = np.minimum(ed, gk.GK_RESULT_MAX_COUNT)
    out[ed == gk.GK_EDITS_UNDEFINED] = gk.GK_RESULT_UNDEFINED
    out[ed == gk.GK_EDITS_INVALID] = gk.GK_RESULT_INVALID
    return out.astype(np.uint8)


def test_pipe_result_bytes_equal_the_oracle():
    """GK_FLAG_RESULT_BYTE through the pipe: one byte per pair and threshold,
    no edit counts moved; each byte is the oracle's count (capped at 253) or
    a sentinel, and decides accept exactly."""
    require_gpu()
    w = synth.config2(scale=0.001, ref_bases=2_000_000)
    ref = gk.gk_load_reference(w.ref)
    bs = batches_of(w, [0, 1500, 3100, w.n_reads])
    max_reads = max(b[1] for b in bs)
    max_pairs = max(b[2].size for b in bs)
    want = {e: oracle_run(w, e) for e in THRESHOLDS}
    with gk.Pipe(ref, max_reads, w.stride, 100, max_pairs, THRESHOLDS, flags=gk.GK_FLAG_RESULT_BYTE) as pipe:
        jobs = []
        for asc, nr, pr, po, idx in bs:
            res = torch.empty(len(THRESHOLDS) * pr.size, dtype=torch.uint8).pin_memory()
            jobs.append((pipe.submit(pinned(asc), nr, pinned(pr), pinned(po), res, None), res, idx))
        pipe.wait(jobs[-1][0])
        for t, res, idx in jobs:
            r = res.numpy().reshape(len(THRESHOLDS), idx.size)
            for i, e in enumerate(THRESHOLDS):
                wa, we = want[e][0][idx], want[e][1][idx]
                assert np.array_equal(r[i], _result_bytes_of(wa, we)), f"batch {t} e={e}"
                acc = accept_of_result_bytes(r[i], e)
                assert np.array_equal(acc, wa), f"batch {t} e={e}"
    with pytest.raises(gk.GKError):
        gk.Pipe(ref, 10, w.stride, 100, 10, (3, 253), flags=gk.GK_FLAG_RESULT_BYTE)
    ref.close()


def test_pipe_read_starts_leave_unclaimed_pairs_invalid():
    """GK_PIPE_READ_STARTS with starts that skip pairs (the first read starts
    at 3, so no read claims pairs 0..2): claimed pairs equal the oracle,
    unclaimed pairs come back invalid (accept 0, GK_EDITS_INVALID; result
    byte GK_RESULT_INVALID)."""
    require_gpu()
    w = synth.config2(scale=0.0002, ref_bases=2_000_000)
    ref = gk.gk_load_reference(w.ref)
    (asc, nr, pr, po, idx), = batches_of(w, [0, 600])
    starts = np.searchsorted(pr, np.arange(nr)).astype(np.uint32)
    assert starts[0] == 0 and starts[1] >= 4
    starts[0] = 3
    claimed = np.arange(pr.size) >= 3
    want = oracle_run(w, 4)
    for flags in (gk.GK_PIPE_READ_STARTS, gk.GK_PIPE_READ_STARTS | gk.GK_FLAG_RESULT_BYTE):
        with gk.Pipe(ref, nr, w.stride, 100, pr.size, (4,), flags=flags) as pipe:
            acc = torch.empty(pr.size, dtype=torch.uint8).pin_memory()
            ed = torch.empty(pr.size, dtype=torch.int16).pin_memory()
            pipe.wait(pipe.submit(pinned(asc), nr, pinned(starts), pinned(po), acc, ed))
            a = acc.numpy()
            if flags & gk.GK_FLAG_RESULT_BYTE:
                assert np.all(a[~claimed] == gk.GK_RESULT_INVALID)
                assert np.array_equal(a[claimed], _result_bytes_of(want[0][idx][claimed], want[1][idx][claimed]))
            else:
                d = ed.numpy().view(np.uint16)
                assert np.all(a[~claimed] == 0) and np.all(d[~claimed] == gk.GK_EDITS_INVALID)
                assert_same((a[claimed], d[claimed]), (want[0][idx][claimed], want[1][idx][claimed]), "claimed")
    ref.close()
