"""Bit-exact parity of the batched persistent filter (gk_filter_batched) with
the oracle, on mixed read lengths and per-pair thresholds, for every
words-per-lane choice; graph replay; agreement with the plain filter."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2103_14978_gb300 import batch, device_data as dd, gk, synth
from tests.gpu_helpers import assert_same, oracle_run, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


class Batched:
    def __init__(self, w: synth.Workload):
        self.w = w
        self.ref = gk.gk_load_reference(w.ref)
        self.reads = dd.upload_reads(w.reads, w.read_len, w.stride)
        self.read_len = dd.as_i16(w.read_len).cuda()
        self.pairs = dd.upload_pairs(w.pair_read, w.pair_off, w.pair_e)

    def filter_(self, tiling, e=None, mode=gk.GK_COUNT_RUNS4, flags=0, err=None):
        if e is None:
            e = self.pairs.pair_e if self.pairs.pair_e is not None else self.w.e
        bf = batch.BatchedFilter(self.ref, self.reads.packed, self.reads.stride_words, self.reads.n_reads,
                                 self.read_len, self.reads.nflag, self.pairs.pair_read, self.pairs.pair_off, e,
                                 tiling, mode, flags, err)
        bf.run()
        torch.cuda.synchronize()
        return bf, (bf.accept.cpu().numpy(), dd.edits_u16(bf.edits))


def mixed_workload(seed, n_pairs=30000, m=(1, 512), rates=(0.0, 0.02, 0.05, 0.10, 0.3, 1.0), n_frac=0.0,
                   read_n_frac=0.0, ref_len=400_000):
    ref = synth.reference(ref_len, seed, 0.05, n_frac)
    return synth.pairs_workload("mixed", seed=seed, ref=ref, n_pairs=n_pairs, m=m, cands=4,
                                e_rates=rates, read_edit_rate=0.04, read_n_frac=read_n_frac, shuffle=True)


@pytest.fixture(scope="module")
def mixed():
    w = mixed_workload(31)
    rng = np.random.default_rng(2)
    w.pair_e[rng.integers(0, w.n_pairs, 300)] = 255
    w.pair_e[rng.integers(0, w.n_pairs, 300)] = 0
    return Batched(w), oracle_run(w)


@pytest.mark.parametrize("wpt", [1, 2, 3, 4, 6, 8])
def test_batched_parity_every_wpt(mixed, wpt):
    b, want = mixed
    _, got = b.filter_((wpt, 256, 2, 8))
    assert_same(got, want, f"batched wpt={wpt}")


@pytest.mark.parametrize("tiling", [(4, 32, 1, 1), (2, 65536, 1, 4), (3, 64, 8, 4), (8, 1024, 1, 8), (1, 32, 2, 8), (1, 4096, 1, 2)])
def test_batched_parity_tilings(mixed, tiling):
    b, want = mixed
    _, got = b.filter_(tiling)
    assert_same(got, want, f"batched tiling={tiling}")


def test_batched_modes_and_variants():
    w = mixed_workload(32, n_pairs=12000, m=(1, 300))
    b = Batched(w)
    for mode, flags in ((gk.GK_COUNT_POPCOUNT, 0), (gk.GK_COUNT_RUNS4, gk.GK_FLAG_NO_EDGE_FIX),
                        (gk.GK_COUNT_POPCOUNT, gk.GK_FLAG_NO_EDGE_FIX)):
        _, got = b.filter_((3, 128, 2, 8), mode=mode, flags=flags)
        assert_same(got, oracle_run(w, None, mode, flags), f"batched mode={mode} flags={flags}")
    for e in (0, 7, 255):  # one scalar threshold for every pair
        _, got = b.filter_((4, 256, 2, 8), e=e)
        assert_same(got, oracle_run(w, e), f"batched scalar e={e}")


def test_batched_result_bytes():
    """GK_FLAG_RESULT_BYTE with per-pair thresholds 0..255: one byte per
    pair (count capped at GK_RESULT_MAX_COUNT, GK_RESULT_UNDEFINED,
    GK_RESULT_INVALID) equal to the oracle's counts in that format, with N
    and invalid pairs, and no edits buffer."""
    w = mixed_workload(34, n_pairs=20000, m=(20, 300), n_frac=0.001, read_n_frac=0.001)
    w.pair_read[:50] = w.n_reads + 7
    b = Batched(w)
    ws = torch.empty(gk.gk_filter_batched_workspace(w.n_pairs), dtype=torch.uint8, device="cuda")
    res, none = gk.gk_filter_batched(b.ref, b.reads.packed, b.reads.stride_words, b.reads.n_reads, b.read_len,
                                     b.reads.nflag, b.pairs.pair_read, b.pairs.pair_off, b.pairs.pair_e,
                                     gk.Tiling(3, 256, 2, 8), ws, flags=gk.GK_FLAG_RESULT_BYTE)
    torch.cuda.synchronize()
    assert none is None
    _, e = oracle_run(w)
    e = e.astype(np.int64)
    want = np.where(e == O.UNDEFINED, gk.GK_RESULT_UNDEFINED,
                    np.where(e == O.INVALID, gk.GK_RESULT_INVALID, np.minimum(e, gk.GK_RESULT_MAX_COUNT)))
    assert np.array_equal(res.cpu().numpy(), want.astype(np.uint8))
    assert (e == O.UNDEFINED).sum() > 50 and (e == O.INVALID).sum() >= 50


def test_batched_undefined_and_invalid():
    w = mixed_workload(33, n_pairs=20000, m=(20, 300), n_frac=0.001, read_n_frac=0.001)
    rng = np.random.default_rng(6)
    L = w.ref.shape[0]
    bad_id = rng.integers(0, w.n_pairs, 150)
    w.pair_read[bad_id] = w.n_reads + rng.integers(0, 100, 150).astype(np.uint32)
    bad_off = rng.integers(0, w.n_pairs, 150)
    w.pair_off[bad_off] = L - 10 + rng.integers(0, 100, 150).astype(np.uint32)
    w.read_len[rng.integers(0, w.n_reads, 20)] = 0  # empty reads
    b = Batched(w)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    _, got = b.filter_((4, 256, 2, 8), err=err)
    want = oracle_run(w)
    assert_same(got, want, "batched N/invalid")
    assert int(err.item()) == int((want[1] == O.INVALID).sum()) > 0
    assert (want[1] == O.UNDEFINED).sum() > 100


def test_graph_replay_and_plain_agreement():
    """One graph-captured launch, replayed twice, equals the plain per-length
    launches over the same pairs (config 4 structure, scaled)."""
    w = synth.config4(scale=0.004, ref_bases=20_000_000)
    b = Batched(w)
    bf = batch.BatchedFilter(b.ref, b.reads.packed, b.reads.stride_words, b.reads.n_reads, b.read_len,
                             b.reads.nflag, b.pairs.pair_read, b.pairs.pair_off, b.pairs.pair_e, (4, 256, 4, 8))
    bf.capture()
    outs = []
    for _ in range(2):
        bf.accept.fill_(7)
        bf.edits.fill_(-7)
        bf.replay()
        torch.cuda.synchronize()
        outs.append((bf.accept.cpu().numpy().copy(), dd.edits_u16(bf.edits).copy()))
    assert_same(outs[0], outs[1], "replay")
    # plain per-length launches over the same pairs
    m_pair = w.read_len[w.pair_read]
    acc = np.empty(w.n_pairs, np.uint8)
    ed = np.empty(w.n_pairs, np.uint16)
    for m in np.unique(m_pair):
        idx = np.nonzero(m_pair == m)[0]
        pr = dd.as_i32(w.pair_read[idx]).cuda()
        po = dd.as_i32(w.pair_off[idx]).cuda()
        pe = torch.from_numpy(w.pair_e[idx]).cuda()
        a, e = gk.gk_filter(b.ref, b.reads.packed, b.reads.stride_words, b.reads.n_reads, b.reads.nflag,
                            int(m), pr, po, pe)
        torch.cuda.synchronize()
        acc[idx] = a.cpu().numpy()
        ed[idx] = dd.edits_u16(e)
    assert_same(outs[0], (acc, ed), "batched vs plain")
    sample = np.random.default_rng(1).choice(w.n_pairs, 40000, replace=False)
    want = oracle_run(w, idx=sample)
    assert_same((outs[0][0][sample], outs[0][1][sample]), want, "batched vs oracle (sample)")


def test_autotuner_picks_a_valid_tiling():
    w = synth.config4(scale=0.002, ref_bases=20_000_000)
    b = Batched(w)
    best, results = batch.autotune(b.ref, b.reads.packed, b.reads.stride_words, b.reads.n_reads, b.read_len,
                                   b.reads.nflag, b.pairs.pair_read, b.pairs.pair_off, b.pairs.pair_e,
                                   reps=1, budget_s=30)
    assert best in results and np.isfinite(results[best])
    assert results[best] == min(v for v in results.values())
    _, got = b.filter_(best)
    sample = np.random.default_rng(2).choice(w.n_pairs, 20000, replace=False)
    assert_same((got[0][sample], got[1][sample]), oracle_run(w, idx=sample), "autotuned")


def test_whole_pair_odd_stride_and_unaligned_reads():
    """One pair per lane with the 8-byte read loads: an odd row stride
    (9 words for reads up to 288 bases), and an even stride whose read buffer
    starts 8 bytes past a 16-byte boundary."""
    w = mixed_workload(34, n_pairs=15000, m=(1, 288))
    want = oracle_run(w)
    b = Batched(w)
    assert b.reads.stride_words == 9
    for tiling in ((1, 256, 2, 8), (4, 256, 2, 8)):
        _, got = b.filter_(tiling)
        assert_same(got, want, f"odd stride {tiling}")
    r10 = dd.upload_reads(w.reads, w.read_len, w.stride, stride_words=10)
    buf = torch.zeros(r10.packed.numel() + 2, dtype=torch.int32, device="cuda")
    buf[2:] = r10.packed
    shifted = buf[2:]
    assert shifted.data_ptr() % 16 == 8
    bf = batch.BatchedFilter(b.ref, shifted, 10, r10.n_reads, b.read_len, r10.nflag, b.pairs.pair_read,
                             b.pairs.pair_off, b.pairs.pair_e, (1, 256, 2, 8))
    bf.run()
    torch.cuda.synchronize()
    assert_same((bf.accept.cpu().numpy(), dd.edits_u16(bf.edits)), want, "unaligned read buffer")


@pytest.mark.parametrize("ref_len", [4096, 4100, 4127])
def test_batched_windows_at_reference_end(ref_len):
    """Windows ending at the genome's last base, for W odd and even and
    window starts in odd and even words (the 16-byte window loads read up to
    the genome's zero tail words)."""
    ref = synth.reference(ref_len, 40, 0.0, 0.0)
    rng = np.random.default_rng(ref_len)
    ms = np.array([1, 31, 32, 33, 63, 64, 65, 95, 96, 97, 100, 128, 150, 250, 255, 288, 300, 320, 416, 500, 512])
    rows, lens, offs = [], [], []
    for m in ms:
        for o in range(ref_len - int(m) - 70, ref_len - int(m) + 1):
            seq = np.frombuffer(bytes(ref[o:o + m]), np.uint8).copy()
            flip = rng.random(m) < 0.03
            seq[flip] = synth.BASES[rng.integers(0, 4, int(flip.sum()))]
            row = np.full(512, ord("N"), np.uint8)
            row[:m] = seq
            rows.append(row)
            lens.append(m)
            offs.append(o)
    n = len(rows)
    pair_e = rng.integers(0, 40, n).astype(np.uint8)
    w = synth.Workload("end-mixed", np.concatenate(rows), np.asarray(lens, np.uint16), 512, ref,
                       np.arange(n, dtype=np.uint32), np.asarray(offs, np.uint32), pair_e=pair_e)
    b = Batched(w)
    want = oracle_run(w)
    for tiling in ((1, 64, 2, 8), (2, 64, 2, 8)):
        _, got = b.filter_(tiling)
        assert_same(got, want, f"end ref_len={ref_len} {tiling}")
