"""Bit-exact parity of the CUDA filter (through the C-ABI) with the CPU
oracle, on seeded synthetic inputs: every accept bit and edit count must be
identical (integer work, tolerance 0)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2103_14978_gb300 import device_data as dd, gk, synth
from tests.gpu_helpers import GpuRun, accept_of_result_bytes, assert_same, oracle_run, require_gpu, small_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def c1():
    w = synth.config1()
    return w, GpuRun(w)


def test_config1_parity(c1):
    """10,000 pairs, 100 bp, e=2: the small configuration, every pair."""
    w, run = c1
    assert_same(run.filter(), oracle_run(w), "c1 e=2")


@pytest.mark.parametrize("mode,flags", [(gk.GK_COUNT_RUNS4, 0), (gk.GK_COUNT_POPCOUNT, 0),
                                        (gk.GK_COUNT_RUNS4, gk.GK_FLAG_NO_EDGE_FIX),
                                        (gk.GK_COUNT_POPCOUNT, gk.GK_FLAG_NO_EDGE_FIX)])
def test_config1_e_sweep_modes(c1, mode, flags):
    w, run = c1
    for e in (0, 1, 3, 5, 10, 99, 100, 255):
        assert_same(run.filter(e=e, mode=mode, flags=flags), oracle_run(w, e, mode, flags),
                    f"c1 e={e} mode={mode} flags={flags}")


LENGTHS = [1, 2, 3, 31, 32, 33, 63, 64, 65, 95, 96, 97, 100, 127, 128, 150, 160, 250, 255, 256,
           300, 320, 384, 416, 448, 480, 500, 511, 512]


@pytest.mark.parametrize("m", LENGTHS)
def test_read_lengths_and_thresholds(m):
    """Every words-per-read template, word-boundary lengths, e from 0 past m."""
    w = small_workload(m, 1500, seed=100 + m)
    run = GpuRun(w)
    for e in sorted({0, 1, 2, max(1, m // 10), min(255, m - 1), min(255, m), min(255, m + 1), 255}):
        assert_same(run.filter(e=e), oracle_run(w, e), f"m={m} e={e}")
    assert_same(run.filter(e=max(1, m // 20), flags=gk.GK_FLAG_NO_EDGE_FIX),
                oracle_run(w, max(1, m // 20), O.RUNS4, O.FLAG_NO_EDGE_FIX), f"m={m} no edge")


def test_per_pair_thresholds():
    w = small_workload(150, 20000, seed=7, e_rates=(0.0, 0.02, 0.05, 0.10, 0.5, 1.0))
    rng = np.random.default_rng(3)
    w.pair_e[rng.integers(0, w.n_pairs, 200)] = 255
    run = GpuRun(w)
    assert_same(run.filter(), oracle_run(w), "per-pair e")
    assert_same(run.filter(mode=gk.GK_COUNT_POPCOUNT), oracle_run(w, None, O.POPCOUNT), "per-pair e popcount")


def test_undefined_bases():
    """'N' at 0.1% of reference and read positions (config 3 structure), plus
    windows with an N exactly at their first or last base."""
    w = small_workload(150, 20000, seed=9, n_frac=0.001, read_n_frac=0.001, cands=(8, 64))
    ref = w.ref.copy()
    rng = np.random.default_rng(4)
    # force N at the first / last base of some windows
    sel = rng.integers(0, w.n_pairs, 300)
    for i, p in enumerate(sel):
        o = int(w.pair_off[p])
        ref[o if i % 2 == 0 else o + 149] = ord("N")
    w.ref = ref
    run = GpuRun(w)
    for e in (0, 2, 4, 8, 15):
        got = run.filter(e=e)
        assert_same(got, oracle_run(w, e), f"N e={e}")
    assert (got[1] == gk.GK_EDITS_UNDEFINED).sum() > 300
    assert run.ref.n_undefined == int((ref == ord("N")).sum())


@pytest.mark.parametrize("m", [64, 100, 180, 200, 250, 300])
def test_undefined_bases_both_layouts(m):
    """A genome and reads with N: thresholds on both sides of the switch
    between one thread per pair and the queue of defined pairs, per-pair
    thresholds, and invalid pairs counted on either side."""
    w = small_workload(m, 6000, seed=900 + m, n_frac=0.001, read_n_frac=0.001, cands=(8, 64),
                       e_rates=(0.0, 0.02, 0.05, 0.10))
    rng = np.random.default_rng(m)
    bad = rng.choice(w.n_pairs, 40, replace=False)
    w.pair_read[bad[:20]] = w.n_reads + 3
    w.pair_off[bad[20:]] = w.ref.shape[0] - m + 1
    run = GpuRun(w)
    for e in (0, 1, 2, 3, 4, 6, 7, 9, 10, 12):
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert_same(run.filter(e=e, err=err), oracle_run(w, e), f"N m={m} e={e}")
        assert int(err.item()) == 40
    assert_same(run.filter(), oracle_run(w), f"N m={m} per-pair e")


@pytest.mark.parametrize("m", [17, 64, 100, 150, 250])
def test_pairs_in_any_order(m):
    """Pairs grouped by read (two neighbours share the read's shifted copies),
    shuffled (each pair on its own) and half-shuffled, with an odd pair count
    and invalid pairs among them."""
    w = small_workload(m, 3001, seed=700 + m, cands=(1, 6))
    rng = np.random.default_rng(m)
    w.pair_read[rng.choice(w.n_pairs, 15, replace=False)] = w.n_reads + 1
    half = np.arange(w.n_pairs)
    half[: w.n_pairs // 2] = rng.permutation(w.n_pairs // 2)
    for name, idx in (("grouped", np.arange(w.n_pairs)), ("shuffled", rng.permutation(w.n_pairs)),
                      ("half", half)):
        ws = w.subset(idx)
        run = GpuRun(ws)
        for e in (2, 3, 7, min(30, m - 1)):
            assert_same(run.filter(e=e), oracle_run(ws, e), f"{name} m={m} e={e}")


@pytest.mark.parametrize("m", [31, 100, 150, 250])
def test_result_byte_format(m):
    """GK_FLAG_RESULT_BYTE: each pair's byte is its count capped at 253, 254
    for undefined and 255 for invalid pairs, on both layouts (genome with N),
    against the split results and the oracle; the flag's argument rules."""
    w = small_workload(m, 5000, seed=1100 + m, n_frac=0.001, read_n_frac=0.001, cands=(1, 8))
    w.pair_read[:25] = w.n_reads + 2
    run = GpuRun(w)
    r = run.reads
    for e in (0, 1, 2, 5, 9, min(252, m - 1), 252):
        a, d = run.filter(e=e)
        res, none = gk.gk_filter(run.ref, r.packed, r.stride_words, r.n_reads, r.nflag, m,
                                 run.pairs.pair_read, run.pairs.pair_off, e, flags=gk.GK_FLAG_RESULT_BYTE)
        torch.cuda.synchronize()
        assert none is None
        d64 = d.astype(np.int64)
        want = np.minimum(d64, 253)
        want[d64 == O.UNDEFINED] = 254
        want[d64 == O.INVALID] = 255
        assert np.array_equal(res.cpu().numpy(), want.astype(np.uint8)), f"m={m} e={e}"
        assert np.array_equal(accept_of_result_bytes(res, e), a)
        assert_same((a, d), oracle_run(w, e), f"m={m} e={e}")
    with pytest.raises(gk.GKError) as exc:
        gk.gk_filter(run.ref, r.packed, r.stride_words, r.n_reads, r.nflag, m, run.pairs.pair_read,
                     run.pairs.pair_off, 253, flags=gk.GK_FLAG_RESULT_BYTE)
    assert exc.value.code == gk.GK_ERANGE
    pe = torch.full((w.n_pairs,), 3, dtype=torch.uint8, device="cuda")
    with pytest.raises(gk.GKError) as exc:
        gk.gk_filter(run.ref, r.packed, r.stride_words, r.n_reads, r.nflag, m, run.pairs.pair_read,
                     run.pairs.pair_off, pe, flags=gk.GK_FLAG_RESULT_BYTE)
    assert exc.value.code == gk.GK_EINVAL


def test_invalid_pairs_and_error_counter():
    w = small_workload(100, 4000, seed=11, ref_len=50_000)
    L = w.ref.shape[0]
    rng = np.random.default_rng(5)
    pr = w.pair_read.copy()
    po = w.pair_off.copy()
    bad_read = rng.integers(0, 4000, 100)
    pr[bad_read] = w.n_reads + rng.integers(0, 1000, 100)
    bad_off = rng.integers(0, 4000, 100)
    po[bad_off] = L - 100 + rng.integers(1, 500, 100)
    po[:10] = L - 100  # the last valid window
    po[10:20] = 0xFFFFFFFF
    w2 = w.subset(np.arange(w.n_pairs))
    w2.pair_read, w2.pair_off = pr, po
    run = GpuRun(w2)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = run.filter(e=3, err=err)
    want = oracle_run(w2, 3)
    assert_same(got, want, "invalid")
    n_invalid = int((want[1] == O.INVALID).sum())
    assert n_invalid >= 200
    assert int(err.item()) == n_invalid
    assert (got[0][want[1] == O.INVALID] == 0).all()


def test_windows_at_reference_end():
    ref = synth.reference(4096, 12, 0.0, 0.0)
    for m in (1, 31, 32, 33, 100, 250, 512):
        offs = np.arange(max(0, 4096 - m - 40), 4096 - m + 1, dtype=np.uint32)
        rng = np.random.default_rng(m)
        reads = np.stack([np.frombuffer(bytes(ref[o:o + m]), np.uint8) for o in offs]).copy()
        flip = rng.random(reads.shape) < 0.03
        reads[flip] = synth.BASES[rng.integers(0, 4, int(flip.sum()))]
        w = synth.Workload("end", reads.reshape(-1), np.full(offs.size, m, np.uint16), m, ref,
                           np.arange(offs.size, dtype=np.uint32), offs, e=0)
        run = GpuRun(w)
        for e in (0, 2, 7):
            assert_same(run.filter(e=e), oracle_run(w, e), f"end m={m} e={e}")


def test_empty_and_zero_length():
    w = small_workload(100, 100, seed=13, ref_len=10_000)
    run = GpuRun(w)
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    acc, ed = gk.gk_filter(run.ref, run.reads.packed, run.reads.stride_words, run.reads.n_reads,
                           run.reads.nflag, 100, empty, empty, 2)
    assert acc.numel() == 0 and ed.numel() == 0
    # m = 0: every valid pair accepted with 0 edits, invalid ones flagged
    po = torch.tensor([0, 10_000, 10_001], dtype=torch.int32, device="cuda")
    pr = torch.tensor([0, 0, 0], dtype=torch.int32, device="cuda")
    acc, ed = gk.gk_filter(run.ref, run.reads.packed, run.reads.stride_words, run.reads.n_reads,
                           run.reads.nflag, 0, pr, po, 5)
    torch.cuda.synchronize()
    assert acc.cpu().tolist() == [1, 1, 0]
    assert dd.edits_u16(ed).tolist() == [0, 0, O.INVALID]


def test_device_encoder_matches_host_encoder():
    rng = np.random.default_rng(8)
    for stride, maxlen in ((100, 100), (150, 150), (301, 300), (512, 512), (1000, 512)):
        n = 777
        lens = rng.integers(0, maxlen + 1, n).astype(np.uint16)
        asc = rng.choice(np.frombuffer(b"ACGTNacgtn", np.uint8), n * stride)
        sw = gk.words_for(maxlen)
        hp, hn = gk.gk_encode(torch.from_numpy(asc), n, stride, lens=dd.as_i16(lens), stride_words=sw)
        dp, dn = gk.gk_encode(torch.from_numpy(asc).cuda(), n, stride, lens=dd.as_i16(lens).cuda(),
                              stride_words=sw)
        torch.cuda.synchronize()
        assert torch.equal(hp, dp.cpu()) and torch.equal(hn, dn.cpu()), stride
        fp, fn = gk.gk_encode(torch.from_numpy(asc).cuda(), n, stride, fixed_len=maxlen, stride_words=sw)
        hp2, hn2 = gk.gk_encode(torch.from_numpy(asc), n, stride, fixed_len=maxlen, stride_words=sw)
        torch.cuda.synchronize()
        assert torch.equal(hp2, fp.cpu()) and torch.equal(hn2, fn.cpu())


def test_device_encoder_every_byte_value_and_rare_undefined_bases():
    """Device encoder against the host encoder where most 32-base words are
    all A/C/G/T in either case (its fast path) and a few hold one other byte;
    and every byte value 0..255 at several positions of a read."""
    rng = np.random.default_rng(9)
    valid = np.frombuffer(b"ACGTacgt", np.uint8)
    others = np.setdiff1d(np.arange(256, dtype=np.uint8), valid)
    for stride, maxlen in ((100, 100), (97, 97), (150, 150), (256, 250), (333, 320)):
        n = 3000
        lens = rng.integers(0, maxlen + 1, n).astype(np.uint16)
        asc = rng.choice(valid, n * stride)
        hit = rng.random(n * stride) < 0.002
        asc[hit] = rng.choice(others, int(hit.sum()))
        sw = gk.words_for(maxlen)
        hp, hn = gk.gk_encode(torch.from_numpy(asc), n, stride, lens=dd.as_i16(lens), stride_words=sw)
        dp, dn = gk.gk_encode(torch.from_numpy(asc).cuda(), n, stride, lens=dd.as_i16(lens).cuda(),
                              stride_words=sw)
        torch.cuda.synchronize()
        assert torch.equal(hp, dp.cpu()) and torch.equal(hn, dn.cpu()), stride
        assert 0 < int(hn.sum()) < n
    # every byte value at positions 0, 13, 31, 32, 63 and 99 of a 100-base read
    pos = (0, 13, 31, 32, 63, 99)
    n = 256 * len(pos)
    asc = rng.choice(valid, n * 100)
    for i, (b, k) in enumerate((b, k) for b in range(256) for k in pos):
        asc[i * 100 + k] = b
    hp, hn = gk.gk_encode(torch.from_numpy(asc), n, 100, fixed_len=100, stride_words=4)
    dp, dn = gk.gk_encode(torch.from_numpy(asc).cuda(), n, 100, fixed_len=100, stride_words=4)
    torch.cuda.synchronize()
    assert torch.equal(hp, dp.cpu()) and torch.equal(hn, dn.cpu())
    assert int(hn.sum()) == len(others) * len(pos)


@pytest.mark.parametrize("stride,m,sw", [(100, 100, 4), (100, 97, 4), (64, 60, 4), (128, 128, 4), (256, 250, 8),
                                         (32, 31, 1), (36, 33, 2), (512, 500, 16), (100, 100, 8)])
def test_device_encoder_one_length_word_per_thread(stride, m, sw):
    """One read length in 4-byte aligned rows with a power-of-two row (the
    one-thread-per-word encoder): the host encoder's words and N flags, with
    rare non-ACGT bytes, lengths not a multiple of 4 or 32 and rows wider
    than the read (words past ceil(m/32) zero)."""
    rng = np.random.default_rng(stride * 1000 + m)
    valid = np.frombuffer(b"ACGTacgt", np.uint8)
    others = np.setdiff1d(np.arange(256, dtype=np.uint8), valid)
    n = 4099
    asc = rng.choice(valid, n * stride)
    hit = rng.random(n * stride) < 0.001
    asc[hit] = rng.choice(others, int(hit.sum()))
    hp, hn = gk.gk_encode(torch.from_numpy(asc), n, stride, fixed_len=m, stride_words=sw)
    dp, dn = gk.gk_encode(torch.from_numpy(asc).cuda(), n, stride, fixed_len=m, stride_words=sw)
    torch.cuda.synchronize()
    assert torch.equal(hp, dp.cpu()) and torch.equal(hn, dn.cpu()), (stride, m, sw)
    assert 0 < int(hn.sum()) < n


def test_config2_structure_scaled():
    """Config 2's structure (duplicated genome regions, 4 candidates per read,
    1 true origin) at 1/500 of its size, over the whole e sweep 0..10."""
    w = synth.config2(scale=0.002, ref_bases=20_000_000)
    run = GpuRun(w)
    for e in range(0, 11):
        assert_same(run.filter(e=e), oracle_run(w, e), f"c2 scaled e={e}")


@pytest.mark.parametrize("m,es", [(150, (0, 4, 10, 15)), (250, (0, 6, 10, 25))])
def test_config3_structure_scaled(m, es):
    w = synth.config3(m, scale=0.002, ref_bases=20_000_000)
    run = GpuRun(w)
    for e in es:
        assert_same(run.filter(e=e), oracle_run(w, e), f"c3 {m}bp scaled e={e}")


@pytest.mark.parametrize("m", [2, 3, 4, 31, 32, 33, 64, 95, 96, 97, 100, 128, 150, 250, 256, 300])
def test_every_threshold_2_to_30(m):
    """One launch per threshold e = 2..30 (the launches whose masks are ANDed
    dilated and eroded once, with end corrections), word-boundary lengths
    included, against the oracle; also with N in reads and genome."""
    w = small_workload(m, 1200, seed=300 + m, n_frac=0.0005, read_n_frac=0.0005)
    run = GpuRun(w)
    for e in range(2, 31):
        assert_same(run.filter(e=e), oracle_run(w, e), f"m={m} e={e}")
    for e in (4, 17, 30):
        assert_same(run.filter(e=e, mode=gk.GK_COUNT_POPCOUNT), oracle_run(w, e, O.POPCOUNT),
                    f"m={m} e={e} popcount")
