"""Bit-exact parity of the bit-sliced batch filter (gk_slice once per batch,
gk_filter_sliced once per threshold, gk_filter_sliced_sweep once per range
of thresholds) with the CPU oracle, through the C-ABI: every accept bit and
edit count identical (integer work, tolerance 0)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2103_14978_gb300 import device_data as dd, gk, synth
from tests.gpu_helpers import GpuRun, assert_same, oracle_run, require_gpu, small_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


class SlicedRun:
    """A workload resident on the device and sliced once."""

    def __init__(self, w: synth.Workload, err=None):
        self.run = GpuRun(w)
        r = self.run
        self.n = w.n_pairs
        self.m = r.m
        self.buf = gk.gk_slice(r.ref, r.reads.packed, r.reads.stride_words, r.reads.n_reads, r.reads.nflag,
                               r.m, r.pairs.pair_read, r.pairs.pair_off, err_count=err)

    def filter(self, e, mode=gk.GK_COUNT_RUNS4, flags=0, accept=None, edits=None):
        acc, ed = gk.gk_filter_sliced(self.buf, self.n, self.m, e, count_mode=mode, flags=flags,
                                      accept=accept, edits=edits)
        torch.cuda.synchronize()
        if flags & gk.GK_FLAG_RESULT_BYTE:
            return acc.cpu().numpy(), None
        return acc.cpu().numpy(), dd.edits_u16(ed)

    def sweep(self, e_lo, e_hi, mode=gk.GK_COUNT_RUNS4, flags=0, err=None):
        """Rows e_lo..e_hi of gk_filter_sliced_sweep as {e: (accept, edits)}."""
        acc, ed = gk.gk_filter_sliced_sweep(self.buf, self.n, self.m, e_lo, e_hi, count_mode=mode, flags=flags,
                                            err_count=err)
        torch.cuda.synchronize()
        out = {}
        for i, e in enumerate(range(e_lo, e_hi + 1)):
            a = acc[i].cpu().numpy()
            out[e] = (a, None) if flags & gk.GK_FLAG_RESULT_BYTE else (a, dd.edits_u16(ed[i]))
        return out


def thresholds(m):
    """Every threshold the compiled shift counts reach: K = min(e, m-1) <= 15."""
    es = list(range(0, gk.GK_SLICED_MAX_SHIFT + 1))
    if m - 1 <= gk.GK_SLICED_MAX_SHIFT:
        es += [m - 1, m, m + 1, 255]
    return sorted({e for e in es if e <= 255})


LENGTHS = [1, 2, 3, 5, 31, 32, 33, 63, 64, 65, 97, 100, 127, 128, 150, 200, 250, 255]


@pytest.mark.parametrize("m", LENGTHS)
def test_sliced_every_threshold(m):
    """Word-boundary lengths, the three compiled lengths (100, 150, 250) and
    the general kernels; N at 0.05% of genome and read bases; a ragged last
    group (n_pairs not a multiple of 32)."""
    w = small_workload(m, 1500 + 13, seed=500 + m, n_frac=0.0005, read_n_frac=0.0005)
    s = SlicedRun(w)
    for e in thresholds(m):
        assert_same(s.filter(e), oracle_run(w, e), f"sliced m={m} e={e}")
    for e in (0, 3, 10):
        assert_same(s.filter(e, mode=gk.GK_COUNT_POPCOUNT), oracle_run(w, e, O.POPCOUNT),
                    f"sliced m={m} e={e} popcount")


@pytest.mark.parametrize("m", [31, 100, 150, 250])
def test_sliced_result_bytes(m):
    w = small_workload(m, 4000, seed=600 + m, n_frac=0.001, read_n_frac=0.001, cands=(8, 64))
    s = SlicedRun(w)
    for e in (0, 2, 7, 10):
        got, _ = s.filter(e, flags=gk.GK_FLAG_RESULT_BYTE)
        acc, ed = oracle_run(w, e)
        want = np.where(ed == O.UNDEFINED, gk.GK_RESULT_UNDEFINED,
                        np.where(ed == O.INVALID, gk.GK_RESULT_INVALID, np.minimum(ed, gk.GK_RESULT_MAX_COUNT)))
        assert (got == want.astype(np.uint8)).all(), f"m={m} e={e}"
        assert (((got <= e) | (got == gk.GK_RESULT_UNDEFINED)) == (acc == 1)).all()


def test_sliced_invalid_pairs_and_error_counter():
    w = small_workload(100, 4000, seed=611, ref_len=50_000)
    L = w.ref.shape[0]
    rng = np.random.default_rng(15)
    pr, po = w.pair_read.copy(), w.pair_off.copy()
    pr[rng.integers(0, 4000, 100)] = w.n_reads + rng.integers(0, 1000, 100)
    po[rng.integers(0, 4000, 100)] = L - 100 + rng.integers(1, 500, 100)
    po[:10] = L - 100  # the last valid window
    po[10:20] = 0xFFFFFFFF
    w2 = w.subset(np.arange(w.n_pairs))
    w2.pair_read, w2.pair_off = pr, po
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = SlicedRun(w2, err=err)
    for e in (0, 3, 10):
        want = oracle_run(w2, e)
        got = s.filter(e)
        assert_same(got, want, f"invalid e={e}")
    n_invalid = int((want[1] == O.INVALID).sum())
    assert n_invalid >= 200
    assert int(err.item()) == n_invalid  # counted once, by the slice


@pytest.mark.parametrize("n", [1, 31, 32, 33, 4096, 4097, 3 * 4096])
def test_sliced_group_and_block_edges(n):
    """Pair counts at group (32) and block (4096 pairs) boundaries."""
    w = small_workload(100, n, seed=700 + n, ref_len=30_000)
    s = SlicedRun(w)
    for e in (0, 4, 10):
        assert_same(s.filter(e), oracle_run(w, e), f"n={n} e={e}")


@pytest.mark.parametrize("m", [100, 150, 70])
def test_sliced_pairs_in_any_order(m):
    """Pairs shuffled (no two candidates of a read side by side, so no read
    is reused between neighbouring pairs), with N and invalid windows."""
    w = small_workload(m, 5000, seed=840 + m, n_frac=0.001, read_n_frac=0.001)
    rng = np.random.default_rng(841)
    perm = rng.permutation(w.n_pairs)
    w2 = w.subset(perm)
    w2.pair_off = w2.pair_off.copy()
    w2.pair_off[rng.integers(0, w2.n_pairs, 40)] = w.ref.shape[0] - m + rng.integers(1, 50, 40)
    s = SlicedRun(w2)
    for e in (0, 1, 5, 10):
        assert_same(s.filter(e), oracle_run(w2, e), f"shuffled m={m} e={e}")


def test_sliced_unaligned_outputs():
    """Result buffers off the 16-byte grid take the scalar stores."""
    w = small_workload(100, 2000, seed=801)
    s = SlicedRun(w)
    abuf = torch.full((w.n_pairs + 8,), 0xAB, dtype=torch.uint8, device="cuda")
    ebuf = torch.full((w.n_pairs + 8,), 0x1234, dtype=torch.int16, device="cuda")
    got = s.filter(6, accept=abuf[3:3 + w.n_pairs], edits=ebuf[1:1 + w.n_pairs])
    assert_same(got, oracle_run(w, 6), "unaligned")
    torch.cuda.synchronize()
    assert abuf[:3].cpu().tolist() == [0xAB] * 3 and abuf[3 + w.n_pairs:].cpu().tolist() == [0xAB] * 5
    assert ebuf[0].item() == 0x1234 and ebuf[1 + w.n_pairs:].cpu().tolist() == [0x1234] * 7


def test_sliced_config2_structure_scaled():
    w = synth.config2(scale=0.002, ref_bases=20_000_000)
    s = SlicedRun(w)
    for e in range(0, 11):
        assert_same(s.filter(e), oracle_run(w, e), f"c2 scaled sliced e={e}")


@pytest.mark.parametrize("m", [150, 250])
def test_sliced_config3_structure_scaled(m):
    w = synth.config3(m, scale=0.002, ref_bases=20_000_000)
    s = SlicedRun(w)
    for e in (0, 1, 4, 10, 13, 15):
        assert_same(s.filter(e), oracle_run(w, e), f"c3 {m}bp scaled sliced e={e}")


def test_sliced_config2_full_size_sampled():
    """Config 2 at its full size (20M pairs, 100 bp), the launch form the
    benchmark times: 20,000 sampled pairs against the oracle at e = 0, 5, 10,
    and every pair against gk_filter."""
    w = synth.config2()
    s = SlicedRun(w)
    rng = np.random.default_rng(2103)
    idx = np.sort(rng.choice(w.n_pairs, 20_000, replace=False))
    for e in (0, 5, 10):
        got = s.filter(e)
        want = oracle_run(w, e, idx=idx)
        assert_same((got[0][idx], got[1][idx]), want, f"c2 full sampled e={e}")
        plain = s.run.filter(e=e)
        assert (plain[0] == got[0]).all() and (plain[1] == got[1]).all(), f"c2 full vs gk_filter e={e}"


def test_sliced_argument_errors_and_empty():
    w = small_workload(100, 64, seed=901, ref_len=10_000)
    s = SlicedRun(w)
    with pytest.raises(gk.GKError) as ex:
        gk.gk_filter_sliced(s.buf, s.n, 100, 16)  # min(e, m-1) = 16 > 15
    assert ex.value.code == gk.GK_ERANGE
    with pytest.raises(gk.GKError) as ex:
        gk.gk_filter_sliced(s.buf, s.n, 100, 3, flags=gk.GK_FLAG_NO_EDGE_FIX)
    assert ex.value.code == gk.GK_EINVAL
    with pytest.raises(gk.GKError) as ex:
        gk.gk_filter_sliced(s.buf[: gk.gk_sliced_bytes(s.n, 100) - 8], s.n, 100, 3)
    assert ex.value.code == gk.GK_EINVAL
    r = s.run
    for m in (0, 256):
        with pytest.raises(gk.GKError) as ex:
            gk.gk_slice(r.ref, r.reads.packed, r.reads.stride_words, r.reads.n_reads, r.reads.nflag, m,
                        r.pairs.pair_read, r.pairs.pair_off, out=s.buf)
        assert ex.value.code == gk.GK_ERANGE
    assert gk.gk_sliced_bytes(0, 100) == 0 and gk.gk_sliced_bytes(10, 0) == 0
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    gk.gk_slice(r.ref, r.reads.packed, r.reads.stride_words, r.reads.n_reads, r.reads.nflag, 100, empty, empty)
    acc, ed = gk.gk_filter_sliced(s.buf, 0, 100, 3)
    assert acc.numel() == 0 and ed.numel() == 0


SWEEPS = [(0, 10), (0, 5), (6, 10), (2, 4), (3, 9), (5, 6), (7, 15), (0, 15), (10, 12), (4, 4)]


@pytest.mark.parametrize("m", [1, 2, 5, 8, 11, 31, 33, 64, 100, 127, 150, 250, 255])
def test_sliced_sweep_matches_oracle(m):
    """gk_filter_sliced_sweep over ranges that start and end inside, at and
    across the compiled shift-count ranges (0..5, 6..10) and past them, at
    lengths where e > m-1 shares K = m-1; N in genome and reads, a ragged
    last group."""
    w = small_workload(m, 1500 + 7, seed=1500 + m, n_frac=0.0005, read_n_frac=0.0005)
    s = SlicedRun(w)
    want = {}
    for lo, hi in SWEEPS + ([(0, m + 2)] if m + 2 <= 15 or m - 1 <= 15 else []):
        got = s.sweep(lo, hi)
        for e in range(lo, hi + 1):
            if e not in want:
                want[e] = oracle_run(w, e)
            assert_same(got[e], want[e], f"sweep m={m} [{lo},{hi}] e={e}")


@pytest.mark.parametrize("m", [100, 150, 70])
def test_sliced_sweep_popcount_and_result_bytes(m):
    w = small_workload(m, 3000, seed=1600 + m, n_frac=0.001, read_n_frac=0.001, cands=(8, 64))
    s = SlicedRun(w)
    got = s.sweep(0, 10, mode=gk.GK_COUNT_POPCOUNT)
    for e in range(0, 11):
        assert_same(got[e], oracle_run(w, e, O.POPCOUNT), f"sweep popcount m={m} e={e}")
    got = s.sweep(1, 12, flags=gk.GK_FLAG_RESULT_BYTE)
    for e in range(1, 13):
        acc, ed = oracle_run(w, e)
        want = np.where(ed == O.UNDEFINED, gk.GK_RESULT_UNDEFINED,
                        np.where(ed == O.INVALID, gk.GK_RESULT_INVALID, np.minimum(ed, gk.GK_RESULT_MAX_COUNT)))
        assert (got[e][0] == want.astype(np.uint8)).all(), f"sweep result bytes m={m} e={e}"


def test_sliced_buffer_header_mismatch():
    """A filter call whose (m, n_pairs) differ from the slice's, or a buffer
    never sliced: every pair gets the invalid result, and the sweep counts
    the pairs in its error counter."""
    w = small_workload(100, 1000, seed=1700, ref_len=20_000)
    s = SlicedRun(w)
    assert_same(s.filter(3), oracle_run(w, 3), "header ok")
    for n, m in ((999, 100), (1000, 99), (1001 - 32, 100)):
        acc, ed = gk.gk_filter_sliced(s.buf, n, m, 3)
        torch.cuda.synchronize()
        assert (acc.cpu().numpy() == 0).all() and (dd.edits_u16(ed) == gk.GK_EDITS_INVALID).all(), (n, m)
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        a2, e2 = gk.gk_filter_sliced_sweep(s.buf, n, m, 0, 10, err_count=err)
        torch.cuda.synchronize()
        assert (a2.cpu().numpy() == 0).all() and (dd.edits_u16(e2) == gk.GK_EDITS_INVALID).all()
        assert int(err.item()) == 2 * n  # two launches (shift counts 0..5 and 6..10), every pair counted
    fresh = torch.zeros_like(s.buf)
    acc, _ = gk.gk_filter_sliced(fresh, 1000, 100, 3, flags=gk.GK_FLAG_RESULT_BYTE)
    torch.cuda.synchronize()
    assert (acc.cpu().numpy() == gk.GK_RESULT_INVALID).all()


def test_sliced_sweep_config2_full_size():
    """Config 2 at its full size (20M pairs, 100 bp) through the launch form
    the benchmark times (one sweep over e = 0..10): every pair equal to the
    per-threshold sliced filter, 20,000 sampled pairs equal to the oracle."""
    w = synth.config2()
    s = SlicedRun(w)
    got = s.sweep(0, 10)
    rng = np.random.default_rng(2104)
    idx = np.sort(rng.choice(w.n_pairs, 20_000, replace=False))
    for e in range(0, 11):
        single = s.filter(e)
        assert (single[0] == got[e][0]).all() and (single[1] == got[e][1]).all(), f"c2 sweep vs single e={e}"
        if e in (0, 3, 6, 10):
            assert_same((got[e][0][idx], got[e][1][idx]), oracle_run(w, e, idx=idx), f"c2 sweep sampled e={e}")


@pytest.mark.parametrize("m", [150, 250])
def test_sliced_config3_full_size_sampled(m):
    """Config 3 at its full size (10M pairs, 8-64 candidates per read, N at
    0.1%), sliced once as the benchmark does: 30,000 sampled pairs against the
    oracle at e = 0, 8, 15 (single thresholds) and the sweep 0..10."""
    w = synth.config3(m)
    s = SlicedRun(w)
    rng = np.random.default_rng(2105 + m)
    idx = np.sort(rng.choice(w.n_pairs, 30_000, replace=False))
    for e in (0, 8, 15):
        got = s.filter(e)
        assert_same((got[0][idx], got[1][idx]), oracle_run(w, e, idx=idx), f"c3 {m}bp full sampled e={e}")
    sw = s.sweep(0, 10)
    for e in (0, 5, 9, 10):
        assert_same((sw[e][0][idx], sw[e][1][idx]), oracle_run(w, e, idx=idx), f"c3 {m}bp sweep sampled e={e}")
