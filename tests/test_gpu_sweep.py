"""Bit-exact parity of the per-pair threshold sweep (gk_filter_sweep: every
threshold of a range in one launch, each pair's masks built once) with the
CPU oracle at every threshold, through the C-ABI: every accept bit and edit
count identical (integer work, tolerance 0)."""
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


def sweep(run, e_lo, e_hi, mode=gk.GK_COUNT_RUNS4, flags=0, err=None, out_stride=None):
    r = run.reads
    acc, ed = gk.gk_filter_sweep(run.ref, r.packed, r.stride_words, r.n_reads, r.nflag, run.m,
                                 run.pairs.pair_read, run.pairs.pair_off, e_lo, e_hi, count_mode=mode, flags=flags,
                                 err_count=err, out_stride=out_stride)
    torch.cuda.synchronize()
    out = {}
    for i, e in enumerate(range(e_lo, e_hi + 1)):
        a = acc[i].cpu().numpy()
        out[e] = (a, None) if flags & gk.GK_FLAG_RESULT_BYTE else (a, dd.edits_u16(ed[i]))
    return out


LENGTHS = [1, 2, 3, 7, 31, 32, 33, 64, 65, 100, 127, 150, 200, 250, 300, 511, 512]


@pytest.mark.parametrize("m", LENGTHS)
def test_sweep_matches_oracle(m):
    """Ranges from 0 (shift counts 0 and 1 finished by the deferred form),
    inside, and up to the limit; thresholds above m-1 sharing K = m-1; N at
    0.05% of genome and reads (one thread per pair); a ragged last warp."""
    w = small_workload(m, 1200 + 11, seed=2000 + m, n_frac=0.0005, read_n_frac=0.0005)
    run = GpuRun(w)
    hi = min(30, max(m + 2, 3)) if m <= 40 else 30
    ranges = [(0, hi), (0, 3), (2, 12), (hi - 4, hi)]
    want = {}
    for lo, h in ranges:
        lo = max(0, lo)
        got = sweep(run, lo, h)
        for e in range(lo, h + 1):
            if e not in want:
                want[e] = oracle_run(w, e)
            assert_same(got[e], want[e], f"sweep m={m} [{lo},{h}] e={e}")


@pytest.mark.parametrize("m", [100, 150, 250])
def test_sweep_dense_n_queue_popcount_and_result_bytes(m):
    """A genome with N at 0.1% (the queue of defined pairs), 8-64 candidates
    per read, invalid pairs counted once; popcount; result bytes."""
    w = small_workload(m, 5000, seed=2100 + m, n_frac=0.001, read_n_frac=0.001, cands=(8, 64))
    w.pair_read[:17] = w.n_reads + 3
    run = GpuRun(w)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = sweep(run, 0, 25, err=err)
    for e in range(0, 26):
        assert_same(got[e], oracle_run(w, e), f"sweep queue m={m} e={e}")
    assert int(err.item()) == 17
    got = sweep(run, 5, 14, mode=gk.GK_COUNT_POPCOUNT)
    for e in range(5, 15):
        assert_same(got[e], oracle_run(w, e, O.POPCOUNT), f"sweep popcount m={m} e={e}")
    got = sweep(run, 3, 20, flags=gk.GK_FLAG_RESULT_BYTE)
    for e in range(3, 21):
        acc, ed = oracle_run(w, e)
        want = np.where(ed == O.UNDEFINED, gk.GK_RESULT_UNDEFINED,
                        np.where(ed == O.INVALID, gk.GK_RESULT_INVALID, np.minimum(ed, gk.GK_RESULT_MAX_COUNT)))
        assert (got[e][0] == want.astype(np.uint8)).all(), f"sweep result bytes m={m} e={e}"


def test_sweep_rows_and_arguments():
    """Rows land out_stride apart and nothing is written between them;
    argument errors are refused before any work."""
    w = small_workload(100, 1000, seed=2200, ref_len=20_000)
    run = GpuRun(w)
    r = run.reads
    stride = 1000 + 40
    acc = torch.full((4 * stride,), 0xAB, dtype=torch.uint8, device="cuda")
    ed = torch.full((4 * stride,), 0x1234, dtype=torch.int16, device="cuda")
    a, e = gk.gk_filter_sweep(run.ref, r.packed, r.stride_words, r.n_reads, r.nflag, 100, run.pairs.pair_read,
                              run.pairs.pair_off, 4, 7, accept=acc, edits=ed, out_stride=stride)
    torch.cuda.synchronize()
    for i, t in enumerate(range(4, 8)):
        assert_same((a[i].cpu().numpy(), dd.edits_u16(e[i])), oracle_run(w, t), f"rows e={t}")
        gap = acc[i * stride + 1000:(i + 1) * stride].cpu().numpy()
        assert (gap == 0xAB).all()
    # an odd row stride and rows off the 4-byte grid: one store per pair
    acc.fill_(0xAB)
    a, e = gk.gk_filter_sweep(run.ref, r.packed, r.stride_words, r.n_reads, r.nflag, 100, run.pairs.pair_read,
                              run.pairs.pair_off, 2, 5, accept=acc[1:], edits=ed[1:], out_stride=1001)
    torch.cuda.synchronize()
    for i, t in enumerate(range(2, 6)):
        assert_same((a[i].cpu().numpy(), dd.edits_u16(e[i])), oracle_run(w, t), f"odd rows e={t}")
    assert acc[0].item() == 0xAB
    for bad in (dict(e_lo=5, e_hi=4), dict(e_lo=0, e_hi=31), dict(e_lo=0, e_hi=10, flags=gk.GK_FLAG_NO_EDGE_FIX),
                dict(e_lo=0, e_hi=10, out_stride=999)):
        with pytest.raises(gk.GKError):
            kw = dict(bad)
            gk.gk_filter_sweep(run.ref, r.packed, r.stride_words, r.n_reads, r.nflag, 100, run.pairs.pair_read,
                               run.pairs.pair_off, kw.pop("e_lo"), kw.pop("e_hi"), **kw)


def test_sweep_config3_250bp_full_size_sampled():
    """Config 3 at 250 bp, full size (10M pairs, 0.1% N), the launch form the
    benchmark times for e = 16..25: 20,000 sampled pairs against the oracle
    at every threshold, and every pair against gk_filter at 16 and 25."""
    w = synth.config3(250)
    run = GpuRun(w)
    got = sweep(run, 16, 25)
    rng = np.random.default_rng(2106)
    idx = np.sort(rng.choice(w.n_pairs, 20_000, replace=False))
    for e in range(16, 26):
        assert_same((got[e][0][idx], got[e][1][idx]), oracle_run(w, e, idx=idx), f"c3 250bp sweep e={e}")
    for e in (16, 25):
        plain = run.filter(e=e)
        assert (plain[0] == got[e][0]).all() and (plain[1] == got[e][1]).all(), f"c3 250bp sweep vs gk_filter e={e}"
