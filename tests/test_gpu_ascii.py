"""gk_filter_ascii (reads as ASCII rows, encoded inside the filter kernel):
bit-exact against the oracle at word-boundary read lengths, with N in reads
and genome, invalid pairs, per-pair thresholds, pairs grouped by read or
shuffled, rows at aligned and unaligned strides, and the result-byte form."""
import numpy as np
import pytest
import torch

from paper_2103_14978_gb300 import gk
from tests.gpu_helpers import GpuRun, assert_same, oracle_run, require_gpu, small_workload

pytestmark = pytest.mark.gpu


def ascii_rows(w, stride, shift=0):
    """The workload's reads as device rows of `stride` bytes, the first row
    `shift` bytes into the buffer."""
    m = int(w.read_len[0])
    rows = np.zeros((w.n_reads, stride), np.uint8)
    rows[:, :m] = w.reads.reshape(w.n_reads, w.stride)[:, :m]
    buf = torch.zeros(w.n_reads * stride + shift + 16, dtype=torch.uint8)
    buf[shift:shift + w.n_reads * stride] = torch.from_numpy(rows.reshape(-1))
    return buf.cuda()[shift:shift + w.n_reads * stride]


@pytest.mark.parametrize("m", [1, 31, 32, 33, 100, 150, 250, 300, 512])
def test_ascii_filter_equals_the_oracle(m):
    require_gpu()
    w = small_workload(m, 2500, seed=1300 + m, n_frac=0.0005, read_n_frac=0.001, cands=(1, 9))
    w.pair_read[:10] = w.n_reads + 4  # invalid pairs
    run = GpuRun(w)
    order = np.random.default_rng(m).permutation(w.n_pairs)
    shuffled = w.subset(order)
    for ws, name in ((w, "grouped"), (shuffled, "shuffled")):
        r = GpuRun(ws, ref=run.ref)
        for stride, shift in ((w.stride, 0), (m + 3, 0), (m + 4, 1)):
            asc = ascii_rows(ws, stride, shift)
            for e in sorted({0, 1, 2, 5, max(1, m // 10), min(30, m), 255}):
                err = torch.zeros(1, dtype=torch.int32, device="cuda")
                a, d = gk.gk_filter_ascii(run.ref, asc, stride, ws.n_reads, m, r.pairs.pair_read, r.pairs.pair_off,
                                          e, err_count=err)
                torch.cuda.synchronize()
                assert_same((a.cpu().numpy(), d.cpu().numpy().view(np.uint16)), oracle_run(ws, e),
                            f"{name} m={m} stride={stride}+{shift} e={e}")
                assert int(err.item()) == 10


def test_ascii_filter_per_pair_thresholds_and_result_bytes():
    require_gpu()
    w = small_workload(150, 6000, seed=1401, n_frac=0.001, read_n_frac=0.001, cands=(4, 16),
                       e_rates=(0.0, 0.02, 0.05, 0.10, 1.0))
    run = GpuRun(w)
    asc = ascii_rows(w, w.stride)
    a, d = gk.gk_filter_ascii(run.ref, asc, w.stride, w.n_reads, 150, run.pairs.pair_read, run.pairs.pair_off,
                              run.pairs.pair_e)
    torch.cuda.synchronize()
    assert_same((a.cpu().numpy(), d.cpu().numpy().view(np.uint16)), oracle_run(w), "per-pair e")
    for e in (3, 12):
        res, _ = gk.gk_filter_ascii(run.ref, asc, w.stride, w.n_reads, 150, run.pairs.pair_read, run.pairs.pair_off,
                                    e, flags=gk.GK_FLAG_RESULT_BYTE)
        a2, d2 = run.filter(e=e)
        want = np.minimum(d2.astype(np.int64), 253)
        want[d2 == gk.GK_EDITS_UNDEFINED] = 254
        want[d2 == gk.GK_EDITS_INVALID] = 255
        torch.cuda.synchronize()
        assert np.array_equal(res.cpu().numpy(), want.astype(np.uint8)), e


def test_ascii_filter_argument_checks():
    require_gpu()
    w = small_workload(100, 100, seed=1402)
    run = GpuRun(w)
    asc = ascii_rows(w, w.stride)
    with pytest.raises(gk.GKError) as exc:
        gk.gk_filter_ascii(run.ref, asc, 99, w.n_reads, 100, run.pairs.pair_read, run.pairs.pair_off, 2)
    assert exc.value.code == gk.GK_EINVAL
    with pytest.raises(gk.GKError) as exc:
        gk.gk_filter_ascii(run.ref, asc, w.stride, w.n_reads, 600, run.pairs.pair_read, run.pairs.pair_off, 2)
    assert exc.value.code == gk.GK_ERANGE
