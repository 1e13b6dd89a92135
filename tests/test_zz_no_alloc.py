"""gk_filter_batched_noalloc: the batched filter for callers that cannot
allocate device memory while they filter (a plugin whose host application
owns all device memory through its own pool, or a latency-bound thread that
must not call cudaMalloc because it can synchronise the device).  It runs on a
fixed scratch array inside the library instead of a caller workspace.

Checked here through the C ABI: two calls in a row, on different inputs, each
give exactly the results of gk_filter_batched on the same inputs (the
second call finds the first call's leftovers in the shared scratch); and a
batch above the stated maximum is refused with GK_ERANGE.
"""
import numpy as np
import pytest
import torch

from paper_2103_14978_gb300 import batch, device_data as dd, gk, synth
from tests.gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu

TILING = (4, 256, 4, 8)


def _workload(seed, n_pairs):
    ref = synth.reference(2_000_000, seed, 0.05, 0.001)
    w = synth.pairs_workload("noalloc", seed=seed, ref=ref, n_pairs=n_pairs, m=(1, 512), cands=4,
                             e_rates=(0.0, 0.02, 0.05, 0.10, 1.0), read_edit_rate=0.04, read_n_frac=0.001,
                             shuffle=True)
    rng = np.random.default_rng(seed)
    w.pair_read[rng.choice(n_pairs, 50, replace=False)] = w.n_reads + 5  # 50 invalid pairs
    return w


def _inputs(w):
    return dict(ref=gk.gk_load_reference(w.ref), reads=dd.upload_reads(w.reads, w.read_len, w.stride),
                read_len=dd.as_i16(w.read_len).cuda(), pairs=dd.upload_pairs(w.pair_read, w.pair_off, w.pair_e))


def _with_workspace(x):
    r, p = x["reads"], x["pairs"]
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    bf = batch.BatchedFilter(x["ref"], r.packed, r.stride_words, r.n_reads, x["read_len"], r.nflag,
                             p.pair_read, p.pair_off, p.pair_e, TILING, err_count=err)
    bf.run()
    torch.cuda.synchronize()
    return bf.accept.cpu().numpy(), dd.edits_u16(bf.edits), int(err.item())


def _without_workspace(x):
    r, p = x["reads"], x["pairs"]
    n = p.n_pairs
    acc = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    ed = torch.full((n,), -7, dtype=torch.int16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    gk.gk_filter_batched_noalloc(x["ref"], r.packed, r.stride_words, r.n_reads, x["read_len"], r.nflag,
                                 p.pair_read, p.pair_off, p.pair_e, gk.Tiling(*TILING), acc, ed,
                                 err_count=err)
    torch.cuda.synchronize()
    return acc.cpu().numpy(), dd.edits_u16(ed), int(err.item())


def test_noalloc_matches_workspace_entry_point_twice():
    require_gpu()
    first = _inputs(_workload(41, 400_000))
    second = _inputs(_workload(42, 150_000))
    for x in (first, second):  # two calls in a row, different sizes
        want = _with_workspace(x)
        got = _without_workspace(x)
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        assert got[2] == want[2] == 50


def test_noalloc_refuses_batches_above_the_limit():
    require_gpu()
    x = _inputs(_workload(43, 1000))
    n = gk.GK_NOALLOC_MAX_PAIRS + 1
    pr = torch.zeros(n, dtype=torch.int32, device="cuda")
    acc = torch.empty(n, dtype=torch.uint8, device="cuda")
    ed = torch.empty(n, dtype=torch.int16, device="cuda")
    r = x["reads"]
    with pytest.raises(gk.GKError) as exc:
        gk.gk_filter_batched_noalloc(x["ref"], r.packed, r.stride_words, r.n_reads, x["read_len"], r.nflag,
                                     pr, pr, 3, gk.Tiling(*TILING), acc, ed)
    assert exc.value.code == gk.GK_ERANGE
    assert "GK_NOALLOC_MAX_PAIRS" in str(exc.value)
