"""Parity at the full sizes of the benchmark configurations, in the launch
configuration bench.py times (one launch over all pairs), checked pair by
pair against the oracle on seeded random samples of the outputs, plus
properties that must hold for every pair."""
import numpy as np
import pytest
import torch

from paper_2103_14978_gb300 import batch, device_data as dd, gk, synth
from tests.gpu_helpers import GpuRun, assert_same, oracle_run, require_gpu

pytestmark = pytest.mark.gpu

SAMPLE = 60_000


def _sample(n, seed):
    return np.sort(np.random.default_rng(seed).choice(n, min(n, SAMPLE), replace=False))


def _whole_output_properties(acc, ed, e):
    valid = ed < gk.GK_EDITS_INVALID
    assert np.array_equal(acc[valid], (ed[valid] <= e).astype(np.uint8))
    assert (acc[ed == gk.GK_EDITS_UNDEFINED] == 1).all()


def test_config2_full_size_sampled():
    require_gpu()
    w = synth.config2()
    assert w.n_pairs == 20_000_000
    run = GpuRun(w)
    for e in (0, 2, 5, 10):
        acc, ed = run.filter(e=e)
        _whole_output_properties(acc, ed, e)
        idx = _sample(w.n_pairs, e)
        assert_same((acc[idx], ed[idx]), oracle_run(w, e, idx=idx), f"config 2 full e={e}")


@pytest.mark.parametrize("m,es", [(150, (0, 4, 15)), (250, (0, 10, 25))])
def test_config3_full_size_sampled(m, es):
    require_gpu()
    w = synth.config3(m)
    assert w.n_pairs == 10_000_000
    run = GpuRun(w)
    for e in es:
        acc, ed = run.filter(e=e)
        _whole_output_properties(acc, ed, e)
        idx = _sample(w.n_pairs, 100 + e)
        assert_same((acc[idx], ed[idx]), oracle_run(w, e, idx=idx), f"config 3 {m} bp full e={e}")


def test_config4_full_size_batched_sampled():
    require_gpu()
    w = synth.config4()
    assert w.n_pairs == 50_000_000
    ref = gk.gk_load_reference(w.ref)
    reads = dd.upload_reads(w.reads, w.read_len, w.stride)
    pairs = dd.upload_pairs(w.pair_read, w.pair_off, w.pair_e)
    bf = batch.BatchedFilter(ref, reads.packed, reads.stride_words, reads.n_reads, dd.as_i16(w.read_len).cuda(),
                             reads.nflag, pairs.pair_read, pairs.pair_off, pairs.pair_e, (6, 256, 2, 8))
    bf.capture()
    bf.replay()
    torch.cuda.synchronize()
    acc, ed = bf.accept.cpu().numpy(), dd.edits_u16(bf.edits)
    valid = ed < gk.GK_EDITS_INVALID
    assert np.array_equal(acc[valid], (ed[valid] <= w.pair_e[valid]).astype(np.uint8))
    idx = _sample(w.n_pairs, 4)
    assert_same((acc[idx], ed[idx]), oracle_run(w, idx=idx), "config 4 full batched")
