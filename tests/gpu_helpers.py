"""Shared helpers of the GPU parity tests: run a workload through the C-ABI
(via the binding) and through the oracle, on the same seeded inputs."""
from __future__ import annotations

import numpy as np
import torch

from oracle import oracle as O
from paper_2103_14978_gb300 import build, device_data as dd, gk, synth


def require_gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    gk.lib()


class GpuRun:
    """A workload resident on the device: reference handle, packed reads, pairs."""

    def __init__(self, w: synth.Workload, ref: gk.Reference | None = None):
        self.w = w
        self.ref = ref or gk.gk_load_reference(w.ref)
        self.reads = dd.upload_reads(w.reads, w.read_len, w.stride)
        self.pairs = dd.upload_pairs(w.pair_read, w.pair_off, w.pair_e)
        lens = np.unique(w.read_len)
        assert lens.shape[0] == 1, "plain filter runs take one read length"
        self.m = int(lens[0])

    def filter(self, e=None, mode=gk.GK_COUNT_RUNS4, flags=0, err=None, stream=None):
        if e is None:
            e = self.pairs.pair_e if self.pairs.pair_e is not None else self.w.e
        ee = e
        acc, ed = gk.gk_filter(self.ref, self.reads.packed, self.reads.stride_words, self.reads.n_reads,
                               self.reads.nflag, self.m, self.pairs.pair_read, self.pairs.pair_off, ee,
                               count_mode=mode, flags=flags, err_count=err, stream=stream)
        torch.cuda.synchronize()
        return acc.cpu().numpy(), dd.edits_u16(ed)


def oracle_run(w: synth.Workload, e=None, mode=O.RUNS4, flags=0, idx=None):
    pr, po = w.pair_read, w.pair_off
    if e is None:
        e = w.pair_e if w.pair_e is not None else w.e
    pe = e
    if idx is not None:
        pr, po = pr[idx], po[idx]
        if not np.isscalar(pe) and pe is not None:
            pe = pe[idx]
    acc, ed, _ = O.filter_batch(w.reads, w.read_start, w.read_len, w.ref, pr, po, pe, mode, flags)
    return acc, ed


def accept_of_result_bytes(res, e: int) -> np.ndarray:
    """Accept bits a reader of GK_FLAG_RESULT_BYTE results derives at
    threshold e (<= 252), as the header documents the format: a count at
    most e, or the undefined sentinel."""
    r = res.cpu().numpy() if isinstance(res, torch.Tensor) else np.asarray(res)
    return ((r <= e) | (r == gk.GK_RESULT_UNDEFINED)).astype(np.uint8)


def assert_same(got, want, what=""):
    ga, ge = got
    wa, we = want
    bad = np.nonzero((ga != wa) | (ge != we))[0]
    assert bad.size == 0, (
        f"{what}: {bad.size} of {ga.size} pairs differ; first {bad[:5].tolist()}: "
        f"gpu {list(zip(ga[bad[:5]].tolist(), ge[bad[:5]].tolist()))} "
        f"oracle {list(zip(wa[bad[:5]].tolist(), we[bad[:5]].tolist()))}")


def small_workload(m: int, n_pairs: int, seed: int, ref_len: int = 200_000, n_frac: float = 0.0,
                   read_n_frac: float = 0.0, cands=4, e=None, e_rates=None, read_edit_rate=0.04):
    if e is None and e_rates is None:
        e = 0
    ref = synth.reference(ref_len, seed, 0.05, n_frac)
    return synth.pairs_workload(f"small-m{m}", seed=seed, ref=ref, n_pairs=n_pairs, m=m, cands=cands,
                                e=e, e_rates=e_rates, read_edit_rate=read_edit_rate,
                                read_n_frac=read_n_frac)
