"""Seeded synthetic workloads shaped like the paper's read/candidate sets.

The paper measures on 30M mrFAST-seeded pairs of real 100/150/250 bp reads
against GRCh37 (Sec. 4.1, Sec. 4.3), none of which is available here; these
generators stand in for them with the same read lengths, pair counts, error
thresholds (e up to 10% of the read length) and structure (a read's
candidates are consecutive pairs; one candidate is the read's true origin, the
rest are elsewhere in the genome; 'N' bases where the configuration asks).

This module holds none of the filter's arithmetic: it only draws bases,
edits, lengths and offsets, and emits plain ASCII.  The CUDA path and the
oracle both consume what it returns.
"""
from __future__ import annotations

import dataclasses
import functools

import numpy as np

SEED_BASE = 2103_14978
BASES = np.frombuffer(b"ACGT", dtype=np.uint8)
N_BYTE = ord("N")


@dataclasses.dataclass
class Workload:
    """Reads, reference and pairs of one synthetic configuration.

    ``reads`` is ``n_reads x stride`` ASCII bytes (row r holds read r in its
    first ``read_len[r]`` bytes, the rest is 'N' padding that no consumer may
    read); ``ref`` is the reference in ASCII; pair p compares read
    ``pair_read[p]`` with ``ref[pair_off[p] : pair_off[p] + read_len]`` at
    threshold ``pair_e[p]`` (or the scalar ``e``)."""

    name: str
    reads: np.ndarray
    read_len: np.ndarray
    stride: int
    ref: np.ndarray
    pair_read: np.ndarray
    pair_off: np.ndarray
    pair_e: np.ndarray | None = None
    e: int | None = None
    seed: int = 0
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_reads(self) -> int:
        return int(self.read_len.shape[0])

    @property
    def n_pairs(self) -> int:
        return int(self.pair_read.shape[0])

    @property
    def read_start(self) -> np.ndarray:
        return np.arange(self.n_reads, dtype=np.uint64) * np.uint64(self.stride)

    def read(self, r: int) -> str:
        return bytes(self.reads[r * self.stride: r * self.stride + int(self.read_len[r])]).decode()

    def window(self, p: int) -> str:
        m = int(self.read_len[self.pair_read[p]])
        o = int(self.pair_off[p])
        return bytes(self.ref[o: o + m]).decode()

    def subset(self, idx: np.ndarray, name: str | None = None) -> "Workload":
        """The same reads and reference with only the pairs ``idx``."""
        return dataclasses.replace(
            self, name=name or self.name + "-subset",
            pair_read=np.ascontiguousarray(self.pair_read[idx]),
            pair_off=np.ascontiguousarray(self.pair_off[idx]),
            pair_e=None if self.pair_e is None else np.ascontiguousarray(self.pair_e[idx]))


def random_bases(rng: np.random.Generator, n: int) -> np.ndarray:
    return BASES[rng.integers(0, 4, int(n), dtype=np.uint8)]


def edited_copies(rng: np.random.Generator, text: np.ndarray, starts: np.ndarray,
                  m: int, n_edits: np.ndarray, lengths: np.ndarray | None = None) -> np.ndarray:
    """Copies of ``text[start : start + ~m]`` of exactly m bases, each with
    ``n_edits`` random edits (substitution, insertion or deletion with equal
    odds, positions uniform over the copy's own length).  Deletions pull in
    the bases that follow the window.  Returns uint8 ``(len(starts), m)``."""
    n = int(starts.shape[0])
    k = np.asarray(n_edits, dtype=np.int64)
    kmax = int(k.max()) if n else 0
    cols = np.arange(m, dtype=np.int64)
    if kmax == 0:
        return text[starts[:, None].astype(np.int64) + cols[None, :]]
    lens = np.full(n, m, np.int64) if lengths is None else np.asarray(lengths, np.int64)
    slot = np.arange(kmax)[None, :] < k[:, None]
    kind = rng.integers(0, 3, (n, kmax))
    pos = (rng.random((n, kmax)) * lens[:, None]).astype(np.int64)
    rows = np.repeat(np.arange(n), kmax).reshape(n, kmax)
    shift = np.zeros((n, m + 1), np.int32)
    ins_mask = np.zeros((n, m), bool)
    sub_mask = np.zeros((n, m), bool)
    d = slot & (kind == 2)
    np.add.at(shift, (rows[d], pos[d]), 1)              # deletion: skip a source base
    i = slot & (kind == 1)
    np.add.at(shift, (rows[i], pos[i] + 1), -1)         # insertion: later bases come one earlier
    ins_mask[rows[i], pos[i]] = True
    s = slot & (kind == 0)
    sub_mask[rows[s], pos[s]] = True
    idx = starts[:, None].astype(np.int64) + cols[None, :] + np.cumsum(shift[:, :m], axis=1)
    idx = np.clip(idx, 0, text.shape[0] - 1)
    out = text[idx]
    if ins_mask.any():
        out[ins_mask] = random_bases(rng, int(ins_mask.sum()))
    if sub_mask.any():
        # a different base: add 1..3 to the base's index in ACGT
        lut = np.zeros(256, np.uint8)
        lut[BASES] = np.arange(4, dtype=np.uint8)
        old = lut[out[sub_mask]]
        out[sub_mask] = BASES[(old + rng.integers(1, 4, old.shape[0], dtype=np.uint8)) % 4]
    return out


@functools.lru_cache(maxsize=4)
def reference(n_bases: int = 100_000_000, seed: int = SEED_BASE, dup_frac: float = 0.05,
              n_frac: float = 0.0) -> np.ndarray:
    """Uniform ACGT genome with ``dup_frac`` of it overwritten by 1-10 kbp
    copies of other positions at 1-3% divergence (substitutions and indels),
    then ``n_frac`` of the positions set to 'N'.  Read-only, cached."""
    rng = np.random.default_rng([seed, n_bases, 1])
    ref = random_bases(rng, n_bases)
    target = int(dup_frac * n_bases)
    copied = 0
    seg_hi = max(2, min(10_000, n_bases // 20))
    seg_lo = max(1, min(1_000, seg_hi // 2))
    while copied < target:
        L = int(rng.integers(seg_lo, seg_hi + 1))
        src = int(rng.integers(0, n_bases - 2 * L))
        dst = int(rng.integers(0, n_bases - L))
        k = int(rng.binomial(L, rng.uniform(0.01, 0.03)))
        seg = edited_copies(rng, ref, np.array([src]), L, np.array([k]))[0]
        ref[dst: dst + L] = seg
        copied += L
    if n_frac > 0:
        nn = int(rng.binomial(n_bases, n_frac))
        ref[rng.integers(0, n_bases, nn)] = N_BYTE
    ref.setflags(write=False)
    return ref


def _layout_reads(rows: np.ndarray, lens: np.ndarray, stride: int) -> np.ndarray:
    n = rows.shape[0]
    out = np.full((n, stride), N_BYTE, np.uint8)
    w = rows.shape[1]
    out[:, :w] = rows
    if (lens < w).any():
        pad = np.arange(w)[None, :] >= lens[:, None]
        out[:, :w][pad] = N_BYTE
    return out.reshape(-1)


def sampled_reads(rng, ref: np.ndarray, n_reads: int, lens: np.ndarray, edit_rate_hi: float,
                  chunk: int = 250_000):
    """Reads sampled at uniform positions of ``ref`` with up to
    ``edit_rate_hi`` x length random edits.  Returns (rows uint8 [n, max_len],
    origin offsets uint32)."""
    mmax = int(lens.max())
    L = ref.shape[0]
    margin = int(np.ceil(edit_rate_hi * mmax)) + 2
    origin = rng.integers(margin, L - mmax - margin, n_reads).astype(np.int64)
    rows = np.empty((n_reads, mmax), np.uint8)
    for a in range(0, n_reads, chunk):
        b = min(n_reads, a + chunk)
        kmax = np.floor(edit_rate_hi * lens[a:b]).astype(np.int64)
        k = (rng.random(b - a) * (kmax + 1)).astype(np.int64)
        rows[a:b] = edited_copies(rng, ref, origin[a:b], mmax, k, lengths=lens[a:b])
    return rows, origin.astype(np.uint32)


def pairs_workload(name: str, *, seed: int, ref: np.ndarray, n_pairs: int, m, cands,
                   e: int | None = None, e_rates=None, read_edit_rate: float = 0.02,
                   read_n_frac: float = 0.0, shuffle: bool = False, chunk: int = 250_000) -> Workload:
    """Reads sampled from ``ref``, each with ``cands`` candidates (an int or an
    inclusive range): the first is the read's true origin, the rest uniform
    random offsets.  ``m`` is an int or an inclusive (lo, hi) length range.
    Per-pair thresholds come from ``e_rates`` (e = ceil(rate x m), rate drawn
    per pair) unless the scalar ``e`` is given.  Exactly ``n_pairs`` pairs."""
    rng = np.random.default_rng([seed, n_pairs, 2])
    L = ref.shape[0]
    if isinstance(cands, tuple):
        lo, hi = cands
        mean = (lo + hi) / 2
        est = int(n_pairs / mean * 1.1) + 16
        c = rng.integers(lo, hi + 1, est)
        cs = np.cumsum(c)
        n_reads = int(np.searchsorted(cs, n_pairs) + 1)
        c = c[:n_reads].copy()
        c[-1] -= int(cs[n_reads - 1] - n_pairs)
    else:
        n_reads = -(-n_pairs // int(cands))
        c = np.full(n_reads, int(cands), np.int64)
        c[-1] -= n_reads * int(cands) - n_pairs
    if isinstance(m, tuple):
        lens = rng.integers(m[0], m[1] + 1, n_reads).astype(np.uint16)
    else:
        lens = np.full(n_reads, int(m), np.uint16)
    mmax = int(lens.max())
    stride = mmax
    rows, origin = sampled_reads(rng, ref, n_reads, lens, read_edit_rate, chunk)
    if read_n_frac > 0:
        nn = int(rng.binomial(rows.size, read_n_frac))
        flat = rows.reshape(-1)
        flat[rng.integers(0, rows.size, nn)] = N_BYTE
    reads = _layout_reads(rows, lens.astype(np.int64), stride)
    pair_read = np.repeat(np.arange(n_reads, dtype=np.uint32), c)
    first = np.zeros(n_pairs, bool)
    first[np.concatenate([[0], np.cumsum(c)[:-1]])] = True
    m_pair = lens[pair_read].astype(np.int64)
    pair_off = (rng.random(n_pairs) * (L - m_pair + 1)).astype(np.uint32)
    pair_off[first] = origin[pair_read[first]]
    pair_e = None
    if e is None:
        rates = np.asarray(e_rates, dtype=np.float64)
        r = rates[rng.integers(0, rates.shape[0], n_pairs)]
        pair_e = np.minimum(np.ceil(np.round(r * m_pair, 9)), 255).astype(np.uint8)
    if shuffle:
        perm = rng.permutation(n_pairs)
        pair_read, pair_off = pair_read[perm], pair_off[perm]
        if pair_e is not None:
            pair_e = pair_e[perm]
    return Workload(name=name, reads=reads, read_len=lens, stride=stride, ref=ref,
                    pair_read=np.ascontiguousarray(pair_read), pair_off=np.ascontiguousarray(pair_off),
                    pair_e=pair_e, e=e, seed=seed,
                    meta={"n_reads": n_reads, "cands": cands, "m": m, "ref_len": int(L),
                          "read_edit_rate": read_edit_rate, "read_n_frac": read_n_frac})


# ---- the five configurations ----------------------------------------------

def config1(seed: int = SEED_BASE + 0, n_pairs: int = 10_000, m: int = 100, e: int = 2) -> Workload:
    """10,000 pairs of 100 bp at e=2: i.i.d. uniform reads; each candidate
    segment is the read with k ~ U{0..6} edits, cut or extended to m, flanked
    by e random bases on each side; the reference is the segments end to end
    and pair i's offset is the start of segment i plus e."""
    rng = np.random.default_rng([seed, n_pairs, 1])
    reads = random_bases(rng, n_pairs * m).reshape(n_pairs, m)
    ext = random_bases(rng, n_pairs * m).reshape(n_pairs, m)
    text = np.concatenate([reads, ext], axis=1).reshape(-1)
    starts = np.arange(n_pairs, dtype=np.int64) * (2 * m)
    k = rng.integers(0, 7, n_pairs)
    seg = edited_copies(rng, text, starts, m, k)
    flank_l = random_bases(rng, n_pairs * e).reshape(n_pairs, e)
    flank_r = random_bases(rng, n_pairs * e).reshape(n_pairs, e)
    ref = np.concatenate([flank_l, seg, flank_r], axis=1).reshape(-1)
    seg_len = m + 2 * e
    pair_off = (np.arange(n_pairs, dtype=np.int64) * seg_len + e).astype(np.uint32)
    return Workload(name="c1-100bp-e2", reads=reads.reshape(-1).copy(),
                    read_len=np.full(n_pairs, m, np.uint16), stride=m, ref=ref,
                    pair_read=np.arange(n_pairs, dtype=np.uint32), pair_off=pair_off,
                    e=e, seed=seed, meta={"edits_per_segment": "U{0..6}", "ref_len": int(ref.shape[0])})


def accuracy_set(m: int, k_max: int, n_pairs: int, seed: int = SEED_BASE + 5, unrelated: float = 0.25,
                 flank: int = 32) -> Workload:
    """Pairs for the accuracy study: i.i.d. uniform reads of m bases.  A share
    ``1 - unrelated`` of the segments is the read with k ~ U{0..k_max} random
    edits (substitution, insertion, deletion with equal odds), so many pairs
    sit near any threshold; the rest are unrelated random segments.  Each
    segment is flanked by ``flank`` random bases; the reference is the
    segments end to end and pair i's offset is segment i's start.
    ``meta["k"]`` holds the edits applied (-1 for unrelated segments)."""
    rng = np.random.default_rng([seed, n_pairs, m, k_max, 6])
    reads = random_bases(rng, n_pairs * m).reshape(n_pairs, m)
    ext = random_bases(rng, n_pairs * m).reshape(n_pairs, m)
    text = np.concatenate([reads, ext], axis=1).reshape(-1)
    starts = np.arange(n_pairs, dtype=np.int64) * (2 * m)
    k = rng.integers(0, k_max + 1, n_pairs)
    seg = edited_copies(rng, text, starts, m, k)
    other = rng.random(n_pairs) < unrelated
    seg[other] = random_bases(rng, int(other.sum()) * m).reshape(-1, m)
    k[other] = -1
    flank_l = random_bases(rng, n_pairs * flank).reshape(n_pairs, flank)
    flank_r = random_bases(rng, n_pairs * flank).reshape(n_pairs, flank)
    ref = np.concatenate([flank_l, seg, flank_r], axis=1).reshape(-1)
    pair_off = (np.arange(n_pairs, dtype=np.int64) * (m + 2 * flank) + flank).astype(np.uint32)
    return Workload(name=f"accuracy-{m}bp-k{k_max}", reads=reads.reshape(-1).copy(),
                    read_len=np.full(n_pairs, m, np.uint16), stride=m, ref=ref,
                    pair_read=np.arange(n_pairs, dtype=np.uint32), pair_off=pair_off, e=0, seed=seed,
                    meta={"k": k})


def config2(scale: float = 1.0, seed: int = SEED_BASE + 1, ref_bases: int = 100_000_000) -> Workload:
    """20M pairs of 100 bp: 5M reads x 4 candidates (the true origin, sampled
    with 0-2% edits, then 3 uniform random offsets) on the 100 Mbp genome.
    The threshold is set per launch (the e sweep 0..10)."""
    n_pairs = int(round(20_000_000 * scale))
    ref = reference(ref_bases, SEED_BASE, 0.05, 0.0)
    return pairs_workload(f"c2-100bp-{n_pairs}", seed=seed, ref=ref, n_pairs=n_pairs, m=100,
                          cands=4, e=0, read_edit_rate=0.02)


def config3(m: int = 150, scale: float = 1.0, seed: int = SEED_BASE + 2,
            ref_bases: int = 100_000_000) -> Workload:
    """10M pairs at 150 or 250 bp, 8-64 candidates per read (1 true origin),
    'N' injected at 0.1% of reference and read positions."""
    n_pairs = int(round(10_000_000 * scale))
    ref = reference(ref_bases, SEED_BASE, 0.05, 0.001)
    return pairs_workload(f"c3-{m}bp-{n_pairs}", seed=seed + m, ref=ref, n_pairs=n_pairs, m=m,
                          cands=(8, 64), e=0, read_edit_rate=0.02, read_n_frac=0.001)


def config4(scale: float = 1.0, seed: int = SEED_BASE + 3, ref_bases: int = 100_000_000) -> Workload:
    """50M pairs, read length U{50..300}, 4 candidates per read, per-pair
    e = ceil(rate x m) with rate in {0.02, 0.05, 0.10}, shuffled order."""
    n_pairs = int(round(50_000_000 * scale))
    ref = reference(ref_bases, SEED_BASE, 0.05, 0.0)
    return pairs_workload(f"c4-mixed-{n_pairs}", seed=seed, ref=ref, n_pairs=n_pairs, m=(50, 300),
                          cands=4, e_rates=(0.02, 0.05, 0.10), read_edit_rate=0.02, shuffle=True)


def serving_requests(n_requests: int, seed: int = SEED_BASE + 4, size_lo: int = 1_000,
                     size_hi: int = 1_000_000, lengths=(100, 150, 250), rates=(0.02, 0.05, 0.10)):
    """Request plan of the serving configuration: log-uniform sizes in
    [size_lo, size_hi] pairs, a read length from ``lengths`` and one
    e = ceil(rate x m) per request.  Returns a list of dicts."""
    rng = np.random.default_rng([seed, n_requests, 5])
    sizes = np.exp(rng.uniform(np.log(size_lo), np.log(size_hi), n_requests)).astype(np.int64)
    ms = np.asarray(lengths)[rng.integers(0, len(lengths), n_requests)]
    rs = np.asarray(rates)[rng.integers(0, len(rates), n_requests)]
    return [{"id": i, "n_pairs": int(sizes[i]), "m": int(ms[i]),
             "e": int(np.ceil(round(rs[i] * ms[i], 9))), "seed": int(seed * 1000 + i)}
            for i in range(n_requests)]
