"""Pins of the CPU oracle against the paper's definitions (arxiv 2103.14978).

Step-level cases are derived by hand from the text; pair-level checks live in
``pins.py``.  None of these expected values comes from the CUDA path.
"""
import random

import numpy as np
import pytest

from tests import pins


# Sec. 2.1: A=00, C=01, G=10, T=11; Sec. 3.3: anything else is undefined.
def test_code_table(oracle_lib):
    L = oracle_lib.lib()
    for ch, code in zip("ACGTacgt", [0, 1, 2, 3, 0, 1, 2, 3]):
        assert L.gko_code(ord(ch)) == code
    for ch in "NnRYKMSWBDHVX-. \0":
        assert L.gko_code(ord(ch)) == -1


# Sec. 2.1: a 0-streak of length 1 or 2 with a 1 on both sides becomes 1s.
AMEND = [
    ("", ""), ("0", "0"), ("1", "1"), ("11", "11"),
    ("101", "111"), ("1001", "1111"), ("10001", "10001"),
    ("0110", "0110"), ("010", "010"), ("00100", "00100"),
    ("0101", "0111"), ("1010", "1110"), ("010010", "011110"),
    ("1101011", "1111111"), ("100101", "111111"), ("1000101", "1000111"),
    ("1100110011", "1111111111"), ("10000001", "10000001"),
]


@pytest.mark.parametrize("raw,amended", AMEND)
def test_amend_cases(oracle_lib, raw, amended):
    assert oracle_lib.amend(raw) == amended


# Sec. 3.4: after amendment, the first s bits (s > 0) or the last |s| bits
# (s < 0) of the shifted mask are set.
@pytest.mark.parametrize("raw,s,fixed", [
    ("00000000", 1, "10000000"), ("00000000", 3, "11100000"),
    ("00000000", -1, "00000001"), ("00000000", -3, "00000111"),
    ("01010101", 0, "01010101"), ("0000", 9, "1111"), ("0000", -9, "1111"),
])
def test_edge_fix_cases(oracle_lib, raw, s, fixed):
    assert oracle_lib.edge_fix(raw, s) == fixed


# Sec. 2.1 window table, read as "number of maximal runs of 1s in the 4-base
# window" (16 entries, written out by hand).
RUNS4_TABLE = {
    "0000": 0,
    "1000": 1, "0100": 1, "0010": 1, "0001": 1,
    "1100": 1, "0110": 1, "0011": 1, "1110": 1, "0111": 1, "1111": 1,
    "1010": 2, "0101": 2, "1001": 2, "1101": 2, "1011": 2,
}


def test_window_table(oracle_lib):
    assert len(RUNS4_TABLE) == 16
    for w, n in RUNS4_TABLE.items():
        assert oracle_lib.count(w, oracle_lib.RUNS4) == n, w
        assert oracle_lib.count(w, oracle_lib.POPCOUNT) == w.count("1")


@pytest.mark.parametrize("F,runs4,pop,runs", [
    ("11111111", 2, 8, 1),       # one run over two windows counts once per window
    ("00011000", 2, 2, 1),       # a run split by the window boundary
    ("10101", 3, 3, 3),          # last window padded with 0s
    ("1", 1, 1, 1), ("", 0, 0, 0), ("000000000", 0, 0, 0),
    ("0110" * 5, 5, 10, 5),
])
def test_count_cases(oracle_lib, F, runs4, pop, runs):
    O = oracle_lib
    assert O.count(F, O.RUNS4) == runs4
    assert O.count(F, O.POPCOUNT) == pop
    assert O.count(F, O.RUNS) == runs


# Mask-by-mask hand derivations of the worked examples in pins.WORKED.
@pytest.mark.parametrize("R,G,s,raw,amended,fixed", [
    ("TCGTACGT", "ACGTACGA", -1, "11111110", "11111110", "11111111"),
    ("TCGTACGT", "ACGTACGA", 0, "10000001", "10000001", "10000001"),
    ("TCGTACGT", "ACGTACGA", 1, "01111111", "01111111", "11111111"),
    ("CTTGCCAG", "ATTGCCAG", 1, "01011011", "01111111", "11111111"),
    ("CTTGCCAG", "ATTGCCAG", -1, "10110111", "11111111", "11111111"),
    ("AAGAACGT", "ACGTACGT", 0, "01010000", "01110000", "01110000"),
    ("ACGTGCAA", "ACGTTGCA", 0, "00001110", "00001110", "00001110"),
    ("ACGTGCAA", "ACGTTGCA", 1, "01110000", "01110000", "11110000"),
    ("ACGTGCAA", "ACGTTGCA", -1, "11111110", "11111110", "11111111"),
    ("ACGTACAGT", "ACGTACGTA", 0, "000000111", "000000111", "000000111"),
    ("ACGTACAGT", "ACGTACGTA", 1, "011111111", "011111111", "111111111"),
    ("ACGTACAGT", "ACGTACGTA", -1, "111111000", "111111000", "111111001"),
])
def test_worked_masks(oracle_lib, R, G, s, raw, amended, fixed):
    O = oracle_lib
    assert O.shifted_mask(R, G, s) == raw
    assert O.amend(raw) == amended
    assert O.edge_fix(amended, s) == fixed


def test_worked_final_vectors(oracle_lib):
    for R, G, e, _, _, F in pins.WORKED:
        assert oracle_lib.final_vector(R, G, e) == F


def _fp(O):
    return lambda R, G, e, mode, flags: O.filter_pair(R, G, e, mode, flags)


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pair_pins(oracle_lib, check):
    check(_fp(oracle_lib))


def test_levenshtein_textbook(oracle_lib):
    O = oracle_lib
    assert O.levenshtein("kitten", "sitting") == 3
    assert O.levenshtein("flaw", "lawn") == 2
    assert O.levenshtein("", "ACG") == 3
    assert O.levenshtein("ACGT", "ACGT") == 0
    assert O.levenshtein("ACGT", "TGCA") == 4
    rng = random.Random(3)
    for _ in range(200):
        a = pins.rand_seq(rng, rng.randint(0, 30))
        b = pins.mutate(rng, a, rng.randint(0, 6))
        assert O.levenshtein(a, b) == pins.levenshtein(a, b)


def test_final_vector_nested_in_e(oracle_lib):
    """Adding the masks of e+1 can only clear bits of the AND (Sec. 2.1)."""
    rng = random.Random(21)
    for _ in range(150):
        m = rng.randint(1, 90)
        R, G = pins.near_pair(rng, m, rng.randint(0, 6))
        prev = None
        for e in range(0, 8):
            F = int(oracle_lib.final_vector(R, G, e)[::-1] or "0", 2)
            if prev is not None:
                assert F & ~prev == 0
            prev = F


def test_e_at_least_m(oracle_lib):
    """A shift by |s| >= m vacates the whole mask, which the edge OR then sets
    to all 1s, so every e >= m - 1 gives the same final vector and the pair is
    accepted (at most ceil(m/2) runs <= m <= e)."""
    rng = random.Random(22)
    for _ in range(100):
        m = rng.randint(1, 24)
        R, G = pins.near_pair(rng, m, rng.randint(0, 8))
        base = oracle_lib.final_vector(R, G, m - 1)
        for e in (m, m + 1, 2 * m + 3, 255):
            assert oracle_lib.final_vector(R, G, e) == base
            assert oracle_lib.filter_pair(R, G, e)[0] == 1


def test_empty_read(oracle_lib):
    assert oracle_lib.filter_pair("", "", 0) == (1, 0)
    assert oracle_lib.filter_pair("", "", 3) == (1, 0)


def test_restatements_agree(oracle_lib):
    """The byte-per-base C oracle and the big-integer restatement agree on
    every mode and variant, including undefined pairs."""
    from oracle import bigint_ref as B

    rng = random.Random(23)
    for _ in range(1500):
        m = rng.randint(0, 140)
        R, G = pins.near_pair(rng, m, rng.randint(0, 10)) if m else ("", "")
        if m and rng.random() < 0.05:
            p = rng.randrange(m)
            R = R[:p] + "N" + R[p + 1:]
        e = rng.randint(0, 14)
        for mode in (0, 1, 2):
            for flags in (0, 1):
                assert oracle_lib.filter_pair(R, G, e, mode, flags) == B.filter_pair(R, G, e, mode, flags), (R, G, e, mode, flags)


def test_batch_matches_single_pairs(oracle_lib):
    """The threaded batch driver returns the per-pair results, the invalid
    sentinel for out-of-range pairs, and honours per-pair e."""
    O = oracle_lib
    rng = np.random.default_rng(5)
    ref = rng.choice(np.frombuffer(b"ACGT", np.uint8), 5000)
    ref[rng.integers(0, 5000, 10)] = ord("N")
    n_reads = 200
    lens = rng.integers(1, 130, n_reads).astype(np.uint16)
    starts = np.concatenate([[0], np.cumsum(lens[:-1].astype(np.uint64))]).astype(np.uint64)
    reads = rng.choice(np.frombuffer(b"ACGT", np.uint8), int(lens.sum()))
    n = 3000
    pr = rng.integers(0, n_reads + 3, n).astype(np.uint32)  # some invalid ids
    po = rng.integers(0, 5000, n).astype(np.uint32)         # some windows overrun
    pe = rng.integers(0, 12, n).astype(np.uint8)
    acc, ed, used = O.filter_batch(reads, starts, lens, ref, pr, po, pe, threads=4)
    assert used == 4
    for p in range(n):
        r = int(pr[p])
        if r >= n_reads or int(po[p]) + int(lens[r]) > 5000:
            assert (acc[p], ed[p]) == (0, O.INVALID)
            continue
        R = bytes(reads[starts[r]: starts[r] + lens[r]]).decode()
        G = bytes(ref[po[p]: po[p] + lens[r]]).decode()
        assert (acc[p], ed[p]) == O.filter_pair(R, G, int(pe[p]))
    acc2, ed2, _ = O.filter_batch(reads, starts, lens, ref, pr, po, 4, threads=3)
    acc3, ed3, _ = O.filter_batch(reads, starts, lens, ref, pr, po, np.full(n, 4, np.uint8), threads=1)
    assert (acc2 == acc3).all() and (ed2 == ed3).all()
