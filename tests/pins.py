"""Pair-level pins of the filter definition, written as checks over any
``filter_pair(R, G, e, mode, flags) -> (accept, edits)`` callable.

They hold for the paper's method (arxiv 2103.14978, Sec. 2.1, 3.3, 3.4) and
do not restate its formula: hand-derived worked examples, closed-form
special cases, symmetries and a theorem checked against the textbook edit
distance.  ``test_oracle_pins`` runs them on the oracle; ``test_pin_strength``
runs them on deliberately broken restatements to show each plausible mistake
fails at least one of them.
"""
from __future__ import annotations

import itertools
import random

RUNS4, POPCOUNT = 0, 1
NO_EDGE = 1
UNDEFINED = 0xFFFF

# Worked examples derived by hand from Sec. 2.1 and Sec. 3.4 (the paper's own
# worked figures, Fig. 2/3 and Sup. Fig. S.1, are not available).  Each entry:
# read, reference segment, e, (accept, edits) with the improvement,
# (accept, edits) without it (the original GateKeeper), the RUNS4 final vector.
#
# 1. Substitutions at both ends, both segment ends are 'A'.  Shift +1 leaves
#    position 0 vacant; its comparison 'A' vs 'A' gives 0, which the AND would
#    let hide the error at 0 (likewise shift -1 at position 7).  With the
#    Sec. 3.4 OR both vacant bits become 1 and the two errors are counted:
#      s=-1 raw 11111110 -> amended 11111110 -> edge 11111111
#      s= 0 raw 10000001 -> amended 10000001
#      s=+1 raw 01111111 -> amended 01111111 -> edge 11111111
#    F = 10000001, windows 1000|0001 -> 2 > e=1 -> reject; true edit
#    distance 2, so GateKeeper (F = 00000000, edits 0) falsely accepts.
# 2. Same pair at e=2: the +-2 masks are all 1s after the edge OR, F is
#    unchanged, 2 <= 2 -> accept.
# 3. One substitution at position 0 ('C' for 'A'):
#      s=+1 raw 01011011 -> amended 01111111 -> edge 11111111
#      s=-1 raw 10110111 -> amended 11111111 -> edge 11111111
#    F = 10000000 -> 1 edit (GateKeeper: F = 0, 0 edits).
# 4. Substitutions at 1 and 3, e=0: H = 01010000, the 0 at 2 is bounded by
#    1s -> 01110000: one run in window 0 -> 1 edit (popcount would say 3).
# 5. The read lacks base 3 of the segment and ends with an extra 'A':
#      s= 0 raw 00001110 (no streak bounded on both sides)
#      s=+1 raw 01110000 -> edge 11110000
#      s=-1 raw 11111110 -> edge 11111111
#    F = 0 -> 0 edits at e=1.
# 6. Substitutions at 1 and 5, e=0: H = 01000100; the 0-streak between them
#    is 3 long and stays, so F = 01000100: 2 edits under both counts.
# 7. Why the edge OR comes after amendment.  m=9, e=1:
#      s= 0 raw 000000111 -> amended 000000111
#      s=+1 raw 011111111 -> amended 011111111 -> edge 111111111
#      s=-1 raw 111111000 -> amended 111111000 (the 0-streak touches the end)
#                                   -> edge 111111001
#    F = 000000001 -> 1 edit.  Setting the vacated bit before amending would
#    bound the streak at 6-7, fill it, and give F = 000000111 -> 2 edits.
WORKED = [
    ("TCGTACGT", "ACGTACGA", 1, (0, 2), (1, 0), "10000001"),
    ("TCGTACGT", "ACGTACGA", 2, (1, 2), (1, 0), "10000001"),
    ("CTTGCCAG", "ATTGCCAG", 1, (1, 1), (1, 0), "10000000"),
    ("AAGAACGT", "ACGTACGT", 0, (0, 1), (0, 1), "01110000"),
    ("ACGTGCAA", "ACGTTGCA", 1, (1, 0), (1, 0), "00000000"),
    ("ACGTACGT", "AAGTAAGT", 0, (0, 2), (0, 2), "01000100"),
    ("ACGTACAGT", "ACGTACGTA", 1, (1, 1), (1, 0), "000000001"),
]


def levenshtein(a: str, b: str) -> int:
    """Textbook unit-cost edit distance (Wagner-Fischer)."""
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j - 1] + (a[i - 1] != b[j - 1]), prev[j] + 1, cur[j - 1] + 1)
        prev = cur
    return prev[-1]


def rand_seq(rng, m):
    return "".join(rng.choice("ACGT") for _ in range(m))


def mutate(rng, s, k):
    s = list(s)
    for _ in range(k):
        t = rng.randrange(3)
        p = rng.randrange(len(s) + 1)
        if t == 0 and p < len(s):
            s[p] = rng.choice("ACGT")
        elif t == 1:
            s.insert(p, rng.choice("ACGT"))
        elif p < len(s):
            del s[p]
    return "".join(s)


def near_pair(rng, m, k):
    R = rand_seq(rng, m)
    G = mutate(rng, R, k)
    G = (G + rand_seq(rng, m))[:m]
    return R, G


# ---- checks: each raises AssertionError on a violation --------------------

def check_worked(fp):
    for R, G, e, improved, original, _ in WORKED:
        assert fp(R, G, e, RUNS4, 0) == improved, (R, G, e)
        assert fp(R, G, e, RUNS4, NO_EDGE) == original, (R, G, e, "no edge fix")
    # example 4 under a plain popcount of the amended vector
    assert fp("AAGAACGT", "ACGTACGT", 0, POPCOUNT, 0) == (0, 3)
    # example 6: a 3-streak is not amended, so the popcount stays 2
    assert fp("ACGTACGT", "AAGTAAGT", 0, POPCOUNT, 0) == (0, 2)


def check_identical(fp, n=60, seed=11):
    rng = random.Random(seed)
    for _ in range(n):
        m = rng.randint(1, 130)
        R = rand_seq(rng, m)
        for e in (0, 1, 3, 7, m - 1, m + 2):
            if e < 0:
                continue
            assert fp(R, R, e, RUNS4, 0) == (1, 0), (R, e)


def check_exact_match_at_e0(fp, n=300, seed=12):
    """e = 0 leaves only the Hamming mask: accept iff the strings are equal."""
    rng = random.Random(seed)
    for _ in range(n):
        m = rng.randint(1, 64)
        R, G = near_pair(rng, m, rng.randint(0, 2))
        a, c = fp(R, G, 0, RUNS4, 0)
        assert a == int(R == G), (R, G)
        assert (c == 0) == (R == G)


def check_single_substitution(fp, n=200, seed=13):
    rng = random.Random(seed)
    for _ in range(n):
        m = rng.randint(1, 100)
        R = rand_seq(rng, m)
        p = rng.randrange(m)
        G = R[:p] + rng.choice([b for b in "ACGT" if b != R[p]]) + R[p + 1:]
        for e in (1, 2, 5):
            a, c = fp(R, G, e, RUNS4, 0)
            assert a == 1 and c <= 1, (R, G, e, c)
        assert fp(R, G, 0, RUNS4, 0) == (0, 1)


def check_undefined(fp, n=60, seed=14):
    rng = random.Random(seed)
    for _ in range(n):
        m = rng.randint(1, 80)
        R, G = near_pair(rng, m, 3)
        p = rng.randrange(m)
        bad = rng.choice("NnRYX-")
        e = rng.randint(0, 5)
        if rng.random() < 0.5:
            assert fp(R[:p] + bad + R[p + 1:], G, e, RUNS4, 0) == (1, UNDEFINED)
        else:
            assert fp(R, G[:p] + bad + G[p + 1:], e, RUNS4, 0) == (1, UNDEFINED)
        assert fp(R.lower(), G, e, RUNS4, 0) == fp(R, G, e, RUNS4, 0)


def check_reversal(fp, n=300, seed=15):
    """Reversing both strings swaps the masks of shifts +s and -s (Sec. 2.1:
    all masks are ANDed) and swaps leading and trailing edges (Sec. 3.4), so
    the final vector is reversed: popcount is invariant always, the 4-base
    window count whenever the windows map onto windows (m % 4 == 0)."""
    rng = random.Random(seed)
    for _ in range(n):
        m = rng.randint(1, 60)
        if rng.random() < 0.5:
            m = 4 * rng.randint(1, 15)
        R, G = near_pair(rng, m, rng.randint(0, 6))
        e = rng.randint(0, 6)
        assert fp(R, G, e, POPCOUNT, 0) == fp(R[::-1], G[::-1], e, POPCOUNT, 0), (R, G, e)
        if m % 4 == 0:
            assert fp(R, G, e, RUNS4, 0) == fp(R[::-1], G[::-1], e, RUNS4, 0), (R, G, e)


def check_popcount_monotone(fp, n=150, seed=16):
    """More masks can only clear bits of the AND, so the popcount is
    non-increasing in e and acceptance is monotone."""
    rng = random.Random(seed)
    for _ in range(n):
        m = rng.randint(1, 60)
        R, G = near_pair(rng, m, rng.randint(0, 8))
        prev = None
        for e in range(0, 9):
            a, c = fp(R, G, e, POPCOUNT, 0)
            if prev is not None:
                assert c <= prev[1] and a >= prev[0], (R, G, e)
            prev = (a, c)


def check_no_false_reject(fp, n=1500, seed=17, exhaustive_m=4):
    """Theorem (derived from the definitions): if the global edit distance d
    of the pair is at most e, the 4-base window count is at most d, so the
    pair is accepted.  Sketch: every base of the segment that an optimal
    alignment matches with shift s is 0 in mask s and stays 0 unless its
    0-streak is 1-2 long and bounded inside the mask; then it sits between two
    edit events.  The final vector has no interior 0-streak shorter than 3, and
    a run holding j unmatched bases and t short matched streaks is at most
    j + 2t long while owning at least max(j, t + 1) edit events, which bounds
    the number of windows it touches.  The paper reports 0 false rejects
    against Edlib (Sec. 5.1)."""
    rng = random.Random(seed)
    for _ in range(n):
        m = rng.randint(1, 110)
        R, G = near_pair(rng, m, rng.randint(0, 7))
        d = levenshtein(R, G)
        e = rng.randint(0, 10)
        a, c = fp(R, G, e, RUNS4, 0)
        if d <= e:
            assert c <= d and a == 1, (R, G, e, d, c)
    m = exhaustive_m
    reads = ["".join(p) for p in itertools.product("ACGT", repeat=m)]
    segs = reads[:: max(1, len(reads) // 24)]
    for G in segs:
        for R in reads:
            d = levenshtein(R, G)
            for e in range(d, min(d + 2, m + 1)):
                a, c = fp(R, G, e, RUNS4, 0)
                assert c <= d and a == 1, (R, G, e, d, c)


ALL_CHECKS = [
    check_worked,
    check_identical,
    check_exact_match_at_e0,
    check_single_substitution,
    check_undefined,
    check_reversal,
    check_popcount_monotone,
    check_no_false_reject,
]
