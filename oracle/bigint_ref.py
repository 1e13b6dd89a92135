"""Second restatement of the GateKeeper-GPU filter with Python big integers.

TEST INFRASTRUCTURE ONLY.  Written independently of ``oracle.c``: here a mask
is one arbitrary-precision integer whose bit i is base i, and every step of
the paper's algorithm is a whole-vector shift or logic operation:

* Sec. 2.1: two bit-planes per sequence (high and low bit of the 2-bit code
  A=00 C=01 G=10 T=11), shifted read planes XORed with the segment planes
  and OR-folded; amendment of 0-streaks of length 1-2 bounded by 1s, written
  as neighbour logic; AND of the 2e+1 masks; windowed error count.
* Sec. 3.3: a non-ACGT byte in either sequence passes the pair undefined.
* Sec. 3.4: vacated positions of each shifted mask are set after amendment.

The two restatements must agree exactly; a disagreement means one of them
misreads the paper.
"""
from __future__ import annotations

RUNS4, POPCOUNT, RUNS = 0, 1, 2
FLAG_NO_EDGE_FIX = 1
UNDEFINED = 0xFFFF

_CODE = {"A": 0, "C": 1, "G": 2, "T": 3}


def planes(S: str):
    """(high plane, low plane) of a sequence, or None if it holds a non-ACGT
    byte (lower case folded)."""
    hi = lo = 0
    for i, ch in enumerate(S.upper()):
        c = _CODE.get(ch)
        if c is None:
            return None
        hi |= ((c >> 1) & 1) << i
        lo |= (c & 1) << i
    return hi, lo


def amend(x: int, m: int) -> int:
    """A zero at i flips when it is a 1-streak (x[i-1] & x[i+1]), the first of
    a 2-streak (x[i-1] & ~x[i+1] & x[i+2]) or the second of one
    (x[i-2] & ~x[i-1] & x[i+1]).  Bits outside [0, m) read as 0, so streaks
    touching an end never flip."""
    full = (1 << m) - 1
    x &= full
    prev1 = (x << 1) & full
    prev2 = (x << 2) & full
    next1 = x >> 1
    next2 = x >> 2
    flip = (prev1 & (next1 | next2)) | (prev2 & (full & ~prev1) & next1)
    return (x | flip) & full


def count(F: int, m: int, mode: int = RUNS4) -> int:
    full = (1 << m) - 1
    F &= full
    if mode == POPCOUNT:
        return bin(F).count("1")
    starts_any = F & ~(F << 1)
    if mode == RUNS:
        return bin(starts_any & full).count("1")
    # RUNS4: a 1 starts a run unless the bit before it is 1 and in the same
    # window; window starts are the multiples of 4.
    window_starts = sum(1 << i for i in range(0, m, 4))
    starts = F & ~((F << 1) & ~window_starts)
    return bin(starts & full).count("1")


def final_vector(R: str, G: str, e: int, flags: int = 0):
    m = len(R)
    pr, pg = planes(R), planes(G)
    if pr is None or pg is None:
        return None
    (rh, rl), (gh, gl) = pr, pg
    full = (1 << m) - 1
    F = full
    for s in range(-e, e + 1):
        if s >= 0:
            sh, sl = (rh << s) & full, (rl << s) & full
        else:
            sh, sl = rh >> (-s), rl >> (-s)
        x = ((sh ^ gh) | (sl ^ gl)) & full
        x = amend(x, m)
        if not (flags & FLAG_NO_EDGE_FIX):
            k = min(abs(s), m)
            if s > 0:
                x |= (1 << k) - 1
            elif s < 0:
                x |= full & ~((1 << (m - k)) - 1)
        F &= x
    return F


def filter_pair(R: str, G: str, e: int, mode: int = RUNS4, flags: int = 0):
    F = final_vector(R, G, e, flags)
    if F is None:
        return 1, UNDEFINED
    c = count(F, len(R), mode)
    return int(c <= e), c


def bits_str(F: int, m: int) -> str:
    return "".join("1" if (F >> i) & 1 else "0" for i in range(m))
