"""The pins must catch plausible mistakes.

Each mutant below is a restatement of the filter with one plausible error
planted (a dropped term, a wrong sign or side, a misplaced step).  The pins in
``pins.py`` pass on the oracle (``test_oracle_pins``) and must fail on every
mutant.  Mutants run on the CPU only.
"""
import pytest

from tests import pins

_CODE = {"A": 0, "C": 1, "G": 2, "T": 3}


def _planes(S):
    hi = lo = 0
    for i, ch in enumerate(S.upper()):
        c = _CODE.get(ch)
        if c is None:
            return None
        hi |= ((c >> 1) & 1) << i
        lo |= (c & 1) << i
    return hi, lo


def make_filter(mut: str):
    """A big-integer filter with the mistake ``mut`` planted ('' = none)."""

    def amend(x, m):
        full = (1 << m) - 1
        if mut == "no_amend":
            return x
        if mut == "amend_ends":  # treat bits outside the mask as 1s
            ext = (x << 2) | 0b11 | (0b11 << (m + 2))
            y = amend_core(ext, m + 4)
            return (y >> 2) & full
        if mut == "amend_len3":
            return amend_len3(x, m)
        return amend_core(x, m)

    def amend_core(x, m):
        full = (1 << m) - 1
        p1, p2, n1, n2 = (x << 1) & full, (x << 2) & full, x >> 1, x >> 2
        return (x | (p1 & (n1 | n2)) | (p2 & ~p1 & n1)) & full

    def amend_len3(x, m):
        bits = [(x >> i) & 1 for i in range(m)]
        i = 0
        while i < m:
            if bits[i]:
                i += 1
                continue
            j = i
            while j < m and not bits[j]:
                j += 1
            if j - i <= 3 and i > 0 and j < m:
                for k in range(i, j):
                    bits[k] = 1
            i = j
        return sum(b << i for i, b in enumerate(bits))

    def fp(R, G, e, mode, flags):
        m = len(R)
        pr = _planes(R)
        if mut == "n_read_only":  # a non-ACGT segment base is read as 'A'
            pg = _planes("".join(c if c.upper() in "ACGT" else "A" for c in G))
        else:
            pg = _planes(G)
        if pr is None or pg is None:
            return 1, 0xFFFF
        (rh, rl), (gh, gl) = pr, pg
        full = (1 << m) - 1
        F = full
        hi_s = e - 1 if mut == "drop_mask" else e
        for s in range(-e, hi_s + 1):
            t = -s if mut == "shift_sign" else s
            if t >= 0:
                sh, sl = (rh << t) & full, (rl << t) & full
            else:
                sh, sl = rh >> (-t), rl >> (-t)
            x = (sh ^ gh) & full if mut == "hi_plane_only" else ((sh ^ gh) | (sl ^ gl)) & full
            k = min(abs(s), m)
            lead = (1 << k) - 1
            trail = full & ~((1 << (m - k)) - 1)
            if mut == "vacated_one":  # vacated bits set before amendment
                x |= lead if s > 0 else (trail if s < 0 else 0)
            if mut == "edge_first" and not flags:
                x |= lead if s > 0 else (trail if s < 0 else 0)
            if not (mut == "no_amend_h0" and s == 0):
                x = amend(x, m)
            if not flags and mut not in ("edge_first",):
                if mut == "edge_wrong_side":
                    x |= trail if s > 0 else (lead if s < 0 else 0)
                else:
                    x |= lead if s > 0 else (trail if s < 0 else 0)
            F &= x
        if mode == 1 or mut == "popcount":
            c = bin(F).count("1")
        else:
            ws = sum(1 << i for i in range(1 if mut == "window_offset" else 0, m, 4))
            if mut == "window_offset":
                ws |= 1
            c = bin(F & ~((F << 1) & ~ws) & full).count("1")
        return int(c <= e), c

    return fp


MUTANTS = [
    "no_amend", "amend_ends", "amend_len3", "drop_mask", "shift_sign",
    "hi_plane_only", "vacated_one", "edge_first", "no_amend_h0",
    "edge_wrong_side", "popcount", "window_offset", "n_read_only",
]


def _small(check):
    """Run a check on a reduced sample (big-integer Python is slow)."""
    name = check.__name__
    if name == "check_no_false_reject":
        return lambda fp: check(fp, n=600, exhaustive_m=4)
    return check


def test_unmutated_restatement_passes_pins():
    fp = make_filter("")
    for check in pins.ALL_CHECKS:
        _small(check)(fp)


@pytest.mark.parametrize("mut", MUTANTS)
def test_mutant_is_caught(mut):
    fp = make_filter(mut)
    caught = []
    for check in pins.ALL_CHECKS:
        try:
            _small(check)(fp)
        except AssertionError:
            caught.append(check.__name__)
    assert caught, f"mutant {mut} passes every pin"
