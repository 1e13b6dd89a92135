"""The accuracy study on a small seeded sample: the oracle against the
global edit distance reproduces the paper's qualitative claims (Sec. 5.1):
no false rejects with the 4-base window count, false accepts rising with e
and falling with the read length, fewer false accepts with the Sec. 3.4
edge OR than without; and the popcount reading does false-reject, which is
why the window count is the default reading of Sec. 2.1."""
import pytest

from oracle import accuracy_study as S


@pytest.fixture(scope="module")
def runs():
    return {m: S.study(m, e_max, 4000, 210314983)[2] for m, e_max in ((100, 10), (150, 15))}


def fa_rate(row, variant):
    e, n_in, n_out, res = row
    return res[variant][0] / max(n_out, 1)


def test_no_false_rejects_with_the_window_count(runs):
    for rows in runs.values():
        assert all(res["runs4"][1] == 0 for _, _, _, res in rows)


def test_popcount_false_rejects_somewhere(runs):
    assert sum(res["popcount"][1] for rows in runs.values() for _, _, _, res in rows) > 0


def test_false_accepts_rise_with_e_and_fall_with_length(runs):
    r100, r150 = runs[100], runs[150]
    assert fa_rate(r100[0], "runs4") == 0.0  # e = 0 accepts exact matches only
    for rows in (r100, r150):
        assert fa_rate(rows[1], "runs4") < fa_rate(rows[5], "runs4") < fa_rate(rows[8], "runs4")
    for e in (2, 5, 8):
        assert fa_rate(r150[e], "runs4") < fa_rate(r100[e], "runs4")


def test_edge_or_reduces_false_accepts(runs):
    for rows in runs.values():
        with_or = sum(res["runs4"][0] for _, _, _, res in rows)
        without = sum(res["runs4-no-edge"][0] for _, _, _, res in rows)
        assert with_or < without
