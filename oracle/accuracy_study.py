"""Accuracy of the filter against the global edit distance: false accepts and
false rejects over the threshold sweeps of the benchmark read lengths, for
the default filter (4-base window run count, Sec. 3.4 edge OR), the popcount
of the final vector, and the filter without the edge OR (the original
GateKeeper of Sec. 2.1).  The paper reports 0 false rejects and false-accept
rates that fall with the read length and rise with e (Sec. 5.1); its own
data sets are not available, so this study uses seeded synthetic pairs
(`synth.accuracy_set`).

Test infrastructure: calls only the oracle (and the seeded input
generator).  `python oracle/accuracy_study.py > oracle/accuracy_results.md`
writes the committed table.
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2103_14978_gb300 import synth  # noqa: E402

VARIANTS = (("runs4", O.RUNS4, 0), ("popcount", O.POPCOUNT, 0), ("runs4-no-edge", O.RUNS4, O.FLAG_NO_EDGE_FIX))
SWEEPS = {100: 10, 150: 15, 250: 25}  # e = 0 .. 10% of m


def study(m: int, e_max: int, n_pairs: int, seed: int):
    """Per e: (pairs with d <= e, pairs with d > e, {variant: (false accepts,
    false rejects)}) on one accuracy set, d the global edit distance."""
    w = synth.accuracy_set(m, 2 * e_max, n_pairs, seed=seed)
    d = O.levenshtein_batch(w.reads, w.read_start, w.read_len, w.ref, w.pair_read, w.pair_off)
    rows = []
    for e in range(e_max + 1):
        within = d <= e
        res = {}
        for name, mode, flags in VARIANTS:
            acc, _, _ = O.filter_batch(w.reads, w.read_start, w.read_len, w.ref, w.pair_read, w.pair_off, e,
                                       mode, flags)
            res[name] = (int(((acc == 1) & ~within).sum()), int(((acc == 0) & within).sum()))
        rows.append((e, int(within.sum()), int((~within).sum()), res))
    return w, d, rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=40_000, help="pairs per read length")
    ap.add_argument("--seed", type=int, default=synth.SEED_BASE + 5)
    args = ap.parse_args()
    print("# Accuracy study: false accepts / false rejects against the global edit distance\n")
    print(f"Written by `python oracle/accuracy_study.py --pairs {args.pairs} --seed {args.seed}`.")
    print("Per read length: `synth.accuracy_set` pairs, 75% a read against itself with k ~ U{0..2 e_max}")
    print("random edits, 25% against an unrelated segment.  d = global edit distance of read and")
    print("window.  FA = accepted with d > e (share of the pairs with d > e), FR = rejected with d <= e.\n")
    for m, e_max in SWEEPS.items():
        _, d, rows = study(m, e_max, args.pairs, args.seed)
        print(f"## {m} bp ({args.pairs} pairs)\n")
        print("| e | d <= e | d > e | FA runs4 | FA popcount | FA no edge OR | FR runs4 | FR popcount | FR no edge OR |")
        print("|---|---|---|---|---|---|---|---|---|")
        for e, n_in, n_out, res in rows:
            fa = [res[v][0] for v, _, _ in VARIANTS]
            fr = [res[v][1] for v, _, _ in VARIANTS]
            rate = lambda x: f"{x} ({100.0 * x / max(n_out, 1):.2f}%)"
            print(f"| {e} | {n_in} | {n_out} | " + " | ".join(rate(x) for x in fa) + " | "
                  + " | ".join(str(x) for x in fr) + " |")
        print()


if __name__ == "__main__":
    main()
