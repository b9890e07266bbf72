"""Write the oracle's cutoffs of the 90-cell sweep at 100,000 replicates per cell.

TEST INFRASTRUCTURE ONLY: this script calls nothing but the CPU oracle (plain
C, binary64) and the seeded cell definitions of ``paper_1305_6738_gb300.inputs``
(which hold no arithmetic of the method).  Its output is the stored expected
table ``tests/golden/sweep_cutoffs_R100000.txt``.

Per cell (exponent alpha, x_min = 1, sample size n, cell id, seed 1, stream tag
0): the oracle draws each replicate's sample, fits the exponent by maximum
likelihood (Eq. 2), takes the KS distance at the fit (Eq. 3), and the cell's
cutoffs are the order statistics floor(R q) of the R distances (Section 3 and
Table 1's construction).  The file also stores the mean of D and of alpha-hat
over the cell's replicates (a check over every replicate, not only the three
order statistics) and the count of fits that did not converge.

Run from the repository root (about an hour on 8 cores):
    python oracle/make_sweep_golden.py [--replicates 100000] [--out PATH]
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


import oracle  # noqa: E402
from paper_1305_6738_gb300 import inputs  # noqa: E402

SEED = 1


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--replicates", type=int, default=100_000)
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "sweep_cutoffs_R100000.txt"))
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    cells = inputs.cutoff_table_sweep(args.replicates)
    qs = inputs.QUANTILES
    # the most expensive cells first, so that progress is visible early
    order = sorted(range(len(cells)), key=lambda k: -cells[k].n)
    rows = {}
    t0 = time.time()
    for k in order:
        c = cells[k]
        D, A, nc = oracle.cell(c.alpha, c.xmin, c.n, c.replicates, seed=SEED, cell_id=c.cell_id,
                               threads=args.threads)
        cut = oracle.quantiles(D, qs)
        rows[k] = (c, cut, math.fsum(D) / D.size, math.fsum(A) / A.size, nc)
        print(f"[{time.time() - t0:7.0f} s] alpha={c.alpha} n={c.n}: {' '.join(f'{v:.6f}' for v in cut)}",
              file=sys.stderr, flush=True)
    tmp = args.out + ".tmp"
    with open(tmp, "w") as f:
        f.write("# Oracle cutoffs of the 90-cell sweep (alpha in {1.5, 1.75, ..., 3.5} x n in\n")
        f.write("# {10, 20, 50, 100, 200, 500, 1000, 2000, 5000, 10000}, x_min = 1), binary64.\n")
        f.write(f"# {args.replicates} replicates per cell, seed {SEED}, stream tag 0, cell id = 10 * (alpha index)"
                " + (n index).\n")
        f.write("# Cutoff q = the order statistic floor(R q) (0-based) of the replicates' KS distances.\n")
        f.write("# Written by: python oracle/make_sweep_golden.py"
                + (f" --replicates {args.replicates}" if args.replicates != 100_000 else "") + "\n")
        f.write(f"# oracle threads: {oracle.max_threads() if args.threads == 0 else args.threads}\n")
        f.write("# columns: alpha n cell_id q90 q95 q99 mean_D mean_alpha_hat nonconverged\n")
        for k in range(len(cells)):
            c, cut, mD, mA, nc = rows[k]
            f.write(f"{c.alpha!r} {c.n} {c.cell_id} " + " ".join(repr(float(v)) for v in cut)
                    + f" {mD!r} {mA!r} {nc}\n")
    os.replace(tmp, args.out)
    print(f"wrote {args.out} in {time.time() - t0:.0f} s", file=sys.stderr)


if __name__ == "__main__":
    main()
