"""Write the oracle's results for the large-n cell (alpha = 2, x_min = 1,
n = 1,000,000, 10,000 replicates, seed 1, cell id 0).

TEST INFRASTRUCTURE ONLY: this script calls nothing but the CPU oracle (plain
C, binary64) and the seeded cell definition of ``paper_1305_6738_gb300.inputs``.
Its output is the stored expected table ``tests/golden/large_n_R10000.txt``:
the order statistics floor(R q) of D for q = .90/.95/.99 (Section 3), the
means of D and of alpha-hat over all replicates, and D and alpha-hat of every
100th replicate.

Run from the repository root (about an hour on 8 cores):
    python oracle/make_large_n_golden.py
"""
from __future__ import annotations

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
STRIDE = 100


def main() -> None:
    out = os.path.join(ROOT, "tests", "golden", "large_n_R10000.txt")
    c = inputs.large_n_cell()[0]
    t0 = time.time()
    D, A, nc = oracle.cell(c.alpha, c.xmin, c.n, c.replicates, seed=SEED, cell_id=c.cell_id)
    cut = oracle.quantiles(D, inputs.QUANTILES)
    tmp = out + ".tmp"
    with open(tmp, "w") as f:
        f.write(f"# Oracle results of the large-n cell: alpha = {c.alpha}, x_min = {c.xmin}, n = {c.n}, "
                f"{c.replicates} replicates,\n")
        f.write(f"# seed {SEED}, stream tag 0, cell id {c.cell_id}; binary64.  Written by: "
                "python oracle/make_large_n_golden.py\n")
        f.write("# cutoffs (order statistics floor(R q) of D, q = .90 .95 .99), mean D, mean alpha-hat, "
                "nonconverged:\n")
        f.write("summary " + " ".join(repr(float(v)) for v in cut)
                + f" {math.fsum(D) / D.size!r} {math.fsum(A) / A.size!r} {nc}\n")
        f.write(f"# replicate D alpha-hat, every {STRIDE}th replicate:\n")
        for r in range(0, c.replicates, STRIDE):
            f.write(f"{r} {float(D[r])!r} {float(A[r])!r}\n")
    os.replace(tmp, out)
    print(f"wrote {out} in {time.time() - t0:.0f} s", file=sys.stderr)


if __name__ == "__main__":
    main()
