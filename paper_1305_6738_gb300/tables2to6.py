"""Reproduce Tables 2-6 of the paper (KS cutoffs of the truncated power law
on 1..K, K = 20, 50, 100, 500, 1000) on the GPU.

Every (K, gamma, N) cell is simulated in 10 runs of 50,000 replicates (run r
uses Philox seed r + 1), fitted by maximum likelihood with the finite scaling
factor, and the order statistics D_(floor(R q)) for q = 0.9, 0.95, 0.99,
0.999 are averaged over the runs (Section 3).  All cells of a run go through
one call of pl_ks_cutoffs_truncated.

    python -m paper_1305_6738_gb300.tables2to6 [--precision fp32-bulk|fp64]
        [--runs 10] [--replicates 50000] [--K 20 50 ...] [--compare TABLES.txt]
        [--json out.json]

With --compare (a file of rows "K gamma N q0.9 q0.95 q0.99 q0.999"), each
cell is printed beside the given values with the difference in units of its
Monte Carlo standard error (the spread of the runs).
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np

from . import inputs


def run_tables(ctx, precision: int, runs: int = inputs.TZ_RUNS, replicates: int = 50_000, Ks=inputs.TZ_KS):
    """Returns (cells, cutoffs[runs, ncells, nq]) from `runs` calls of pl_ks_cutoffs_truncated."""
    from . import pl
    cells = [pl.TCell(c.gamma, c.K, c.n, c.replicates, c.cell_id) for c in inputs.tables2to6_cells(replicates, Ks)]
    out = np.empty((runs, len(cells), len(inputs.TZ_QUANTILES)))
    for r in range(runs):
        out[r] = ctx.pl_ks_cutoffs_truncated(cells, r + 1, list(inputs.TZ_QUANTILES), precision)
    return cells, out


def summarise(cells, cut: np.ndarray):
    """Mean over runs and the standard error of that mean, per cell and quantile."""
    mean = cut.mean(axis=0)
    se = cut.std(axis=0, ddof=1) / math.sqrt(cut.shape[0]) if cut.shape[0] > 1 else np.zeros_like(mean)
    return {(c.K, c.gamma, c.n): (mean[i], se[i]) for i, c in enumerate(cells)}


def load_rows(path: str) -> dict:
    rows = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            K, g, n, *q = line.split()
            rows[(int(K), float(g), int(n))] = tuple(float(v) for v in q)
    return rows


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--precision", choices=["fp32-bulk", "fp64"], default="fp32-bulk")
    ap.add_argument("--runs", type=int, default=inputs.TZ_RUNS)
    ap.add_argument("--replicates", type=int, default=50_000)
    ap.add_argument("--K", type=int, nargs="+", default=list(inputs.TZ_KS))
    ap.add_argument("--compare", default="")
    ap.add_argument("--json", default="")
    args = ap.parse_args(argv)
    from . import pl
    ctx = pl.Context(0)
    prec = pl.PL_FP32_BULK if args.precision == "fp32-bulk" else pl.PL_FP64
    cells, cut = run_tables(ctx, prec, args.runs, args.replicates, tuple(args.K))
    table = summarise(cells, cut)
    ref = load_rows(args.compare) if args.compare else {}
    print("   K gamma      N   " + "   ".join(f"q{q:<7}" for q in inputs.TZ_QUANTILES)
          + ("   (given, difference in SE)" if ref else ""))
    for (K, g, n), (m, se) in table.items():
        line = f"{K:4d} {g:5.2f} {n:6d}   " + "  ".join(f"{v:.4f}" for v in m)
        if (K, g, n) in ref:
            z = [(m[j] - ref[(K, g, n)][j]) / max(se[j], 1e-12) for j in range(len(m))]
            line += "   | " + " ".join(f"{v:.4f}" for v in ref[(K, g, n)]) + "  z=" + " ".join(f"{v:+.1f}" for v in z)
        print(line)
    if args.json:
        with open(args.json, "w") as f:
            json.dump({f"{K} {g} {n}": {"mean": list(map(float, m)), "se": list(map(float, se))}
                       for (K, g, n), (m, se) in table.items()}, f, indent=1)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
