"""The cutoff-table sweep at full size against the oracle's stored cutoffs.

The stored table (tests/golden/sweep_cutoffs_R100000.txt, written by
oracle/make_sweep_golden.py, which calls only the CPU oracle) holds, for each
of the 90 cells (alpha in {1.5, ..., 3.5} x n in {10, ..., 10000}, x_min = 1,
100,000 replicates, seed 1), the order statistics floor(R q) of D for
q = .90/.95/.99 (Section 3 and Table 1's construction) and the means of D and
of alpha-hat over the cell's replicates.  Here the library runs the same
9,000,000 replicates in the benchmark's launch configuration in both precision
forms: every cutoff must match the stored one (binary64 form within 1e-12;
binary32-bulk form within 1e-6, inside the 1e-4 bar), and so must the means
(a check over every replicate of every cell).  Every replicate of the n = 10
and n = 100 cells (1.8 million) is also compared one by one with the oracle,
computed here.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1305_6738_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sweep_cutoffs_R100000.txt")
R = 100_000
Q = list(inputs.QUANTILES)
# per-replicate bars (alpha-hat relative, D absolute) of the two precision forms
TOL = {0: (1e-10, 1e-12), 1: (1e-6, 1e-6)}


def load_golden():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            a, n, cid, q90, q95, q99, mD, mA, nc = line.split()
            rows[(float(a), int(n))] = (int(cid), np.array([float(q90), float(q95), float(q99)]),
                                        float(mD), float(mA), int(nc))
    return rows


@pytest.fixture(scope="module")
def sweep():
    from paper_1305_6738_gb300 import pl
    cells = inputs.cutoff_table_sweep(R)
    ctx = pl.Context(0)
    out = {}
    for prec in (0, 1):
        D = torch.empty(len(cells) * R, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
        A = torch.empty(len(cells) * R, dtype=torch.float64, device="cuda")
        cut = torch.empty(len(cells) * len(Q), dtype=torch.float64, device="cuda")
        ctx.pl_ks_cutoffs([pl.Cell(c.alpha, c.xmin, c.n, c.replicates, c.cell_id) for c in cells], 1, Q, prec,
                          cutoffs=cut, D=D, alpha_hat=A)
        ctx.pl_sync()
        out[prec] = (cut.cpu().numpy().reshape(len(cells), len(Q)), D.double().cpu().numpy(), A.cpu().numpy())
    counters = ctx.pl_counters()
    ctx.close()
    return cells, out, counters


def test_golden_table_is_the_sweep():
    g = load_golden()
    cells = inputs.cutoff_table_sweep(R)
    assert len(g) == len(cells) == 90
    for c in cells:
        cid, _, _, _, nc = g[(c.alpha, c.n)]
        assert cid == c.cell_id and nc == 0


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32bulk"])
def test_full_size_cutoffs_and_means_match_the_oracle(sweep, prec):
    cells, out, counters = sweep
    g = load_golden()
    cut, D, A = out[prec]
    tol_a, tol_d = TOL[prec]
    assert counters["newton_capped"] == 0
    worst = 0.0
    for k, c in enumerate(cells):
        _, gq, mD, mA, _ = g[(c.alpha, c.n)]
        err = np.max(np.abs(cut[k] - gq))
        worst = max(worst, err)
        assert err <= tol_d, (c.alpha, c.n, cut[k], gq)
        d = D[k * R:(k + 1) * R]
        a = A[k * R:(k + 1) * R]
        assert abs(np.mean(d) - mD) <= tol_d, (c.alpha, c.n)
        assert abs(np.mean(a) / mA - 1.0) <= tol_a, (c.alpha, c.n)
    assert worst <= 1e-4  # the cutoff bar of the method's statement


@pytest.mark.parametrize("n", [10, 100])
def test_every_replicate_of_small_cells_matches_the_oracle(sweep, n):
    cells, out, _ = sweep
    for k, c in enumerate(cells):
        if c.n != n:
            continue
        D_or, A_or, nc = oracle.cell(c.alpha, c.xmin, c.n, R, seed=1, cell_id=c.cell_id)
        assert nc == 0
        for prec in (0, 1):
            _, D, A = out[prec]
            tol_a, tol_d = TOL[prec]
            d = D[k * R:(k + 1) * R]
            a = A[k * R:(k + 1) * R]
            assert np.max(np.abs(a / A_or - 1.0)) < tol_a, (c.alpha, prec)
            assert np.max(np.abs(d - D_or)) < tol_d, (c.alpha, prec)
