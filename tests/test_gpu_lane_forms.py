"""The lane-form sampler and the shortened histograms against the oracle,
replicate by replicate, in both precision forms.

Cells are chosen so that every path of the two optimisations runs: a light
tail drawn in the lane form into 64 bins although its size alone would give
128 (at least 32,768 replicates), a heavy tail drawn so too with several
spills per replicate and draws beyond the threshold table, a small sample
drawn in the lane form at its own size, and a larger sample kept in the warp
form with a shortened histogram whose replicates lanes finish with spills.
The draws are the Philox streams of the method's sampling (Section 4 of the
paper: inverse CDF of the law of Eq. 1), so D (Eq. 3) and alpha-hat (Eq. 2)
must equal the oracle's for every replicate: binary64 form within 1e-12 (D)
and 1e-10 relative (alpha-hat), binary32-bulk form within 1e-6.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# (alpha, xmin, n, replicates, cell_id)
CELLS = [(2.5, 1, 50, 32768, 41),    # light tail: 64 bins instead of 128, lane form
         (1.5, 1, 60, 40000, 42),    # heavy tail: 64 bins, ~6 spills per replicate, lane form
         (3.0, 2, 20, 5000, 43),     # 64 bins by its size: lane form with few replicates
         (2.0, 1, 800, 4000, 44)]    # 64 bins instead of 1,024, warp form, lanes finish with spills
TOL = {0: (1e-10, 1e-12), 1: (1e-6, 1e-6)}


@pytest.fixture(scope="module")
def results():
    from paper_1305_6738_gb300 import pl
    cells = [pl.Cell(*c) for c in CELLS]
    tot = sum(c.replicates for c in cells)
    ctx = pl.Context(0)
    out = {}
    for prec in (0, 1):
        D = torch.empty(tot, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
        A = torch.empty(tot, dtype=torch.float64, device="cuda")
        ctx.pl_ks_cutoffs(cells, 3, [0.9, 0.99], prec, D=D, alpha_hat=A)
        ctx.pl_sync()
        out[prec] = (D.double().cpu().numpy(), A.cpu().numpy())
    counters = ctx.pl_counters()
    ctx.close()
    return out, counters


@pytest.mark.parametrize("k", range(len(CELLS)))
def test_every_replicate_matches_the_oracle(results, k):
    out, counters = results
    a, xmin, n, R, cid = CELLS[k]
    off = sum(c[3] for c in CELLS[:k])
    D_or, A_or, nc = oracle.cell(a, xmin, n, R, seed=3, cell_id=cid)
    assert nc == 0
    for prec in (0, 1):
        D, A = out[prec]
        tol_a, tol_d = TOL[prec]
        d = D[off:off + R]
        al = A[off:off + R]
        assert np.max(np.abs(al / A_or - 1.0)) < tol_a, (CELLS[k], prec)
        assert np.max(np.abs(d - D_or)) < tol_d, (CELLS[k], prec)


def test_heavy_tail_cell_reaches_the_tail_paths(results):
    # the alpha = 1.5 cell draws values beyond its 64 bins in almost every
    # replicate and some beyond the threshold table (FP64 tail inversion)
    _, counters = results
    assert counters["tail_draws"] > 0
