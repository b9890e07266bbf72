"""The large-n cell at full size (alpha = 2, x_min = 1, n = 1,000,000, 10,000
replicates, seed 1; the block-per-replicate form the benchmark times) against
the oracle's stored results (tests/golden/large_n_R10000.txt, written by
oracle/make_large_n_golden.py, which calls only the CPU oracle): the three
cutoffs and the means of D and alpha-hat over every replicate, and D and
alpha-hat of every 100th replicate, in both precision forms."""
import os

import numpy as np
import pytest

from paper_1305_6738_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large_n_R10000.txt")
TOL = {0: (1e-10, 1e-12), 1: (1e-6, 1e-6)}


def load():
    summary, rows = None, {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = line.split()
            if w[0] == "summary":
                summary = (np.array([float(v) for v in w[1:4]]), float(w[4]), float(w[5]), int(w[6]))
            else:
                rows[int(w[0])] = (float(w[1]), float(w[2]))
    return summary, rows


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="stored large-n results not written")
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32bulk"])
def test_large_n_cell_matches_the_stored_oracle_results(prec):
    from paper_1305_6738_gb300 import pl
    (gcut, gmD, gmA, nc), rows = load()
    assert nc == 0 and len(rows) == 100
    c = inputs.large_n_cell()[0]
    R = c.replicates
    ctx = pl.Context(0)
    D = torch.empty(R, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    A = torch.empty(R, dtype=torch.float64, device="cuda")
    cut = torch.empty(3, dtype=torch.float64, device="cuda")
    ctx.pl_ks_cutoffs([pl.Cell(c.alpha, c.xmin, c.n, R, c.cell_id)], 1, list(inputs.QUANTILES), prec,
                      cutoffs=cut, D=D, alpha_hat=A)
    ctx.pl_sync()
    ctx.close()
    tol_a, tol_d = TOL[prec]
    D, A = D.double().cpu().numpy(), A.cpu().numpy()
    assert np.max(np.abs(cut.cpu().numpy() - gcut)) <= tol_d
    assert abs(np.mean(D) - gmD) <= tol_d
    assert abs(np.mean(A) / gmA - 1) <= tol_a
    for r, (d, a) in rows.items():
        assert abs(D[r] - d) <= tol_d, r
        assert abs(A[r] / a - 1) <= tol_a, r
