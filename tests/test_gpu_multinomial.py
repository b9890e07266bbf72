"""GPU parity of the multinomial histogram sampler (pl_ks_cutoffs_multinomial)
against the oracle's (oracle.mn_cell, stream tag 3): per replicate alpha-hat
within 1e-10 relative and D within 1e-12 (FP64 form) or 1e-6 (FP32-bulk
form), which holds only when the histograms agree value for value; cutoffs as
order statistics.  Cells from n = 1 to 10^6, all-ones atoms, heavy tails and
lower ends above 1; and the cutoffs of a cell agree with the inverse-CDF
sampler's within their Monte Carlo error."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {0: (1e-10, 1e-12), 1: (1e-6, 1e-6)}


@pytest.fixture(scope="module")
def pl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_6738_gb300 import build
    build.build()
    from paper_1305_6738_gb300 import pl as _pl
    return _pl


@pytest.fixture(scope="module")
def ctx(pl):
    c = pl.Context(0)
    yield c
    c.close()


CELLS = [
    (2.5, 1, 100, 300, 0),
    (2.0, 1, 5000, 60, 1),
    (1.5, 3, 2000, 40, 2),       # heavy tail, lower end above 1
    (3.5, 1, 10, 200, 3),        # all-ones atoms
    (2.0, 2, 1, 50, 4),          # n = 1
    (2.0, 1, 1_000_000, 3, 5),   # large n: ~780 binomials and ~780 single draws
    (8.0, 1, 3000, 30, 6),       # light tail: the thresholds reach 1 within the head
]


@pytest.fixture(scope="module")
def mn_oracle():
    return [oracle.mn_cell(a, xm, n, R, seed=1, cell_id=cid)[:2] for a, xm, n, R, cid in CELLS]


@pytest.mark.parametrize("prec", [0, 1])
def test_multinomial_cells_match_oracle(ctx, pl, mn_oracle, prec):
    cells = [pl.Cell(*c) for c in CELLS]
    total = sum(c[3] for c in CELLS)
    D = torch.empty(total, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    A = torch.empty(total, dtype=torch.float64, device="cuda")
    q = [0.9, 0.95, 0.99]
    cut = ctx.pl_ks_cutoffs_multinomial(cells, 1, q, prec, D=D, alpha_hat=A)
    ctx.pl_sync()
    Dg, Ag = D.double().cpu().numpy(), A.cpu().numpy()
    off = 0
    for ci, (a, xm, n, R, cid) in enumerate(CELLS):
        D_or, A_or = mn_oracle[ci]
        assert np.max(np.abs(Ag[off:off + R] / A_or - 1)) < TOL[prec][0], ci
        assert np.max(np.abs(Dg[off:off + R] - D_or)) < TOL[prec][1], ci
        assert np.max(np.abs(cut[ci] - oracle.quantiles(D_or, q))) < TOL[prec][1] + 1e-15
        off += R


def test_multinomial_cutoffs_agree_with_inverse_cdf(ctx, pl):
    cell = pl.Cell(2.0, 1, 20000, 20000, 7)
    q = [0.5, 0.9, 0.95, 0.99]
    a = ctx.pl_ks_cutoffs_multinomial([cell], 1, q, 0)[0]
    b = ctx.pl_ks_cutoffs([cell], 1, q, 0)[0]
    D = torch.empty(20000, dtype=torch.float64, device="cuda")
    ctx.pl_ks_cutoffs([cell], 2, q, 0, D=D)
    d = np.sort(D.cpu().numpy())
    for j, qq in enumerate(q):
        # standard error of an order statistic from the spacing of the sorted D
        i = int(qq * len(d))
        se = (d[min(i + 100, len(d) - 1)] - d[max(i - 100, 0)]) / 200 * np.sqrt(qq * (1 - qq) * len(d))
        assert abs(a[j] - b[j]) < 5 * np.sqrt(2) * se + 1e-6, (qq, a[j], b[j], se)
