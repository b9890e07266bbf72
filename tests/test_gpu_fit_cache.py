"""The context's fit tables (the exponent of Eq. 2 as a function of the mean
log, one table per xmin) are built once and copied on the device by later
calls, for the first 16 values of xmin a context meets; tables of further
values are built by every call.  Results must not depend on which path a
table took: the same call twice in one context, and once in a fresh context,
gives bit-identical D and alpha-hat, and the replicates match the oracle
(Section 4's simulation; binary64 form within 1e-12 for D, 1e-10 relative for
alpha-hat).
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ALPHA, N, R = 2.5, 50, 256
XMINS = list(range(1, 19))   # 18 values: 16 cached, 2 built by every call
CHECKED = [1, 16, 17, 18]    # against the oracle: cached and uncached tables


def run(ctx, pl):
    cells = [pl.Cell(ALPHA, x, N, R, 100 + x) for x in XMINS]
    D = torch.empty(R * len(cells), dtype=torch.float64, device="cuda")
    A = torch.empty(R * len(cells), dtype=torch.float64, device="cuda")
    ctx.pl_ks_cutoffs(cells, 5, [0.9, 0.99], pl.PL_FP64, D=D, alpha_hat=A)
    ctx.pl_sync()
    return D.cpu().numpy(), A.cpu().numpy()


@pytest.fixture(scope="module")
def results():
    from paper_1305_6738_gb300 import pl
    ctx = pl.Context(0)
    first = run(ctx, pl)
    second = run(ctx, pl)
    ctx.close()
    fresh_ctx = pl.Context(0)
    fresh = run(fresh_ctx, pl)
    fresh_ctx.close()
    return first, second, fresh


def test_cached_tables_give_identical_results(results):
    first, second, fresh = results
    for k in range(2):
        assert np.array_equal(first[k], second[k])
        assert np.array_equal(first[k], fresh[k])


@pytest.mark.parametrize("xmin", CHECKED)
def test_replicates_match_the_oracle(results, xmin):
    _, (D, A), _ = results
    i = XMINS.index(xmin)
    D_or, A_or, nc = oracle.cell(ALPHA, xmin, N, R, seed=5, cell_id=100 + xmin)
    assert nc == 0
    d = D[i * R:(i + 1) * R]
    a = A[i * R:(i + 1) * R]
    assert np.max(np.abs(d - D_or)) < 1e-12
    assert np.max(np.abs(a / A_or - 1.0)) < 1e-10
