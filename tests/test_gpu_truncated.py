"""GPU parity of the truncated law on 1..K (Tables 2-6) through the C ABI
against the CPU oracle.

Tolerances as for the untruncated law: sampled integers bit-exact; gamma-hat
within 1e-10 relative (the fit is binary64 in both precision forms); D within
1e-12 absolute (FP64 form) or 1e-6 (FP32-bulk form); cutoffs within the same
D tolerance of the oracle's order statistics.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DTOL = {0: 1e-12, 1: 1e-6}


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


@pytest.mark.parametrize("gamma,K,seed,cell,purpose,rep0,nrep,n", [
    (1.0, 20, 1, 0, 0, 0, 3, 5001),
    (0.25, 1024, 7, 5, 0, 10, 2, 20000),
    (4.0, 50, 3, 99, 1, 0, 2, 777),
    (2.5, 2, 9, 1, 2, 2**32 - 3, 3, 64),
    (0.01, 1000, 2**40 + 3, 2**32 - 1, 0, 5, 1, 30000),
])
def test_sample_bit_exact(ctx, gamma, K, seed, cell, purpose, rep0, nrep, n):
    out = torch.empty(nrep * n, dtype=torch.int64, device="cuda")
    ctx.pl_sample_truncated(gamma, K, seed, cell, purpose, rep0, nrep, n, out)
    ctx.pl_sync()
    got = out.cpu().numpy().view(np.uint64).reshape(nrep, n)
    assert got.min() >= 1 and got.max() <= K
    for r in range(nrep):
        ref = oracle.tz_sample(gamma, K, seed, cell, rep0 + r, purpose, n)
        bad = np.nonzero(got[r] != ref)[0]
        assert bad.size == 0, (r, bad[:5], got[r][bad[:5]], ref[bad[:5]])


# (gamma, K, n, R, cell_id)
CELLS = [
    (0.25, 20, 10, 600, 0),      # small samples: many negative gamma-hat
    (1.0, 50, 100, 300, 1),
    (4.0, 20, 10, 500, 2),       # all-ones samples (the ln 2 rule)
    (2.5, 1000, 2000, 40, 3),
    (1.75, 2, 7, 300, 4),        # smallest support
    (3.0, 100, 1, 200, 5),       # n = 1
    (0.25, 3, 1, 200, 6),        # n = 1 at x = K: gamma-hat at the end -64
    (0.5, 500, 5000, 33, 7),     # ragged last run of a work item
    (1.5, 1024, 65535, 2, 8),    # largest support and sample
    (64.0, 10, 50, 20, 9),       # largest exponent
]


@pytest.fixture(scope="module")
def cells_oracle():
    return [oracle.tz_cell(g, K, n, R, seed=1, cell_id=cid)[:2] for g, K, n, R, cid in CELLS]


@pytest.mark.parametrize("prec", [0, 1])
def test_cutoffs_match_oracle(ctx, pl, cells_oracle, prec):
    cells = [pl.TCell(*c) for c in CELLS]
    total = sum(c[3] for c in CELLS)
    D = torch.empty(total, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    G = torch.empty(total, dtype=torch.float64, device="cuda")
    q = [0.9, 0.95, 0.99, 0.999]
    before = ctx.pl_counters()["newton_capped"]
    cut = ctx.pl_ks_cutoffs_truncated(cells, 1, q, prec, D=D, gamma_hat=G)
    ctx.pl_sync()
    assert ctx.pl_counters()["newton_capped"] == before
    Dg = D.double().cpu().numpy()
    Gg = G.cpu().numpy()
    off = 0
    for ci, (g, K, n, R, cid) in enumerate(CELLS):
        D_or, G_or = cells_oracle[ci]
        dg, gg = Dg[off:off + R], Gg[off:off + R]
        rel = np.abs(gg - G_or) / np.maximum(np.abs(G_or), 1.0)
        assert rel.max() < 1e-10, (ci, rel.max(), gg[rel.argmax()], G_or[rel.argmax()])
        assert np.abs(dg - D_or).max() < DTOL[prec], (ci, np.abs(dg - D_or).max())
        ref = oracle.quantiles(D_or, q)
        assert np.abs(cut[ci] - ref).max() < DTOL[prec] + 1e-15
        off += R
    # the edge cells reach what they are there for
    o6 = sum(c[3] for c in CELLS[:6])
    assert (Gg[o6:o6 + 200] == -64.0).any()
    o0 = 0
    assert (Gg[o0:o0 + 600] < 0).any()


def test_cells_alone_equal_cells_together(ctx, pl):
    cells = [pl.TCell(*c) for c in CELLS[:4]]
    total = sum(c[3] for c in CELLS[:4])
    D_all = torch.empty(total, dtype=torch.float64, device="cuda")
    ctx.pl_ks_cutoffs_truncated(cells, 5, [0.5], 0, D=D_all)
    off = 0
    for c in cells:
        D1 = torch.empty(c.replicates, dtype=torch.float64, device="cuda")
        ctx.pl_ks_cutoffs_truncated([c], 5, [0.5], 0, D=D1)
        assert torch.equal(D1, D_all[off:off + c.replicates])
        off += c.replicates


def test_full_size_cell_sampled(ctx, pl):
    """A Table 2-6 cell at its full size (50,000 replicates of N = 10,000 on
    K = 1000): replicates sampled across the range against the oracle."""
    g, K, n, R, cid = 1.25, 1000, 10000, 50000, 11
    D = torch.empty(R, dtype=torch.float64, device="cuda")
    G = torch.empty(R, dtype=torch.float64, device="cuda")
    ctx.pl_ks_cutoffs_truncated([pl.TCell(g, K, n, R, cid)], 3, [0.9, 0.95, 0.99, 0.999], 0, D=D, gamma_hat=G)
    Dg, Gg = D.cpu().numpy(), G.cpu().numpy()
    for r in [0, 1, 4095, 4096, 25000, 49998, 49999]:
        d_or, g_or = oracle.tz_cell(g, K, n, 1, seed=3, cell_id=cid, rep0=r)[:2]
        assert abs(Gg[r] / g_or[0] - 1) < 1e-10
        assert abs(Dg[r] - d_or[0]) < 1e-12
    # the fitted exponents centre on the simulated one
    assert abs(np.median(Gg) - g) < 0.01


@pytest.mark.parametrize("bad", [
    dict(gamma=0.0), dict(gamma=65.0), dict(K=1), dict(K=1025), dict(n=0), dict(n=65536),
    dict(replicates=0), dict(cell_id=2**32),
])
def test_cutoffs_reject_invalid(ctx, pl, bad):
    c = dict(gamma=1.0, K=20, n=10, replicates=10, cell_id=0)
    c.update(bad)
    with pytest.raises(pl.PLError) as e:
        ctx.pl_ks_cutoffs_truncated([pl.TCell(**c)], 1, [0.9])
    assert e.value.status == pl.PL_EINVAL
