"""A bounded device wait that runs out is reported, and the GPU stays usable.

The table staging waits (bounded) on an mbarrier for its bulk copies.  The
test hook PL_TEST_WAIT_CYCLES, read when a context is created, makes that
context's first staging wait of every block wait instead on a second
mbarrier at which nothing ever arrives, for that many cycles: the wait runs
out, the block latches the timeout in the status word, waits with the full
bound for its own copies to land and returns, and no kernel takes further
work items.  The next pl_sync reports PL_ETIMEOUT (and clears the status);
a fresh context then runs a cell that matches the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_wait_timeout_is_reported_and_the_gpu_stays_usable(monkeypatch):
    import oracle
    from paper_1305_6738_gb300 import pl
    q = [0.9, 0.95, 0.99]
    cells = [pl.Cell(2.5, 1, 100, 2000, 0)]
    monkeypatch.setenv("PL_TEST_WAIT_CYCLES", "100000")
    ctx = pl.Context(0)
    monkeypatch.delenv("PL_TEST_WAIT_CYCLES")
    cut = torch.zeros(len(q), dtype=torch.float64, device="cuda")
    D = torch.zeros(2000, dtype=torch.float64, device="cuda")
    ctx.pl_ks_cutoffs(cells, 1, q, pl.PL_FP64, cutoffs=cut, D=D)  # device outputs: enqueued only
    with pytest.raises(pl.PLError) as e:
        ctx.pl_sync()
    assert e.value.status == pl.PL_ETIMEOUT
    ctx.pl_sync()  # reported once, then cleared
    ctx.close()
    # a fresh context on the same GPU: results match the oracle
    ctx = pl.Context(0)
    ctx.pl_ks_cutoffs(cells, 1, q, pl.PL_FP64, cutoffs=cut, D=D)
    ctx.pl_sync()
    ctx.close()
    D_or, _, _ = oracle.cell(2.5, 1, 100, 2000, seed=1, cell_id=0)
    assert np.max(np.abs(D.cpu().numpy() - D_or)) < 1e-12
    assert np.max(np.abs(cut.cpu().numpy() - oracle.quantiles(D_or, q))) < 1e-12
