"""The allocation-free entry point (for callers that cannot let a library call
cudaMalloc) against the context-based entry points, through the C ABI, on
several calls in a row (the fixed scratch keeps the previous call's contents)."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_6738_gb300 import build
    build.build()
    from paper_1305_6738_gb300 import pl as _pl
    return _pl


def test_noalloc_matches_context_entry_points(pl):
    ctx = pl.Context(0)
    sets = [
        (1, oracle.sample(1.5, 1, 5, 1, 0, 2, 20000)),   # values beyond the on-chip bins
        (1, oracle.sample(2.5, 1, 5, 0, 0, 2, 1000)),
        (1, np.ones(20, dtype=np.uint64)),                # all-equal rule
        (5, oracle.sample(3.2, 5, 5, 2, 0, 2, 333)),
    ]
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    for prec, (atol_a, atol_d) in [(0, (1e-10, 1e-12)), (1, (1e-6, 1e-6))]:
        for xmin, x in sets:  # back-to-back calls sharing the fixed scratch
            xt = torch.tensor(x.astype(np.int32), device="cuda")
            pl.pl_fit_ks_noalloc(xt, xmin, math.nan, out, prec)
            torch.cuda.synchronize()
            a_ref = ctx.pl_fit_mle(xt, xmin)
            d_ref = ctx.pl_ks_stat(xt, xmin, a_ref, prec)
            got = out.cpu().numpy()
            assert abs(got[0] / a_ref - 1) < 1e-10
            assert abs(got[1] - d_ref) < atol_d
            # D at a given exponent
            pl.pl_fit_ks_noalloc(xt, xmin, 2.2, out, prec)
            torch.cuda.synchronize()
            assert abs(out[1].item() - ctx.pl_ks_stat(xt, xmin, 2.2, prec)) < atol_d
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(pl):
    x = torch.ones(262145, dtype=torch.int32, device="cuda")
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(pl.PLError) as e:
        pl.pl_fit_ks_noalloc(x, 1, math.nan, out)
    assert e.value.status == pl.PL_EINVAL
