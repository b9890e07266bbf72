"""GPU parity of the lower-end estimate by KS minimisation against the
oracle: every candidate's x_min and tail size exactly, its alpha-hat within
1e-10 relative and D within 1e-12, and the chosen candidate (the same one,
or one whose D ties the oracle's minimum within 1e-12)."""
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


@pytest.fixture(scope="module")
def ctx(pl):
    c = pl.Context(0)
    yield c
    c.close()


def _planted(x0, alpha, seed, n_tail, n_body):
    rng = np.random.default_rng(seed)
    tail = oracle.sample(alpha, x0, 11 + seed, x0, 0, 2, n_tail)
    body = rng.integers(1, x0, n_body).astype(np.uint64)
    return np.concatenate([body, tail])


def _sets():
    return [
        (_planted(10, 2.5, 0, 20000, 10000), 200, 10),
        (oracle.sample(2.5, 1, 5, 0, 0, 2, 20000), 100, 10),
        (np.minimum(oracle.sample(1.5, 3, 6, 1, 0, 2, 50000), 2**31 - 1), 300, 20),  # values beyond the shared bins
        (np.array([1, 1, 2, 3, 3, 3, 50], dtype=np.uint64), 10, 3),
        (np.full(40, 7, dtype=np.uint64), 5, 1),                                   # one value: all-equal rule
    ]


@pytest.mark.parametrize("k", range(5))
def test_estimate_xmin_matches_oracle(ctx, k):
    x, mc, mt = _sets()[k]
    xt = torch.tensor(x.astype(np.int64).astype(np.int32), device="cuda")
    cx = torch.zeros(mc, dtype=torch.int64, device="cuda")
    ca = torch.zeros(mc, dtype=torch.float64, device="cuda")
    cd = torch.zeros(mc, dtype=torch.float64, device="cuda")
    cn = torch.zeros(mc, dtype=torch.int64, device="cuda")
    r = ctx.pl_estimate_xmin(xt, mc, mt, cx, ca, cd, cn)
    b, xm, a, d, nt = oracle.estimate_xmin(x, mc, mt)
    m = len(xm)
    assert r["candidates"] == m
    gx, ga, gd, gn = (t.cpu().numpy()[:m] for t in (cx, ca, cd, cn))
    assert np.array_equal(gx.astype(np.uint64), xm)
    assert np.array_equal(gn, nt)
    nan = np.isnan(d)
    assert np.array_equal(np.isnan(gd), nan)
    ok = ~nan
    assert np.max(np.abs(ga[ok] / a[ok] - 1), initial=0) < 1e-10
    assert np.max(np.abs(gd[ok] - d[ok]), initial=0) < 1e-12
    if b < 0:
        assert r["xmin"] == 0 and math.isnan(r["D"])
    else:
        assert abs(r["D"] - d[b]) < 1e-12
        assert r["xmin"] == xm[b] or abs(d[list(xm).index(r["xmin"])] - d[b]) < 1e-12
        assert r["n_tail"] == nt[list(xm).index(r["xmin"])]


def test_estimate_xmin_rejects_bad_values(ctx, pl):
    xt = torch.tensor([3, 1, 0, 2], dtype=torch.int32, device="cuda")
    with pytest.raises(pl.PLError) as e:
        ctx.pl_estimate_xmin(xt, 10, 1)
    assert e.value.status == pl.PL_EINVAL
