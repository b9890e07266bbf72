"""The serving engine (pl_server_*) through the C ABI: every request's
result in a mix of concurrent requests equals, bit for bit, the result of the
same request run alone through pl_bootstrap_pvalue on a fresh context; a
request with bad data fails alone; work of different requests overlaps on the
GPU; the device budget is respected."""
import numpy as np
import pytest

from paper_1305_6738_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

B = 400
SEED = 11


@pytest.fixture(scope="module")
def pl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_6738_gb300 import build
    build.build()
    from paper_1305_6738_gb300 import pl as _pl
    return _pl


def _power_law(pl, ctx, alpha, n, rid):
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    ctx.pl_sample(alpha, 1, 4, rid, inputs.PURPOSE_TESTDATA, 0, 1, n, out)
    ctx.pl_sync()
    return inputs.as_request_data(out.cpu().numpy())


def _mix(pl, ctx):
    rng = np.random.default_rng(5)
    reqs = []
    # two large requests first (block form for n above the split), then a spread of sizes
    for rid, (alpha, n) in enumerate([(2.2, 150_000), (1.8, 100_000), (2.5, 50), (3.1, 700),
                                      (1.6, 5000), (2.0, 20_000), (2.9, 123), (1.5, 3000),
                                      (2.4, 40_000), (3.4, 64)]):
        reqs.append((rid, _power_law(pl, ctx, alpha, n, rid)))
    reqs.append((10, inputs.rounded_lognormal(rng, 8000)))
    reqs.append((11, inputs.rounded_lognormal(rng, 77)))
    bad = _power_law(pl, ctx, 2.5, 500, 12)
    bad[17] = 0  # below xmin = 1
    reqs.append((12, bad))
    return reqs


def _drain(srv, count, budget=None, timeout_s=120.0):
    got = {}
    t_end = srv.pl_server_now() + timeout_s
    while len(got) < count and srv.pl_server_now() < t_end:
        for r in srv.pl_server_poll(64, 0.05):
            got[r["request_id"]] = r
        if budget is not None:
            assert srv.pl_server_load()[2] <= budget
    assert len(got) == count
    return got


@pytest.mark.parametrize("prec", [0, 1])
def test_server_mix_equals_alone(pl, prec):
    ctx = pl.Context(0)
    reqs = _mix(pl, ctx)
    budget = 8 << 30
    srv = pl.Server(0, budget, workers=3, prec=prec, seed=SEED, B=B)
    for rid, x in reqs:
        srv.pl_server_submit(rid, x, 1)
    got = _drain(srv, len(reqs), budget)
    srv.close()
    for rid, x in reqs:
        r = got[rid]
        assert r["n"] == x.size
        assert r["submit_s"] <= r["start_s"] <= r["done_s"]
        if rid == 12:
            assert r["status"] == pl.PL_EINVAL
            continue
        assert r["status"] == pl.PL_OK, rid
        alone = pl.Context(0)  # fresh context: no cached fit tables, no earlier workspace
        a, d, p = alone.pl_bootstrap_pvalue(torch.tensor(x, device="cuda"), 1, B, SEED, rid, prec)
        alone.close()
        assert (r["alpha_hat"], r["D"], r["p"]) == (a, d, p), rid
    # the two large requests, submitted together to idle workers, ran at the same time
    r0, r1 = got[0], got[1]
    assert r0["start_s"] < r1["done_s"] and r1["start_s"] < r0["done_s"]
    # lognormal data are rejected at this size
    assert got[10]["p"] == 0.0
    ctx.close()


def test_server_budget_and_errors(pl):
    srv = pl.Server(0, 1 << 20, workers=2, prec=1, seed=1, B=64)  # 1 MiB: nothing fits
    x = np.full(1000, 3, dtype=np.int32)
    srv.pl_server_submit(7, x, 1)
    srv.pl_server_submit(8, x[:10], 1)
    got = _drain(srv, 2, 1 << 20)
    assert got[7]["status"] == pl.PL_ENOMEM and got[8]["status"] == pl.PL_ENOMEM
    with pytest.raises(pl.PLError):
        srv.pl_server_submit(2**32, x, 1)  # request ids key 32-bit streams
    with pytest.raises(pl.PLError):
        srv.pl_server_submit(9, x, 0)
    srv.close()
