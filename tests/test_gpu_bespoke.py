"""GPU parity of the paper's procedure for one data set (Section 3): fit,
D, and the cutoff for the sample's own N and fitted exponent, simulated
("bespoke"), for the untruncated and the truncated law, plus the truncated
law's data-set fit and the lookup of tabulated cutoffs at a fitted exponent.
The oracle side composes the oracle's own fit, D and cell simulation."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {0: (1e-10, 1e-12), 1: (1e-6, 1e-6)}  # precision -> (exponent rel, D abs)


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


def _dev(x):
    return torch.tensor(np.asarray(x, dtype=np.int64).astype(np.int32), device="cuda")


# ----------------------------------------------------------------------------- truncated data sets
def _tz_sets():
    return [
        (20, oracle.tz_sample(1.0, 20, 5, 0, 0, 2, 100)),
        (1000, oracle.tz_sample(0.5, 1000, 5, 1, 0, 2, 5000)),
        (1024, oracle.tz_sample(2.0, 1024, 5, 2, 0, 2, 100000)),   # n beyond the simulation's 65,535
        (3, np.array([3, 3, 2])),                                   # negative estimate
        (50, np.ones(20, dtype=np.int64)),                           # all ones
        (2, np.array([2, 2, 2])),                                    # all K: the -64 end
    ]


@pytest.mark.parametrize("k", range(6))
@pytest.mark.parametrize("prec", [0, 1])
def test_truncated_fit_and_ks_match_oracle(ctx, k, prec):
    K, x = _tz_sets()[k]
    xu = np.asarray(x, dtype=np.uint64)
    g_or = oracle.tz_mle(xu, K)
    g, d = ctx.pl_fit_ks_truncated(_dev(x), K, prec=prec)
    assert abs(g - g_or) / max(abs(g_or), 1.0) < 1e-10, (g, g_or)
    assert abs(d - oracle.tz_ks(xu, K, g_or)) < TOL[prec][1]
    g2, d2 = ctx.pl_fit_ks_truncated(_dev(x), K, gamma=1.3, prec=prec)
    assert g2 == 1.3
    assert abs(d2 - oracle.tz_ks(xu, K, 1.3)) < TOL[prec][1]


def test_truncated_data_outside_support_rejected(ctx, pl):
    for bad in ([1, 2, 0], [1, 21, 3]):
        with pytest.raises(pl.PLError) as e:
            ctx.pl_fit_ks_truncated(_dev(bad), 20)
        assert e.value.status == pl.PL_EINVAL


# ----------------------------------------------------------------------------- bespoke cutoffs
Q = [0.9, 0.95, 0.99]


def _near_ties(Db, d, tol):
    return int(np.sum(np.abs(Db - d) <= tol))


@pytest.mark.parametrize("prec", [0, 1])
def test_bespoke_cutoffs_match_oracle(ctx, pl, prec):
    x = oracle.sample(2.2, 1, 5, 0, 0, 2, 500)
    xu = x.astype(np.uint64)
    R, seed, rid = 3000, 9, 77
    a, d, p, cut = ctx.pl_bespoke_cutoffs(_dev(x), 1, R, seed, rid, Q, prec)
    a_or = oracle.mle(xu, 1)
    d_or = oracle.ks(xu, 1, a_or)
    Db, _, _ = oracle.cell(a_or, 1, 500, R, seed=seed, cell_id=rid, purpose=1)
    assert abs(a / a_or - 1) < TOL[prec][0]
    assert abs(d - d_or) < TOL[prec][1]
    assert np.abs(cut - oracle.quantiles(Db, Q)).max() < TOL[prec][1] + 1e-15
    assert abs(p - np.mean(Db >= d_or)) <= _near_ties(Db, d_or, 2 * TOL[prec][1]) / R
    # the same simulation as the bootstrap p-value of the data set
    a2, d2, p2 = ctx.pl_bootstrap_pvalue(_dev(x), 1, R, seed, rid, prec)
    assert (a2, d2, p2) == (a, d, p)


@pytest.mark.parametrize("K,x", [
    (100, oracle.tz_sample(1.0, 100, 5, 3, 0, 2, 300)),
    (1000, oracle.tz_sample(2.5, 1000, 5, 4, 0, 2, 2000)),
    (10, np.array([10, 9, 10, 8, 10, 7, 9, 10])),                # negative estimate: simulated below 0
])
@pytest.mark.parametrize("prec", [0, 1])
def test_bespoke_cutoffs_truncated_match_oracle(ctx, K, x, prec):
    xu = np.asarray(x, dtype=np.uint64)
    n, R, seed, rid = len(x), 2000, 9, 78
    g, d, p, cut = ctx.pl_bespoke_cutoffs_truncated(_dev(x), K, R, seed, rid, Q, prec)
    g_or = oracle.tz_mle(xu, K)
    d_or = oracle.tz_ks(xu, K, g_or)
    Db, _, _ = oracle.tz_cell(g_or, K, n, R, seed=seed, cell_id=rid, purpose=1)
    assert abs(g - g_or) / max(abs(g_or), 1.0) < 1e-10
    assert abs(d - d_or) < TOL[prec][1]
    assert np.abs(cut - oracle.quantiles(Db, Q)).max() < TOL[prec][1] + 1e-15
    assert abs(p - np.mean(Db >= d_or)) <= _near_ties(Db, d_or, 2 * TOL[prec][1]) / R
    if K == 10:
        assert g < 0


def test_bespoke_rejects_invalid(ctx, pl):
    x = _dev([1, 2, 3])
    for kw in (dict(q=[1.0]), dict(q=[0.5], R=0)):
        args = dict(R=10, q=[0.9])
        args.update(kw)
        with pytest.raises(pl.PLError):
            ctx.pl_bespoke_cutoffs(x, 1, args["R"], 1, 0, args["q"])
        with pytest.raises(pl.PLError):
            ctx.pl_bespoke_cutoffs_truncated(x, 5, args["R"], 1, 0, args["q"])


# ----------------------------------------------------------------------------- table lookup
def test_cutoff_lookup_matches_oracle(ctx, pl):
    GA = [1.5, 2.0, 2.5, 3.0]
    GN = [10, 100, 1000]
    cells = [pl.Cell(a, 1, n, 2000, 10 * i + k) for i, a in enumerate(GA) for k, n in enumerate(GN)]
    table = torch.empty(len(cells) * len(Q), dtype=torch.float64, device="cuda")
    ctx.pl_ks_cutoffs(cells, 1, Q, 0, cutoffs=table)
    rng = np.random.default_rng(6)
    qa = list(rng.uniform(1.3, 3.3, 200)) + GA + [2.0, 2.25]
    qn = list(np.exp(rng.uniform(math.log(5), math.log(5000), 200)).astype(np.int64)) + [100] * 4 + [10, 31]
    qa_t = torch.tensor(qa, dtype=torch.float64, device="cuda")
    qn_t = torch.tensor(qn, dtype=torch.int64, device="cuda")
    out = torch.empty(len(qa) * len(Q), dtype=torch.float64, device="cuda")
    ctx.pl_cutoff_lookup(GA, GN, table, len(Q), qa_t, qn_t, out)
    got = out.cpu().numpy().reshape(len(qa), len(Q))
    tab = table.cpu().numpy().reshape(len(GA), len(GN), len(Q))
    for m in range(len(qa)):
        ref = oracle.cutoff_lookup(GA, GN, tab, qa[m], qn[m])
        assert np.abs(got[m] - ref).max() < 1e-14, (m, qa[m], qn[m], got[m], ref)
    # grid points give the tabulated values exactly
    for i in range(len(GA)):
        assert np.array_equal(got[200 + i], tab[i, 1])


@pytest.mark.parametrize("prec", [0, 1])
def test_bespoke_batch_equals_single_calls(ctx, pl, prec):
    specs = [(2.2, 1, 500), (1.8, 1, 3000), (2.6, 2, 50), (2.0, 1, 20000), (3.0, 1, 10), (2.4, 3, 1000)]
    xs = [_dev(oracle.sample(a, xm, 5, 10 + i, 0, 2, n)) for i, (a, xm, n) in enumerate(specs)]
    xmins = [xm for _, xm, _ in specs]
    rids = [100 + i for i in range(len(specs))]
    a, d, p, cut = ctx.pl_bespoke_cutoffs_batch(xs, xmins, 2000, 9, rids, Q, prec)
    for i in range(len(specs)):
        a1, d1, p1, c1 = ctx.pl_bespoke_cutoffs(xs[i], xmins[i], 2000, 9, rids[i], Q, prec)
        assert (a[i], d[i], p[i]) == (a1, d1, p1), i
        assert np.array_equal(cut[i], c1), i


def test_bespoke_batch_rejects_bad_data(ctx, pl):
    xs = [_dev([1, 2, 3]), _dev([3, 0, 2])]
    with pytest.raises(pl.PLError) as e:
        ctx.pl_bespoke_cutoffs_batch(xs, [1, 1], 100, 1, [0, 1], Q)
    assert e.value.status == pl.PL_EINVAL
