"""The allocation-free entry point, for callers that cannot let a library call
cudaMalloc (a runtime that owns all device memory through its own pool, or a
loop that must never reach the allocator).  Through the C ABI, several calls
in a row share the library's fixed scratch, which keeps the previous call's
contents: every call is checked against the CPU oracle (fit, D and
zeta(alpha, xmin)) and against the context-based entry points, a call with
bad data (NaN outputs) is followed by good calls, the largest accepted sample
(every value beyond the on-chip bins) runs, and the device's free memory does
not change across the calls.  Collected last (file name) so that a failure
here stops a -x run only after every other test has run."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {0: (1e-10, 1e-12), 1: (1e-6, 1e-6)}  # (alpha-hat relative, D absolute) per precision form


@pytest.fixture(scope="module")
def pl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_6738_gb300 import build
    build.build()
    from paper_1305_6738_gb300 import pl as _pl
    return _pl


def _sets():
    rng = np.random.default_rng(31)
    big = (1 + 8192 + rng.integers(0, 1 << 20, 262144)).astype(np.uint64)  # n at the limit, all beyond the bins
    return [
        (1, oracle.sample(1.5, 1, 5, 1, 0, 2, 20000)),   # values beyond the on-chip bins
        (1, oracle.sample(2.5, 1, 5, 0, 0, 2, 1000)),
        (1, np.ones(20, dtype=np.uint64)),                # all-equal rule
        (5, oracle.sample(3.2, 5, 5, 2, 0, 2, 333)),
        (1, big),
    ]


def _check(pl, ctx, out, x, xmin, prec):
    """One fitted call and one call at a given exponent against the oracle and
    the context entry points."""
    atol_a, atol_d = TOL[prec]
    xu = x.astype(np.uint64)
    xt = torch.tensor(x.astype(np.int32), device="cuda")
    pl.pl_fit_ks_noalloc(xt, xmin, math.nan, out, prec)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    a_or = oracle.mle(xu, xmin)
    assert abs(got[0] / a_or - 1) < atol_a
    assert abs(got[1] - oracle.ks(xu, xmin, got[0])) < atol_d
    assert abs(got[2] / oracle.hurwitz(got[0], xmin) - 1) < 1e-12
    a_ref = ctx.pl_fit_mle(xt, xmin)
    assert abs(got[0] / a_ref - 1) < 1e-10
    assert abs(got[1] - ctx.pl_ks_stat(xt, xmin, a_ref, prec)) < atol_d
    pl.pl_fit_ks_noalloc(xt, xmin, 2.2, out, prec)  # D at a given exponent
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[0] == 2.2
    assert abs(got[1] - oracle.ks(xu, xmin, 2.2)) < atol_d
    assert abs(got[2] / oracle.hurwitz(2.2, xmin) - 1) < 1e-12


def test_noalloc_matches_oracle_and_context_calls_in_a_row(pl):
    ctx = pl.Context(0)
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    for prec in (0, 1):
        for xmin, x in _sets():  # back-to-back calls sharing the fixed scratch
            _check(pl, ctx, out, x, xmin, prec)
    ctx.close()


def test_noalloc_bad_data_then_good_data(pl):
    ctx = pl.Context(0)
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    bad = torch.tensor([3, 4, 1, 7], dtype=torch.int32, device="cuda")  # a value below xmin = 2
    pl.pl_fit_ks_noalloc(bad, 2, math.nan, out)
    torch.cuda.synchronize()
    assert np.isnan(out.cpu().numpy()).all()
    xmin, x = _sets()[1]
    _check(pl, ctx, out, x, xmin, 0)  # the latched error of the bad call does not leak into this one
    _check(pl, ctx, out, x, xmin, 0)
    ctx.close()


def test_noalloc_allocates_nothing(pl):
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    xmin, x = _sets()[0]
    xt = torch.tensor(x.astype(np.int32), device="cuda")
    pl.pl_fit_ks_noalloc(xt, xmin, math.nan, out)  # first call on the device: looks up the scratch address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for prec in (0, 1, 0):
        pl.pl_fit_ks_noalloc(xt, xmin, math.nan, out, prec)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_scratch(pl):
    x = torch.ones(262145, dtype=torch.int32, device="cuda")
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(pl.PLError) as e:
        pl.pl_fit_ks_noalloc(x, 1, math.nan, out)
    assert e.value.status == pl.PL_EINVAL
    with pytest.raises(ValueError):  # the binding checks the tensors it passes
        pl.pl_fit_ks_noalloc(x.cpu(), 1, math.nan, out)
