"""Pins for the oracle's lower-end estimate by KS minimisation (the procedure
of Clauset, Shalizi & Newman that the paper's tables are used with,
Section 3).

* Each candidate's fit and D equal the pinned single-data-set routines on
  the tail: D against the brute force over every integer, the fit against
  the log-likelihood grid argmax.
* A planted lower end: a flat body below x0 and a power law from x0 give an
  estimate at or a few values above x0 (never below: the body's mass would
  raise D) with the tail exponent within 0.05; a pure power law from 1 gives
  an estimate near 1.
* Candidates with a short tail are skipped; the estimate is the argmin.
"""
import math

import numpy as np
import pytest

import oracle


def _planted(x0, alpha, seed, n_tail=20000, n_body=10000):
    rng = np.random.default_rng(seed)
    tail = oracle.sample(alpha, x0, 11 + seed, x0, 0, 2, n_tail)
    body = rng.integers(1, x0, n_body).astype(np.uint64)
    return np.concatenate([body, tail])


@pytest.mark.parametrize("x0,alpha,seed", [(10, 2.5, 0), (5, 2.0, 1), (20, 3.0, 2)])
def test_planted_lower_end_is_found(x0, alpha, seed):
    x = _planted(x0, alpha, seed)
    b, xm, a, d, nt = oracle.estimate_xmin(x, 200, 10)
    assert x0 <= xm[b] <= x0 + 8
    assert abs(a[b] - alpha) < 0.05
    assert d[b] == np.nanmin(d)


def test_pure_power_law_estimate_is_low():
    x = oracle.sample(2.5, 1, 5, 0, 0, 2, 20000)
    b, xm, a, d, nt = oracle.estimate_xmin(x, 200, 10)
    assert xm[b] <= 3 and abs(a[b] - 2.5) < 0.05


def test_candidates_match_single_data_set_routines():
    x = oracle.sample(2.2, 1, 9, 1, 0, 2, 400)
    b, xm, a, d, nt = oracle.estimate_xmin(x, 12, 5)
    assert list(xm) == sorted(set(int(v) for v in x))[:12]
    for j in range(len(xm)):
        tail = x[x >= xm[j]]
        assert nt[j] == tail.size
        if tail.size < 5:
            assert math.isnan(d[j])
            continue
        assert d[j] == pytest.approx(oracle.ks(tail, int(xm[j]), a[j], brute=True), abs=1e-14)
        # the fit maximises the log-likelihood of the tail (grid around it)
        L = oracle.log_sum(tail, int(xm[j]))
        ll = lambda s: -s * L - tail.size * math.log(oracle.hurwitz(s, float(xm[j])))  # noqa: E731
        assert ll(a[j]) >= max(ll(a[j] - 1e-3), ll(a[j] + 1e-3))


def test_short_tails_are_skipped():
    x = np.array([1, 1, 2, 3, 3, 3, 50], dtype=np.uint64)
    b, xm, a, d, nt = oracle.estimate_xmin(x, 10, 3)
    assert list(nt) == [7, 5, 4, 1]
    assert math.isnan(d[3]) and not math.isnan(d[2])
    assert b == int(np.nanargmin(d))
