"""Pins for the oracle's law, survival function and inverse-CDF sampler.

The law is Eq. 1 of the paper generalised to a lower end xmin,
p(k) = k^-alpha / zeta(alpha, xmin).  Checks: the pmf sums to one, the
survival function agrees with an mpmath partial sum, the inverse CDF equals a
brute-force linear search over the cumulative pmf (the paper's own sampler,
Section 4) on small cases, and a chi-square test of sampled frequencies.
"""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("alpha,xmin", [(1.5, 1), (2.0, 1), (2.5, 1), (3.5, 1), (1.6, 2), (3.2, 5)])
def test_pmf_sums_to_one(alpha, xmin):
    Z = oracle.hurwitz(alpha, float(xmin))
    for K in [xmin, xmin + 10, xmin + 1000, xmin + 100000]:
        k = np.arange(xmin, K + 1, dtype=np.float64)
        partial = math.fsum(k ** (-alpha)) / Z
        tail = oracle.survival(alpha, xmin, K, Z)
        assert abs(partial + tail - 1.0) < 1e-14


def test_survival_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for alpha, xmin in [(1.5, 1), (2.5, 1), (3.2, 5)]:
        Z = mpmath.zeta(alpha, xmin)
        for k in [xmin - 1, xmin, xmin + 1, xmin + 30, 10 ** 6, 10 ** 12]:
            ref = 1 - mpmath.fsum(mpmath.mpf(j) ** (-alpha) for j in range(xmin, k + 1)) / Z \
                if k < xmin + 40 else mpmath.zeta(alpha, k + 1) / Z
            got = oracle.survival(alpha, xmin, k)
            assert got == pytest.approx(float(ref), rel=5e-15, abs=1e-300)


def _linear_search(alpha, xmin, v, kmax):
    """The paper's sampler: the smallest k whose cumulative probability reaches v,
    evaluated with exact rationals of the mpmath pmf (no survival function)."""
    import mpmath
    Z = mpmath.zeta(alpha, xmin)
    c = mpmath.mpf(0)
    for k in range(xmin, kmax):
        c += mpmath.mpf(k) ** (-alpha) / Z
        # X = min{k : Q(k) < v} = min{k : 1 - C(k) < v}
        if 1 - c < v:
            return k
    return None


def test_inverse_cdf_matches_linear_search():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(11)
    for alpha, xmin in [(2.5, 1), (1.75, 1), (3.0, 2)]:
        Z = oracle.hurwitz(alpha, float(xmin))
        ms = [2 ** 53, 2 ** 53 - 1, 1 + 2 ** 52] + [int(v) for v in rng.integers(2 ** 40, 2 ** 53, 40)]
        for m in ms:
            v = mpmath.mpf(m) / mpmath.mpf(2) ** 53
            ref = _linear_search(alpha, xmin, v, 5000)
            if ref is None:
                continue
            assert oracle.invert(alpha, xmin, m, Z) == ref, (alpha, xmin, m)


def test_inverse_cdf_edges():
    Z = oracle.hurwitz(2.5, 1.0)
    assert oracle.invert(2.5, 1, 2 ** 53, Z) == 1         # v = 1 -> xmin
    big = oracle.invert(1.5, 1, 1, oracle.hurwitz(1.5, 1.0))  # v = 2^-53
    assert big == oracle.XCAP                              # ~1e31 > 2^62 -> saturates
    x = oracle.invert(2.5, 1, 1, Z)                        # v = 2^-53 at alpha 2.5
    # Q(x) < v <= Q(x-1)
    v = 2.0 ** -53
    assert oracle.survival(2.5, 1, x, Z) < v <= oracle.survival(2.5, 1, x - 1, Z)
    # monotone: larger uniform -> smaller value
    ms = sorted(int(m) for m in np.random.default_rng(3).integers(1, 2 ** 53, 200))
    xs = [oracle.invert(2.0, 1, m, oracle.hurwitz(2.0, 1.0)) for m in ms]
    assert all(a >= b for a, b in zip(xs, xs[1:]))


@pytest.mark.parametrize("alpha,xmin", [(1.5, 1), (2.5, 1), (3.5, 1), (2.0, 5)])
def test_sampler_chi_square(alpha, xmin):
    n = 400_000
    reps = 8
    x = np.concatenate([oracle.sample(alpha, xmin, 1234, 3, r, 2, n // reps) for r in range(reps)])
    assert x.min() >= xmin
    Z = oracle.hurwitz(alpha, float(xmin))
    # bins: single values while expected >= 50, then one pooled tail bin
    edges = []
    k = xmin
    while True:
        e = n * oracle.pmf(alpha, xmin, k)
        if e < 50:
            break
        edges.append(k)
        k += 1
    obs = [int((x == k).sum()) for k in edges]
    exp = [n * oracle.pmf(alpha, xmin, k) for k in edges]
    obs.append(int((x > edges[-1]).sum()))
    exp.append(n * oracle.survival(alpha, xmin, edges[-1], Z))
    obs = np.array(obs, float)
    exp = np.array(exp)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    dof = len(obs) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)
    # heavy tail: fraction above 1000 matches Q(1000)
    q = oracle.survival(alpha, xmin, 1000, Z)
    frac = (x > 1000).mean()
    assert abs(frac - q) < 6 * math.sqrt(q * (1 - q) / n) + 1e-9
