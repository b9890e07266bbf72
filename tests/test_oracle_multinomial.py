"""Pins for the oracle's multinomial histogram sampler (a large-n variant:
bin counts by conditional binomials, the tail value by value).

* The binomial probabilities against SciPy's.
* The binomial sampler is an inversion along a fixed order of the outcomes,
  so a stratified grid of N uniforms gives every outcome N P(k) times to
  within one: checked against SciPy's pmf on both branches (from 0 and from
  the mode), including p near 0 and near 1 and a mode (n+1) p that is an
  integer (p = 64/113, n = 112).
* The thresholds realise the inverse-CDF test: X(T[i]) <= xmin + i < X(T[i] - 1).
* A replicate has n values >= xmin; pooled bin counts follow p(k) (chi-square);
  the distribution of D equals the inverse-CDF sampler's (two-sample KS test),
  which is what makes the sampler a drop-in for the cutoff simulation.
"""
import numpy as np
import pytest

import oracle

stats = pytest.importorskip("scipy.stats")


@pytest.mark.parametrize("n,p", [(10, 0.3), (1000, 0.5), (10**6, 0.6), (50, 0.999), (10**5, 1e-4),
                                 (40, 0.7), (7, 0.02)])
def test_binomial_pmf_against_scipy(n, p):
    mean = n * p
    for x in {0, 1, int(mean), int(mean) + 3, max(int(mean) - 5, 0), n - 1, n}:
        ref = stats.binom.pmf(x, n, p)
        if ref > 1e-200:
            assert oracle.binom_pmf(x, n, p) == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("n,num,den,N", [(10, 3, 10, 20000), (40, 7, 10, 20000), (1000, 1, 2, 20000),
                                         (10**6, 3, 5, 4000), (10**5, 1, 10000, 20000), (50, 999, 1000, 20000),
                                         (7, 1, 50, 20000), (112, 64, 113, 20000)])
def test_binomial_sampler_is_an_inversion(n, num, den, N):
    p = num / den
    counts = {}
    for i in range(N):
        k = oracle.binomial(n, num, den, (i + 0.5) / N)
        assert 0 <= k <= n
        counts[k] = counts.get(k, 0) + 1
    for k, c in counts.items():
        assert abs(c - N * stats.binom.pmf(k, n, p)) <= 1.0 + 1e-9 * N, (k, c, N * stats.binom.pmf(k, n, p))
    # every outcome with N P(k) >= 2 appears
    lo, hi = stats.binom.ppf(1e-6, n, p), stats.binom.ppf(1 - 1e-6, n, p)
    for k in range(int(lo), int(hi) + 1):
        if N * stats.binom.pmf(k, n, p) >= 2:
            assert k in counts


def test_thresholds_realise_the_inverse_cdf():
    alpha, xmin = 2.3, 2
    T = oracle.thresholds(alpha, xmin, 64)
    assert np.all(np.diff(T.astype(np.float64)) <= 0) and T[0] <= 2**53
    for i in range(0, 64, 7):
        assert oracle.invert(alpha, xmin, int(T[i])) <= xmin + i
        assert oracle.invert(alpha, xmin, int(T[i]) - 1) > xmin + i


@pytest.mark.parametrize("alpha,xmin,n", [(2.5, 1, 1), (2.5, 1, 2), (2.0, 1, 5000), (1.5, 3, 3000), (3.5, 1, 200)])
def test_replicate_has_n_values_of_the_law(alpha, xmin, n):
    x = oracle.mn_sample(alpha, xmin, 1, 2, 3, oracle.PURPOSE_MULTINOMIAL, n)
    assert x.size == n and x.min() >= xmin


def test_pooled_bins_follow_the_law():
    alpha, n, R = 2.0, 3000, 200
    T = oracle.thresholds(alpha, 1)
    cnt = np.zeros(12)
    for r in range(R):
        x = oracle.mn_sample(alpha, 1, 7, 0, r, oracle.PURPOSE_MULTINOMIAL, n, T)
        b = np.minimum(x, 12).astype(np.int64) - 1
        cnt += np.bincount(b, minlength=12)
    p = np.array([oracle.pmf(alpha, 1, k) for k in range(1, 12)])
    p = np.append(p, oracle.survival(alpha, 1, 11))
    chi2 = ((cnt - n * R * p) ** 2 / (n * R * p)).sum()
    assert stats.chi2.sf(chi2, 11) > 1e-4


@pytest.mark.parametrize("alpha,n", [(2.5, 500), (1.75, 2000)])
def test_D_distribution_matches_the_inverse_cdf_sampler(alpha, n):
    R = 1500
    D_mn, A_mn, _ = oracle.mn_cell(alpha, 1, n, R, seed=3, cell_id=1)
    D_ic, A_ic, _ = oracle.cell(alpha, 1, n, R, seed=3, cell_id=1)
    assert stats.ks_2samp(D_mn, D_ic).pvalue > 1e-3
    assert stats.ks_2samp(A_mn, A_ic).pvalue > 1e-3
