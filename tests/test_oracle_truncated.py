"""Pins for the oracle's truncated Zipf law (support 1..K, Section 1's second
version) and its cutoffs (Tables 2-6).

* The scaling factor zeta_K(gamma): K at gamma = 0, the harmonic number at
  gamma = 1, the generalised harmonic number zeta(s) - zeta(s, K+1) (SciPy /
  mpmath) elsewhere; the survival runs from 1 to 0.
* Draws: the inverse CDF against a linear search of the CDF, and a
  chi-square test of the draws against p(k).
* MLE: uniform data give gamma-hat = 0; the estimate is the argmax of the
  log-likelihood on a grid; E[ln X] at the estimate equals the sample mean log.
* D: brute force over every t against the definition with a sorted sample.
* Tables 2-6: simulated cutoffs within the order statistic's Monte Carlo
  interval of the printed values; the K = 20, gamma = 4, N = 10 atom.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tables2to6_truncated.txt")


def load_tables():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            K, g, n, *q = line.split()
            out[(int(K), float(g), int(n))] = tuple(float(v) for v in q)
    return out


def test_golden_tables_complete():
    t = load_tables()
    assert len(t) == 5 * 12 * 15
    assert t[(20, 1.0, 100)] == (0.0671, 0.0742, 0.0886, 0.1059)


@pytest.mark.parametrize("K", [2, 20, 1000])
def test_scaling_factor_closed_forms(K):
    _, z0 = oracle.tz_survival(1e-300, K)
    assert z0 == pytest.approx(K, rel=1e-14)
    _, z1 = oracle.tz_survival(1.0, K)
    assert z1 == pytest.approx(sum(1.0 / k for k in range(1, K + 1)), rel=1e-14)
    special = pytest.importorskip("scipy.special")
    _, z2 = oracle.tz_survival(2.0, K)
    assert z2 == pytest.approx(math.pi ** 2 / 6 - special.polygamma(1, K + 1), rel=1e-13)
    mpmath = pytest.importorskip("mpmath")
    _, zh = oracle.tz_survival(0.5, K)
    assert zh == pytest.approx(float(mpmath.zeta(0.5) - mpmath.zeta(0.5, K + 1)), rel=1e-12)


def test_survival_runs_from_one_to_zero():
    Q, z = oracle.tz_survival(0.75, 50)
    assert Q[0] == pytest.approx(1.0, abs=1e-15) and Q[50] == 0.0
    assert np.all(np.diff(Q) < 0)
    p = np.arange(1, 51, dtype=float) ** -0.75 / z
    assert np.allclose(-np.diff(Q), p, rtol=1e-13, atol=1e-16)


def test_inverse_cdf_matches_linear_search():
    K, g = 37, 1.3
    Q, _ = oracle.tz_survival(g, K)
    rng = np.random.default_rng(2)
    for m in list(rng.integers(1, 2 ** 53, 2000)) + [1, 2 ** 53]:
        v = math.ldexp(float(m), -53)
        lin = next(k for k in range(1, K + 1) if Q[k] < v)
        assert oracle.tz_invert(Q, K, int(m)) == lin


def test_draws_chi_square():
    stats = pytest.importorskip("scipy.stats")
    K, g, n = 20, 1.0, 200_000
    x = oracle.tz_sample(g, K, 7, 3, 0, 2, n)
    assert x.min() >= 1 and x.max() <= K
    cnt = np.bincount(x.astype(np.int64), minlength=K + 1)[1:]
    Q, z = oracle.tz_survival(g, K)
    exp = n * np.arange(1, K + 1, dtype=float) ** -g / z
    chi2 = float(((cnt - exp) ** 2 / exp).sum())
    assert stats.chi2.sf(chi2, K - 1) > 1e-4


def test_mle_uniform_data_gives_zero():
    for K in (5, 20, 100):
        assert abs(oracle.tz_mle(np.arange(1, K + 1, dtype=np.uint64), K)) < 1e-12


@pytest.mark.parametrize("x,K", [([1, 1, 2, 5], 10), ([3, 7, 7, 20, 1, 2], 20), ([50, 49, 1], 50)])
def test_mle_is_loglikelihood_argmax(x, K):
    x = np.array(x, dtype=np.uint64)
    g = oracle.tz_mle(x, K)
    L = float(np.log(x.astype(float)).sum())
    ks = np.arange(1, K + 1, dtype=float)

    def ll(gg):
        return -gg * L - len(x) * math.log(float((ks ** -gg).sum()))
    grid = np.arange(g - 0.5, g + 0.5, 1e-4)
    best = grid[int(np.argmax([ll(v) for v in grid]))]
    assert abs(best - g) <= 1e-4
    w = ks ** -g
    assert float((np.log(ks) * w).sum() / w.sum()) == pytest.approx(L / len(x), rel=1e-12)


def test_ks_definition():
    K, g = 30, 0.9
    x = np.array([1, 1, 2, 3, 3, 3, 9, 17, 30, 4], dtype=np.uint64)
    Q, z = oracle.tz_survival(g, K)
    s = np.sort(x.astype(np.int64))
    best = 0.0
    for t in range(1, K + 1):
        S = np.searchsorted(s, t, side="right") / len(s)
        best = max(best, abs((1.0 - Q[t]) - S))
    assert oracle.tz_ks(x, K, g) == pytest.approx(best, abs=1e-15)


def _rank_interval(R, q, z=4.0):
    i = oracle.quantile_index(R, q)
    h = z * math.sqrt(R * q * (1 - q))
    return max(0, int(i - h)), min(R - 1, int(math.ceil(i + h)))


@pytest.mark.parametrize("K,g,n", [(20, 0.25, 10), (20, 1.0, 100), (50, 0.5, 50), (100, 2.0, 100),
                                   (500, 1.5, 30), (1000, 3.0, 20)])
def test_cutoffs_match_tables(K, g, n):
    tables = load_tables()
    R = 20_000
    D, A, nc = oracle.tz_cell(g, K, n, R, seed=1, cell_id=0)
    assert nc == 0
    s = np.sort(D)
    for col, q in enumerate([0.90, 0.95, 0.99]):
        lo, hi = _rank_interval(R, q)
        printed = tables[(K, g, n)][col]
        assert s[lo] - 5e-5 <= printed <= s[hi] + 5e-5, (K, g, n, q, s[lo], printed, s[hi])


def test_atom_k20_gamma4_n10():
    # all-ones samples (probability ~0.87^10 = 0.25 at gamma = 4) give one D
    # value; Table 2 prints .0821 at q = 0.9 and 0.95
    ones = np.ones(10, dtype=np.uint64)
    atom = oracle.tz_ks(ones, 20, oracle.tz_mle(ones, 20))
    assert round(atom, 4) == 0.0821
    D, _, _ = oracle.tz_cell(4.0, 20, 10, 10_000, seed=1, cell_id=5)
    assert oracle.quantiles(D, [0.9])[0] == atom


@pytest.mark.parametrize("K", [2, 20, 1000])
def test_negative_exponents(K):
    """On a finite support the law is defined for every real exponent (the
    fitted exponent of a small sample can be negative): zeta_K(-1) and
    zeta_K(-2) are the sums of k and k^2, and draws at gamma = -1 follow
    p(k) = 2k / (K(K+1))."""
    _, z1 = oracle.tz_survival(-1.0, K)
    assert z1 == pytest.approx(K * (K + 1) / 2, rel=1e-14)
    _, z2 = oracle.tz_survival(-2.0, K)
    assert z2 == pytest.approx(K * (K + 1) * (2 * K + 1) / 6, rel=1e-14)
    D, G, nc = oracle.tz_cell(-1.5, K, 50, 20, seed=1, cell_id=3)
    assert nc == 0 and np.all(np.isfinite(D))


def test_draws_at_negative_exponent_chi_square():
    stats = pytest.importorskip("scipy.stats")
    K, n = 12, 120_000
    x = oracle.tz_sample(-1.0, K, 5, 1, 0, 1, n).astype(np.int64)
    cnt = np.bincount(x, minlength=K + 1)[1:]
    p = np.arange(1, K + 1) / (K * (K + 1) / 2)
    chi2 = ((cnt - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, K - 1) > 1e-4
