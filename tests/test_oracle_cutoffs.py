"""Pins for the oracle's cutoffs (order statistics of simulated D) and the
bootstrap p-value.

* Index rule: the 0-based index floor(R*q) equals the integer forms
  R*9/10, R*95/100, R*99/100, R*999/1000 the paper's code reads.
* Table 1 cells: simulated cutoffs agree with the printed values within the
  Monte Carlo uncertainty of an order statistic (distribution-free binomial
  interval of the rank) plus the 4-decimal rounding.
* The atom: at alpha = 3.5, n = 10 the 90% cutoff is exactly D of the
  all-ones sample (Table 1 prints .0819).
* Bootstrap p: uniform under the null; near 0 for lognormal data.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1305_6738_gb300 import inputs


@pytest.mark.parametrize("R", [10_000, 50_000, 100_000, 12_345, 1, 7])
def test_quantile_index_rule(R):
    assert oracle.quantile_index(R, 0.90) == min(R * 9 // 10, R - 1)
    assert oracle.quantile_index(R, 0.95) == min(R * 95 // 100, R - 1)
    assert oracle.quantile_index(R, 0.99) == min(R * 99 // 100, R - 1)
    assert oracle.quantile_index(R, 0.999) == min(R * 999 // 1000, R - 1)


def test_quantiles_are_order_statistics():
    rng = np.random.default_rng(1)
    D = rng.random(1001)
    q = [0.5, 0.9, 0.95, 0.99]
    s = np.sort(D)
    assert list(oracle.quantiles(D, q)) == [s[int(1001 * v)] for v in q]


def _rank_interval(R, q, z=4.0):
    i = oracle.quantile_index(R, q)
    h = z * math.sqrt(R * q * (1 - q))
    return max(0, int(i - h)), min(R - 1, int(math.ceil(i + h)))


@pytest.mark.parametrize("alpha,n", [(2.5, 100), (2.0, 100), (3.0, 50), (1.75, 20), (2.0, 500)])
def test_cutoffs_match_table1(table1, alpha, n):
    R = 20_000
    D, A, nc = oracle.cell(alpha, 1, n, R, seed=1, cell_id=0)
    assert nc == 0
    s = np.sort(D)
    for col, q in enumerate([0.90, 0.95, 0.99]):
        lo, hi = _rank_interval(R, q)
        printed = table1[(alpha, n)][col]
        assert s[lo] - 5e-5 <= printed <= s[hi] + 5e-5, (alpha, n, q, s[lo], printed, s[hi])


def test_atom_cutoff_alpha35_n10(table1):
    R = 10_000
    D, A, _ = oracle.cell(3.5, 1, 10, R, seed=1, cell_id=60)
    atom = oracle.ks(np.ones(10, dtype=np.uint64), 1, oracle.mle(np.ones(10, dtype=np.uint64), 1))
    cut = oracle.quantiles(D, [0.9])[0]
    assert cut == atom
    assert round(cut, 4) == table1[(3.5, 10)][0]
    # the atom's mass is the all-ones probability zeta(3.5)^-10
    frac = float((D == atom).mean())
    p = oracle.hurwitz(3.5, 1.0) ** -10
    assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / R)


def test_bootstrap_p_uniform_under_null():
    # requests drawn from the law itself: p is (discretely) uniform
    B, n = 40, 40
    ps = []
    for r in range(160):
        x = oracle.sample(2.5, 1, 99, r, 0, 2, n).astype(np.int32)
        _, _, p, _ = oracle.bootstrap_pvalue(x, 1, B, seed=3, request_id=r)
        ps.append(p)
    ps = np.array(ps)
    counts = np.histogram(ps, bins=[0, 0.2, 0.4, 0.6, 0.8, 1.0001])[0]
    exp = len(ps) / 5
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 4 + 6 * math.sqrt(8), counts


def test_bootstrap_p_small_for_lognormal():
    x = inputs.rounded_lognormal(np.random.default_rng(4), 10_000, mu=2.0, sigma=1.0, xmin=1)
    a, D, p, Db = oracle.bootstrap_pvalue(x, 1, 20, seed=3, request_id=0)
    assert p == 0.0
    assert D > Db.max()


def test_bootstrap_ties_count_as_exceeding():
    # all-ones data at n = 10: the observed D is the atom; replicates that are
    # all ones reproduce it exactly and count toward p
    x = np.ones(10, dtype=np.int32)
    a, D, p, Db = oracle.bootstrap_pvalue(x, 1, 400, seed=5, request_id=1)
    assert (Db == D).sum() > 0
    assert p == pytest.approx(float((Db >= D).mean()))
    assert p >= float((Db == D).mean())
