"""Pins for the oracle's maximum-likelihood fit (Eq. 2) and KS distance (Eq. 3).

* The MLE equals the argmax of the log-likelihood
  l(alpha) = -alpha * sum ln x_i - n ln zeta(alpha, xmin), found by a grid
  search plus golden-section refinement over SciPy's Hurwitz zeta.
* The MLE equals an mpmath root of zeta'/zeta + mean(ln x) at 40 digits.
* The all-ones samples at n = 10 and n = 20 give D equal to the exact atoms
  Table 1 prints (.0819 at gamma = 3.5/4.0, N = 10; .0440 at gamma = 4,
  N = 20), which pins the all-ones rule and the untruncated normaliser.
* D over distinct values equals the brute-force maximum over every integer.
* For n <= 4 the oracle's Monte Carlo distribution of D matches the exact
  distribution obtained by enumerating every multiset of small values.
"""
import itertools
import math

import numpy as np
import pytest

import oracle


def _loglik(sp, alpha, L, n, xmin):
    return -alpha * L - n * math.log(float(sp.zeta(alpha, xmin)))


def _grid_argmax(sp, x, xmin):
    L = float(np.log(x.astype(np.float64)).sum())
    n = x.size
    grid = np.arange(1.0005, 12.0, 1e-3)
    vals = [_loglik(sp, a, L, n, xmin) for a in grid]
    i = int(np.argmax(vals))
    lo, hi = grid[max(i - 1, 0)], grid[min(i + 1, len(grid) - 1)]
    g = (math.sqrt(5) - 1) / 2
    for _ in range(80):
        c, d = hi - g * (hi - lo), lo + g * (hi - lo)
        if _loglik(sp, c, L, n, xmin) > _loglik(sp, d, L, n, xmin):
            hi = d
        else:
            lo = c
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("xmin,data", [
    (1, [1, 1, 2, 5]),
    (2, [2, 2, 3, 7, 11]),
    (1, [1, 2, 3, 4, 5, 6, 7, 100]),
    (1, [1] * 30 + [2] * 8 + [3, 4, 9]),
    (5, [5, 5, 6, 8, 13, 40, 41]),
])
def test_mle_is_loglik_argmax(xmin, data):
    sp = pytest.importorskip("scipy.special")
    x = np.array(data, dtype=np.uint64)
    assert oracle.mle(x, xmin) == pytest.approx(_grid_argmax(sp, x, xmin), abs=2e-7)


def test_mle_against_mpmath_root():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(5)
    cases = [(1, np.array([1, 1, 2, 5])), (2, np.array([2, 2, 3, 7, 11]))]
    for alpha in [1.5, 2.5, 3.5]:
        cases.append((1, oracle.sample(alpha, 1, 77, 1, int(rng.integers(1000)), 2, 300)))
    for xmin, x in cases:
        x = np.asarray(x, dtype=np.uint64)
        mbar = mpmath.fsum(mpmath.log(int(v)) for v in x) / len(x)
        f = lambda a: mpmath.zeta(a, xmin, 1) / mpmath.zeta(a, xmin) + mbar
        root = mpmath.findroot(f, oracle.mle(x, xmin))
        assert oracle.mle(x, xmin) == pytest.approx(float(root), rel=1e-14)


@pytest.mark.parametrize("n,gamma,col", [(10, 3.5, 0), (10, 4.0, 0), (10, 4.0, 1), (20, 4.0, 0)])
def test_all_ones_atoms_match_table1(table1, n, gamma, col):
    # Table 1 prints these cutoffs; they are D of the all-ones sample (an atom of D's law
    # holding more than the remaining quantile mass), so the 4-decimal value is exact.
    x = np.ones(n, dtype=np.uint64)
    a = oracle.mle(x, 1)
    D = oracle.ks(x, 1, a)
    assert round(D, 4) == pytest.approx(table1[(gamma, n)][col], abs=1e-12)
    # all-ones rule: alpha-hat solves zeta'/zeta = -ln2/n
    z = oracle.hurwitz3(a, 1.0)
    assert z[1] / z[0] == pytest.approx(-math.log(2) / n, rel=1e-13)


def test_all_ones_rule_general_xmin():
    x = np.full(7, 3, dtype=np.uint64)
    a = oracle.mle(x, 3)
    z = oracle.hurwitz3(a, 3.0)
    assert z[1] / z[0] == pytest.approx(-(7 * math.log(3) + math.log(4 / 3)) / 7, rel=1e-13)


def test_ks_distinct_equals_brute_force():
    rng = np.random.default_rng(9)
    for trial in range(40):
        alpha = float(rng.uniform(1.6, 4.0))
        xmin = int(rng.choice([1, 2, 5]))
        n = int(rng.integers(1, 60))
        x = oracle.sample(alpha, xmin, 5, 9, trial, 2, n)
        if x.max() > 200000:
            continue
        for a in [alpha, oracle.mle(x, xmin), 1.3, 6.0]:
            assert oracle.ks(x, xmin, a) == oracle.ks(x, xmin, a, brute=True)


def test_ks_simple_values():
    # one point at xmin: S jumps to 1 at xmin, D = 1 - p(xmin) = Q(xmin)
    x = np.array([1], dtype=np.uint64)
    assert oracle.ks(x, 1, 2.0) == pytest.approx(1 - 1 / oracle.hurwitz(2.0, 1.0), rel=1e-15)
    # one point at 3: D = max(F(2), 1 - F(3))
    Z = oracle.hurwitz(2.0, 1.0)
    F2 = (1 + 2 ** -2) / Z
    F3 = (1 + 2 ** -2 + 3 ** -2) / Z
    assert oracle.ks(np.array([3], dtype=np.uint64), 1, 2.0) == pytest.approx(max(F2, 1 - F3), rel=1e-14)


def test_worked_example_values():
    # {1,1,2,5}: alpha-hat and D at 30 digits with mpmath
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    x = np.array([1, 1, 2, 5], dtype=np.uint64)
    mbar = mpmath.log(10) / 4
    root = mpmath.findroot(lambda a: mpmath.zeta(a, 1, 1) / mpmath.zeta(a, 1) + mbar, 2.0)
    Z = mpmath.zeta(root, 1)
    F = lambda t: 1 - mpmath.zeta(root, t + 1) / Z
    S = {0: 0, 1: 0.5, 2: 0.75, 3: 0.75, 4: 0.75, 5: 1.0}
    D = max(abs(F(t) - S[t]) for t in range(1, 6))
    assert oracle.mle(x, 1) == pytest.approx(float(root), rel=1e-14)
    assert oracle.ks(x, 1, oracle.mle(x, 1)) == pytest.approx(float(D), abs=1e-14)


def _exact_D_distribution(alpha, n, kmax, edges):
    """Exact law of D for samples of size n: enumerate every multiset of values in
    [1, kmax] with its multinomial probability; multisets with any value > kmax go to a
    separate 'other' category with the remaining mass."""
    Z = oracle.hurwitz(alpha, 1.0)
    p = {k: k ** (-alpha) / Z for k in range(1, kmax + 1)}
    probs = np.zeros(len(edges) + 1)
    covered = 0.0
    for ms in itertools.combinations_with_replacement(range(1, kmax + 1), n):
        counts = {}
        for v in ms:
            counts[v] = counts.get(v, 0) + 1
        pr = math.factorial(n)
        for v, c in counts.items():
            pr *= p[v] ** c / math.factorial(c)
        x = np.array(ms, dtype=np.uint64)
        D = oracle.ks(x, 1, oracle.mle(x, 1))
        probs[np.searchsorted(edges, D, side="right")] += pr
        covered += pr
    return probs, 1.0 - covered


@pytest.mark.parametrize("alpha,n,kmax", [(3.0, 3, 40), (2.5, 2, 300), (3.5, 4, 14)])
def test_D_distribution_matches_exact_enumeration(alpha, n, kmax):
    edges = np.linspace(0.0, 1.0, 41)[1:-1]
    probs, other = _exact_D_distribution(alpha, n, kmax, edges)
    R = 60_000
    D, A, _ = oracle.cell(alpha, 1, n, R, seed=21, cell_id=4, purpose=2)
    # replicates with a value > kmax form the 'other' category
    mx = np.array([oracle.sample(alpha, 1, 21, 4, r, 2, n).max() for r in range(R)])
    obs = np.zeros(len(edges) + 1)
    np.add.at(obs, np.searchsorted(edges, D[mx <= kmax], side="right"), 1)
    obs_other = int((mx > kmax).sum())
    expc = probs * R
    keep = expc >= 20
    o = np.concatenate([obs[keep], [obs[~keep].sum() + obs_other]])
    e = np.concatenate([expc[keep], [expc[~keep].sum() + other * R]])
    chi2 = ((o - e) ** 2 / e).sum()
    dof = len(o) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)
