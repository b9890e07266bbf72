"""Pins for the oracle's cutoff-table lookup (the use of the tables at a
close value of the exponent, Section 3): bilinear in (exponent, ln N) between
the surrounding grid cells, clamped to the grid's edges."""
import math

import numpy as np

import oracle

GA = [1.25, 1.5, 1.75, 2.0, 2.5, 3.0, 3.5, 4.0]
GN = [10, 20, 30, 40, 50, 100, 500, 1000, 2000, 3000, 4000, 5000, 10000, 20000, 50000]


def _table(f, nq=3):
    t = np.zeros((len(GA), len(GN), nq))
    for i, a in enumerate(GA):
        for k, n in enumerate(GN):
            for j in range(nq):
                t[i, k, j] = f(a, math.log(n)) + j
    return t


def test_grid_points_are_exact():
    rng = np.random.default_rng(3)
    t = rng.random((len(GA), len(GN), 4))
    for i, a in enumerate(GA):
        for k, n in enumerate(GN):
            assert np.array_equal(oracle.cutoff_lookup(GA, GN, t, a, n), t[i, k])


def test_bilinear_functions_are_reproduced():
    f = lambda a, l: 0.3 - 0.05 * a + 0.02 * l - 0.004 * a * l  # noqa: E731
    t = _table(f)
    rng = np.random.default_rng(4)
    for _ in range(300):
        a = rng.uniform(GA[0], GA[-1])
        n = int(math.exp(rng.uniform(math.log(GN[0]), math.log(GN[-1]))))
        got = oracle.cutoff_lookup(GA, GN, t, a, n)
        assert np.allclose(got, [f(a, math.log(n)) + j for j in range(3)], rtol=0, atol=1e-13)
    # a function that is not bilinear is not reproduced between grid points
    g = lambda a, l: a * a  # noqa: E731
    tg = _table(g, 1)
    assert oracle.cutoff_lookup(GA, GN, tg, 1.375, 100)[0] > 1.375 ** 2 + 1e-3


def test_clamped_outside_the_grid():
    rng = np.random.default_rng(5)
    t = rng.random((len(GA), len(GN), 2))
    assert np.array_equal(oracle.cutoff_lookup(GA, GN, t, 0.5, 5), t[0, 0])
    assert np.array_equal(oracle.cutoff_lookup(GA, GN, t, 9.0, 10 ** 6), t[-1, -1])
    assert np.array_equal(oracle.cutoff_lookup(GA, GN, t, 2.0, 10 ** 6), t[3, -1])


def test_single_row_grids():
    t = np.arange(6, dtype=float).reshape(1, 3, 2)
    got = oracle.cutoff_lookup([2.0], [10, 100, 1000], t, 7.0, 100)
    assert np.array_equal(got, t[0, 1])
    got = oracle.cutoff_lookup([2.0], [10, 100, 1000], t, 2.0, 31)
    w = (math.log(31) - math.log(10)) / (math.log(100) - math.log(10))
    assert np.allclose(got, (1 - w) * t[0, 0] + w * t[0, 1], rtol=0, atol=1e-15)
