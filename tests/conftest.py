import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled library")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_table1():
    """Table 1 of the paper as {(gamma, N): (q90, q95, q99, q999)}."""
    out = {}
    with open(os.path.join(GOLDEN, "table1_pure_power_law.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            g, n, *q = line.split()
            out[(float(g), int(n))] = tuple(float(v) for v in q)
    return out


@pytest.fixture(scope="session")
def table1():
    return load_table1()


def load_tables2to6():
    """Tables 2-6 of the paper as {(K, gamma, N): (q90, q95, q99, q999)}."""
    out = {}
    with open(os.path.join(GOLDEN, "tables2to6_truncated.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            K, g, n, *q = line.split()
            out[(int(K), float(g), int(n))] = tuple(float(v) for v in q)
    return out


@pytest.fixture(scope="session")
def tables2to6():
    return load_tables2to6()
