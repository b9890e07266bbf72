"""The benchmark's per-cell lines (host arithmetic only, no GPU)."""
import math

import bench


def test_cell_line_rates_and_fraction():
    d = bench.cell_line(2.0, 100, 100_000, 10.0, 6.0, 3.0, 10068.48)
    assert d["replicates_per_s"] == 1e7 and d["samples_per_s"] == 1e9
    assert math.isclose(d["finisher_ns_per_replicate"], 30.0)
    # sampler: MUL_PER_DRAW multiplies per draw over the sampler's own time, against the peak in Gmul/s
    assert math.isclose(d["sampler_frac"], bench.MUL_PER_DRAW * 1e7 / 6e-3 / 1e9 / 10068.48)
    assert bench.cell_line(2.0, 10, 1, 1.0, 0.0, 0.0, 1.0)["sampler_frac"] is None
