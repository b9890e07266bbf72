"""The issue-rate probe (pl_probe_rates) on the GPU: the rates it reports
are those of real units (plausible per-SM-per-clock counts, an SM clock
inside the part's range), and Philox words per second agree with the
multiply rate (20 wide multiplies per block of four words)."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    from paper_1305_6738_gb300 import pl
    ctx = pl.Context(0)
    p = ctx.pl_probe_rates()
    ctx.close()
    assert p["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 300.0 < p["sm_clock_mhz"] < 3500.0
    assert 8.0 <= p["mul_wide_per_sm_clk"] <= 128.0
    assert 16.0 <= p["lop3_per_sm_clk"] <= 256.0
    assert 0.25 <= p["dfma_per_sm_clk"] <= 128.0
    # a Philox block is 20 wide multiplies: its word rate cannot beat the multiply rate
    mul_per_s = p["mul_wide_per_sm_clk"] * p["sms"] * p["sm_clock_mhz"] * 1e6
    assert p["philox_words_per_s"] <= 1.1 * mul_per_s / 5.0
    assert p["philox_words_per_s"] >= 0.25 * mul_per_s / 5.0
