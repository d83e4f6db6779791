"""The roofline denominators bench.py reports, against their closed forms.

The combined FP32 + SFU bound balances instruction issue against MUFU time:
(5 + 3 p + 17 (1 - p)) / 128 = 2 p / 16 gives p = 11/15 and 8 / p = 120/11
updates per clock per SM; the SFU bound is 16 / 2 = 8.  At 152 SMs and
2070 MHz these are 3431.1 and 2517.12 G updates/s."""
import pytest

from paper_1003_1140_gb300 import roofline as rl


def test_bounds_match_their_closed_forms():
    assert rl.sfu_per_clk() == 8.0
    comb, p = rl.combined_per_clk()
    assert p == pytest.approx(11 / 15, abs=1e-3)
    assert comb == pytest.approx(120 / 11, rel=2e-3)
    assert comb <= 120 / 11 + 1e-12          # the grid search cannot beat the balance point
    # a free polynomial would put everything on the FMA pipe: 128 / 5 per clock
    comb0, p0 = rl.combined_per_clk(poly_fp32=0.0)
    assert p0 == 0.0 and comb0 == pytest.approx(128 / 5)


def test_accum32_roofline_at_the_bench_clock():
    upd, ms = 1.0e12, 500.0                   # 2000 G updates/s
    r = rl.accum32_roofline(upd, ms, 152, 2070.0)
    assert r["achieved"] == pytest.approx(2000.0)
    assert r["peak_sfu"] == pytest.approx(152 * 2070e6 * 8 / 1e9)       # 2517.12
    assert r["peak"] == pytest.approx(152 * 2.070 * 120 / 11, rel=2e-3)  # 3431
    assert r["frac"] == pytest.approx(2000.0 / r["peak"])
    assert r["frac_sfu"] == pytest.approx(2000.0 / 2517.12)
    assert r["bound"] == "alu" and r["unit"] == "G updates/s"
    # no clock sample: the maximum SM clock
    assert rl.accum32_roofline(upd, ms, 152, None)["peak_sfu"] == pytest.approx(2517.12)
