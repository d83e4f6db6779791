"""The roofline denominators bench.py reports, against their closed forms.

Algorithmic bound (`peak`): (7 + 10 (1 - p)) / 128 = 2 p / 16 gives p = 17/26
and 8 / p = 208/17 updates per clock per SM.  This kernel's issue model:
(5 + 3 p + 17 (1 - p)) / 128 = 2 p / 16 gives p = 11/15 and 120/11.  The SFU
bound is 16 / 2 = 8.  At 152 SMs and 2070 MHz: 3849.8, 3431.1 and 2517.12
G updates/s."""
import pytest

from paper_1003_1140_gb300 import roofline as rl


def test_bounds_match_their_closed_forms():
    assert rl.sfu_per_clk() == 8.0
    alg, pa = rl.algorithmic_per_clk()
    assert pa == pytest.approx(17 / 26, abs=1e-4)
    assert alg == pytest.approx(208 / 17, rel=2e-4)
    assert alg <= 208 / 17 + 1e-12           # the grid search cannot beat the balance point
    comb, p = rl.combined_per_clk()
    assert p == pytest.approx(11 / 15, abs=1e-4)
    assert comb == pytest.approx(120 / 11, rel=2e-4)
    assert comb <= 120 / 11 + 1e-12
    # a free polynomial would put everything on the FMA pipe
    comb0, p0 = rl.combined_per_clk(poly_fp32=0.0)
    assert p0 == 0.0 and comb0 == pytest.approx(128 / 5)
    alg0, pa0 = rl.algorithmic_per_clk(poly=0.0)
    assert pa0 == 0.0 and alg0 == pytest.approx(128 / 7)


def test_accum32_roofline_at_the_bench_clock():
    upd, ms = 1.0e12, 500.0                   # 2000 G updates/s
    r = rl.accum32_roofline(upd, ms, 152, 2070.0)
    assert r["achieved"] == pytest.approx(2000.0)
    assert r["peak"] == pytest.approx(152 * 2.070 * 208 / 17, rel=2e-4)         # 3849.8
    assert r["peak_sfu"] == pytest.approx(152 * 2070e6 * 8 / 1e9)              # 2517.12
    assert r["peak_issue_model"] == pytest.approx(152 * 2.070 * 120 / 11, rel=2e-4)  # 3431
    assert r["frac"] == pytest.approx(2000.0 / r["peak"])
    assert r["frac_sfu"] == pytest.approx(2000.0 / 2517.12)
    assert r["frac_issue_model"] == pytest.approx(2000.0 / r["peak_issue_model"])
    assert r["bound"] == "alu" and r["unit"] == "G updates/s"
    # no clock sample: the maximum SM clock
    assert rl.accum32_roofline(upd, ms, 152, None)["peak_sfu"] == pytest.approx(2517.12)
