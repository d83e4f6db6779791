"""Roofline of the FP32 split-phase accumulation kernel (an ALU-bound kernel).

The kernel's work is an update per (particle, sample, direction, omega): one
FFMA for the phase theta = fma(w, dphi, Theta), four FFMA to add V e^{i theta}
to two complex accumulators, and e^{i theta} itself -- two special-function
(MUFU) operations, or an FMA-pipe polynomial.  The bound follows from the
per-SM unit counts of sm_103a:

    FP32 (FFMA) lanes        128 / clock / SM
    MUFU sin/cos lanes        16 / clock / SM   (measured on GB300: 16.4 at 1.91 GHz)
    instruction issue        128 thread-instructions / clock / SM (4 x 32)

* SFU bound: every e^{i theta} on the MUFU pipe, 2 MUFU per update ->
  R_SFU = SMs * f * 16 / 2 = 8 updates / clock / SM.
* Combined FP32 + SFU bound: a fraction p of the updates on the MUFU pipe
  (1 FMUL argument scale + 2 MUFU) and 1 - p on a POLY_FP32-instruction
  FMA-pipe polynomial; the best p balances issue and MUFU time:
      t(p) = max((5 + 3 p + POLY_FP32 (1 - p)) / 128,  2 p / 16)  clocks / update / SM.
f is the SM clock sampled during the timed region (falling back to the
maximum SM clock, 2070 MHz, when no sample exists).
"""
from __future__ import annotations

FP32_PER_CLK = 128.0
MUFU_PER_CLK = 16.0
ISSUE_PER_CLK = 128.0
COMMON_FP32 = 5.0          # phase FFMA + 4 accumulate FFMA
SFU_PATH_ISSUE = 3.0       # argument-scale FMUL + MUFU.SIN + MUFU.COS
POLY_FP32 = 17.0           # Cody-Waite half-turn reduction (4), y^2 (1), sin deg 9 (5),
                           # cos deg 8 (4), double angle (3)
SM_MAX_MHZ = 2070.0


def sfu_per_clk() -> float:
    return MUFU_PER_CLK / 2.0


def combined_per_clk(poly_fp32: float = POLY_FP32):
    """Best updates/clock/SM over the SFU fraction p, and that p."""
    best, best_p = 0.0, 1.0
    for i in range(1001):
        p = i / 1000.0
        issue = (COMMON_FP32 + SFU_PATH_ISSUE * p + poly_fp32 * (1.0 - p)) / ISSUE_PER_CLK
        mufu = 2.0 * p / MUFU_PER_CLK
        r = 1.0 / max(issue, mufu)
        if r > best:
            best, best_p = r, p
    return best, best_p


def accum32_roofline(updates_per_launch: float, ms_per_launch: float, sms: int,
                     sm_mhz: float | None, options: dict | None = None) -> dict:
    f = (sm_mhz or SM_MAX_MHZ) * 1e6
    achieved = updates_per_launch / (ms_per_launch * 1e-3) / 1e9 if ms_per_launch > 0 else 0.0
    comb, p = combined_per_clk()
    peak_comb = sms * f * comb / 1e9
    peak_sfu = sms * f * sfu_per_clk() / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak_comb, "unit": "G updates/s",
            "frac": achieved / peak_comb if peak_comb else None, "traffic": None,
            "peak_kind": f"combined FP32+SFU bound, {comb:.2f} updates/clk/SM at p_sfu={p:.2f}, "
                         f"{sms} SMs x {f / 1e6:.0f} MHz (sampled SM clock)",
            "peak_sfu": peak_sfu, "frac_sfu": achieved / peak_sfu if peak_sfu else None,
            "ms_per_launch": ms_per_launch, "updates_per_launch": updates_per_launch}
