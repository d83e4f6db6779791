"""Roofline of the FP32 split-phase accumulation kernel (an ALU-bound kernel).

The work unit is an update per (particle, sample, direction, omega).  The
algorithmic minimum per update is one FFMA for the phase theta = w dphi +
Theta, six FFMA to add V e^{i theta} to the three complex components of the
amplitude, and e^{i theta} itself: two special-function (MUFU) operations
(sin, cos), or an FMA-pipe polynomial of P instructions.  Per-SM unit counts
of sm_103a:

    FP32 (FFMA) lanes        128 / clock / SM
    MUFU sin/cos lanes        16 / clock / SM   (measured on GB300: 16.4 at 1.91 GHz)
    instruction issue        128 thread-instructions / clock / SM (4 x 32)

* Algorithmic bound (the denominator `peak`): a fraction p of the updates
  takes its e^{i theta} from the MUFU pipe and 1 - p from a P = 10
  instruction polynomial on the FP32 pipe; the best p balances the two pipes:
      t(p) = max((7 + P (1 - p)) / 128,  2 p / 16)  clocks / update / SM,
  p = 17/26 and 8 / p = 208/17 = 12.24 updates / clock / SM.
* SFU bound: every e^{i theta} on the MUFU pipe, 2 MUFU per update ->
  16 / 2 = 8 updates / clock / SM.
* Issue model of this kernel's own instruction stream (reported beside the
  others): 5 FFMA (V has two components on a basis normal to n, so the
  amplitude needs two complex accumulators: 4 FFMA, plus the phase), the
  argument-scale FMUL and 2 MUFU on the SFU path or a 17-instruction
  polynomial, all counted against instruction issue:
      t(p) = max((5 + 3 p + 17 (1 - p)) / 128,  2 p / 16),
  p = 11/15 and 120/11 = 10.91 updates / clock / SM.
Updates per second = SMs x f x (updates / clock / SM), f the SM clock sampled
during the timed region (the maximum SM clock, 2070 MHz, when no sample
exists).
"""
from __future__ import annotations

FP32_PER_CLK = 128.0
MUFU_PER_CLK = 16.0
ISSUE_PER_CLK = 128.0
# algorithmic count
ALG_FP32 = 7.0             # phase FFMA + 6 accumulate FFMA
ALG_POLY = 10.0            # FMA-pipe sin/cos polynomial of the algorithmic bound
# this kernel's instruction stream
COMMON_FP32 = 5.0          # phase FFMA + 4 accumulate FFMA
SFU_PATH_ISSUE = 3.0       # argument-scale FMUL + MUFU.SIN + MUFU.COS
POLY_FP32 = 17.0           # Cody-Waite half-turn reduction (4), y^2 (1), sin deg 9 (5),
                           # cos deg 8 (4), double angle (3)
SM_MAX_MHZ = 2070.0


def sfu_per_clk() -> float:
    return MUFU_PER_CLK / 2.0


def _best(time_of_p):
    best, best_p = 0.0, 1.0
    for i in range(100001):
        p = i / 100000.0
        r = 1.0 / time_of_p(p)
        if r > best:
            best, best_p = r, p
    return best, best_p


def algorithmic_per_clk(fp32: float = ALG_FP32, poly: float = ALG_POLY):
    """Best updates/clock/SM of the algorithmic count over the SFU fraction p, and p."""
    return _best(lambda p: max((fp32 + poly * (1.0 - p)) / FP32_PER_CLK,
                               2.0 * p / MUFU_PER_CLK))


def combined_per_clk(poly_fp32: float = POLY_FP32):
    """Best updates/clock/SM of this kernel's issue model over p, and that p."""
    return _best(lambda p: max((COMMON_FP32 + SFU_PATH_ISSUE * p + poly_fp32 * (1.0 - p))
                               / ISSUE_PER_CLK, 2.0 * p / MUFU_PER_CLK))


def accum32_roofline(updates_per_launch: float, ms_per_launch: float, sms: int,
                     sm_mhz: float | None, options: dict | None = None) -> dict:
    f = (sm_mhz or SM_MAX_MHZ) * 1e6
    achieved = updates_per_launch / (ms_per_launch * 1e-3) / 1e9 if ms_per_launch > 0 else 0.0
    alg, p_alg = algorithmic_per_clk()
    comb, p = combined_per_clk()
    peak = sms * f * alg / 1e9
    peak_issue = sms * f * comb / 1e9
    peak_sfu = sms * f * sfu_per_clk() / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G updates/s",
            "frac": achieved / peak if peak else None, "traffic": None,
            "peak_kind": f"algorithmic FP32+SFU bound: 7 FFMA + 2 MUFU per update, "
                         f"P=10 polynomial share {1 - p_alg:.3f}, {alg:.2f} updates/clk/SM, "
                         f"{sms} SMs x {f / 1e6:.0f} MHz (sampled SM clock)",
            "peak_sfu": peak_sfu, "frac_sfu": achieved / peak_sfu if peak_sfu else None,
            "peak_issue_model": peak_issue,
            "frac_issue_model": achieved / peak_issue if peak_issue else None,
            "issue_model_kind": f"this kernel's stream: 5 FFMA + (FMUL + 2 MUFU | 17-op "
                                f"polynomial), {comb:.2f} updates/clk/SM at p_sfu={p:.2f}",
            "ms_per_launch": ms_per_launch, "updates_per_launch": updates_per_launch}
