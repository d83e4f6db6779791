"""The FMA-pipe e^{i theta} of the MIX kernel variant (Cody-Waite half-angle
reduction, minimax sin/cos on [-pi/2, pi/2], double angle): its coefficients,
read from the kernel source, evaluated by a float32 emulation of the kernel's
instruction sequence, stay within 1e-6 of cos/sin over |theta| <= 2000 (the
special-function unit's sine is specified to about 2^-20.9 absolute)."""
import os
import re
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1003_1140_gb300", "csrc")


def kernel_constants():
    src = open(os.path.join(CSRC, "rad_accum32.cuh")).read()
    get = lambda n: np.float32(float(re.search(rf"\b{n} = ([-+0-9.e]+)f", src).group(1)))
    S = np.array([get("kS3"), get("kS5"), get("kS7"), get("kS9")], np.float32)
    C = np.array([get("kC2"), get("kC4"), get("kC6"), get("kC8")], np.float32)
    return S, C, get("kPiHi"), get("kPiLo")


def test_polynomial_error_bound():
    sys.path.insert(0, CSRC)
    import fit_sincos as f
    S, C, pi_hi, pi_lo = kernel_constants()
    assert pi_hi == f.PI_HI and pi_lo == f.PI_LO
    err = f.max_error(S, C, n=400_001, lim=2000.0)
    assert err < 1e-6, err


def test_coefficients_are_the_fit():
    sys.path.insert(0, CSRC)
    import fit_sincos as f
    S, C, _, _ = kernel_constants()
    S2, C2 = f.fit()
    np.testing.assert_allclose(S, S2, rtol=1e-6)
    np.testing.assert_allclose(C, C2, rtol=1e-6)
