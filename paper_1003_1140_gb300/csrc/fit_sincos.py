"""Fit the FMA-pipe e^{i theta} polynomials used by the MIX variant.

Method (written from the mathematics, not from any library's code):
  * half-angle reduction: theta/2 = k pi + y, |y| <= pi/2 (Cody & Waite two-
    constant subtraction of k pi), so e^{i theta} = (cos y + i sin y)^2;
  * sin y ~ y + y^3 (S3 + y^2 S5 + y^4 S7 + y^6 S9),
    cos y ~ 1 + y^2 (C2 + y^2 C4 + y^4 C6 + y^6 C8):
    minimax (equioscillating absolute error) polynomials on [0, pi/2] found by
    a Remez exchange on the even/odd parts, in float64;
  * double angle: cos theta = c^2 - s^2, sin theta = 2 c s.

Running this module prints the float32 coefficients for rad_accum32.cuh and
the error of the complete float32 evaluation; the unit test re-runs the
float32 emulation and checks the bound.
"""
from __future__ import annotations

import numpy as np

HALF_PI = np.pi / 2


def _remez(basis, target, weight, a, b, n_iter=40):
    """Minimax fit of target(x) ~ sum c_i basis_i(x) with weight(x) on [a, b]."""
    m = len(basis)
    # initial reference: Chebyshev extrema
    ref = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(np.pi * np.arange(m + 1)[::-1] / m)
    xs = np.linspace(a, b, 20001)
    coef = None
    for _ in range(n_iter):
        A = np.zeros((m + 1, m + 1))
        for i, x in enumerate(ref):
            A[i, :m] = [f(x) for f in basis]
            A[i, m] = (-1) ** i / weight(x)
        sol = np.linalg.solve(A, np.array([target(x) for x in ref]))
        coef = sol[:m]
        err = (np.array([sum(c * f(x) for c, f in zip(coef, basis)) for x in xs]) -
               np.array([target(x) for x in xs])) * np.array([weight(x) for x in xs])
        # new reference: extrema of the error between sign changes
        sgn = np.sign(err)
        idx = []
        start = 0
        for i in range(1, len(xs)):
            if sgn[i] != sgn[i - 1] and sgn[i] != 0:
                seg = slice(start, i)
                idx.append(start + int(np.argmax(np.abs(err[seg]))))
                start = i
        idx.append(start + int(np.argmax(np.abs(err[start:]))))
        if len(idx) >= m + 1:
            # keep the m+1 largest alternating extrema
            while len(idx) > m + 1:
                if abs(err[idx[0]]) < abs(err[idx[-1]]):
                    idx.pop(0)
                else:
                    idx.pop()
            ref = xs[idx]
    return coef


def fit():
    # sin: s(y) = y + y^3 P(y^2); fit P on u = y^2 in [0, (pi/2)^2] for minimax abs error in s
    def sbasis(k):
        return lambda y: y ** (2 * k + 3)
    S = _remez([sbasis(k) for k in range(4)], lambda y: np.sin(y) - y, lambda y: 1.0,
               1e-6, HALF_PI)
    def cbasis(k):
        return lambda y: y ** (2 * k + 2)
    C = _remez([cbasis(k) for k in range(4)], lambda y: np.cos(y) - 1.0, lambda y: 1.0,
               0.0, HALF_PI)
    return np.float32(S), np.float32(C)


PI_HI = np.float32(np.pi)
PI_LO = np.float32(np.pi - float(PI_HI))
INV_PI = np.float32(1.0 / np.pi)
MAGIC = np.float32(12582912.0)   # 1.5 * 2^23: adding it rounds to an integer


def eval_f32(theta, S, C):
    """float32 emulation of the kernel's sequence (numpy float32, fma by float64 rounding)."""
    f = np.float32
    th = (np.asarray(theta, np.float32) * f(0.5)).astype(np.float32)
    fma = lambda a, b, c: (a.astype(np.float64) * b + c).astype(np.float32)
    t = fma(th, np.full_like(th, INV_PI), np.full_like(th, MAGIC))
    k = (t - MAGIC).astype(np.float32)
    y = fma(k, np.full_like(k, -PI_HI), th)
    y = fma(k, np.full_like(k, -PI_LO), y)
    y2 = (y * y).astype(np.float32)
    p = fma(y2, np.full_like(y2, S[3]), np.full_like(y2, S[2]))
    p = fma(y2, p, np.full_like(y2, S[1]))
    p = fma(y2, p, np.full_like(y2, S[0]))
    y3 = (y * y2).astype(np.float32)
    s = fma(y3, p, y)
    q = fma(y2, np.full_like(y2, C[3]), np.full_like(y2, C[2]))
    q = fma(y2, q, np.full_like(y2, C[1]))
    q = fma(y2, q, np.full_like(y2, C[0]))
    c = fma(y2, q, np.ones_like(y2))
    s2 = (s * s).astype(np.float32)
    cos_t = fma(c, c, -s2)
    sin_half = (c * s).astype(np.float32)       # sin(theta) / 2
    return cos_t, sin_half


def max_error(S, C, n=2_000_001, lim=2000.0):
    th = np.linspace(-lim, lim, n).astype(np.float32)
    ct, sh = eval_f32(th, S, C)
    t64 = th.astype(np.float64)
    return max(np.abs(ct - np.cos(t64)).max(), np.abs(2 * sh.astype(np.float64) - np.sin(t64)).max())


if __name__ == "__main__":
    S, C = fit()
    print("S3, S5, S7, S9 =", ", ".join(f"{v:.9e}f" for v in S))
    print("C2, C4, C6, C8 =", ", ".join(f"{v:.9e}f" for v in C))
    print("PI_HI, PI_LO =", f"{PI_HI:.9e}f, {PI_LO:.9e}f")
    print("max |error| of e^{i theta}, |theta| <= 2000:", max_error(S, C))
