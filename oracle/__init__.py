"""FP64 CPU oracle for the in-situ radiation spectrum -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never imports it,
and the two share no code: this package wraps ``rad_oracle.c`` (plain C, FP64,
libm ``sin``/``cos``) through ctypes and adds the bookkeeping that maps the
library's windows / species / frequency grids onto the plain per-window sum.

The formula (Frederiksen et al., Sec. 2.2, discretised P_omega integral, with
the Lienard-Wiechert integrand of Jackson eq. 14.67 that the paper cites via
Rybicki & Lightman):

    S_w(n, omega) = 1/(4 pi^2 c) * sum_j |A_j|^2          (incoherent)
                  = 1/(4 pi^2 c) * |sum_j A_j|^2          (coherent)
    A_j = sum_{m in [s0, s1)} q_j V_m exp(i omega (m dt - n.r_m)) dt
    V   = n x ((n - beta) x betadot) / (1 - n.beta)^2

Parity status: pinned by the CPU tests in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rad_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile rad_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, FP64).

    No fast-math and no FP contraction, so the arithmetic is exactly what the
    source writes on both x86-64 and aarch64.
    """
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            lib.rado_samples.restype = ctypes.c_int
            lib.rado_samples.argtypes = [ctypes.c_int64, ctypes.c_int64, _dp, _dp,
                                         ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
            lib.rado_field.restype = None
            lib.rado_field.argtypes = [_dp, _dp, _dp, _dp]
            lib.rado_amplitude.restype = None
            lib.rado_amplitude.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double,
                                           ctypes.c_double, _dp, ctypes.c_int32, _dp, _dp, _dp]
            lib.rado_spectrum.restype = ctypes.c_int
            lib.rado_spectrum.argtypes = [ctypes.c_int64, ctypes.c_int64, _dp, _dp, _dp, _dp,
                                          ctypes.POINTER(ctypes.c_ubyte), ctypes.c_double,
                                          ctypes.c_int32, _dp, ctypes.c_int32, _dp,
                                          ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _dp]
            lib.rado_num_threads.restype = ctypes.c_int
            lib.rado_set_num_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def num_threads() -> int:
    return int(_load().rado_num_threads())


def set_num_threads(n: int) -> None:
    _load().rado_set_num_threads(int(n))


def samples(x, u, dt, box_L=0.0):
    """Leapfrog states -> trajectory samples (r, beta, betadot).

    x, u: [n_calls, 3, N] (call s carries x_s and u_{s-1/2}).  Returns three
    arrays of shape [n_calls - 1, 3, N]; sample m needs calls m and m + 1.
    """
    x, px = _c(x)
    u, pu = _c(u)
    if x.ndim != 3 or x.shape[1] != 3 or u.shape != x.shape:
        raise ValueError("x and u must both be [n_calls, 3, N]")
    nc, _, N = x.shape
    if nc < 2:
        raise ValueError("need at least two calls for one sample")
    out = [np.empty((nc - 1, 3, N)) for _ in range(3)]
    rc = _load().rado_samples(nc, N, px, pu, float(dt), float(box_L),
                              *[o.ctypes.data_as(_dp) for o in out])
    if rc != 0:
        raise ValueError("rado_samples rejected its arguments")
    return tuple(out)


def field(n, beta, betadot):
    """V = n x ((n - beta) x betadot) / (1 - n.beta)^2 for single 3-vectors."""
    n, pn = _c(n)
    b, pb = _c(beta)
    bd, pbd = _c(betadot)
    V = np.empty(3)
    _load().rado_field(pn, pb, pbd, V.ctypes.data_as(_dp))
    return V


def amplitude(r, beta, betadot, j, m0, m1, dt, q, n, omega):
    """Vector amplitude A_j(n, omega) over samples [m0, m1): complex [nf, 3]."""
    r, pr = _c(r)
    b, pb = _c(beta)
    bd, pbd = _c(betadot)
    n, pn = _c(n)
    om, pom = _c(np.atleast_1d(omega))
    N = r.shape[2]
    Are = np.empty((om.size, 3))
    Aim = np.empty((om.size, 3))
    _load().rado_amplitude(N, int(j), int(m0), int(m1), pr, pb, pbd, float(dt), float(q), pn,
                           om.size, pom, Are.ctypes.data_as(_dp), Aim.ctypes.data_as(_dp))
    return Are + 1j * Aim


def window_spectrum(r, beta, betadot, charge, dt, dirs, omega, s0, s1, coherent=False,
                    include=None):
    """Spectrum [D, nf] of one window [s0, s1) from sample arrays [n_samp, 3, N]."""
    r, pr = _c(r)
    b, pb = _c(beta)
    bd, pbd = _c(betadot)
    q, pq = _c(charge)
    dirs, pd = _c(np.reshape(dirs, (-1, 3)))
    om, pom = _c(np.atleast_1d(omega))
    n_samp, _, N = r.shape
    if q.shape != (N,):
        raise ValueError("charge must be [N]")
    inc_ptr = ctypes.POINTER(ctypes.c_ubyte)()
    if include is not None:
        inc = np.ascontiguousarray(include, dtype=np.uint8)
        inc_ptr = inc.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    D = dirs.shape[0]
    S = np.empty((D, om.size))
    rc = _load().rado_spectrum(N, n_samp, pr, pb, pbd, pq, inc_ptr, float(dt), D, pd, om.size,
                               pom, int(s0), int(s1), 1 if coherent else 0,
                               S.ctypes.data_as(_dp))
    if rc != 0:
        raise ValueError("rado_spectrum rejected its arguments")
    return S


def spectra(x, u, dt, dirs, grids, windows, species, coherent=False, box_L=0.0):
    """Full diagnostic, in the library's terms, as a list of [D, len(grid)] arrays.

    x, u     : [n_calls, 3, N_total] leapfrog states (species concatenated).
    dirs     : [D, 3] unit vectors.
    grids    : list of 1-D frequency arrays.
    windows  : list of (s0, s1, species_mask, grid_index).
    species  : list of (count, charge).
    """
    r, beta, bdot = samples(x, u, dt, box_L)
    counts = [int(c) for c, _ in species]
    N = int(sum(counts))
    if r.shape[2] != N:
        raise ValueError("species counts do not add up to the particle axis")
    sp_index = np.repeat(np.arange(len(species)), counts)
    charge = np.repeat(np.array([float(q) for _, q in species]), counts)
    out = []
    for (s0, s1, mask, g) in windows:
        include = ((int(mask) >> sp_index) & 1).astype(np.uint8)
        out.append(window_spectrum(r, beta, bdot, charge, dt, dirs, grids[g], s0, s1,
                                   coherent=coherent, include=include))
    return out
