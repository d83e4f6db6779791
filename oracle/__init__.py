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


def subsamples(x, u, dt, box_L, nsub):
    """Sub-cycled samples (Sec. 2.2: tracked particles sub-cycled at a fraction of
    the PIC step), nsub per PIC sample m, at times (m + tau_k) dt with
    tau_k = (k + 1/2)/nsub - 1/2:
      u(tau)       = ubar_m + tau (u_{m+1/2} - u_{m-1/2})       (linear in time)
      beta(tau)    = u / gamma(u),  gamma = sqrt(1 + u.u)
      betadot(tau) = udot / gamma - u (u . udot) / gamma^3,  udot = (u_{m+1/2} - u_{m-1/2}) / dt
      r(tau)       = r_m + dt (tau / 6) (beta(0) + 4 beta(tau/2) + beta(tau))   (Simpson)
    Returns r, beta, betadot of shape [(n_calls - 1) nsub, 3, N]; sub-sample
    M = m nsub + k is spaced dt / nsub from its neighbours.
    """
    r, _, _ = samples(x, u, dt, box_L)
    u = np.asarray(u, dtype=np.float64)
    um, up = u[:-1], u[1:]
    ubar = 0.5 * (um + up)
    du = up - um

    def beta_of(uu):
        return uu / np.sqrt(1.0 + (uu * uu).sum(1, keepdims=True))

    b0 = beta_of(ubar)
    n_s, _, N = r.shape
    R = np.empty((n_s, nsub, 3, N))
    B = np.empty_like(R)
    BD = np.empty_like(R)
    for k in range(nsub):
        tau = (k + 0.5) / nsub - 0.5
        uk = ubar + tau * du
        uh = ubar + 0.5 * tau * du
        gk = np.sqrt(1.0 + (uk * uk).sum(1, keepdims=True))
        udot = du / dt
        B[:, k] = uk / gk
        BD[:, k] = udot / gk - uk * (uk * udot).sum(1, keepdims=True) / gk ** 3
        R[:, k] = r + dt * (tau / 6.0) * (b0 + 4.0 * beta_of(uh) + uk / gk)
    shape = (n_s * nsub, 3, N)
    return R.reshape(shape), B.reshape(shape), BD.reshape(shape)


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


def selector_mask(x, u, sel):
    """Per-sample selection [n_calls - 1, N] (Sec. 2.2 regions for spectral
    collection; the momentum pitch cone of Sec. 3.2):
      box : lo <= x_m < hi per component, x_m the position handed over for step m;
      cone: cos(angle(ubar_m, axis)) in [cos(theta_c + dtheta), cos(theta_c - dtheta)]
            (angles clamped to [0, pi]), ubar_m = (u_{m-1/2} + u_{m+1/2}) / 2,
            cos = ((ubar_x a_x + ubar_y a_y) + ubar_z a_z) / sqrt((ubar_x^2 + ubar_y^2) + ubar_z^2).
    """
    x = np.asarray(x, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    xm = x[:-1]
    if sel["kind"] == "box":
        lo = np.asarray(sel["lo"], dtype=np.float64)
        hi = np.asarray(sel["hi"], dtype=np.float64)
        ok = np.ones(xm.shape[0:1] + xm.shape[2:], dtype=bool)
        for q in range(3):
            ok &= (xm[:, q] >= lo[q]) & (xm[:, q] < hi[q])
        return ok
    a = np.asarray(sel["axis"], dtype=np.float64)
    a = a / np.sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2])
    ub = 0.5 * (u[:-1] + u[1:])
    par = (ub[:, 0] * a[0] + ub[:, 1] * a[1]) + ub[:, 2] * a[2]
    nrm = np.sqrt((ub[:, 0] * ub[:, 0] + ub[:, 1] * ub[:, 1]) + ub[:, 2] * ub[:, 2])
    with np.errstate(invalid="ignore", divide="ignore"):
        cs = par / nrm
    c_lo = np.cos(min(np.pi, sel["theta_c"] + sel["dtheta"]))
    c_hi = np.cos(max(0.0, sel["theta_c"] - sel["dtheta"]))
    return (cs >= c_lo) & (cs <= c_hi)


def spectra(x, u, dt, dirs, grids, windows, species, coherent=False, box_L=0.0,
            selectors=None, window_selector=None, subcycle=1):
    """Full diagnostic, in the library's terms, as a list of [D, len(grid)] arrays.

    x, u     : [n_calls, 3, N_total] leapfrog states (species concatenated).
    dirs     : [D, 3] unit vectors.
    grids    : list of 1-D frequency arrays.
    windows  : list of (s0, s1, species_mask, grid_index) or (s0, s1, species_mask,
               grid_index, direction indices): a window's spectrum is [len(its
               directions), len(grid)], rows in the order of its direction list.
    species  : list of (count, charge).
    selectors, window_selector: optional sample selectors (see selector_mask) and,
               per window, the selector index or -1; a selected-out sample
               contributes nothing (its V is zero).
    """
    nsub = max(1, int(subcycle))
    if nsub == 1:
        r, beta, bdot = samples(x, u, dt, box_L)
    else:
        r, beta, bdot = subsamples(x, u, dt, box_L, nsub)
    masks = [np.repeat(selector_mask(x, u, sdef), nsub, axis=0) for sdef in (selectors or [])]
    counts = [int(c) for c, _ in species]
    N = int(sum(counts))
    if r.shape[2] != N:
        raise ValueError("species counts do not add up to the particle axis")
    sp_index = np.repeat(np.arange(len(species)), counts)
    charge = np.repeat(np.array([float(q) for _, q in species]), counts)
    out = []
    dirs = np.reshape(np.asarray(dirs, dtype=np.float64), (-1, 3))
    for wi, wdef in enumerate(windows):
        s0, s1, mask, g = wdef[:4]
        wdirs = dirs if len(wdef) < 5 or wdef[4] is None else dirs[np.asarray(wdef[4], int)]
        include = ((int(mask) >> sp_index) & 1).astype(np.uint8)
        bd = bdot
        if window_selector is not None and window_selector[wi] >= 0:
            bd = bdot * masks[window_selector[wi]][:, None, :]   # V is linear in betadot
        out.append(window_spectrum(r, beta, bd, charge, dt / nsub, wdirs, grids[g], s0 * nsub,
                                   s1 * nsub, coherent=coherent, include=include))
    return out
