"""Seeded synthetic trajectories for the radiation diagnostic (input generator).

This module serves both the CUDA library's tests/benchmark and the FP64 CPU
oracle; it holds none of the radiation method's arithmetic.  It only makes
the leapfrog states (x_s, u_{s-1/2}) a PIC code would hand to the diagnostic.

Workload recipe (a frozen-field stand-in for the paper's filamentation runs,
Sec. 2.1 "frozen" EM fields, units c = m_e = q_e = 1, t in 1/omega_pe):

* static magnetic field B = curl(A_x(y, z) x_hat) = (0, dA_x/dz, -dA_x/dy) in a
  periodic cube of side L = 40, with A_x = sum of 64 modes a cos(k.(y,z) + psi),
  k = 2 pi (n_y, n_z) / L for integer n with |k| in [0.3, 3], drawn without
  +-k duplicates; equal amplitudes a set so that the box rms |B| is B_rms
  (<|B|^2> = sum a^2 |k|^2 / 2);
* two counter-streaming beams along +-x (even particle index: +x): a
  rest-frame Maxwell-Juttner momentum at temperature theta (drawn by a
  tabulated inverse CDF of u^2 exp(-(gamma-1)/theta); the Sobol rejection
  method is impractical at theta = 0.01), isotropic direction, then a Lorentz
  boost of each particle's 4-momentum to the beam gamma; uniform positions;
* Boris push with E = 0 (per-species q/m), positions wrapped into [0, L).

All random draws are counter-based per particle (Philox keyed by
(seed, stream)), so particle j's initial state depends on (seed, j) only and
not on N.  The GPU pusher (``trajgen/push.cu``) runs the same steps in FP32
arithmetic; the NumPy pusher here runs them in FP64.  The two agree
statistically, not bitwise: every test that compares the CUDA library with
the oracle hands both the same generated arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

L_BOX = 40.0


# ---------------------------------------------------------------------------
# counter-based random streams
# ---------------------------------------------------------------------------
def _stream(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


def uniforms(seed: int, stream: int, n: int) -> np.ndarray:
    """First n U[0,1) draws of stream (seed, stream); entry j depends on j only."""
    return _stream(seed, stream).random(n)


# ---------------------------------------------------------------------------
# static field
# ---------------------------------------------------------------------------
@dataclass
class FieldModes:
    ky: np.ndarray
    kz: np.ndarray
    psi: np.ndarray
    amp: np.ndarray
    L: float = L_BOX

    def B(self, y, z):
        """B = (0, dA/dz, -dA/dy) at points (y, z); returns (By, Bz)."""
        ph = np.multiply.outer(y, self.ky) + np.multiply.outer(z, self.kz) + self.psi
        s = np.sin(ph) * self.amp
        By = -(s * self.kz).sum(-1)
        Bz = (s * self.ky).sum(-1)
        return By, Bz


def make_field(seed: int, n_modes: int = 64, kmin: float = 0.3, kmax: float = 3.0,
               b_rms: float = 0.1, L: float = L_BOX) -> FieldModes:
    """Draw n_modes distinct periodic modes with |k| in [kmin, kmax]."""
    nmax = int(math.ceil(kmax * L / (2 * math.pi)))
    cand = []
    for ny in range(0, nmax + 1):
        for nz in range(-nmax, nmax + 1):
            if ny == 0 and nz <= 0:
                continue  # canonical half plane: no +-k duplicates
            kk = 2 * math.pi * math.hypot(ny, nz) / L
            if kmin <= kk <= kmax:
                cand.append((ny, nz))
    cand = np.array(cand, dtype=np.int64)
    if len(cand) < n_modes:
        raise ValueError("not enough periodic modes in the |k| band")
    rng = _stream(seed, 1000)
    pick = cand[rng.permutation(len(cand))[:n_modes]]
    ky = 2 * math.pi * pick[:, 0] / L
    kz = 2 * math.pi * pick[:, 1] / L
    psi = 2 * math.pi * _stream(seed, 1001).random(n_modes)
    k2 = ky ** 2 + kz ** 2
    a = b_rms / math.sqrt(0.5 * k2.sum())
    return FieldModes(ky=ky, kz=kz, psi=psi, amp=np.full(n_modes, a), L=L)


# ---------------------------------------------------------------------------
# initial conditions
# ---------------------------------------------------------------------------
def mj_momentum(uni: np.ndarray, theta: float) -> np.ndarray:
    """Rest-frame Maxwell-Juttner |u| by tabulated inverse CDF of u^2 e^{-(g-1)/theta}."""
    umax = math.sqrt((1.0 + 60.0 * theta) ** 2 - 1.0)
    grid = np.linspace(0.0, umax, 200001)
    g = np.sqrt(1.0 + grid ** 2)
    pdf = grid ** 2 * np.exp(-(g - 1.0) / theta)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    return np.interp(uni, cdf, grid)


def beam_particles(seed: int, N: int, gamma_beam: float, theta: float = 0.01,
                   L: float = L_BOX, first_index: int = 0):
    """Positions [3, N] and momenta u_{-1/2} [3, N] of two +-x beams."""
    idx = np.arange(first_index, first_index + N)
    s = int(seed)
    # counter-based: draw first_index + N values and keep the tail
    def U(stream):
        return uniforms(s, stream, first_index + N)[first_index:]
    x = np.stack([U(0) * L, U(1) * L, U(2) * L])
    umag = mj_momentum(U(3), theta)
    mu = 2.0 * U(4) - 1.0
    ph = 2.0 * math.pi * U(5)
    st = np.sqrt(np.maximum(0.0, 1.0 - mu ** 2))
    ur = np.stack([umag * mu, umag * st * np.cos(ph), umag * st * np.sin(ph)])
    gr = np.sqrt(1.0 + umag ** 2)
    sign = np.where(idx % 2 == 0, 1.0, -1.0)
    Gb = float(gamma_beam)
    bb = math.sqrt(1.0 - 1.0 / Gb ** 2) if Gb > 1.0 else 0.0
    ux = Gb * (ur[0] + sign * bb * gr)
    u = np.stack([ux, ur[1], ur[2]])
    return x, u


# ---------------------------------------------------------------------------
# Boris push (E = 0), FP64 NumPy version
# ---------------------------------------------------------------------------
def boris_push(x0, u0, qm, fieldm: FieldModes, dt: float, n_calls: int, L: float = L_BOX):
    """Return X, U of shape [n_calls, 3, N]: call s holds x_s and u_{s-1/2}.

    qm: charge-to-mass ratio per particle [N] (or scalar).
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    u = np.array(u0, dtype=np.float64, copy=True)
    N = x.shape[1]
    qm = np.broadcast_to(np.asarray(qm, dtype=np.float64), (N,))
    X = np.empty((n_calls, 3, N))
    U = np.empty((n_calls, 3, N))
    for s in range(n_calls):
        X[s] = x
        U[s] = u
        if s == n_calls - 1:
            break
        By, Bz = fieldm.B(x[1], x[2])
        g = np.sqrt(1.0 + (u * u).sum(0))
        f = 0.5 * dt * qm / g
        t = np.stack([np.zeros(N), f * By, f * Bz])
        t2 = (t * t).sum(0)
        sv = 2.0 * t / (1.0 + t2)
        up = u + np.cross(u, t, axis=0)
        u = u + np.cross(up, sv, axis=0)
        g = np.sqrt(1.0 + (u * u).sum(0))
        x = x + dt * u / g
        x = x - L * np.floor(x / L)
    return X, U


# ---------------------------------------------------------------------------
# observer directions
# ---------------------------------------------------------------------------
def healpix_centres(nside: int) -> np.ndarray:
    """HEALPix RING-scheme pixel centres [12 nside^2, 3] (Gorski et al. 2005)."""
    npix = 12 * nside * nside
    ncap = 2 * nside * (nside - 1)
    out = np.empty((npix, 3))
    for p in range(npix):
        if p < ncap:  # north polar cap
            i = int(math.floor(0.5 * (1.0 + math.sqrt(1.0 + 2.0 * p))))
            j = p + 1 - 2 * i * (i - 1)
            z = 1.0 - i * i / (3.0 * nside * nside)
            phi = math.pi / (2.0 * i) * (j - 0.5)
        elif p < npix - ncap:  # equatorial belt
            q = p - ncap
            i = q // (4 * nside) + nside
            j = q % (4 * nside) + 1
            s = (i - nside + 1) % 2
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * nside)
            phi = math.pi / (2.0 * nside) * (j - 0.5 * s)
        else:  # south polar cap
            q = npix - p - 1
            i = int(math.floor(0.5 * (1.0 + math.sqrt(1.0 + 2.0 * q))))
            j = 4 * i - (q - 2 * i * (i - 1))
            z = -(1.0 - i * i / (3.0 * nside * nside))
            phi = math.pi / (2.0 * i) * (j - 0.5)
        st = math.sqrt(max(0.0, 1.0 - z * z))
        out[p] = (st * math.cos(phi), st * math.sin(phi), z)
    return out


def axis_and_oblique_dirs() -> np.ndarray:
    """+-x, +-y, +-z and two oblique directions (1,1,0)/sqrt2, (1,1,1)/sqrt3."""
    d = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
         (1 / math.sqrt(2), 1 / math.sqrt(2), 0), (1 / math.sqrt(3),) * 3]
    return np.array(d, dtype=np.float64)


def paper_observers(axis=(1.0, 0.0, 0.0), perp=(0.0, 0.0, 1.0), count: int = 6) -> np.ndarray:
    """Six observers at angles m pi/10, m = 0..5, from the streaming axis
    ("0" head-on, "5" edge-on), in the plane spanned by axis and perp."""
    a = np.asarray(axis, float)
    b = np.asarray(perp, float)
    th = np.arange(count) * (math.pi / (2 * (count - 1)))
    return np.cos(th)[:, None] * a + np.sin(th)[:, None] * b


def log_grid(lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(np.linspace(math.log(lo), math.log(hi), n))


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    species: list            # [(count, charge, mass, gamma_beam)]
    n_calls: int             # PIC calls; samples = n_calls - 1
    dt: float
    dirs: np.ndarray
    grids: list
    windows: list            # [(s0, s1, species_mask, grid)]
    coherent: bool = False
    field_seed: int = 11
    particle_seed: int = 23
    theta: float = 0.01
    b_rms: float = 0.1
    L: float = L_BOX
    notes: str = ""

    @property
    def n_total(self) -> int:
        return int(sum(s[0] for s in self.species))

    def updates(self) -> int:
        """particle * sample * omega * direction updates over all windows."""
        tot = 0
        D = len(self.dirs)
        for (s0, s1, mask, g) in self.windows:
            n = sum(sp[0] for i, sp in enumerate(self.species) if (mask >> i) & 1)
            tot += n * (s1 - s0) * D * len(self.grids[g])
        return int(tot)

    def initial_state(self, first: int = 0, count: int | None = None):
        """x0, u_{-1/2} [3, N] and q/m [N] for particles [first, first+count)."""
        xs, us, qms = [], [], []
        off = 0
        for si, (cnt, q, m, gb) in enumerate(self.species):
            lo, hi = off, off + cnt
            off = hi
            a = max(lo, first)
            b = min(hi, first + (self.n_total if count is None else count))
            if b <= a:
                continue
            x, u = beam_particles(self.particle_seed + 7919 * si, b - a, gb, self.theta,
                                  self.L, first_index=a - lo)
            xs.append(x)
            us.append(u)
            qms.append(np.full(b - a, q / m))
        return np.concatenate(xs, 1), np.concatenate(us, 1), np.concatenate(qms)

    def field(self) -> FieldModes:
        return make_field(self.field_seed, b_rms=self.b_rms, L=self.L)

    def trajectory_numpy(self, first: int = 0, count: int | None = None, n_calls=None):
        x0, u0, qm = self.initial_state(first, count)
        return boris_push(x0, u0, qm, self.field(), self.dt,
                          self.n_calls if n_calls is None else n_calls, self.L)


def config(k: int, scale_particles: float = 1.0) -> Workload:
    """The five workloads (1-based), optionally with the particle counts scaled."""
    def n(c):
        return max(1, int(round(c * scale_particles)))
    if k == 1:
        return Workload("plain-fp64-1024e-2000s-1dir-256w", [(n(1024), -1.0, 1.0, 3.0)], 2001,
                        0.05, np.array([[0.0, 1.0, 0.0]]), [log_grid(0.1, 300.0, 256)],
                        [(0, 2000, 1, 0)])
    if k == 2:
        return Workload("fp64-scale-65536e-4096s-8dir-1024w", [(n(65536), -1.0, 1.0, 3.0)],
                        4097, 0.05, axis_and_oblique_dirs(), [log_grid(0.1, 1000.0, 1024)],
                        [(0, 4096, 1, 0)])
    if k == 3:
        return Workload("precision-1M-e-gamma10-4096s-8dir-1024w",
                        [(n(1048576), -1.0, 1.0, 10.0)], 4097, 0.05, axis_and_oblique_dirs(),
                        [log_grid(0.1, 1000.0, 1024)], [(0, 4096, 1, 0)])
    if k == 4:
        grids = [log_grid(0.01, 30.0, 512), log_grid(0.1, 300.0, 1024),
                 log_grid(0.1, 1000.0, 2048)]
        wins = [(0, 4096, 1, 2), (0, 2048, 1, 1), (1024, 1536, 1, 0),
                (0, 4096, 2, 1), (2048, 2560, 2, 0)]
        return Workload("batched-512Ke-32Kions-192dir-3grids",
                        [(n(524288), -1.0, 1.0, 3.0), (n(32768), 1.0, 16.0, 3.0)], 4097, 0.05,
                        healpix_centres(4), grids, wins)
    if k == 5:
        return Workload("learned-1024e-2000s-192dir-2048w", [(n(1024), -1.0, 1.0, 3.0)], 2001,
                        0.05, healpix_centres(4), [log_grid(0.1, 1000.0, 2048)],
                        [(0, 2000, 1, 0)])
    raise ValueError("workloads are numbered 1..5")


# ---------------------------------------------------------------------------
# initial state of the live two-stream PIC (Sec. 2.1 setup)
# ---------------------------------------------------------------------------
@dataclass
class TwoStream:
    """Two equal-density neutral beams streaming against each other along
    `axis` in a periodic 2D3V box of n x n cells of size d (Sec. 2.1: the
    filamentation setup, with the paper's reduced mass ratio 64 for the
    baryonic case, or pairs).  Every electron has a partner of the other
    species at the same position with the same bulk momentum, so the initial
    charge density vanishes identically; thermal momenta are drawn
    independently (Gaussian per component, spread u_th for electrons and
    u_th (m_partner / m_e)^(1/2) for partners: equal temperatures), and their
    current noise seeds the instability.  Densities follow the
    paper's normalisation: the relativistic electron plasma frequency
    (n_e / gamma)^(1/2) is 1 (n_e summed over both beams)."""
    n: int = 64
    d: float = 0.1
    dt: float = 0.05
    ppc: int = 4                # electron-partner pairs per cell and beam
    gamma: float = 3.0
    u_th: float = 0.01          # Gaussian thermal spread of each momentum component
    mass_ratio: float = 64.0    # partner mass (1: pair plasma)
    axis: int = 0               # streaming axis (0 = x, out of the simulation plane)
    seed: int = 11

    @property
    def L(self) -> float:
        return self.n * self.d

    @property
    def n_particles(self) -> int:
        return 2 * 2 * self.ppc * self.n * self.n

    def particles(self):
        """x, u [3][N] and per-particle charge, mass, macro weight [N].  Order:
        the 2 ppc n^2 electrons (even index: beam +, odd: beam -), then their
        partners in the same order (partner i starts on electron i)."""
        ne = 2 * self.ppc * self.n * self.n
        L = self.L
        x = np.stack([uniforms(self.seed, c, ne) * L for c in range(3)])
        ue = np.stack([self.u_th * _stream(self.seed, 3 + c).standard_normal(ne) for c in range(3)])
        up = np.stack([self.u_th * math.sqrt(self.mass_ratio) *
                       _stream(self.seed, 6 + c).standard_normal(ne) for c in range(3)])
        gb = float(self.gamma)
        u0 = math.sqrt(gb * gb - 1.0)
        sign = np.where(np.arange(ne) % 2 == 0, 1.0, -1.0)   # beams alternate by index
        for u in (ue, up):
            u[self.axis] += sign * u0
        n_e = gb                                   # (n_e / gamma)^(1/2) = 1
        w = n_e * self.d * self.d / (2 * self.ppc)  # electrons per cell: 2 ppc
        X = np.concatenate([x, x], 1)
        U = np.concatenate([ue, up], 1)
        q = np.concatenate([-np.ones(ne), np.ones(ne)])
        m = np.concatenate([np.ones(ne), self.mass_ratio * np.ones(ne)])
        return X, U, q, m, np.full(2 * ne, w)
