"""FP64 reference of the small two-stream PIC that drives the in-situ coupling.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing in the product path).

Sec. 2.1 sets up the filamentation instability as two equal-density neutral
plasma beams streaming through each other in a fully periodic box, in the PIC
units c = m_e = q_e = 1 with time in 1/omega_pe; Sec. 2.2 collects the
radiation from the particle histories as the simulation runs.  The paper's
production code (PhotonPlasma, 6th-order solver, spline shapes) is not given;
this reference states the textbook second-order scheme the GPU PIC implements:

  * 2D3V: fields and positions in the (y, z) plane vary, nothing depends on x;
    particles carry all three position components (x drifts freely) and all
    three momentum components.  Square cells of size d, n x n cells, box
    L = n d, periodic in x, y and z.
  * Yee staggering (node (j, k) at (j d, k d)): E_x at (j, k), E_y at
    (j + 1/2, k), E_z at (j, k + 1/2), B_x at (j + 1/2, k + 1/2), B_y at
    (j, k + 1/2), B_z at (j + 1/2, k).  Units with eps0 = mu0 = c = 1:
        dB/dt = -curl E,   dE/dt = curl B - J.
    Step n -> n + 1: B^{n+1/2} = B^n - dt/2 curl E^n;
    E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2}); B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1}.
  * Gather: linear (cloud-in-cell) weights from each component's own staggered
    points to the particle position at step n.
  * Push: relativistic Boris rotation (Boris 1970; Birdsall & Langdon Sec. 15-4):
    half electric kick, magnetic rotation with t = (q dt / 2 m gamma^-) B,
    s = 2 t / (1 + t^2), half electric kick; x^{n+1} = x^n + dt u^{n+1/2} / gamma^{n+1/2}.
  * Deposit: charge-conserving current of a linear-shape particle moving from
    its old to its new position (Esirkepov 2001, 2D form with the
    out-of-plane current): with S0, S1 the CIC node weights before and after
    the move and dS = S1 - S0,
        W_y = dS_y (S0_z + S1_z) / 2,  W_z = (S0_y + S1_y) dS_z / 2,
        W_x = S0_y S0_z + dS_y S0_z / 2 + S0_y dS_z / 2 + dS_y dS_z / 3,
    J_y(j + 1/2, k) = -(q w / (d dt)) sum_{j' <= j} W_y(j', k) (and J_z alike),
    J_x(j, k) = (q w / d^2) v_x W_x, so that
        (rho^{n+1} - rho^n)/dt + div J = 0 on the nodes exactly.

Particles: arrays x, u [3][N]; per particle charge q, mass m and macro weight
w (charge density q w / d^2 per particle on the 2D grid).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Grid:
    n: int          # cells per axis (y and z)
    d: float        # cell size
    dt: float

    @property
    def L(self) -> float:
        return self.n * self.d


def cic(s):
    """Lower node index and fraction of a coordinate s in cell units."""
    i = np.floor(s)
    return i.astype(np.int64), s - i


def gather(E, B, y, z, g: Grid):
    """E and B [3][N] at the particles from their staggered Yee points."""
    n = g.n
    sy, sz = y / g.d, z / g.d
    jn, fyn = cic(sy)            # nodes
    jh, fyh = cic(sy - 0.5)      # half points (j + 1/2)
    kn, fzn = cic(sz)
    kh, fzh = cic(sz - 0.5)

    def interp(F, j, fy, k, fz):
        j0, j1 = j % n, (j + 1) % n
        k0, k1 = k % n, (k + 1) % n
        return ((1 - fy) * (1 - fz) * F[j0, k0] + fy * (1 - fz) * F[j1, k0] +
                (1 - fy) * fz * F[j0, k1] + fy * fz * F[j1, k1])

    Ep = np.stack([interp(E[0], jn, fyn, kn, fzn),      # E_x (j, k)
                   interp(E[1], jh, fyh, kn, fzn),      # E_y (j+1/2, k)
                   interp(E[2], jn, fyn, kh, fzh)])     # E_z (j, k+1/2)
    Bp = np.stack([interp(B[0], jh, fyh, kh, fzh),      # B_x (j+1/2, k+1/2)
                   interp(B[1], jn, fyn, kh, fzh),      # B_y (j, k+1/2)
                   interp(B[2], jh, fyh, kn, fzn)])     # B_z (j+1/2, k)
    return Ep, Bp


def boris(u, Ep, Bp, qm, dt):
    """u^{n-1/2} -> u^{n+1/2} (relativistic Boris)."""
    um = u + 0.5 * qm * dt * Ep
    gm = np.sqrt(1.0 + np.sum(um * um, axis=0))
    t = (0.5 * qm * dt / gm) * Bp
    s = 2.0 * t / (1.0 + np.sum(t * t, axis=0))
    up = um + np.cross(um, t, axis=0)
    uplus = um + np.cross(up, s, axis=0)
    return uplus + 0.5 * qm * dt * Ep


def node_weights(s, base):
    """CIC weights of coordinates s (cell units) on the 4 nodes base .. base + 3."""
    i, f = cic(s)
    W = np.zeros((4,) + s.shape)
    a = i - base
    for off, wt in ((0, 1.0 - f), (1, f)):
        idx = a + off
        for c in range(4):
            W[c] += np.where(idx == c, wt, 0.0)
    return W


def deposit(y0, z0, y1, z1, vx, qw, g: Grid):
    """Charge-conserving current J [3][n][n] of the moves (y0, z0) -> (y1, z1)
    (unwrapped, each less than one cell per axis)."""
    n, d, dt = g.n, g.d, g.dt
    s0y, s0z, s1y, s1z = y0 / d, z0 / d, y1 / d, z1 / d
    by = np.floor(s0y).astype(np.int64) - 1
    bz = np.floor(s0z).astype(np.int64) - 1
    S0y, S1y = node_weights(s0y, by), node_weights(s1y, by)
    S0z, S1z = node_weights(s0z, bz), node_weights(s1z, bz)
    dSy, dSz = S1y - S0y, S1z - S0z
    J = np.zeros((3, n, n))
    for a in range(4):
        for b in range(4):
            Wy = dSy[a] * (S0z[b] + S1z[b]) * 0.5
            Wz = (S0y[a] + S1y[a]) * dSz[b] * 0.5
            Wx = (S0y[a] * S0z[b] + 0.5 * dSy[a] * S0z[b] + 0.5 * S0y[a] * dSz[b] +
                  dSy[a] * dSz[b] / 3.0)
            j, k = (by + a) % n, (bz + b) % n
            np.add.at(J[0], (j, k), qw * vx * Wx / (d * d))
            # J_y at (j + 1/2, k): running sum over a' <= a of W_y(a', b)
            cy = np.zeros_like(qw)
            cz = np.zeros_like(qw)
            for a2 in range(a + 1):
                cy += dSy[a2] * (S0z[b] + S1z[b]) * 0.5
            for b2 in range(b + 1):
                cz += (S0y[a] + S1y[a]) * dSz[b2] * 0.5
            np.add.at(J[1], (j, k), -qw * cy / (d * dt))
            np.add.at(J[2], (j, k), -qw * cz / (d * dt))
    return J


def curl_E(E, d):
    """curl E on the B points."""
    Ex, Ey, Ez = E
    up = lambda F, ax: np.roll(F, -1, axis=ax)   # F at index + 1
    # d/dx = 0: curl E = (dEz/dy - dEy/dz, dEx/dz, -dEx/dy)
    cx = (up(Ez, 0) - Ez) / d - (up(Ey, 1) - Ey) / d      # at (j+1/2, k+1/2)
    cy = (up(Ex, 1) - Ex) / d                            # at (j, k+1/2)
    cz = -(up(Ex, 0) - Ex) / d                           # at (j+1/2, k)
    return np.stack([cx, cy, cz])


def curl_B(B, d):
    """curl B on the E points."""
    Bx, By, Bz = B
    dn = lambda F, ax: np.roll(F, 1, axis=ax)    # F at index - 1
    # d/dx = 0: curl B = (dBz/dy - dBy/dz, dBx/dz, -dBx/dy)
    cx = (Bz - dn(Bz, 0)) / d - (By - dn(By, 1)) / d      # at (j, k)
    cy = (Bx - dn(Bx, 1)) / d                            # at (j+1/2, k)
    cz = -(Bx - dn(Bx, 0)) / d                           # at (j, k+1/2)
    return np.stack([cx, cy, cz])


def step(x, u, E, B, q, m, w, g: Grid):
    """One PIC step: (x^n, u^{n-1/2}, E^n, B^n) -> (x^{n+1}, u^{n+1/2}, E^{n+1}, B^{n+1})."""
    Ep, Bp = gather(E, B, x[1], x[2], g)
    u1 = boris(u, Ep, Bp, q / m, g.dt)
    gam = np.sqrt(1.0 + np.sum(u1 * u1, axis=0))
    v = u1 / gam
    x1 = x + g.dt * v
    J = deposit(x[1], x[2], x1[1], x1[2], v[0], q * w, g)
    x1 = np.mod(x1, g.L)
    Bh = B - 0.5 * g.dt * curl_E(E, g.d)
    E1 = E + g.dt * (curl_B(Bh, g.d) - J)
    B1 = Bh - 0.5 * g.dt * curl_E(E1, g.d)
    return x1, u1, E1, B1, J


def charge_density(y, z, qw, g: Grid):
    """rho on the nodes (CIC)."""
    n = g.n
    j, fy = cic(y / g.d)
    k, fz = cic(z / g.d)
    rho = np.zeros((n, n))
    for dj, wy in ((0, 1 - fy), (1, fy)):
        for dk, wz in ((0, 1 - fz), (1, fz)):
            np.add.at(rho, ((j + dj) % n, (k + dk) % n), qw * wy * wz / (g.d * g.d))
    return rho


def div_E(E, d):
    """div E on the nodes."""
    return (E[1] - np.roll(E[1], 1, axis=0)) / d + (E[2] - np.roll(E[2], 1, axis=1)) / d


def energies(u, E, B, m, w, d):
    """Field energy (E^2 + B^2)/2 summed over cells x d^2, and kinetic energy
    sum of w m (gamma - 1).  B should be the integer-time field."""
    ef = 0.5 * (np.sum(E * E) + np.sum(B * B)) * d * d
    gam = np.sqrt(1.0 + np.sum(u * u, axis=0))
    return ef, float(np.sum(w * m * (gam - 1.0)))
