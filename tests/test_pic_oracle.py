"""Pins of the FP64 reference PIC (oracle/pic.py) against what the mathematics
fixes: the Boris rotation angle, exact interpolation of linear fields at each
component's staggered points, the exact discrete dispersion of vacuum waves on
the Yee grid, exact discrete charge continuity of the current deposition,
Gauss's law over a run, and the cold-beam filamentation growth rate."""
import math

import numpy as np
import pytest

import trajgen
from oracle import pic


def test_boris_gyration_angle():
    """Uniform B along x, E = 0: each step turns (u_y, u_z) by
    -2 atan(q B dt / (2 m gamma)) (the Boris rotation's exact angle) at fixed |u|."""
    rng = np.random.default_rng(1)
    u = np.array([[0.3], [1.7], [-0.8]])
    B0, qm, dt = 0.7, -1.0, 0.05
    gam = math.sqrt(1.0 + float(np.sum(u * u)))
    z0 = u[1, 0] + 1j * u[2, 0]
    Bp = np.array([[B0], [0.0], [0.0]])
    Ep = np.zeros((3, 1))
    N = 1000
    for _ in range(N):
        u = pic.boris(u, Ep, Bp, qm, dt)
    theta = -2.0 * math.atan(qm * B0 * dt / (2.0 * gam))
    z_exp = z0 * np.exp(1j * N * theta)
    assert abs(u[1, 0] + 1j * u[2, 0] - z_exp) <= 1e-10 * abs(z0)
    assert abs(u[0, 0] - 0.3) <= 1e-14
    assert rng is not None


def test_boris_electric_kick():
    """B = 0: u advances by (q/m) E dt exactly."""
    u = np.array([[0.1], [0.2], [0.3]])
    E = np.array([[0.5], [-1.0], [2.0]])
    out = pic.boris(u, E, np.zeros((3, 1)), 2.0, 0.25)
    assert np.allclose(out, u + 2.0 * 0.25 * E, rtol=0, atol=1e-15)


def test_gather_reproduces_linear_fields_at_staggered_points():
    """Each component set to a linear function of its own Yee coordinates is
    returned exactly at any interior particle position: this fixes the
    half-cell offsets of all six components."""
    g = pic.Grid(16, 0.25, 0.1)
    n, d = g.n, g.d
    j = np.arange(n)[:, None] * np.ones((1, n))
    k = np.ones((n, 1)) * np.arange(n)[None, :]
    offs = {"Ex": (0, 0), "Ey": (0.5, 0), "Ez": (0, 0.5),
            "Bx": (0.5, 0.5), "By": (0, 0.5), "Bz": (0.5, 0)}
    coef = {c: (1.0 + i, 0.3 * (i + 1), -0.2 * (i + 2)) for i, c in enumerate(offs)}
    F = {c: coef[c][0] + coef[c][1] * (j + oy) * d + coef[c][2] * (k + oz) * d
         for c, (oy, oz) in offs.items()}
    E = np.stack([F["Ex"], F["Ey"], F["Ez"]])
    B = np.stack([F["Bx"], F["By"], F["Bz"]])
    rng = np.random.default_rng(2)
    y = rng.uniform(2 * d, g.L - 2 * d, 50)
    z = rng.uniform(2 * d, g.L - 2 * d, 50)
    Ep, Bp = pic.gather(E, B, y, z, g)
    for i, c in enumerate(("Ex", "Ey", "Ez")):
        assert np.allclose(Ep[i], coef[c][0] + coef[c][1] * y + coef[c][2] * z, rtol=0, atol=1e-12), c
    for i, c in enumerate(("Bx", "By", "Bz")):
        assert np.allclose(Bp[i], coef[c][0] + coef[c][1] * y + coef[c][2] * z, rtol=0, atol=1e-12), c


@pytest.mark.parametrize("case", ["Ex_Bz_y", "Ez_Bx_y", "Ex_By_z", "Ey_Bx_z"])
def test_vacuum_wave_follows_discrete_dispersion(case):
    """A plane wave initialised as the Yee grid's discrete eigenmode keeps its
    shape and advances with the discrete frequency
    sin(w dt/2)/dt = sin(k d/2)/d.  B at integer steps is the mean of the
    half-step Yee values, hence the factor cos(w dt/2)."""
    g = pic.Grid(32, 0.1, 0.05)
    n, d, dt = g.n, g.d, g.dt
    kw = 2 * math.pi * 3 / g.L
    w = 2.0 / dt * math.asin(dt / d * math.sin(kw * d / 2))
    c = math.cos(w * dt / 2)
    idx = np.arange(n)
    E = np.zeros((3, n, n))
    B = np.zeros((3, n, n))
    # (E component, B component, axis, sign of B relative to E for propagation along +axis)
    comp = {"Ex_Bz_y": (0, 2, 0, -1.0), "Ez_Bx_y": (2, 0, 0, 1.0),
            "Ex_By_z": (0, 1, 1, 1.0), "Ey_Bx_z": (1, 0, 1, -1.0)}[case]
    ei, bi, ax, sg = comp
    shape = (n, 1) if ax == 0 else (1, n)
    E[ei] = np.cos(kw * idx * d).reshape(shape) * np.ones((n, n))
    B[bi] = sg * c * np.cos(kw * (idx + 0.5) * d).reshape(shape) * np.ones((n, n))
    empty = np.zeros((3, 0))
    x, u = empty.copy(), empty.copy()
    z = np.zeros(0)
    N = 200
    for _ in range(N):
        x, u, E, B, _ = pic.step(x, u, E, B, z, z + 1.0, z, g)
    exp = np.cos(kw * idx * d - w * N * dt).reshape(shape) * np.ones((n, n))
    assert np.abs(E[ei] - exp).max() <= 1e-11
    others = [i for i in range(3) if i != ei]
    assert np.abs(E[others]).max() <= 1e-14


def test_deposit_satisfies_discrete_continuity():
    """(rho^{n+1} - rho^n)/dt + div J = 0 on every node for arbitrary moves of
    under one cell, across the periodic boundary too; the out-of-plane
    current sums to sum q w v_x."""
    g = pic.Grid(12, 0.5, 0.1)
    rng = np.random.default_rng(3)
    N = 300
    y0 = rng.uniform(0, g.L, N)
    z0 = rng.uniform(0, g.L, N)
    y1 = y0 + rng.uniform(-0.95, 0.95, N) * g.d
    z1 = z0 + rng.uniform(-0.95, 0.95, N) * g.d
    qw = rng.normal(size=N)
    vx = rng.uniform(-0.9, 0.9, N)
    J = pic.deposit(y0, z0, y1, z1, vx, qw, g)
    r0 = pic.charge_density(y0, z0, qw, g)
    r1 = pic.charge_density(np.mod(y1, g.L), np.mod(z1, g.L), qw, g)
    divJ = (J[1] - np.roll(J[1], 1, 0)) / g.d + (J[2] - np.roll(J[2], 1, 1)) / g.d
    resid = (r1 - r0) / g.dt + divJ
    assert np.abs(resid).max() <= 1e-11 * np.abs(divJ).max()
    assert abs(J[0].sum() * g.d * g.d - np.sum(qw * vx)) <= 1e-12 * np.sum(np.abs(qw * vx))


def _run(ts, steps, record=None):
    X, U, q, m, w = ts.particles()
    g = pic.Grid(ts.n, ts.d, ts.dt)
    E = np.zeros((3, ts.n, ts.n))
    B = np.zeros((3, ts.n, ts.n))
    for s in range(steps):
        X, U, E, B, _ = pic.step(X, U, E, B, q, m, w, g)
        if record is not None:
            record(s + 1, X, U, E, B)
    return X, U, E, B, q, m, w, g


def test_gauss_law_holds_over_a_run():
    """Neutral beams start with rho = 0 and E = 0; the charge-conserving
    deposition keeps div E = rho on the nodes as the species separate."""
    ts = trajgen.TwoStream(n=16, ppc=2, gamma=3.0, u_th=0.05, seed=4)
    X, U, E, B, q, m, w, g = _run(ts, 40)
    rho = pic.charge_density(X[1], X[2], q * w, g)
    assert np.abs(rho).max() > 1e-3          # the species have separated
    assert np.abs(pic.div_E(E, g.d) - rho).max() <= 1e-10 * np.abs(rho).max()


def test_plasma_oscillation_frequency():
    """Cold electrons on a lattice (quiet start) over immobile ions, with a
    small velocity perturbation of the longest wavelength: the field
    oscillates at the plasma frequency (n_e q^2 / m)^(1/2).  At k d = 0.2 the
    shape-factor and leapfrog corrections are below 0.3%."""
    n, d, dt = 32, 0.1, 0.05
    g = pic.Grid(n, d, dt)
    pps = 2
    s = (np.arange(n * pps) + 0.5) * d / pps
    Y, Z = np.meshgrid(s, s, indexing="ij")
    Y, Z = Y.ravel(), Z.ravel()
    N = Y.size
    ne = 2.0
    k = 2 * math.pi / g.L
    xe = np.stack([np.zeros(N), Y, Z])
    ue = np.stack([np.zeros(N), 1e-5 * np.sin(k * Y), np.zeros(N)])
    X, U = np.concatenate([xe, xe], 1), np.concatenate([ue, 0 * ue], 1)
    q = np.concatenate([-np.ones(N), np.ones(N)])
    m = np.concatenate([np.ones(N), 1e12 * np.ones(N)])
    w = np.full(2 * N, ne * d * d / pps ** 2)
    E = np.zeros((3, n, n))
    B = np.zeros((3, n, n))
    ey = []
    for _ in range(360):
        X, U, E, B, _ = pic.step(X, U, E, B, q, m, w, g)
        ey.append(np.fft.fft(E[1].mean(axis=1))[1].imag)
    ey = np.array(ey)
    t = dt * np.arange(1, len(ey) + 1)
    i = np.nonzero(np.sign(ey[1:]) != np.sign(ey[:-1]))[0]
    zc = t[i] + dt * ey[i] / (ey[i] - ey[i + 1])
    omega = math.pi * (len(zc) - 1) / (zc[-1] - zc[0])
    assert len(zc) >= 7
    assert abs(omega / math.sqrt(ne) - 1.0) <= 5e-3, omega


def test_filamentation_growth_rate_and_energy():
    """Beams along x (out of the plane): only the filamentation mode (k
    perpendicular to the beams) exists.  Cold symmetric beams, all species
    with the same velocity, give
        w^4 - w^2 (k^2 + W^2/g^3) - k^2 b^2 W^2/g = 0,  W^2 = sum of the
    species' squared plasma frequencies,
    so Gamma(k) rises to b W / g^(1/2) at large k.  The magnetic energy of the
    noise-seeded run grows at twice the rate of its dominant modes; the CIC
    shape factor weakens the short-wavelength modes, so the measured rate
    lies somewhat below 2 Gamma(inf) -- the band [0.75, 1.05] x 2 Gamma(inf)
    excludes a plasma frequency off by 2^(1/2) or a missing gamma.  Total
    energy (fields + kinetic) is conserved to 1e-4 of the beam energy."""
    ts = trajgen.TwoStream(n=32, d=0.1, dt=0.05, ppc=4, gamma=3.0, u_th=1e-3, seed=5)
    g = pic.Grid(ts.n, ts.d, ts.dt)
    eb, et = [], []

    def rec(s, X, U, E, B):
        eb.append(0.5 * float(np.sum(B * B)))
        ef, ek = pic.energies(U, E, B, m, w, g.d)
        et.append(ef + ek)
    X, U, q, m, w = ts.particles()
    _run(ts, 100, record=rec)
    t = ts.dt * np.arange(1, len(eb) + 1)
    lg = np.log(np.array(eb))
    i0, i1 = np.searchsorted(t, 1.5), np.searchsorted(t, 3.5)
    rate = np.polyfit(t[i0:i1], lg[i0:i1], 1)[0]
    g0 = ts.gamma
    b0 = math.sqrt(1 - 1 / g0 ** 2)
    W2 = g0 * (1.0 + 1.0 / ts.mass_ratio)          # n_e = gamma, partners add n_e / m_p
    gam_inf = b0 * math.sqrt(W2 / g0)
    assert 0.75 * 2 * gam_inf <= rate <= 1.05 * 2 * gam_inf, (rate, 2 * gam_inf)
    assert eb[-1] > 1e2 * eb[20]                   # several e-foldings observed
    assert abs(et[-1] - et[0]) <= 1e-4 * et[0]
