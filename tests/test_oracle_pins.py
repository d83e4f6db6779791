"""Pins for the FP64 CPU oracle (no GPU).

Each test checks the oracle against something other than itself: closed forms
derived by hand for special geometries, trigonometric identities, the
discrete Parseval identity, the textbook synchrotron single-pass spectrum and
the Lienard power, and exact invariants.  A dropped term, a wrong sign, a
wrong power of (1 - n.beta), a transposed cross product or a shifted sample
index fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle

PI = math.pi


def geom_sum(x, m0, M):
    """sum_{m=m0}^{m0+M-1} exp(i x m), closed form."""
    x = np.asarray(x, dtype=np.float64)
    num = 1.0 - np.exp(1j * x * M)
    den = 1.0 - np.exp(1j * x)
    return np.exp(1j * x * m0) * num / den


# ---------------------------------------------------------------------------
# (a) uniform motion radiates nothing, bitwise
# ---------------------------------------------------------------------------
def test_uniform_motion_is_exactly_zero():
    rng = np.random.default_rng(1)
    N, nc, dt = 5, 40, 0.05
    u0 = rng.normal(size=(3, N)) * 2.0
    g = np.sqrt(1 + (u0 ** 2).sum(0))
    U = np.broadcast_to(u0, (nc, 3, N)).copy()
    X = np.stack([rng.uniform(0, 40, (3, N)) + s * dt * u0 / g for s in range(nc)])
    X = X - 40.0 * np.floor(X / 40.0)
    r, b, bd = oracle.samples(X, U, dt, 40.0)
    assert np.all(bd == 0.0)
    dirs = np.array([[1.0, 0, 0], [0, 0.6, 0.8], [-1.0, 0, 0]])
    om = np.array([0.1, 3.0, 300.0])
    for coh in (False, True):
        S = oracle.window_spectrum(r, b, bd, -np.ones(N), dt, dirs, om, 0, nc - 1, coherent=coh)
        assert np.all(S == 0.0)


# ---------------------------------------------------------------------------
# samples(): time-centring of beta, betadot and r
# ---------------------------------------------------------------------------
def test_beta_centring_pythagorean():
    # u alternates 4/3 (beta = 4/5) and 5/12 (beta = 5/13) along x, so
    # ubar = 7/8 for every sample and beta_m = (7/8)/sqrt(1 + 49/64) = 7/sqrt(113);
    # betadot_m = (beta_{m+1/2} - beta_{m-1/2})/dt = -+ (4/5 - 5/13)/dt = -+ (27/65)/dt.
    nc, dt = 9, 0.1
    U = np.zeros((nc, 3, 1))
    U[0::2, 0, 0] = 4.0 / 3.0
    U[1::2, 0, 0] = 5.0 / 12.0
    X = np.zeros((nc, 3, 1))
    r, b, bd = oracle.samples(X, U, dt)
    np.testing.assert_allclose(b[:, 0, 0], 7.0 / math.sqrt(113.0), rtol=1e-15)
    assert np.all(b[:, 1:, 0] == 0.0)
    expect = np.where(np.arange(nc - 1) % 2 == 0, -27.0 / 65.0, 27.0 / 65.0) / dt
    np.testing.assert_allclose(bd[:, 0, 0], expect, rtol=1e-14)


def test_positions_unwrapped_and_on_their_own_call():
    # straight line x_s = x0 + s d in a box of side 10, raw positions wrapped:
    # sample m must be at x0 + m d (the position of call m), unwrapped.
    nc, L = 60, 10.0
    x0 = np.array([1.0, 9.5, 5.0])
    d = np.array([0.7, -0.3, 0.05])
    line = x0[None, :] + np.arange(nc)[:, None] * d[None, :]
    X = (line - L * np.floor(line / L))[:, :, None]
    U = np.zeros_like(X)
    r, _, _ = oracle.samples(X, U, 0.05, L)
    np.testing.assert_allclose(r[:, :, 0], line[:-1], atol=1e-12)


def test_dipole_betadot_identity():
    # beta_{s-1/2} = b cos(w0 (s-1/2) dt) x  =>  betadot_m = -(2b/dt) sin(w0 m dt) sin(w0 dt/2)
    nc, dt, b, w0 = 300, 0.05, 0.3, 1.7
    s = np.arange(nc)
    beta_half = b * np.cos(w0 * (s - 0.5) * dt)
    U = np.zeros((nc, 3, 1))
    U[:, 0, 0] = beta_half / np.sqrt(1 - beta_half ** 2)
    X = np.zeros_like(U)
    _, _, bd = oracle.samples(X, U, dt)
    m = np.arange(nc - 1)
    expect = -(2 * b / dt) * np.sin(w0 * m * dt) * math.sin(w0 * dt / 2)
    np.testing.assert_allclose(bd[:, 0, 0], expect, atol=1e-12)
    assert np.all(bd[:, 1:, 0] == 0.0)


# ---------------------------------------------------------------------------
# field(): hand-derived V = n x ((n-beta) x betadot)/(1-n.beta)^2
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,beta,bdot,expect", [
    # n = z, beta = (0.3, 0, 0.5): n - beta = (-0.3, 0, 0.5), kappa = 0.5
    ((0, 0, 1), (0.3, 0, 0.5), (0, 1, 0), (0, -2.0, 0)),     # (n-b) x y = (-0.5, 0, -0.3)
    ((0, 0, 1), (0.3, 0, 0.5), (1, 0, 0), (-2.0, 0, 0)),     # (n-b) x x = (0, 0.5, 0)
    ((0, 0, 1), (0.3, 0, 0.5), (0, 0, 1), (-1.2, 0, 0)),     # (n-b) x z = (0, 0.3, 0)
    # n = x, beta = (0.5, 0.3, 0): (n-b) x z = (-0.3, -0.5, 0); x cross it = (0, 0, -0.5)
    ((1, 0, 0), (0.5, 0.3, 0), (0, 0, 1), (0, 0, -2.0)),
    # receding: n = z, beta = (0, 0, -0.5), kappa = 1.5: z x (1.5 y) = -1.5 x; / 2.25
    ((0, 0, 1), (0, 0, -0.5), (1, 0, 0), (-2.0 / 3.0, 0, 0)),
])
def test_field_hand_derived(n, beta, bdot, expect):
    V = oracle.field(np.array(n, float), np.array(beta, float), np.array(bdot, float))
    np.testing.assert_allclose(V, expect, atol=1e-15)


# ---------------------------------------------------------------------------
# amplitude(): exact geometric sums for prescribed samples with kappa != 1
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("edir,W", [((0, 1, 0), (0, -2.0, 0)), ((1, 0, 0), (-2.0, 0, 0)),
                                    ((0, 0, 1), (-1.2, 0, 0))])
def test_amplitude_oblique_closed_form(edir, W):
    # beta_m = (0.3, 0, 0.5) constant, r_m = beta m dt, betadot_m = b sin(w0 m dt) e, n = z.
    # Then phi_m = m dt - 0.5 m dt = 0.5 m dt and V_m = b sin(w0 m dt) W, so
    # A(w) = q dt b W sum_m sin(w0 m dt) e^{i w m dt/2}
    #      = q dt b W [G(w dt/2 + w0 dt) - G(w dt/2 - w0 dt)] / (2i).
    dt, b, w0, q = 0.05, 0.2, 2.3, -1.0
    ns, m0, m1 = 400, 37, 351
    beta0 = np.array([0.3, 0.0, 0.5])
    m = np.arange(ns)
    r = (beta0[None, :] * (m * dt)[:, None])[:, :, None]
    beta = np.broadcast_to(beta0[None, :, None], (ns, 3, 1)).copy()
    bd = (b * np.sin(w0 * m * dt))[:, None, None] * np.array(edir, float)[None, :, None]
    om = np.array([0.01, 0.7, 4.7, 19.0, 123.0])
    A = oracle.amplitude(r, beta, bd, 0, m0, m1, dt, q, np.array([0, 0, 1.0]), om)
    M = m1 - m0
    s = (geom_sum(om * dt / 2 + w0 * dt, m0, M) - geom_sum(om * dt / 2 - w0 * dt, m0, M)) / 2j
    expect = q * dt * b * s[:, None] * np.array(W)[None, :]
    np.testing.assert_allclose(A, expect, rtol=1e-11, atol=1e-13 * np.abs(expect).max())


def test_dipole_spectrum_through_whole_chain():
    # beta_{s-1/2} = b cos(w0 (s-1/2) dt) x, particle at the origin, n = y:
    # kappa = 1, phi_m = m dt, V_m = -betadot_m = (2b/dt) sin(w0 m dt) sin(w0 dt/2) x, so
    # S = |q 2b sin(w0 dt/2) sum_m sin(w0 m dt) e^{i w m dt}|^2 / (4 pi^2).
    nc, dt, b, w0 = 801, 0.05, 0.05, 1.3
    s = np.arange(nc)
    bh = b * np.cos(w0 * (s - 0.5) * dt)
    U = np.zeros((nc, 3, 2))
    U[:, 0, :] = (bh / np.sqrt(1 - bh ** 2))[:, None]
    X = np.zeros_like(U)
    om = np.linspace(0.2, 3.0, 29)
    s0, s1 = 100, 700
    M = s1 - s0
    ssum = (geom_sum(om * dt + w0 * dt, s0, M) - geom_sum(om * dt - w0 * dt, s0, M)) / 2j
    single = np.abs(2 * b * math.sin(w0 * dt / 2) * ssum) ** 2 / (4 * PI ** 2)
    r, be, bd = oracle.samples(X, U, dt)
    for q, coh, factor in [(-1.0, False, 2.0), (-1.0, True, 4.0), (2.0, False, 8.0)]:
        S = oracle.window_spectrum(r, be, bd, np.full(2, q), dt, np.array([[0, 1.0, 0]]), om,
                                   s0, s1, coherent=coh)
        np.testing.assert_allclose(S[0], factor * single, rtol=1e-9, atol=1e-12 * single.max())
    # the line sits at w0 for b << 1
    S = oracle.window_spectrum(r, be, bd, np.full(2, -1.0), dt, np.array([[0, 1.0, 0]]),
                               np.linspace(0.5, 2.5, 201), s0, s1)
    assert abs(np.linspace(0.5, 2.5, 201)[np.argmax(S[0])] - w0) < 0.011


# ---------------------------------------------------------------------------
# (d) discrete Parseval: uniform phase spacing h makes |A|^2 a trigonometric
# polynomial of degree < M in w h, whose mean over P >= M equispaced points of
# one period 2 pi / h equals sum_m |a_m|^2 exactly.
# ---------------------------------------------------------------------------
def test_discrete_parseval_prefactor():
    dt, b, w0, q = 0.04, 0.3, 3.1, -1.0
    ns = 250
    beta0 = np.array([0.3, 0.0, 0.5])            # n = z: phi_m = 0.5 m dt, h = dt/2
    m = np.arange(ns)
    r = (beta0[None, :] * (m * dt)[:, None])[:, :, None]
    beta = np.broadcast_to(beta0[None, :, None], (ns, 3, 1)).copy()
    bd = (b * np.sin(w0 * m * dt))[:, None, None] * np.array([0, 1.0, 0])[None, :, None]
    h = dt / 2
    P = 2 * ns
    om = np.arange(P) * (2 * PI / h) / P
    S = oracle.window_spectrum(r, beta, bd, np.array([q]), dt, np.array([[0, 0, 1.0]]), om, 0, ns)
    integral = S[0].mean() * (2 * PI / h)                    # int over one period of S dw
    # |V_m| = 2 b |sin(w0 m dt)| (hand-derived W = (0, -2, 0)); a_m = q V_m dt
    sum_a2 = np.sum((q * dt * 2 * b * np.sin(w0 * m * dt)) ** 2)
    expect = (2 * PI / h) * sum_a2 / (4 * PI ** 2)
    np.testing.assert_allclose(integral, expect, rtol=1e-11)


# ---------------------------------------------------------------------------
# (b) synchrotron: single-pass spectrum of a relativistic electron on a Boris
# circle in uniform B against Jackson's closed form in K_{2/3}, K_{1/3}
# (Classical Electrodynamics eq. 14.79) and, integrated over elevation, the
# synchrotron function F(x) = x int_x^inf K_{5/3} (Jackson 14.91; Rybicki &
# Lightman Sec. 6.4).
# ---------------------------------------------------------------------------
def _boris_circle(gamma, B0, dt):
    """Electron (q/m = -1) in B = B0 z, velocity -x at call 0, one full turn."""
    u = math.sqrt(gamma ** 2 - 1)
    alpha = 2 * math.atan(B0 * dt / (2 * gamma))    # Boris rotation per step
    nsteps = int(round(2 * PI / alpha))
    nc = nsteps + 1
    X = np.zeros((nc, 3, 1))
    U = np.zeros((nc, 3, 1))
    ang = -PI - alpha / 2
    uu = np.array([u * math.cos(ang), u * math.sin(ang), 0.0])
    x = np.zeros(3)
    for s in range(nc):
        X[s, :, 0] = x
        U[s, :, 0] = uu
        g = math.sqrt(1 + uu @ uu)
        t = np.array([0, 0, -0.5 * dt * B0 / g])
        sv = 2 * t / (1 + t @ t)
        up = uu + np.cross(uu, t)
        uu = uu + np.cross(up, sv)
        x = x + dt * uu / math.sqrt(1 + uu @ uu)
    return X, U, nsteps, u / B0


def _jackson_single_pass(w, theta, gamma, rho):
    from scipy.special import kv
    a = 1.0 / gamma ** 2 + theta ** 2
    xi = w * rho / 3.0 * a ** 1.5
    return (1.0 / (3 * PI ** 2)) * (w * rho) ** 2 * a ** 2 * (
        kv(2.0 / 3.0, xi) ** 2 + theta ** 2 / a * kv(1.0 / 3.0, xi) ** 2)


@pytest.fixture(scope="module")
def synchrotron_samples():
    gamma, B0, dt = 20.0, 1.0, 0.002
    X, U, ns, rho = _boris_circle(gamma, B0, dt)
    r, b, bd = oracle.samples(X, U, dt)
    return dict(gamma=gamma, rho=rho, dt=dt, ns=ns, r=r, b=b, bd=bd)


def test_synchrotron_single_pass(synchrotron_samples):
    pytest.importorskip("scipy")
    d = synchrotron_samples
    gamma, rho = d["gamma"], d["rho"]
    wc = 1.5 * gamma ** 3 / rho
    om = wc * np.array([0.05, 0.1, 0.3, 0.6, 1.0, 2.0])
    for th in (0.0, 0.5 / gamma, 1.0 / gamma):
        n = np.array([[math.cos(th), 0.0, math.sin(th)]])
        S = oracle.window_spectrum(d["r"], d["b"], d["bd"], np.array([-1.0]), d["dt"], n, om,
                                   0, d["ns"])[0]
        J = _jackson_single_pass(om, th, gamma, rho)
        np.testing.assert_allclose(S, J, rtol=0.03)


def test_synchrotron_function_F(synchrotron_samples):
    pytest.importorskip("scipy")
    from scipy.integrate import quad
    from scipy.special import kv
    d = synchrotron_samples
    gamma, rho = d["gamma"], d["rho"]
    wc = 1.5 * gamma ** 3 / rho
    xs = np.array([0.1, 0.3, 1.0, 2.0])
    om = wc * xs
    # integrate the single-pass spectrum over elevation (Gauss-Legendre in theta)
    tmax = 6.0 / gamma
    nodes, weights = np.polynomial.legendre.leggauss(48)
    th = nodes * tmax
    dirs = np.stack([np.cos(th), np.zeros_like(th), np.sin(th)], 1)
    S = oracle.window_spectrum(d["r"], d["b"], d["bd"], np.array([-1.0]), d["dt"], dirs, om,
                               0, d["ns"])
    per_turn = 2 * PI * (weights[:, None] * S).sum(0) * tmax
    F = np.array([x * quad(lambda t: kv(5.0 / 3.0, t), x, np.inf)[0] for x in xs])
    expect = math.sqrt(3.0) * gamma * F
    np.testing.assert_allclose(per_turn, expect, rtol=0.03)


# ---------------------------------------------------------------------------
# (d) energy over the sphere and frequency = time-integrated Lienard power
#     (2 q^2 / 3c) gamma^6 [betadot^2 - (beta x betadot)^2]
# ---------------------------------------------------------------------------
def test_lienard_sphere_integral():
    import trajgen
    gamma, dt, nc = 2.0, 0.02, 801
    u = math.sqrt(gamma ** 2 - 1)
    X = np.zeros((nc, 3, 1))
    U = np.zeros((nc, 3, 1))
    x = np.array([-7.0, 0.0, 0.0])
    uu = np.array([u, 0.0, 0.0])
    for s in range(nc):                       # electron through a Gaussian B_z bump
        X[s, :, 0] = x
        U[s, :, 0] = uu
        g = math.sqrt(1 + uu @ uu)
        Bz = 1.0 * math.exp(-(x[0] / 1.0) ** 2)
        t = np.array([0, 0, -0.5 * dt * Bz / g])
        sv = 2 * t / (1 + t @ t)
        up = uu + np.cross(uu, t)
        uu = uu + np.cross(up, sv)
        x = x + dt * uu / math.sqrt(1 + uu @ uu)
    r, b, bd = oracle.samples(X, U, dt)
    ns = nc - 1
    dirs = trajgen.healpix_centres(8)
    om = np.linspace(0.0, 60.0, 481)
    S = oracle.window_spectrum(r, b, bd, np.array([-1.0]), dt, dirs, om, 0, ns)
    per_dir = np.trapezoid(S, om, axis=1)
    total = per_dir.sum() * 4 * PI / len(dirs)
    bb = b[:, :, 0]
    bdd = bd[:, :, 0]
    g2 = 1.0 / (1.0 - (bb ** 2).sum(1))
    cr = np.cross(bb, bdd)
    lienard = np.sum((2.0 / 3.0) * g2 ** 3 * ((bdd ** 2).sum(1) - (cr ** 2).sum(1))) * dt
    np.testing.assert_allclose(total, lienard, rtol=0.02)


# ---------------------------------------------------------------------------
# invariants of the definition
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_traj():
    import trajgen
    w = trajgen.config(1, 6 / 1024)
    X, U = w.trajectory_numpy(n_calls=161)
    return w, X, U


def test_invariants_permutation_and_conjugation(small_traj):
    w, X, U = small_traj
    N = X.shape[2]
    dirs = np.array([[0, 1.0, 0], [0.6, 0, 0.8]])
    om = np.array([0.3, 2.0, 17.0])
    base = oracle.spectra(X, U, w.dt, dirs, [om], [(3, 150, 1, 0)], [(N, -1.0)], box_L=w.L)[0]
    perm = np.random.default_rng(4).permutation(N)
    p = oracle.spectra(X[:, :, perm], U[:, :, perm], w.dt, dirs, [om], [(3, 150, 1, 0)],
                       [(N, -1.0)], box_L=w.L)[0]
    np.testing.assert_allclose(p, base, rtol=1e-12)
    neg = oracle.spectra(X, U, w.dt, dirs, [-om], [(3, 150, 1, 0)], [(N, -1.0)], box_L=w.L)[0]
    np.testing.assert_allclose(neg, base, rtol=1e-12)


def test_invariant_joint_rotation(small_traj):
    w, X, U = small_traj
    N = X.shape[2]
    r, _, _ = oracle.samples(X, U, w.dt, w.L)        # unwrapped, so rotation is legal
    Xu = np.concatenate([r, r[-1:] ], 0)
    Q, _ = np.linalg.qr(np.random.default_rng(7).normal(size=(3, 3)))
    dirs = np.array([[0, 1.0, 0], [0.6, 0, 0.8], [1.0, 0, 0]])
    om = np.array([0.3, 2.0, 17.0])
    a = oracle.spectra(Xu, U, w.dt, dirs, [om], [(0, 150, 1, 0)], [(N, -1.0)])[0]
    Xr = np.einsum("ij,sjn->sin", Q, Xu)
    Ur = np.einsum("ij,sjn->sin", Q, U)
    b = oracle.spectra(Xr, Ur, w.dt, dirs @ Q.T, [om], [(0, 150, 1, 0)], [(N, -1.0)])[0]
    np.testing.assert_allclose(b, a, rtol=1e-9)


def test_invariant_time_shift(small_traj):
    w, X, U = small_traj
    N = X.shape[2]
    dirs = np.array([[0, 1.0, 0], [1.0, 0, 0]])
    om = np.array([0.5, 5.0, 50.0])
    a = oracle.spectra(X, U, w.dt, dirs, [om], [(10, 140, 1, 0)], [(N, -1.0)], box_L=w.L)[0]
    k = 7  # the same history, 7 calls later
    Xs = np.concatenate([np.repeat(X[:1], k, 0), X], 0)
    Us = np.concatenate([np.repeat(U[:1], k, 0), U], 0)
    b = oracle.spectra(Xs, Us, w.dt, dirs, [om], [(10 + k, 140 + k, 1, 0)], [(N, -1.0)],
                       box_L=w.L)[0]
    np.testing.assert_allclose(b, a, rtol=1e-10)


def test_coherent_relations_and_charge_cancellation(small_traj):
    w, X, U = small_traj
    dirs = np.array([[0, 1.0, 0]])
    om = np.array([0.5, 5.0, 50.0])
    one = (X[:, :, :1], U[:, :, :1])
    inc = oracle.spectra(*one, w.dt, dirs, [om], [(0, 150, 1, 0)], [(1, -1.0)], box_L=w.L)[0]
    coh = oracle.spectra(*one, w.dt, dirs, [om], [(0, 150, 1, 0)], [(1, -1.0)], coherent=True,
                         box_L=w.L)[0]
    np.testing.assert_allclose(coh, inc, rtol=1e-13)
    two = (np.repeat(X[:, :, :1], 2, 2), np.repeat(U[:, :, :1], 2, 2))
    pair = oracle.spectra(*two, w.dt, dirs, [om], [(0, 150, 3, 0)], [(1, -1.0), (1, 1.0)],
                          coherent=True, box_L=w.L)[0]
    assert np.all(pair == 0.0)
    only_first = oracle.spectra(*two, w.dt, dirs, [om], [(0, 150, 1, 0)],
                                [(1, -1.0), (1, 1.0)], box_L=w.L)[0]
    np.testing.assert_allclose(only_first, inc, rtol=1e-13)


def test_window_additivity_in_amplitude(small_traj):
    w, X, U = small_traj
    r, b, bd = oracle.samples(X, U, w.dt, w.L)
    n = np.array([0.0, 0.6, 0.8])
    om = np.array([0.2, 4.0, 40.0])
    a = oracle.amplitude(r, b, bd, 2, 5, 90, w.dt, -1.0, n, om)
    c = oracle.amplitude(r, b, bd, 2, 90, 155, w.dt, -1.0, n, om)
    t = oracle.amplitude(r, b, bd, 2, 5, 155, w.dt, -1.0, n, om)
    np.testing.assert_allclose(a + c, t, rtol=1e-12, atol=1e-14 * np.abs(t).max())


def test_empty_window_and_empty_species():
    X = np.zeros((5, 3, 2))
    U = np.ones((5, 3, 2)) * np.array([0.1, 0.2, 0.3])[None, :, None]
    U[2] *= 2.0
    S = oracle.spectra(X, U, 0.1, np.array([[1.0, 0, 0]]), [np.array([1.0, 2.0])],
                       [(2, 2, 1, 0), (0, 4, 0, 0)], [(2, -1.0)])
    assert np.all(S[0] == 0.0) and np.all(S[1] == 0.0)


# ---------------------------------------------------------------------------
# precision: FP64 oracle vs a 50-digit evaluation on a tiny input (this
# re-evaluates the same sum, so it checks rounding, not the formula).
# ---------------------------------------------------------------------------
def test_fp64_rounding_against_mpmath(small_traj):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    w, X, U = small_traj
    r, b, bd = oracle.samples(X[:11, :, :2], U[:11, :, :2], w.dt, w.L)
    n = np.array([0.0, 0.6, 0.8])
    om = np.array([0.3, 30.0, 300.0])
    S = oracle.window_spectrum(r, b, bd, np.array([-1.0, -1.0]), w.dt, n[None, :], om, 0, 10)[0]
    for k, wk in enumerate(om):
        tot = mp.mpf(0)
        for j in range(2):
            A = [mp.mpc(0)] * 3
            for m in range(10):
                nv = [mp.mpf(float(v)) for v in n]
                bv = [mp.mpf(float(v)) for v in b[m, :, j]]
                dv = [mp.mpf(float(v)) for v in bd[m, :, j]]
                rv = [mp.mpf(float(v)) for v in r[m, :, j]]
                nmb = [nv[i] - bv[i] for i in range(3)]
                inner = [nmb[1] * dv[2] - nmb[2] * dv[1], nmb[2] * dv[0] - nmb[0] * dv[2],
                         nmb[0] * dv[1] - nmb[1] * dv[0]]
                outer = [nv[1] * inner[2] - nv[2] * inner[1], nv[2] * inner[0] - nv[0] * inner[2],
                         nv[0] * inner[1] - nv[1] * inner[0]]
                kap = 1 - sum(nv[i] * bv[i] for i in range(3))
                phi = m * mp.mpf(w.dt) - sum(nv[i] * rv[i] for i in range(3))
                e = mp.expj(mp.mpf(float(wk)) * phi)
                for i in range(3):
                    A[i] += -outer[i] / kap ** 2 * e * mp.mpf(w.dt)
            tot += sum(abs(a) ** 2 for a in A)
        ref = float(tot / (4 * mp.pi ** 2))
        assert abs(S[k] - ref) <= 1e-11 * abs(ref) + 1e-300


# ---------------------------------------------------------------------------
# sample selectors (regions / pitch cones)
# ---------------------------------------------------------------------------
def test_selector_box_and_cone_hand_cases():
    # three calls, one particle: x_0 = (1, 1, 1), x_1 = (5, 1, 1); u along x then along y
    X = np.zeros((3, 3, 1))
    X[0, :, 0] = [1, 1, 1]
    X[1, :, 0] = [5, 1, 1]
    U = np.zeros((3, 3, 1))
    U[0, 0, 0] = 2.0
    U[1, 0, 0] = 2.0
    U[2, 1, 0] = 2.0
    box = {"kind": "box", "lo": [0, 0, 0], "hi": [4, 4, 4]}
    assert oracle.selector_mask(X, U, box)[:, 0].tolist() == [True, False]
    # ubar_0 = (2, 0, 0): angle 0 from x; ubar_1 = (1, 1, 0): 45 degrees
    cone = {"kind": "cone", "axis": [1, 0, 0], "theta_c": 0.0, "dtheta": 0.1}
    assert oracle.selector_mask(X, U, cone)[:, 0].tolist() == [True, False]
    cone45 = {"kind": "cone", "axis": [3, 0, 0], "theta_c": math.pi / 4, "dtheta": 0.01}
    assert oracle.selector_mask(X, U, cone45)[:, 0].tolist() == [False, True]


def test_selector_everything_and_complementary_boxes(small_traj):
    w, X, U = small_traj
    N = X.shape[2]
    dirs = np.array([[0, 1.0, 0], [0.6, 0, 0.8]])
    om = np.array([0.5, 5.0, 50.0])
    full = oracle.spectra(X, U, w.dt, dirs, [om], [(0, 150, 1, 0)], [(N, -1.0)], box_L=w.L)[0]
    every = oracle.spectra(X, U, w.dt, dirs, [om], [(0, 150, 1, 0)], [(N, -1.0)], box_L=w.L,
                           selectors=[{"kind": "box", "lo": [-1] * 3, "hi": [41] * 3}],
                           window_selector=[0])[0]
    np.testing.assert_array_equal(every, full)
    # complementary halves x < 20, x >= 20: amplitudes (not spectra) add up
    r, b, bd = oracle.samples(X, U, w.dt, w.L)
    lo = oracle.selector_mask(X, U, {"kind": "box", "lo": [-1, -1, -1], "hi": [20, 41, 41]})
    hi = oracle.selector_mask(X, U, {"kind": "box", "lo": [20, -1, -1], "hi": [41, 41, 41]})
    assert np.all(lo ^ hi)
    for j in range(N):
        a = oracle.amplitude(r, b, bd * lo[:, None, :], j, 0, 150, w.dt, -1.0, dirs[1], om)
        c = oracle.amplitude(r, b, bd * hi[:, None, :], j, 0, 150, w.dt, -1.0, dirs[1], om)
        t = oracle.amplitude(r, b, bd, j, 0, 150, w.dt, -1.0, dirs[1], om)
        np.testing.assert_allclose(a + c, t, rtol=1e-12, atol=1e-14 * np.abs(t).max())


# ---------------------------------------------------------------------------
# sub-cycling
# ---------------------------------------------------------------------------
def test_subsamples_reduce_to_textbook_cases():
    # uniform motion: every sub-sample has betadot exactly zero and r on the line
    u0 = np.array([0.6, -0.2, 0.3])
    g = math.sqrt(1 + u0 @ u0)
    nc, dt, n = 6, 0.1, 4
    U = np.broadcast_to(u0[None, :, None], (nc, 3, 1)).copy()
    X = (np.arange(nc)[:, None] * dt * u0 / g)[:, :, None]
    r, b, bd = oracle.subsamples(X, U, dt, 0.0, n)
    assert np.all(bd == 0.0)
    t = ((np.arange(nc - 1)[:, None] + ((np.arange(n) + 0.5) / n - 0.5)[None, :]).reshape(-1))
    np.testing.assert_allclose(r[:, :, 0], t[:, None] * dt * u0 / g, atol=1e-15)
    # constant force along x from rest-ish: u linear in time, so betadot is the
    # derivative of u/sqrt(1+u^2) = 1/(1+u^2)^{3/2} * udot
    U = np.zeros((nc, 3, 1))
    U[:, 0, 0] = 0.2 + 0.5 * (np.arange(nc) - 0.5) * dt      # u_{s-1/2}
    X = np.zeros_like(U)
    r, b, bd = oracle.subsamples(X, U, dt, 0.0, n)
    ut = 0.2 + 0.5 * t * dt
    np.testing.assert_allclose(b[:, 0, 0], ut / np.sqrt(1 + ut ** 2), rtol=1e-14)
    np.testing.assert_allclose(bd[:, 0, 0], 0.5 / (1 + ut ** 2) ** 1.5, rtol=1e-13)


def _constant_force_history(ux0, uy, a, dt, nc):
    """Leapfrog states of u(t) = (ux0 + a t, uy, 0) (a constant force along x on a
    particle that also moves along y, so beta turns), with the exact positions
    x(t) = int beta dt: gamma = sqrt(1 + u^2) changes as dgamma/dt = a u_x / gamma, so
    r_x(t) = (gamma(t) - gamma(0)) / a and
    r_y(t) = (u_y / a) (asinh(u_x(t) / c) - asinh(u_x(0) / c)), c = sqrt(1 + u_y^2)."""
    c = math.sqrt(1.0 + uy * uy)

    def ux(t):
        return ux0 + a * t

    def pos(t):
        g = np.sqrt(1.0 + ux(t) ** 2 + uy * uy)
        g0 = math.sqrt(1.0 + ux0 * ux0 + uy * uy)
        return np.stack([(g - g0) / a, (uy / a) * (np.arcsinh(ux(t) / c) - math.asinh(ux0 / c)),
                         np.zeros_like(g)])

    s = np.arange(nc) * dt
    X = pos(s).T[:, :, None].copy()                       # x_s at t = s dt
    U = np.zeros((nc, 3, 1))
    U[:, 0, 0] = ux(s - 0.5 * dt)                          # u_{s-1/2}
    U[:, 1, 0] = uy
    return X, U, pos


@pytest.mark.parametrize("uy", [0.0, 1.3])
def test_subsample_positions_follow_the_exact_path(uy):
    """Sec. 2.2 sub-cycling: with u exactly linear in time the sub-sample positions
    must be the exact path integral r(t) = r_m + int_{t_m}^{t} beta dt' at every
    sub-sample time (m + tau_k) dt.  Simpson's rule over a step of |tau| dt <= dt / 2
    is exact to h^5 max|beta''''| / 2880 ~ 1e-11 here, so a 1e-10 bound fails for a
    trapezoid rule (error ~ h^3 beta'' ~ 1e-5), for beta(tau / 2) taken at tau, or
    for a wrong sub-sample time."""
    dt, nc, n, a = 0.1, 7, 5, 0.5
    X, U, pos = _constant_force_history(-0.4, uy, a, dt, nc)
    r, b, bd = oracle.subsamples(X, U, dt, 0.0, n)
    tau = (np.arange(n) + 0.5) / n - 0.5
    t = ((np.arange(nc - 1)[:, None] + tau[None, :]) * dt).reshape(-1)
    exact = pos(t).T
    np.testing.assert_allclose(r[:, :, 0], exact, rtol=0, atol=1e-10)
    # beta and betadot of the same path (u = u(t), betadot = d(u/gamma)/dt)
    u = np.stack([-0.4 + a * t, np.full_like(t, uy), np.zeros_like(t)], 1)
    g = np.sqrt(1.0 + (u * u).sum(1, keepdims=True))
    np.testing.assert_allclose(b[:, :, 0], u / g, rtol=0, atol=1e-14)
    udot = np.array([a, 0.0, 0.0])
    bdot = udot / g - u * (u @ udot)[:, None] / g ** 3
    np.testing.assert_allclose(bd[:, :, 0], bdot, rtol=0, atol=1e-13)


def _circle_history(u0, omega, dt, nc):
    """Leapfrog states of uniform circular motion, u(t) = u0 (cos wt, sin wt, 0)
    (a uniform magnetic field), and its exact arc r(t) = (u0 / (gamma w)) (sin wt,
    1 - cos wt, 0)."""
    g = math.sqrt(1.0 + u0 * u0)

    def pos(t):
        return np.stack([u0 / (g * omega) * np.sin(omega * t),
                         u0 / (g * omega) * (1.0 - np.cos(omega * t)), np.zeros_like(t)])

    s = np.arange(nc) * dt
    th = omega * (s - 0.5 * dt)
    X = pos(s).T[:, :, None].copy()
    U = np.zeros((nc, 3, 1))
    U[:, 0, 0] = u0 * np.cos(th)                           # u_{s-1/2}
    U[:, 1, 0] = u0 * np.sin(th)
    return X, U, pos


def test_subsample_positions_on_a_circle():
    """Sec. 2.2 sub-cycling on a uniform circle (u turns at constant |u|).  (a) The
    sub-sample positions are r_m plus the integral of beta along the linearly
    interpolated u, here checked against adaptive quadrature of that integral (not
    Simpson's rule) to 1e-8: Simpson's error h^5 max|beta^(4)| / 2880 is ~1e-9 for
    this tight turn (|du/dt| = 3), a trapezoid rule's ~1e-5.  (b) They converge to
    the exact circular arc: halving dt divides the largest distance from the arc by
    at least 3.5 (8 measured: the interpolated u is second-order accurate and each
    sub-step integrates it over a fraction of dt)."""
    from scipy.integrate import quad
    u0, omega, n = 2.0, 1.5, 4
    err = []
    for dt in (0.1, 0.05):
        nc = int(round(0.6 / dt)) + 1
        X, U, pos = _circle_history(u0, omega, dt, nc)
        r, _, _ = oracle.subsamples(X, U, dt, 0.0, n)
        tau = (np.arange(n) + 0.5) / n - 0.5
        if dt == 0.1:
            for m in range(nc - 1):
                um, up = U[m, :, 0], U[m + 1, :, 0]
                ub, du = 0.5 * (um + up), up - um
                for k in range(n):
                    for c in range(2):
                        def bc(s, c=c):
                            uu = ub + (s / dt) * du
                            return uu[c] / math.sqrt(1.0 + uu @ uu)
                        q, _ = quad(bc, 0.0, tau[k] * dt, epsabs=1e-14, epsrel=1e-14)
                        assert abs(r[m * n + k, c, 0] - (X[m, c, 0] + q)) < 1e-8, (m, k, c)
        t = ((np.arange(nc - 1)[:, None] + tau[None, :]) * dt).reshape(-1)
        err.append(np.abs(r[:, :, 0] - pos(t).T).max())
    assert err[0] / err[1] >= 3.5, err


def test_subsample_position_pin_catches_a_trapezoid_rule():
    """The 1e-10 bound above is tight enough: the same sub-sample positions by a
    trapezoid rule over [0, tau] (weights 1/2, 1/2), or by Simpson's rule with the
    midpoint velocity taken at the end point, miss the exact path by far more."""
    dt, nc, n, a, uy = 0.1, 7, 5, 0.5, 1.3
    X, U, pos = _constant_force_history(-0.4, uy, a, dt, nc)
    r, _, _ = oracle.samples(X, U, dt, 0.0)
    tau = (np.arange(n) + 0.5) / n - 0.5
    ub = 0.5 * (U[:-1] + U[1:])
    du = U[1:] - U[:-1]

    def beta(uu):
        return uu / np.sqrt(1.0 + (uu * uu).sum(1, keepdims=True))

    t = ((np.arange(nc - 1)[:, None] + tau[None, :]) * dt)
    exact = np.stack([pos(t[:, k]).T for k in range(n)], 1)          # [m, k, 3]
    trap = np.stack([(r + dt * tau[k] * 0.5 * (beta(ub) + beta(ub + tau[k] * du)))[:, :, 0]
                     for k in range(n)], 1)
    late_mid = np.stack([(r + dt * (tau[k] / 6.0) * (beta(ub) + 4.0 * beta(ub + tau[k] * du)
                                                      + beta(ub + tau[k] * du)))[:, :, 0]
                         for k in range(n)], 1)
    assert np.abs(trap - exact).max() > 1e-7
    assert np.abs(late_mid - exact).max() > 1e-4


def test_subcycling_resolves_what_the_coarse_step_aliases():
    """A gamma = 3 circle sampled coarsely: sub-cycled spectra approach the spectrum of
    a 10x finer PIC step at frequencies above the coarse Nyquist frequency."""
    def circle(dt, nsteps):
        B0, u = 1.0, math.sqrt(8.0)
        X = np.zeros((nsteps + 1, 3, 1))
        U = np.zeros((nsteps + 1, 3, 1))
        x = np.zeros(3)
        uu = np.array([u, 0.0, 0.0])
        for s in range(nsteps + 1):
            X[s, :, 0] = x
            U[s, :, 0] = uu
            g = math.sqrt(1 + uu @ uu)
            tt = np.array([0, 0, -0.5 * dt * B0 / g])
            sv = 2 * tt / (1 + tt @ tt)
            up = uu + np.cross(uu, tt)
            uu = uu + np.cross(up, sv)
            x = x + dt * uu / math.sqrt(1 + uu @ uu)
        return X, U
    T = 12.0
    om = np.linspace(8.0, 60.0, 27)      # coarse dt = 0.2: Nyquist ~ pi/0.2 = 16
    n = np.array([[0.0, 1.0, 0.0]])
    Xf, Uf = circle(0.02, 600)
    fine = oracle.spectra(Xf, Uf, 0.02, n, [om], [(0, 600, 1, 0)], [(1, -1.0)])[0][0]
    Xc, Uc = circle(0.2, 60)
    coarse = oracle.spectra(Xc, Uc, 0.2, n, [om], [(0, 60, 1, 0)], [(1, -1.0)])[0][0]
    sub = oracle.spectra(Xc, Uc, 0.2, n, [om], [(0, 60, 1, 0)], [(1, -1.0)], subcycle=10)[0][0]
    e_coarse = np.linalg.norm(np.log(coarse / fine))
    e_sub = np.linalg.norm(np.log(sub / fine))
    assert e_sub < 0.5 * e_coarse, (e_sub, e_coarse)
