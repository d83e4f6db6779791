"""The seeded input generator against the recipe it states (CPU): periodic
field modes with the requested rms |B| (exact on a grid fine enough for the
modes to be orthogonal) and zero divergence; the Maxwell-Juttner sampler's
mean gamma against its closed form K_1(1/theta)/K_2(1/theta) + 3 theta; the
boosted beams; counter-based draws (particle j's state does not depend on N);
and the E = 0 Boris push, which only rotates u."""
import math

import numpy as np
import pytest

import trajgen


def test_field_modes_periodic_distinct_and_rms():
    f = trajgen.make_field(seed=7, b_rms=0.2)
    L = f.L
    ny = f.ky * L / (2 * math.pi)
    nz = f.kz * L / (2 * math.pi)
    np.testing.assert_allclose(ny, np.round(ny), atol=1e-12)      # periodic in the box
    np.testing.assert_allclose(nz, np.round(nz), atol=1e-12)
    k = np.hypot(f.ky, f.kz)
    assert len(k) == 64 and k.min() >= 0.3 and k.max() <= 3.0
    pairs = {(int(round(a)), int(round(b))) for a, b in zip(ny, nz)}
    assert len(pairs) == 64
    assert not any((-a, -b) in pairs for a, b in pairs)          # no +-k duplicates
    # |n| <= 20 per axis, so a 64-point grid resolves every product of two modes
    g = (np.arange(64) + 0.5) * L / 64
    Y, Z = np.meshgrid(g, g, indexing="ij")
    By, Bz = f.B(Y, Z)
    assert np.mean(By ** 2 + Bz ** 2) == pytest.approx(0.04, rel=1e-12)
    # B = curl(A_x x) has zero divergence: dBy/dy + dBz/dz, term by term
    ph = np.multiply.outer(Y, f.ky) + np.multiply.outer(Z, f.kz) + f.psi
    div = (np.cos(ph) * f.amp * (-f.kz * f.ky + f.ky * f.kz)).sum(-1)
    assert np.abs(div).max() <= 1e-15


def test_maxwell_juttner_mean_gamma():
    scipy_special = pytest.importorskip("scipy.special")
    theta = 0.01
    u = trajgen.mj_momentum(trajgen.uniforms(3, 0, 400000), theta)
    g = np.sqrt(1.0 + u * u)
    x = 1.0 / theta
    exact = scipy_special.kve(1, x) / scipy_special.kve(2, x) + 3.0 * theta
    se = g.std() / math.sqrt(len(g))
    assert abs(g.mean() - exact) <= 4 * se + 1e-6


def test_beams_boosted_and_counter_based():
    x, u = trajgen.beam_particles(seed=11, N=20000, gamma_beam=3.0, theta=0.01)
    assert np.all((x >= 0) & (x < trajgen.L_BOX))
    g = np.sqrt(1.0 + (u * u).sum(0))
    even, odd = u[0, 0::2], u[0, 1::2]
    assert np.all(even > 0) and np.all(odd < 0)                    # +x and -x beams
    # boosted mean gamma = gamma_beam * <gamma_rest> (the boost mixes in the
    # rest-frame u_x, whose mean is zero)
    assert g.mean() == pytest.approx(3.0 * (1.0 + 1.5 * 0.01), rel=2e-3)
    # particle j's state depends on (seed, j) only
    x2, u2 = trajgen.beam_particles(seed=11, N=7, gamma_beam=3.0, theta=0.01, first_index=100)
    np.testing.assert_array_equal(x2, x[:, 100:107])
    np.testing.assert_array_equal(u2, u[:, 100:107])


def test_boris_push_only_rotates_u():
    w = trajgen.Workload("t", [(40, -1.0, 1.0, 3.0), (8, 1.0, 16.0, 3.0)], 301, 0.05,
                         np.array([[0.0, 1.0, 0.0]]), [trajgen.log_grid(1.0, 2.0, 4)],
                         [(0, 300, 3, 0)], b_rms=0.3)
    X, U = w.trajectory_numpy()
    assert X.shape == U.shape == (301, 3, 48)
    umag = np.linalg.norm(U, axis=1)
    np.testing.assert_allclose(umag, np.broadcast_to(umag[0], umag.shape), rtol=1e-12)
    assert np.all((X >= 0) & (X < w.L))
    assert np.abs(U[-1] - U[0]).max() > 1e-3                       # the field did act


def test_log_grid():
    g = trajgen.log_grid(0.1, 1000.0, 5)
    np.testing.assert_allclose(g, [0.1, 1.0, 10.0, 100.0, 1000.0], rtol=1e-14)
