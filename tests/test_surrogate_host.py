"""Host-side pieces of the learned surrogate, on the CPU: the HEALPix direction
grid (Gorski et al. 2005), the sparse subset (a literal subset of the dense
grid), the log/standardise transform, the interpolation baseline the network is
judged against, and the error measures."""
import math

import numpy as np
import pytest

import trajgen
from paper_1003_1140_gb300 import surrogate as su


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_healpix_centres_closed_forms(nside):
    c = trajgen.healpix_centres(nside)
    assert c.shape == (12 * nside * nside, 3)
    np.testing.assert_allclose(np.linalg.norm(c, axis=1), 1.0, rtol=0, atol=1e-14)
    # the grid is symmetric under z -> -z and under rotations by pi/2 about z
    np.testing.assert_allclose(c.sum(0), 0.0, atol=1e-12)
    # ring latitudes: z = 1 - i^2 / (3 nside^2) on the polar caps (i < nside),
    # 4/3 - 2 i / (3 nside) on the belt; each polar ring holds 4 i pixels
    zs = np.round(c[:, 2], 12)
    for i in range(1, nside):
        z = 1.0 - i * i / (3.0 * nside * nside)
        assert np.sum(np.isclose(zs, z, atol=1e-12)) == 4 * i
        assert np.sum(np.isclose(zs, -z, atol=1e-12)) == 4 * i
    for i in range(nside, 3 * nside + 1):
        z = 4.0 / 3.0 - 2.0 * i / (3.0 * nside)
        assert np.sum(np.isclose(zs, z, atol=1e-12)) == 4 * nside
    if nside == 1:
        # the 12 base pixels: 4 at z = 2/3, 4 on the equator, 4 at z = -2/3
        for z in (2 / 3, 0.0, -2 / 3):
            assert np.sum(np.isclose(c[:, 2], z, atol=1e-12)) == 4


def test_sparse_set_is_a_literal_subset_of_the_dense_grid():
    spec = su.SurrogateSpec()
    om = spec.omegas()
    fi = spec.sparse_omega_index()
    assert len(om) == 2048 and len(fi) == 64 and np.all(np.diff(fi) == 32) and fi[0] == 0
    np.testing.assert_array_equal(om[fi], trajgen.log_grid(0.1, 1000.0, 2048)[::32])
    si = spec.sparse_dir_index()
    dense = spec.dense_dirs()
    assert len(dense) == 192 and len(si) == 12 and len(set(si.tolist())) == 12
    # every base-pixel centre has one of its nearest dense directions in the
    # sparse set (a centre between two rings has two equally near ones)
    base = trajgen.healpix_centres(1)
    for b in base:
        cos = dense @ b
        assert np.any(cos[si] >= cos.max() - 1e-12)


def test_normaliser_round_trip_and_floor():
    rng = np.random.default_rng(3)
    data = 10.0 ** rng.uniform(-8, 2, size=(5, 4, 7))
    n = su.Normaliser(data)
    z = n.forward(data)
    assert z.shape == (5, 28) and z.dtype == np.float32
    np.testing.assert_allclose(z.mean(0), 0.0, atol=1e-5)
    np.testing.assert_allclose(n.inverse(z).reshape(data.shape), data, rtol=1e-5)
    # zeros are taken at the floor, not as -inf
    zero = np.zeros((1, 4, 7))
    assert np.all(np.isfinite(n.forward(zero)))


def test_interpolation_baseline_is_exact_for_power_laws_and_nearest_in_direction():
    spec = su.SurrogateSpec(dirs_subset=48)
    om = spec.omegas()
    si = spec.sparse_dir_index()
    fi = spec.sparse_omega_index()
    amp = 1.0 + np.arange(len(si), dtype=float)             # one amplitude per sparse direction
    slope = -1.7
    sparse = (amp[:, None] * om[fi][None, :] ** slope)[None]
    out = su.interpolate_baseline(spec, sparse)[0]
    dense = spec.dense_dirs()
    nearest = np.argmax(dense @ dense[si].T, axis=1)
    inside = om <= om[fi[-1]]
    expect = amp[nearest][:, None] * om[None, :] ** slope
    np.testing.assert_allclose(out[:, inside], expect[:, inside], rtol=1e-12)
    # beyond the last sparse frequency the interpolation holds the last value
    np.testing.assert_allclose(out[:, ~inside], expect[:, [np.flatnonzero(inside)[-1]]].repeat(
        int((~inside).sum()), axis=1), rtol=1e-12)


def test_error_measures():
    rng = np.random.default_rng(4)
    true = 10.0 ** rng.uniform(-3, 1, size=(3, 5, 11))
    lin, dex = su.errors(true, true)
    assert np.all(lin == 0.0) and np.all(dex == 0.0)
    lin, dex = su.errors(2.0 * true, true)
    np.testing.assert_allclose(lin, 1.0, rtol=1e-12)
    np.testing.assert_allclose(dex, math.log10(2.0), rtol=1e-12)
