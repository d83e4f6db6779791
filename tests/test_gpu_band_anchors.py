"""Anchor interval per frequency band (FP32 split path).

The offset phase w dphi of an update is rounded in FP32, |dphi| <= (K - 1) dt
inside an anchor block of K samples, so its rounding grows with w K.  Under a
phase budget b the context anchors the ring at the K that the highest frequency
needs (the longest of 8, 16, 32 with w_max (K - 1) dt 2^-24 <= b, 8 at least)
and lets each frequency tile take the longest such interval for its own highest
frequency, as a multiple of the ring's.  Checked here, on gamma = 10 electrons
(the precision workload's beams) and a grid whose three 256-frequency tiles get
K = 32, 16 and 8:

* every direction of every window against the oracle within the FP32 path's
  1e-4 relative L2;
* the top tile, at the ring's own K, reproduces the uniform K = 8 context (the
  same arithmetic, up to the order of the FP64 sums);
* each lower tile is as accurate against the oracle as the uniform context at
  the K it was given -- its blocks combine several ring blocks, with the ring
  anchors' offsets n . (r_a - r_A) added in float-float, at no loss;
* the precise-phase variant under a budget takes the precise phase only in the
  tiles that need it.
"""
import numpy as np
import pytest

import oracle
import trajgen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FIXED = {"variant": 1, "freq_per_lane": 8, "blocks_per_sm": 2}   # 256 frequencies per tile


def _band_K(wmax, dt, budget):
    for K in (32, 16):
        if wmax * (K - 1) * dt * 2.0 ** -24 <= budget:
            return K
    return 8


@pytest.fixture(scope="module")
def beams():
    w = trajgen.config(3, 128 / 1048576)
    X, U = w.trajectory_numpy(n_calls=2049)
    grid = trajgen.log_grid(10.0, 100.0, 768)
    wins = [(0, 2048, 1, 0), (37, 1990, 1, 0)]
    ref = oracle.spectra(X, U, w.dt, w.dirs, [grid], wins, [(X.shape[2], -1.0)], box_L=w.L)
    return w, X, U, grid, wins, ref


def _run(R, w, X, U, grid, wins, opts):
    with R.Radiation(w.dirs, [grid], w.dt, [(X.shape[2], -1.0, 1.0)], wins,
                     precision=R.RAD_FP32_SPLIT, box_L=w.L, options=opts) as r:
        r.accumulate_steps(0, torch.as_tensor(X, device="cuda"), torch.as_tensor(U, device="cuda"))
        return r.finalize(), r.options()


def test_anchor_interval_per_band(beams):
    import paper_1003_1140_gb300 as R
    w, X, U, grid, wins, ref = beams
    budget = 720 * w.dt * 2.0 ** -24                       # K = 32, 16, 8 on the three tiles
    tiles = [slice(256 * t, 256 * t + 256) for t in range(3)]
    Ks = [_band_K(np.abs(grid[s]).max(), w.dt, budget) for s in tiles]
    assert Ks == [32, 16, 8]
    band, o = _run(R, w, X, U, grid, wins, dict(FIXED, phase_budget=budget))
    assert o["anchor_K"] == 8 and abs(o["phase_budget"] - budget) < 1e-9
    uni = {K: _run(R, w, X, U, grid, wins, dict(FIXED, anchor_K=K))[0] for K in (8, 16, 32)}
    # without a budget, the fixed kernel choice keeps the one interval of 32
    assert _run(R, w, X, U, grid, wins, FIXED)[1]["anchor_K"] == 32
    for wi in range(len(wins)):
        e = ref[wi]
        for d in range(e.shape[0]):
            err = np.linalg.norm(band[wi][d] - e[d]) / np.linalg.norm(e[d])
            assert err <= 1e-4, (wi, d, err)
        top = tiles[2]
        np.testing.assert_allclose(band[wi][:, top], uni[8][wi][:, top], rtol=1e-9,
                                   atol=1e-12 * np.abs(e).max())
        for t, K in ((0, 32), (1, 16)):
            s = tiles[t]
            eb = np.linalg.norm(band[wi][:, s] - e[:, s], axis=1) / np.linalg.norm(e[:, s], axis=1)
            eu = np.linalg.norm(uni[K][wi][:, s] - e[:, s], axis=1) / np.linalg.norm(e[:, s], axis=1)
            print(f"window {wi} tile {t} (K {K}): per-band {eb.max():.2e}, uniform {eu.max():.2e}")
            assert np.all(eb <= 2.0 * eu + 1e-7), (wi, t, eb, eu)
            # and the tile's spectra are the uniform context's up to that accuracy
            db = np.linalg.norm(band[wi][:, s] - uni[K][wi][:, s], axis=1) / \
                np.linalg.norm(e[:, s], axis=1)
            assert np.all(db <= 2.0 * eu + 1e-7), (wi, t, db, eu)


def test_precise_phase_per_band(beams):
    """The precise-phase variant under a phase budget takes the precise phase only in
    the frequency tiles whose rounding bound at K = 32, w_max 31 dt 2^-24, exceeds the
    budget (here the upper two of three).  Those tiles equal the all-precise context's
    (the same arithmetic, up to the order of the FP64 sums); the lowest tile runs the
    SFU path and is as accurate against the oracle as the default context."""
    import paper_1003_1140_gb300 as R
    w, X, U, grid, wins, ref = beams
    budget = 3e-6
    tiles = [slice(256 * t, 256 * t + 256) for t in range(3)]
    bound = [np.abs(grid[s]).max() * 31 * w.dt * 2.0 ** -24 for s in tiles]
    assert [b > budget for b in bound] == [False, True, True]
    base = {"freq_per_lane": 8, "blocks_per_sm": 3}
    hyb, o = _run(R, w, X, U, grid, wins, dict(base, variant=3, phase_budget=budget))
    assert o["variant"] == 3 and o["anchor_K"] == 32
    allp, _ = _run(R, w, X, U, grid, wins, dict(base, variant=3))
    dflt, _ = _run(R, w, X, U, grid, wins, dict(base, variant=1, anchor_K=32))
    for wi in range(len(wins)):
        e = ref[wi]
        for d in range(e.shape[0]):
            err = np.linalg.norm(hyb[wi][d] - e[d]) / np.linalg.norm(e[d])
            assert err <= 1e-4, (wi, d, err)
        up = slice(256, 768)
        np.testing.assert_allclose(hyb[wi][:, up], allp[wi][:, up], rtol=1e-9,
                                   atol=1e-12 * np.abs(e).max())
        s = tiles[0]
        eh = np.linalg.norm(hyb[wi][:, s] - e[:, s], axis=1) / np.linalg.norm(e[:, s], axis=1)
        ed = np.linalg.norm(dflt[wi][:, s] - e[:, s], axis=1) / np.linalg.norm(e[:, s], axis=1)
        print(f"window {wi} SFU tile: per-band precise {eh.max():.2e}, default {ed.max():.2e}")
        assert np.all(eh <= 2.0 * ed + 1e-7), (wi, eh, ed)
    # a budget no tile exceeds leaves the SFU path everywhere
    _, o0 = _run(R, w, X, U, grid, wins, dict(base, variant=3, phase_budget=1e-4))
    assert o0["variant"] == 1


def test_phase_budget_must_not_be_negative():
    import paper_1003_1140_gb300 as R
    w = trajgen.config(3, 8 / 1048576)
    with pytest.raises(R.RadError):
        with R.Radiation(w.dirs, w.grids, w.dt, [(8, -1.0, 1.0)], w.windows,
                         precision=R.RAD_FP32_SPLIT, box_L=w.L,
                         options={"phase_budget": -1e-6}):
            pass
