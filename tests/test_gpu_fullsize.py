"""Full-size and high-gamma parity.

* The FP64-at-scale workload at full size (65,536 electrons x 4096 samples x 8
  directions x 1024 omega): the FP64 GPU path against the oracle on 64 sampled
  output bins (two in every frequency tile of every direction) that the oracle
  computes over all particles, and the FP32 split path against the FP64 path
  on the whole spectra (the parity chain oracle <-> FP64 GPU <-> FP32 split).
* The precision workload's particles (two gamma = 10 beams, where
  1 - n.beta ~ 1/(2 gamma^2) makes the head-on directions sensitive to
  cancellation) with all 4096 samples, 8 directions and 1024 omega on 256
  particles, both precisions against the oracle.
* The precision workload's upper decade on 65,536 particles, bin by bin, by default,
  under a phase budget (anchor interval per frequency band) and with the precise
  phase, against the FP64 path.
* The batched workload's full structure (electrons + ions, 192 HEALPix
  directions, three grids of 512/1024/2048 omega, five uneven windows of
  512 to 4096 steps) fed one step per call through the per-step CUDA graphs
  and the autotuned persistent launch, on a particle sample, checked on 64
  sampled bins against the oracle.
"""
import numpy as np
import pytest

import oracle
import trajgen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sample_check(got, ref, what):
    """FP32 split path on sampled bins: relative L2 over the sample within the
    metric's 1e-4, and no single bin off by more than 5e-3 (a broken frequency or
    direction tile is off by O(1); single upper-decade bins of aliased spectra are
    small sums of large cancelling terms, where FP32 phases are least accurate)."""
    got, ref = np.asarray(got), np.asarray(ref)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    worst = np.max(np.abs(got - ref) / np.abs(ref))
    print(f"{what}: sampled-bin rel-L2 {rel:.2e}, worst bin {worst:.2e}")
    assert rel <= 1e-4, (what, rel)
    assert worst <= 5e-3, (what, worst)


def test_workload2_full_size_sampled_bins():
    import paper_1003_1140_gb300 as R
    from trajgen import gpu as tg
    w = trajgen.config(2)
    X, U = tg.trajectory_gpu(w)
    sp = [(s[0], s[1], s[2]) for s in w.species]
    S = {}
    for prec in (R.RAD_FP32_SPLIT, R.RAD_FP64):
        with R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows, precision=prec,
                         box_L=w.L) as r:
            r.accumulate_steps(0, X, U)
            S[prec] = r.finalize()[0]
        assert np.all(np.isfinite(S[prec])) and np.all(S[prec] >= 0)
    # FP32 split against FP64 at full size: the metric's comparison
    rel = np.linalg.norm(S[R.RAD_FP32_SPLIT] - S[R.RAD_FP64], axis=1) / \
        np.linalg.norm(S[R.RAD_FP64], axis=1)
    print("FP32 vs FP64 rel-L2 per direction", rel)
    assert rel.max() <= 1e-4
    Xh = X.cpu().numpy()
    Uh = U.cpu().numpy()
    del X, U
    torch.cuda.empty_cache()
    rb, bb, bdb = oracle.samples(Xh, Uh, w.dt, w.L)
    del Xh, Uh
    rng = np.random.default_rng(5)
    om = w.grids[0]
    # two bins in every 256-omega tile of every direction (tile = the FP32 kernel's
    # frequency tile, 8 per lane x 32 lanes)
    picks = [(d, 256 * t + int(k)) for d in range(len(w.dirs)) for t in range(4)
             for k in rng.choice(256, 2, replace=False)]
    q = np.full(w.n_total, w.species[0][1])
    ref = np.array([oracle.window_spectrum(rb, bb, bdb, q, w.dt, w.dirs[d:d + 1], om[k:k + 1],
                                           w.windows[0][0], w.windows[0][1])[0, 0]
                    for d, k in picks])
    g64 = np.array([S[R.RAD_FP64][d, k] for d, k in picks])
    np.testing.assert_allclose(g64, ref, rtol=1e-10, atol=0)
    g32 = np.array([S[R.RAD_FP32_SPLIT][d, k] for d, k in picks])
    _sample_check(g32, ref, "workload 2 FP32")


def test_gamma10_all_samples():
    import paper_1003_1140_gb300 as R
    w = trajgen.config(3, 256 / 1048576)
    X, U = w.trajectory_numpy()
    assert X.shape == (4097, 3, 256)
    sp = [(w.n_total, -1.0, 1.0)]
    ref = oracle.spectra(X, U, w.dt, w.dirs, w.grids, w.windows, [(w.n_total, -1.0)],
                         box_L=w.L)[0]
    Xd, Ud = torch.as_tensor(X, device="cuda"), torch.as_tensor(U, device="cuda")
    for prec, tol, opts in ((R.RAD_FP64, 1e-10, None), (R.RAD_FP32_SPLIT, 1e-4, None),
                            (R.RAD_FP32_SPLIT, 1e-4, {"variant": 2}),
                            (R.RAD_FP32_SPLIT, 1e-4, {"anchor_K": 8}),
                            (R.RAD_FP32_SPLIT, 1e-4, {"anchor_K": 32})):
        with R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows, precision=prec, box_L=w.L,
                         options=opts) as r:
            r.accumulate_steps(0, Xd, Ud)
            S = r.finalize()[0]
        for d in range(len(w.dirs)):
            e = np.linalg.norm(S[d] - ref[d]) / np.linalg.norm(ref[d])
            assert e <= tol, (prec, opts, d, e)


def test_gamma10_upper_decade_bins():
    """65,536 electrons of the precision workload (gamma = 10), all 4096 samples, 8
    directions, 1024 omega, against the FP64 GPU path bin by bin: the FP32 split path
    by default (anchor blocks of 32 samples), under a 2.1e-5-rad phase budget (blocks
    of 8 samples for the upper decade's frequency tile, 32 below) and with the precise
    phase.  Every spectrum within 1e-6 relative L2; in the upper decade the budget at
    least halves the default's worst bin, and the precise phase keeps every bin within
    1e-5."""
    import paper_1003_1140_gb300 as R
    from trajgen import gpu as tg
    w = trajgen.config(3, 65536 / 1048576)
    X, U = tg.trajectory_gpu(w)
    sp = [(w.n_total, -1.0, 1.0)]
    S = {}
    for name, prec, opts in (("fp64", R.RAD_FP64, None), ("default", R.RAD_FP32_SPLIT, None),
                             ("budget", R.RAD_FP32_SPLIT, {"phase_budget": 2.1e-5}),
                             ("precise", R.RAD_FP32_SPLIT, {"variant": R.RAD_VARIANT_PRECISE})):
        with R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows, precision=prec, box_L=w.L,
                         options=opts) as r:
            r.accumulate_steps(0, X, U)
            S[name] = r.finalize()[0]
            if name == "budget":
                assert r.options()["anchor_K"] == 8
    up = w.grids[0] >= 100.0
    assert up.sum() == 256
    ref = S["fp64"]
    worst = {}
    for name in ("default", "budget", "precise"):
        worst[name] = (np.abs(S[name] - ref) / ref)[:, up].max()
        rel = np.linalg.norm(S[name] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        print(f"{name}: upper-decade worst bin {worst[name]:.2e}, rel-L2 {rel.max():.2e}")
        assert rel.max() <= 1e-6
    assert worst["budget"] <= 0.6 * worst["default"]
    assert worst["precise"] <= 1e-5


def test_batched_workload4_full_structure_per_step_graphs():
    """Every window, direction and grid of the batched workload, one rad_accumulate per
    step (use_graph: each step's ingest, and at the closing steps the persistent
    accumulation launch, replayed as CUDA graphs), autotuned kernel, on 2048 electrons
    + 128 ions; 64 sampled (window, direction, omega) bins against the oracle."""
    import paper_1003_1140_gb300 as R
    from trajgen import gpu as tg
    w = trajgen.config(4, 2048 / 524288)
    assert [s[0] for s in w.species] == [2048, 128]
    X, U = tg.trajectory_gpu(w)
    sp = [(s[0], s[1], s[2]) for s in w.species]
    with R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows, precision=R.RAD_FP32_SPLIT,
                     box_L=w.L, options={"use_graph": 1}) as r:
        for s in range(X.shape[0]):
            r.accumulate(s, X[s], U[s])
        got = r.finalize()
        t = r.timing()
        assert r.options()["use_graph"] == 1
    assert t["accum_launches"] == 4          # closing steps 1536, 2048, 2560, 4096
    Xh, Uh = X.cpu().numpy(), U.cpu().numpy()
    rb, bb, bdb = oracle.samples(Xh, Uh, w.dt, w.L)
    counts = [s[0] for s in w.species]
    sp_index = np.repeat(np.arange(2), counts)
    q = np.repeat([s[1] for s in w.species], counts)
    rng = np.random.default_rng(11)
    picks = []
    for wi, (s0, s1, mask, g) in enumerate(w.windows):
        nb = 16 if wi < 4 else 0
        for _ in range(nb):
            picks.append((wi, int(rng.integers(192)), int(rng.integers(len(w.grids[g])))))
    assert len(picks) == 64
    ref, g32 = [], []
    for wi, d, k in picks:
        s0, s1, mask, g = w.windows[wi]
        inc = ((mask >> sp_index) & 1).astype(np.uint8)
        ref.append(oracle.window_spectrum(rb, bb, bdb, q, w.dt, w.dirs[d:d + 1],
                                          w.grids[g][k:k + 1], s0, s1, include=inc)[0, 0])
        g32.append(got[wi][d, k])
    _sample_check(g32, ref, "workload 4 structure")
