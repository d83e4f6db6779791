"""CUDA path (through the C ABI) against the FP64 CPU oracle on identical inputs.

Tolerances: FP64 GPU path within 1e-10 relative L2 of the oracle; FP32
split-phase path within 1e-4 relative L2 per (window, direction) spectrum.
Sizes span several particle tiles (8), frequency tiles (256 / 128) and
sample chunks (32 / 16), each with a ragged tail.
"""
import math

import numpy as np
import pytest

import oracle
import trajgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rad():
    import paper_1003_1140_gb300 as R
    return R


def relL2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def two_species():
    """29 electrons (gamma 3) + 11 ions (m = 16, q = +1), 301 calls."""
    w = trajgen.Workload("two-species", [(29, -1.0, 1.0, 3.0), (11, 1.0, 16.0, 3.0)], 301, 0.05,
                         np.array([[0.0, 1.0, 0.0], [1.0, 0, 0], [-1.0, 0, 0],
                                   [0.6, 0.0, 0.8], [1 / math.sqrt(3)] * 3]),
                         [trajgen.log_grid(0.1, 300.0, 300), np.linspace(0.5, 20.0, 37)],
                         [(0, 300, 3, 0), (17, 250, 1, 1), (100, 100, 3, 0), (33, 64, 2, 0)],
                         b_rms=0.3)
    X, U = w.trajectory_numpy()
    species = [(s[0], s[1]) for s in w.species]
    ref = {}
    for coh in (False, True):
        ref[coh] = oracle.spectra(X, U, w.dt, w.dirs, w.grids, w.windows, species,
                                  coherent=coh, box_L=w.L)
    return w, X, U, ref


def _run(w, X, U, precision, coherent=False, options=None, device_inputs=True, steps=True):
    R = _rad()
    sp = [(s[0], s[1], s[2]) for s in w.species]
    r = R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows,
                    mode=R.RAD_COHERENT if coherent else R.RAD_INCOHERENT,
                    precision=precision, box_L=w.L, options=options)
    if device_inputs:
        Xi = torch.as_tensor(X, device="cuda")
        Ui = torch.as_tensor(U, device="cuda")
    else:
        Xi, Ui = np.ascontiguousarray(X), np.ascontiguousarray(U)
    if steps:
        r.accumulate_steps(0, Xi, Ui)
    else:
        for s in range(X.shape[0]):
            r.accumulate(s, Xi[s], Ui[s])
    out = r.finalize()
    r.close()
    return out


def _check(got, ref, tol, per_direction):
    for g, e in zip(got, ref):
        assert g.shape == e.shape
        if not np.any(e):
            assert np.all(g == 0.0)
            continue
        if per_direction:
            for d in range(e.shape[0]):
                assert relL2(g[d], e[d]) <= tol, (d, relL2(g[d], e[d]))
        else:
            assert relL2(g, e) <= tol, relL2(g, e)


@pytest.mark.parametrize("coherent", [False, True])
def test_fp64_matches_oracle(two_species, coherent):
    R = _rad()
    w, X, U, ref = two_species
    got = _run(w, X, U, R.RAD_FP64, coherent)
    _check(got, ref[coherent], 1e-10, per_direction=True)


@pytest.mark.parametrize("coherent", [False, True])
@pytest.mark.parametrize("K", [8, 16, 32])
def test_fp32_split_matches_oracle(two_species, coherent, K):
    R = _rad()
    w, X, U, ref = two_species
    got = _run(w, X, U, R.RAD_FP32_SPLIT, coherent, options={"anchor_K": K})
    _check(got, ref[coherent], 1e-4, per_direction=True)


@pytest.mark.parametrize("variant,ft,mb", [(1, 16, 2), (1, 8, 3), (2, 8, 2), (2, 8, 3),
                                           (2, 16, 2), (1, 4, 4), (3, 8, 2), (3, 8, 3)])
@pytest.mark.parametrize("coherent", [False, True])
def test_fp32_split_kernel_variants(two_species, variant, ft, mb, coherent):
    """SFU-only, SFU + FMA-polynomial (MIX) and precise-phase kernels, 4, 8 or 16
    frequencies per thread, built for 2, 3 or 4 resident blocks per SM."""
    R = _rad()
    w, X, U, ref = two_species
    got = _run(w, X, U, R.RAD_FP32_SPLIT, coherent,
               options={"variant": variant, "freq_per_lane": ft, "blocks_per_sm": mb})
    _check(got, ref[coherent], 1e-4, per_direction=True)


@pytest.mark.parametrize("precision", [0, 1])
def test_host_inputs_and_single_steps_agree(two_species, precision):
    w, X, U, _ = two_species
    a = _run(w, X, U, precision, device_inputs=True, steps=True)
    b = _run(w, X, U, precision, device_inputs=False, steps=False)
    for g, e in zip(a, b):
        np.testing.assert_allclose(g, e, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("precision", [0, 1])
def test_defer_matches_eager(two_species, precision):
    w, X, U, _ = two_species
    a = _run(w, X, U, precision)
    b = _run(w, X, U, precision, options={"defer": 1})
    for g, e in zip(a, b):
        np.testing.assert_allclose(g, e, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("precision", [0, 1])
def test_uniform_motion_is_exactly_zero_on_gpu(precision):
    R = _rad()
    rng = np.random.default_rng(3)
    N, nc, dt = 13, 70, 0.05
    u0 = rng.normal(size=(3, N))
    g = np.sqrt(1 + (u0 ** 2).sum(0))
    U = np.ascontiguousarray(np.broadcast_to(u0, (nc, 3, N)))
    X = np.stack([rng.uniform(0, 40, (3, N)) + s * dt * u0 / g for s in range(nc)])
    X = np.ascontiguousarray(X - 40.0 * np.floor(X / 40.0))
    for coh in (R.RAD_INCOHERENT, R.RAD_COHERENT):
        with R.Radiation(trajgen.axis_and_oblique_dirs(), [trajgen.log_grid(0.1, 300, 50)], dt,
                         [(N, -1.0)], [(0, nc - 1, 1, 0)], mode=coh, precision=precision,
                         box_L=40.0) as r:
            r.accumulate_steps(0, X, U)
            S = r.finalize()[0]
        assert np.all(S == 0.0)


def test_finalize_twice_and_reset(two_species):
    R = _rad()
    w, X, U, ref = two_species
    sp = [(s[0], s[1], s[2]) for s in w.species]
    with R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows, precision=R.RAD_FP64, box_L=w.L,
                     options={"defer": 1}) as r:
        for _ in range(2):
            r.accumulate_steps(0, X, U)
            a = r.finalize()
            b = r.finalize()
            for g, e, o in zip(a, b, ref[False]):
                np.testing.assert_array_equal(g, e)
                if np.any(o):
                    assert relL2(g, o) <= 1e-10
            r.reset()


def test_error_codes(two_species):
    R = _rad()
    w, X, U, _ = two_species
    sp = [(s[0], s[1], s[2]) for s in w.species]
    with R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows, precision=R.RAD_FP64, box_L=w.L) as r:
        with pytest.raises(R.RadError) as ei:
            r.accumulate(1, X[1], U[1])
        assert ei.value.code == -4
        r.accumulate_steps(0, X[:10], U[:10])
        with pytest.raises(R.RadError) as ei:
            r.finalize()
        assert ei.value.code == -5
        with pytest.raises(R.RadError) as ei:
            r.set_options(anchor_K=4)
        assert ei.value.code in (-1, -8)
    with pytest.raises(R.RadError) as ei:
        R.Radiation(w.dirs, w.grids, -1.0, sp, w.windows)
    assert ei.value.code == -1
    with pytest.raises(R.RadError):
        R.Radiation(w.dirs, w.grids, w.dt, sp, [(5, 3, 1, 0)])
    with pytest.raises(R.RadError):
        R.Radiation(w.dirs, w.grids, w.dt, sp, [(0, 3, 1, 7)])
    with pytest.raises(R.RadError):
        R.Radiation(np.zeros((1, 3)), w.grids, w.dt, sp, [(0, 3, 1, 0)])


def test_check_inputs_flags_nan(two_species):
    R = _rad()
    w, X, U, _ = two_species
    sp = [(s[0], s[1], s[2]) for s in w.species]
    Xb = X.copy()
    Xb[5, 1, 3] = np.nan
    with R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows, precision=R.RAD_FP32_SPLIT,
                     box_L=w.L, options={"check_inputs": 1}) as r:
        r.accumulate_steps(0, Xb, U)
        with pytest.raises(R.RadError) as ei:
            r.finalize()
        assert ei.value.code == -7


def test_workload1_full_fp64_and_fp32():
    """1024 e-, 2000 samples, n = y, 256 log-spaced omega in [0.1, 300]."""
    R = _rad()
    w = trajgen.config(1)
    X, U = w.trajectory_numpy()
    ref = oracle.spectra(X, U, w.dt, w.dirs, w.grids, w.windows,
                         [(s[0], s[1]) for s in w.species], box_L=w.L)
    f64 = _run(w, X, U, R.RAD_FP64)
    f32 = _run(w, X, U, R.RAD_FP32_SPLIT)
    assert relL2(f64[0], ref[0]) <= 1e-10
    assert relL2(f32[0], ref[0]) <= 1e-4


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_workload4_structure(precision):
    """Workload 4's structure, scaled: electrons + ions (m = 16, q = +1), 192 HEALPix
    directions, three log grids, five uneven windows over both species -- all evaluated in
    one deferred persistent launch -- against the oracle."""
    R = _rad()
    w = trajgen.config(4, 40 / 524288)            # 40 electrons, 2-3 ions
    scale = 16                                   # windows / 16: 256, 128, 32, 256, 32 samples
    wins = [(s0 // scale, s1 // scale, m, g) for (s0, s1, m, g) in w.windows]
    grids = [g[::8] for g in w.grids]            # 64, 128, 256 omegas
    nc = max(s1 for _, s1, _, _ in wins) + 1
    X, U = w.trajectory_numpy(n_calls=nc)
    sp = [(s[0], s[1], s[2]) for s in w.species]
    ref = oracle.spectra(X, U, w.dt, w.dirs, grids, wins, [(s[0], s[1]) for s in w.species],
                         box_L=w.L)
    with R.Radiation(w.dirs, grids, w.dt, sp, wins, precision=precision, box_L=w.L,
                     options={"defer": 1}) as r:
        r.accumulate_steps(0, torch.as_tensor(X, device="cuda"), torch.as_tensor(U, device="cuda"))
        got = r.finalize()
        t = r.timing()
    assert t["accum_launches"] == 1
    _check(got, ref, 1e-10 if precision == 0 else 1e-4, per_direction=True)


@pytest.mark.parametrize("coherent", [False, True])
def test_step_graphs_match_batched_steps(two_species, coherent):
    """use_graph: one rad_accumulate per step replayed as CUDA graphs (a plain-step
    graph and one per closing step) gives the batched result."""
    R = _rad()
    w, X, U, ref = two_species
    a = _run(w, X, U, R.RAD_FP32_SPLIT, coherent, device_inputs=True, steps=True)
    b = _run(w, X, U, R.RAD_FP32_SPLIT, coherent, options={"use_graph": 1},
             device_inputs=True, steps=False)
    for g, e in zip(b, a):
        np.testing.assert_allclose(g, e, rtol=1e-9, atol=1e-300)
    _check(b, ref[coherent], 1e-4, per_direction=True)


def test_autotuner_times_caches_and_reuses(tmp_path, monkeypatch):
    """variant AUTO on a problem large enough to tune: the choice is written to the
    on-disk cache, a second context with the same shape reads it back, and the
    tuned kernel stays within the FP32 tolerance of the fixed default."""
    R = _rad()
    from trajgen import gpu as tg
    cache = tmp_path / "tune.tsv"
    monkeypatch.setenv("RAD_AUTOTUNE_CACHE", str(cache))
    w = trajgen.config(2, 4096 / 65536)
    X, U = tg.trajectory_gpu(w)
    sp = [(s[0], s[1], s[2]) for s in w.species]

    def run(opts):
        with R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows, precision=R.RAD_FP32_SPLIT,
                         box_L=w.L, options=opts) as r:
            r.accumulate_steps(0, X, U)
            return r.finalize()[0], r.options()

    s_fixed, _ = run({"variant": 1, "anchor_K": 32})
    s_auto, o1 = run(None)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1 and "\t" in lines[0]
    s_auto2, o2 = run(None)
    assert len(cache.read_text().strip().splitlines()) == 1     # reused, not re-tuned
    assert o1 == o2
    for S in (s_auto, s_auto2):
        err = np.linalg.norm(S - s_fixed, axis=1) / np.linalg.norm(s_fixed, axis=1)
        assert err.max() <= 1e-4


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("coherent", [False, True])
def test_particle_shards_combine_to_the_whole(two_species, precision, coherent):
    """Two contexts over disjoint particle halves: their partial sums combine (host
    reduction) to the spectrum of one context over all particles."""
    R = _rad()
    from paper_1003_1140_gb300 import shard
    w, X, U, ref = two_species
    Ne = w.species[0][0]
    halves = [(0, Ne // 2), (Ne // 2, Ne - Ne // 2)]
    parts = []
    for first, n in halves:
        Xs = np.ascontiguousarray(X[:, :, first:first + n])
        Us = np.ascontiguousarray(U[:, :, first:first + n])
        win = [(0, 300, 1, 0)]
        with R.Radiation(w.dirs, w.grids, w.dt, [(n, -1.0, 1.0)], win,
                         mode=R.RAD_COHERENT if coherent else R.RAD_INCOHERENT,
                         precision=precision, box_L=w.L) as r:
            r.accumulate_steps(0, Xs, Us)
            parts.append(r.partial_sums())
    S = shard.combine(parts, coherent).reshape(len(w.dirs), -1)
    Xa, Ua = np.ascontiguousarray(X[:, :, :Ne]), np.ascontiguousarray(U[:, :, :Ne])
    with R.Radiation(w.dirs, w.grids, w.dt, [(Ne, -1.0, 1.0)], [(0, 300, 1, 0)],
                     mode=R.RAD_COHERENT if coherent else R.RAD_INCOHERENT,
                     precision=precision, box_L=w.L) as r:
        r.accumulate_steps(0, Xa, Ua)
        whole = r.finalize()[0]
    np.testing.assert_allclose(S, whole, rtol=1e-9, atol=1e-12 * np.abs(whole).max())


@pytest.mark.parametrize("precision,opts", [(0, None), (1, None), (1, {"variant": 3})])
@pytest.mark.parametrize("coherent", [False, True])
def test_selectors_match_oracle(two_species, precision, opts, coherent):
    """Windows restricted to a spatial box and to a momentum pitch cone about the
    streaming axis (and one unrestricted window) against the oracle."""
    R = _rad()
    w, X, U, _ = two_species
    sels = [{"kind": "box", "lo": [0, 10, 0], "hi": [40, 30, 25]},
            {"kind": "cone", "axis": [1, 0, 0], "theta_c": 0.0, "dtheta": 0.2},
            {"kind": "cone", "axis": [-1, 0, 0], "theta_c": math.pi / 8, "dtheta": 0.3}]
    wins = [(0, 300, 3, 0), (17, 250, 1, 1), (0, 300, 1, 0), (10, 290, 3, 0)]
    wsel = [0, 1, 2, -1]
    sp = [(s[0], s[1], s[2]) for s in w.species]
    ref = oracle.spectra(X, U, w.dt, w.dirs, w.grids, wins, [(s[0], s[1]) for s in w.species],
                         coherent=coherent, box_L=w.L, selectors=sels, window_selector=wsel)
    with R.Radiation(w.dirs, w.grids, w.dt, sp, wins,
                     mode=R.RAD_COHERENT if coherent else R.RAD_INCOHERENT,
                     precision=precision, box_L=w.L, options=opts) as r:
        r.set_selectors(sels, wsel)
        r.accumulate_steps(0, torch.as_tensor(X, device="cuda"), torch.as_tensor(U, device="cuda"))
        got = r.finalize()
    _check(got, ref, 1e-10 if precision == 0 else 1e-4, per_direction=True)


@pytest.mark.parametrize("precision,opts", [(0, {}), (1, {}), (1, {"variant": 3})])
@pytest.mark.parametrize("coherent", [False, True])
def test_subcycling_matches_oracle(two_species, precision, opts, coherent):
    """Sub-cycling (4 sub-samples per PIC sample) with a selector, several windows
    and both species, against the oracle's sub-cycled sum."""
    R = _rad()
    w, X, U, _ = two_species
    sels = [{"kind": "box", "lo": [0, 10, 0], "hi": [40, 30, 25]}]
    wsel = [-1, 0, -1, -1]
    sp = [(s[0], s[1], s[2]) for s in w.species]
    ref = oracle.spectra(X, U, w.dt, w.dirs, w.grids, w.windows, [(s[0], s[1]) for s in w.species],
                         coherent=coherent, box_L=w.L, selectors=sels, window_selector=wsel,
                         subcycle=4)
    with R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows,
                     mode=R.RAD_COHERENT if coherent else R.RAD_INCOHERENT,
                     precision=precision, box_L=w.L, options=dict(opts, subcycle=4)) as r:
        r.set_selectors(sels, wsel)
        r.accumulate_steps(0, torch.as_tensor(X, device="cuda"), torch.as_tensor(U, device="cuda"))
        got = r.finalize()
    _check(got, ref, 1e-10 if precision == 0 else 1e-4, per_direction=True)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("coherent", [False, True])
def test_host_blocked_transfer(precision, coherent):
    """Host inputs of one species over 2050 particles: the particle-blocked
    transfer (blocks of 8, 32, 128 and 89 tiles; windows closing at three calls
    inside the batch; a 1 MiB staging cap so a block's segment arrives in
    several chunks) gives the device-input and the deferred single-launch
    results (FP64 summation order aside) and the oracle's."""
    R = _rad()
    w = trajgen.Workload("blocked", [(2050, -1.0, 1.0, 3.0)], 181, 0.05,
                         np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.6, 0.0, 0.8]]),
                         [trajgen.log_grid(0.1, 200.0, 64)],
                         [(0, 180, 1, 0), (30, 120, 1, 0), (100, 100, 1, 0), (60, 90, 1, 0)],
                         b_rms=0.3)
    X, U = w.trajectory_numpy()
    dev = _run(w, X, U, precision, coherent)           # device inputs: one launch
    host = _run(w, X, U, precision, coherent, options={"host_stage_mib": 1}, device_inputs=False)
    whole = _run(w, X, U, precision, coherent, options={"defer": 1})   # one launch, all particles
    for g, e in zip(host, whole):
        np.testing.assert_allclose(g, e, rtol=1e-11, atol=1e-300)
    for g, e in zip(dev, whole):
        np.testing.assert_allclose(g, e, rtol=1e-11, atol=1e-300)
    ref = oracle.spectra(X, U, w.dt, w.dirs, w.grids, w.windows, [(2050, -1.0)],
                         coherent=coherent, box_L=w.L)
    _check(host, ref, 1e-10 if precision == R.RAD_FP64 else 1e-4, per_direction=True)


@pytest.mark.parametrize("precision", [0, 1])
def test_host_blocked_transfer_with_subcycling_and_selector(precision):
    """The particle-blocked host transfer with 3 sub-samples per PIC sample
    and a region selector on one window, against the oracle's sub-cycled,
    selected sum (2050 particles, 1 MiB staging cap, windows closing inside
    the batch; the particle blocks' ingest is also split in time)."""
    R = _rad()
    w = trajgen.Workload("blocked-sub", [(2050, -1.0, 1.0, 3.0)], 161, 0.05,
                         np.array([[0.0, 1.0, 0.0], [0.6, 0.0, 0.8]]),
                         [trajgen.log_grid(0.1, 200.0, 48)],
                         [(0, 160, 1, 0), (40, 100, 1, 0)], b_rms=0.3)
    X, U = w.trajectory_numpy()
    sels = [{"kind": "box", "lo": [0, 5, 0], "hi": [40, 35, 30]}]
    wsel = [-1, 0]
    ref = oracle.spectra(X, U, w.dt, w.dirs, w.grids, w.windows, [(2050, -1.0)], box_L=w.L,
                         selectors=sels, window_selector=wsel, subcycle=3)
    with R.Radiation(w.dirs, w.grids, w.dt, [(2050, -1.0, 1.0)], w.windows, precision=precision,
                     box_L=w.L, options={"subcycle": 3, "host_stage_mib": 1}) as r:
        r.set_selectors(sels, wsel)
        r.accumulate_steps(0, np.ascontiguousarray(X), np.ascontiguousarray(U))
        got = r.finalize()
    _check(got, ref, 1e-10 if precision == 0 else 1e-4, per_direction=True)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("host", [False, True])
def test_batches_across_calls(precision, host):
    """The same 181 calls handed over in three batches of uneven length (67, 70,
    44), windows opening in one batch and closing in another: the per-particle
    ingest state (raw position, image count, u) carries across batches through
    the blocked host transfer and the time-segmented ingest alike."""
    R = _rad()
    w = trajgen.Workload("batches", [(2050, -1.0, 1.0, 3.0)], 181, 0.05,
                         np.array([[0.0, 1.0, 0.0], [0.6, 0.0, 0.8]]),
                         [trajgen.log_grid(0.1, 200.0, 48)],
                         [(0, 180, 1, 0), (50, 120, 1, 0), (10, 60, 1, 0)], b_rms=0.3)
    X, U = w.trajectory_numpy()
    ref = oracle.spectra(X, U, w.dt, w.dirs, w.grids, w.windows, [(2050, -1.0)], box_L=w.L)
    with R.Radiation(w.dirs, w.grids, w.dt, [(2050, -1.0, 1.0)], w.windows, precision=precision,
                     box_L=w.L, options={"host_stage_mib": 1}) as r:
        s = 0
        for n in (67, 70, 44):
            xs, us = np.ascontiguousarray(X[s:s + n]), np.ascontiguousarray(U[s:s + n])
            if not host:
                xs, us = torch.as_tensor(xs, device="cuda"), torch.as_tensor(us, device="cuda")
            r.accumulate_steps(s, xs, us)
            s += n
        got = r.finalize()
    _check(got, ref, 1e-10 if precision == 0 else 1e-4, per_direction=True)


@pytest.mark.parametrize("precision", [0, 1])
def test_host_blocked_transfer_two_species(precision):
    """Host inputs of two species (1701 electrons + 390 ions, m = 16, q = +1):
    every block carries a share of each species; windows over electrons only,
    ions only and both close inside the batch; a 1 MiB staging cap splits the
    copies.  Against the device-input result and the oracle."""
    R = _rad()
    w = trajgen.Workload("blocked-2sp", [(1701, -1.0, 1.0, 3.0), (390, 1.0, 16.0, 3.0)], 151, 0.05,
                         np.array([[0.0, 1.0, 0.0], [0.6, 0.0, 0.8]]),
                         [trajgen.log_grid(0.1, 200.0, 40), np.linspace(0.5, 20.0, 23)],
                         [(0, 150, 3, 0), (20, 110, 1, 1), (40, 150, 2, 0), (70, 90, 3, 1)],
                         b_rms=0.3)
    X, U = w.trajectory_numpy()
    species = [(s[0], s[1]) for s in w.species]
    dev = _run(w, X, U, precision)
    host = _run(w, X, U, precision, options={"host_stage_mib": 1}, device_inputs=False)
    for g, e in zip(host, dev):
        np.testing.assert_allclose(g, e, rtol=1e-11, atol=1e-300)
    ref = oracle.spectra(X, U, w.dt, w.dirs, w.grids, w.windows, species, box_L=w.L)
    _check(host, ref, 1e-10 if precision == 0 else 1e-4, per_direction=True)
