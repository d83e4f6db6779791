"""Particle shards through one context (rad_next_shard) and per-window direction
subsets (rad_window.dir_set), through the C ABI against the FP64 CPU oracle.

* Shards: a context sized for one shard of the particles receives the shards
  one after another; the accumulators add them, so the spectrum equals the
  oracle's over the union (Sec. 2.2's sum over the tracked particles).  This
  is how a population whose whole-window ring does not fit beside its inputs
  runs on one GPU.
* Direction sets: windows of a batched two-species configuration (HEALPix
  directions, two log grids, uneven windows) each take their own subset of
  the directions (Sec. 2.2's multiple far-field observers); every window's
  spectrum has one row per listed direction, in the listed order.

Tolerances as everywhere: FP64 path 1e-10, FP32 split path 1e-4 relative L2
per (window, direction).
"""
import numpy as np
import pytest

import oracle
import trajgen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rad():
    import paper_1003_1140_gb300 as R
    return R


def _check(got, ref, tol):
    for g, e in zip(got, ref):
        assert g.shape == e.shape
        for d in range(e.shape[0]):
            err = np.linalg.norm(g[d] - e[d]) / np.linalg.norm(e[d])
            assert err <= tol, (d, err)


@pytest.fixture(scope="module")
def sharded():
    """43 electrons (gamma 10: the precision workload's beams) and 301 calls in three
    shards of 15, 15 and 13 particles (ragged against the 8-particle tile)."""
    w = trajgen.config(3, 43 / 1048576)
    X, U = w.trajectory_numpy(n_calls=301)
    dirs = w.dirs
    grid = trajgen.log_grid(0.1, 1000.0, 300)
    wins = [(0, 300, 1, 0), (37, 211, 1, 0)]
    ref = {coh: oracle.spectra(X, U, w.dt, dirs, [grid], wins, [(X.shape[2], -1.0)],
                               coherent=coh, box_L=w.L) for coh in (False, True)}
    return w, X, U, dirs, grid, wins, ref


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("coherent", [False, True])
@pytest.mark.parametrize("mode", ["device", "host", "defer"])
def test_next_shard_sums_particle_shards(sharded, precision, coherent, mode):
    R = _rad()
    w, X, U, dirs, grid, wins, ref = sharded
    cuts = [(0, 15), (15, 30), (30, 43)]
    # one context of the largest shard's size; a smaller last shard is handed over
    # as that size with its missing particles at rest (uniform motion radiates
    # exactly nothing)
    n = max(b - a for a, b in cuts)
    opts = {"defer": 1} if mode == "defer" else None
    with R.Radiation(dirs, [grid], w.dt, [(n, -1.0, 1.0)], wins,
                     mode=R.RAD_COHERENT if coherent else R.RAD_INCOHERENT,
                     precision=precision, box_L=w.L, options=opts) as r:
        for i, (a, b) in enumerate(cuts):
            Xs = np.zeros((X.shape[0], 3, n))
            Us = np.zeros((X.shape[0], 3, n))
            Xs[:, :, :b - a] = X[:, :, a:b]
            Us[:, :, :b - a] = U[:, :, a:b]
            Xs[:, :, b - a:] = 1.0
            if i:
                r.next_shard()
            if mode == "host":
                r.accumulate_steps(0, Xs, Us)
            else:
                r.accumulate_steps(0, torch.as_tensor(Xs, device="cuda"),
                                   torch.as_tensor(Us, device="cuda"))
        got = r.finalize()
    _check(got, ref[coherent], 1e-10 if precision == 0 else 1e-4)


def test_next_shard_needs_complete_windows(sharded):
    R = _rad()
    w, X, U, dirs, grid, wins, ref = sharded
    with R.Radiation(dirs, [grid], w.dt, [(8, -1.0, 1.0)], wins, box_L=w.L) as r:
        Xd = torch.as_tensor(np.ascontiguousarray(X[:100, :, :8]), device="cuda")
        Ud = torch.as_tensor(np.ascontiguousarray(U[:100, :, :8]), device="cuda")
        r.accumulate_steps(0, Xd, Ud)
        with pytest.raises(R.RadError) as ei:
            r.next_shard()
        assert ei.value.code == R.rad.RAD_EINCOMPLETE
        # a reset context starts a fresh first shard
        r.reset()
        r.accumulate_steps(0, Xd, Ud)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("coherent", [False, True])
def test_window_direction_sets(precision, coherent):
    """A scaled batched configuration: 37 electrons + 5 ions (m = 16, q = +1), the 192
    HEALPix Nside-4 directions, two log grids, windows with their own direction subsets
    (a ring of 12, a handful with a repeat, all of them), eager windows."""
    R = _rad()
    w = trajgen.config(4, 37 / 524288)
    w.species[1] = (5,) + tuple(w.species[1][1:])
    grids = [trajgen.log_grid(0.01, 30.0, 64), trajgen.log_grid(0.1, 1000.0, 300)]
    ring12 = list(range(0, 192, 16))
    few = [191, 3, 96, 3, 40]
    wins = [(0, 256, 1, 1, ring12), (64, 192, 3, 0, few), (32, 96, 2, 1), (0, 128, 3, 0, [7])]
    X, U = w.trajectory_numpy(n_calls=257)
    species = [(s[0], s[1]) for s in w.species]
    ref = oracle.spectra(X, U, w.dt, w.dirs, grids, wins, species, coherent=coherent,
                         box_L=w.L)
    sp = [(s[0], s[1], s[2]) for s in w.species]
    with R.Radiation(w.dirs, grids, w.dt, sp, wins,
                     mode=R.RAD_COHERENT if coherent else R.RAD_INCOHERENT,
                     precision=precision, box_L=w.L) as r:
        assert r.spectrum_size() == 12 * 300 + 5 * 64 + 192 * 300 + 1 * 64
        assert r.updates() == (37 * 256 * 12 * 300 + 42 * 128 * 5 * 64 + 5 * 64 * 192 * 300
                               + 42 * 128 * 1 * 64)
        r.accumulate_steps(0, torch.as_tensor(X, device="cuda"), torch.as_tensor(U, device="cuda"))
        got = r.finalize()
    _check(got, ref, 1e-10 if precision == 0 else 1e-4)
    # the repeated direction gives the same row twice (up to the order of the FP64
    # atomic additions of the work items' particle sums)
    np.testing.assert_allclose(got[1][1], got[1][3], rtol=1e-12, atol=0)


@pytest.mark.parametrize("coherent", [False, True])
def test_spectrum_from_summed_partials_on_the_device(sharded, coherent):
    """The exchange step of the multi-GPU path, on one GPU: two contexts over disjoint
    particle halves export their partial sums into device buffers, the sums are added
    (what an all-reduce does across ranks) and rad_spectrum_from_sums forms the
    spectrum of the union on the device; it equals the oracle's."""
    R = _rad()
    w, X, U, dirs, grid, wins, ref = sharded
    mode = R.RAD_COHERENT if coherent else R.RAD_INCOHERENT
    halves = [(0, 21), (21, 43)]
    total = None
    for a, b in halves:
        with R.Radiation(dirs, [grid], w.dt, [(b - a, -1.0, 1.0)], wins, mode=mode,
                         precision=R.RAD_FP64, box_L=w.L) as r:
            r.accumulate_steps(0, torch.as_tensor(np.ascontiguousarray(X[:, :, a:b]), device="cuda"),
                               torch.as_tensor(np.ascontiguousarray(U[:, :, a:b]), device="cuda"))
            part = torch.empty(r.spectrum_size() * (4 if coherent else 1), dtype=torch.float64,
                               device="cuda")
            r.partial_sums(part)
            total = part if total is None else total + part
    out = torch.empty(total.numel() // (4 if coherent else 1), dtype=torch.float64, device="cuda")
    R.spectrum_from_sums(total, mode, out)
    got = out.cpu().numpy()
    n0 = len(dirs) * len(grid)
    _check([got[:n0].reshape(len(dirs), -1), got[n0:].reshape(len(dirs), -1)], ref[coherent],
           1e-10)
    # host memory is refused (no CPU path)
    with pytest.raises(R.RadError):
        R.spectrum_from_sums(total.cpu(), mode, out.cpu())


def test_direction_sets_through_every_path():
    """Windows with direction subsets through each way the library takes inputs: device
    inputs in one batch, host inputs through the particle-blocked transfer (2048 particles,
    blocks of whole tiles with their own work lists), one call per step replayed as CUDA
    graphs, deferred windows, and two particle shards -- all against the oracle, and with
    each other up to the order of the FP64 sums."""
    R = _rad()
    w = trajgen.config(2, 2048 / 65536)
    X, U = w.trajectory_numpy(n_calls=129)
    N = X.shape[2]
    grids = [trajgen.log_grid(0.1, 300.0, 64)]
    wins = [(0, 128, 1, 0, [6, 0, 2]), (40, 100, 1, 0, [7]), (0, 64, 1, 0)]
    ref = oracle.spectra(X, U, w.dt, w.dirs, grids, wins, [(N, -1.0)], box_L=w.L)
    Xd, Ud = torch.as_tensor(X, device="cuda"), torch.as_tensor(U, device="cuda")

    def run(inputs, options=None, per_step=False):
        with R.Radiation(w.dirs, grids, w.dt, [(N, -1.0, 1.0)], wins, box_L=w.L,
                         options=options) as r:
            Xi, Ui = inputs
            if per_step:
                for s in range(Xi.shape[0]):
                    r.accumulate(s, Xi[s], Ui[s])
            else:
                r.accumulate_steps(0, Xi, Ui)
            return r.finalize()

    out = {"device": run((Xd, Ud)),
           "host blocked": run((np.ascontiguousarray(X), np.ascontiguousarray(U))),
           "graphs": run((Xd, Ud), {"use_graph": 1}, per_step=True),
           "deferred": run((Xd, Ud), {"defer": 1})}
    half = N // 2
    with R.Radiation(w.dirs, grids, w.dt, [(half, -1.0, 1.0)], wins, box_L=w.L) as r:
        for i in range(2):
            if i:
                r.next_shard()
            sl = slice(i * half, (i + 1) * half)
            r.accumulate_steps(0, torch.as_tensor(np.ascontiguousarray(X[:, :, sl]), device="cuda"),
                               torch.as_tensor(np.ascontiguousarray(U[:, :, sl]), device="cuda"))
        out["two shards"] = r.finalize()
    for name, got in out.items():
        assert [g.shape for g in got] == [(3, 64), (1, 64), (8, 64)], name
        _check(got, ref, 1e-4)
        for g, e in zip(got, out["device"]):
            np.testing.assert_allclose(g, e, rtol=1e-9, atol=1e-12 * np.abs(e).max(),
                                       err_msg=name)
