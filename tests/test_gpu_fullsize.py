"""Full-size and high-gamma parity.

* The benchmark's workload at full size (65,536 electrons x 4096 samples x 8
  directions x 1024 omega) in the launch configuration bench.py times, checked
  on sampled output bins that the FP64 oracle computes over all particles.
* A gamma = 10 two-beam load (the precision workload's particles), where
  1 - n.beta ~ 1/(2 gamma^2) makes the head-on directions sensitive to
  cancellation, at full samples / directions / omegas on a particle subset.
"""
import numpy as np
import pytest

import oracle
import trajgen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_workload2_full_size_sampled_bins():
    import paper_1003_1140_gb300 as R
    from trajgen import gpu as tg
    w = trajgen.config(2)
    X, U = tg.trajectory_gpu(w)
    sp = [(s[0], s[1], s[2]) for s in w.species]
    with R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows, precision=R.RAD_FP32_SPLIT,
                     box_L=w.L) as r:
        r.accumulate_steps(0, X, U)
        S = r.finalize()[0]
    assert np.all(np.isfinite(S)) and np.all(S >= 0)
    Xh = X.cpu().numpy()
    Uh = U.cpu().numpy()
    del X, U
    torch.cuda.empty_cache()
    rb, bb, bdb = oracle.samples(Xh, Uh, w.dt, w.L)
    del Xh, Uh
    rng = np.random.default_rng(5)
    om = w.grids[0]
    picks = [(0, 0), (2, 511), (6, 1023), (int(rng.integers(8)), int(rng.integers(1024)))]
    q = np.full(w.n_total, w.species[0][1])
    for d, k in picks:
        ref = oracle.window_spectrum(rb, bb, bdb, q, w.dt, w.dirs[d:d + 1], om[k:k + 1],
                                     w.windows[0][0], w.windows[0][1])[0, 0]
        assert abs(S[d, k] - ref) <= 1e-4 * abs(ref), (d, k, S[d, k], ref)


def test_gamma10_precision_workload_subset():
    import paper_1003_1140_gb300 as R
    w = trajgen.config(3, 48 / 1048576)
    X, U = w.trajectory_numpy(n_calls=1025)
    win = [(0, 1024, 1, 0)]
    sp = [(w.n_total, -1.0, 1.0)]
    ref = oracle.spectra(X, U, w.dt, w.dirs, w.grids, win, [(w.n_total, -1.0)], box_L=w.L)[0]
    Xd, Ud = torch.as_tensor(X, device="cuda"), torch.as_tensor(U, device="cuda")
    for prec, tol, opts in ((R.RAD_FP64, 1e-10, None), (R.RAD_FP32_SPLIT, 1e-4, None),
                            (R.RAD_FP32_SPLIT, 1e-4, {"variant": 2}),
                            (R.RAD_FP32_SPLIT, 1e-4, {"anchor_K": 32})):
        with R.Radiation(w.dirs, w.grids, w.dt, sp, win, precision=prec, box_L=w.L,
                         options=opts) as r:
            r.accumulate_steps(0, Xd, Ud)
            S = r.finalize()[0]
        for d in range(len(w.dirs)):
            e = np.linalg.norm(S[d] - ref[d]) / np.linalg.norm(ref[d])
            assert e <= tol, (prec, opts, d, e)
