"""The live GPU PIC against the FP64 reference PIC, its invariants at a larger
size, and the diagnostic driven in situ by it against the oracle on the
recorded particle histories."""
import math

import numpy as np
import pytest

import oracle
import trajgen
from oracle import pic as ref

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _periodic_diff(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


@pytest.mark.parametrize("mass_ratio", [64.0, 1.0])
def test_pic_matches_reference_pic(mass_ratio):
    """20 steps of a small two-stream box (baryonic or pair partners), field and
    particle state against the NumPy reference from the same initial state (the
    GPU's atomic current sums differ in the last bits only)."""
    from paper_1003_1140_gb300 import pic
    ts = trajgen.TwoStream(n=16, ppc=2, gamma=3.0, u_th=0.05, mass_ratio=mass_ratio, seed=21)
    X, U, q, m, w = ts.particles()
    g = ref.Grid(ts.n, ts.d, ts.dt)
    E = np.zeros((3, ts.n, ts.n))
    B = np.zeros((3, ts.n, ts.n))
    with pic.Pic.two_stream(ts) as p:
        for _ in range(20):
            X, U, E, B, _ = ref.step(X, U, E, B, q, m, w, g)
        p.step(20)
        assert p.steps_done == 20
        Eg, Bg = p.fields()
        xg, ug = p.particles()
    assert np.abs(_periodic_diff(xg, X, ts.L)).max() <= 1e-10 * ts.L
    assert np.abs(ug - U).max() <= 1e-10 * np.abs(U).max()
    assert np.abs(Eg - E).max() <= 1e-9 * np.abs(E).max()
    assert np.abs(Bg - B).max() <= 1e-9 * np.abs(B).max()


def test_pic_fields_from_set_fields_follow_vacuum_dispersion():
    """A Yee eigenmode loaded through rad_pic_set_fields advances with the
    discrete dispersion (no particles)."""
    from paper_1003_1140_gb300 import pic
    n, d, dt = 32, 0.1, 0.05
    kw = 2 * math.pi * 3 / (n * d)
    om = 2.0 / dt * math.asin(dt / d * math.sin(kw * d / 2))
    idx = np.arange(n)
    E = np.zeros((3, n, n))
    B = np.zeros((3, n, n))
    E[0] = np.cos(kw * idx * d)[:, None] * np.ones((1, n))
    B[2] = -math.cos(om * dt / 2) * np.cos(kw * (idx + 0.5) * d)[:, None] * np.ones((1, n))
    empty = np.zeros((3, 1))
    with pic.Pic(n, d, dt, [(1, -1.0, 1.0, 0.0)], empty + 0.5, empty) as p:
        p.set_fields(E, B)
        p.step(200)
        Eg, _ = p.fields()
    exp = np.cos(kw * idx * d - om * 200 * dt)[:, None] * np.ones((1, n))
    assert np.abs(Eg[0] - exp).max() <= 1e-11


def test_pic_gauss_law_and_energy_at_scale():
    """64 x 64 cells, 65,536 particles, 200 steps through the linear growth:
    div E = rho on the nodes to rounding, total energy conserved to 1e-4."""
    from paper_1003_1140_gb300 import pic
    ts = trajgen.TwoStream(n=64, d=0.1, dt=0.05, ppc=4, gamma=3.0, u_th=1e-3, seed=22)
    _, _, q, _, w = ts.particles()
    g = ref.Grid(ts.n, ts.d, ts.dt)
    with pic.Pic.two_stream(ts) as p:
        e0 = sum(p.energy())
        eb = []
        for _ in range(10):
            p.step(20)
            E, B = p.fields()
            eb.append(0.5 * float(np.sum(B * B)))
        e1 = sum(p.energy())
        x, _ = p.particles()
    rho = ref.charge_density(x[1], x[2], q * w, g)
    assert np.abs(ref.div_E(E, g.d) - rho).max() <= 1e-9 * np.abs(rho).max()
    assert abs(e1 - e0) <= 1e-4 * e0
    assert eb[-1] > 100 * eb[1]           # the filamentation grew


def _rad_setup(N_track, S):
    dirs = trajgen.paper_observers(axis=(1.0, 0.0, 0.0), perp=(0.0, 0.0, 1.0))
    grids = [trajgen.log_grid(0.1, 50.0, 96)]
    windows = [(0, S, 1, 0), (S // 2, S, 1, 0)]
    return dirs, grids, windows, [(N_track, -1.0)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("coherent", [False, True])
def test_in_situ_spectrum_matches_oracle(precision, coherent):
    """The PIC hands the first 96 electrons to the diagnostic every step (device
    buffers, no host copy on the path); the spectra equal the oracle's on the
    recorded histories of the same particles: <= 1e-10 (FP64), <= 1e-4 (FP32 split)."""
    from paper_1003_1140_gb300 import pic
    from paper_1003_1140_gb300 import rad as R
    ts = trajgen.TwoStream(n=16, ppc=2, gamma=3.0, u_th=0.05, seed=23)
    Nt, S = 96, 48
    dirs, grids, windows, species = _rad_setup(Nt, S)
    prec = R.RAD_FP64 if precision == "fp64" else R.RAD_FP32_SPLIT
    xt = torch.empty((3, Nt), dtype=torch.float64, device="cuda")
    ut = torch.empty_like(xt)
    hx, hu = [], []
    with pic.Pic.two_stream(ts) as p, \
            R.Radiation(dirs, grids, ts.dt, [(Nt, -1.0, 1.0)], windows, precision=prec,
                        mode=R.RAD_COHERENT if coherent else R.RAD_INCOHERENT,
                        box_L=ts.L) as r:
        for s in range(S + 1):
            p.tracked(0, Nt, xt, ut)
            r.accumulate(s, xt, ut)
            hx.append(xt.cpu().numpy().copy())
            hu.append(ut.cpu().numpy().copy())
            if s < S:
                p.step(1)
        got = r.finalize()
    exp = oracle.spectra(np.stack(hx), np.stack(hu), ts.dt, dirs, grids, windows, species,
                         coherent=coherent, box_L=ts.L)
    tol = 1e-10 if precision == "fp64" else 1e-4
    for gw, ew in zip(got, exp):
        for d in range(len(dirs)):
            assert np.linalg.norm(gw[d] - ew[d]) <= tol * np.linalg.norm(ew[d]), d
    assert max(np.abs(e).max() for e in exp) > 0


def test_run_coupled_matches_manual_coupling():
    """rad_pic_run_coupled (the PIC calling the diagnostic from C each step,
    final state included) gives the spectrum of the step-by-step coupling, and
    a second run continues the same windows without handing a state twice."""
    from paper_1003_1140_gb300 import pic
    from paper_1003_1140_gb300 import rad as R
    ts = trajgen.TwoStream(n=16, ppc=2, gamma=3.0, u_th=0.05, seed=24)
    Nt, S = 64, 40
    dirs, grids, windows, _ = _rad_setup(Nt, S)
    xt = torch.empty((3, Nt), dtype=torch.float64, device="cuda")
    ut = torch.empty_like(xt)
    with pic.Pic.two_stream(ts) as p, \
            R.Radiation(dirs, grids, ts.dt, [(Nt, -1.0, 1.0)], windows, precision=R.RAD_FP64,
                        box_L=ts.L) as r:
        for s in range(S + 1):
            p.tracked(0, Nt, xt, ut)
            r.accumulate(s, xt, ut)
            if s < S:
                p.step(1)
        manual = r.finalize()
    with pic.Pic.two_stream(ts) as p, \
            R.Radiation(dirs, grids, ts.dt, [(Nt, -1.0, 1.0)], windows, precision=R.RAD_FP64,
                        box_L=ts.L) as r:
        p.run_coupled(r, 0, Nt, S // 2)
        p.run_coupled(r, 0, Nt, S - S // 2)
        assert p.steps_done == S
        coupled = r.finalize()
    for a, b in zip(coupled, manual):
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)


def test_pic_rejects_bad_arguments():
    from paper_1003_1140_gb300 import pic
    ts = trajgen.TwoStream(n=8, ppc=1, seed=25)
    with pic.Pic.two_stream(ts) as p:
        xt = torch.empty((3, 4), dtype=torch.float64, device="cuda")
        with pytest.raises(RuntimeError):
            p.tracked(p.N - 2, 4, xt, xt.clone())          # range past the end
        with pytest.raises(RuntimeError):
            p.tracked(0, 4, np.empty((3, 4)), np.empty((3, 4)))   # host buffers
    with pytest.raises(RuntimeError):
        pic.Pic(16, 0.1, 0.1, [(1, -1.0, 1.0, 1.0)], np.zeros((3, 1)), np.zeros((3, 1)))  # Courant
    # a coupled run must hand over exactly the radiation context's particle count
    from paper_1003_1140_gb300 import rad as R
    with pic.Pic.two_stream(ts) as p, \
            R.Radiation(np.array([[0.0, 1.0, 0.0]]), [np.linspace(1.0, 2.0, 8)], ts.dt,
                        [(16, -1.0, 1.0)], [(0, 4, 1, 0)], box_L=ts.L) as r:
        with pytest.raises(RuntimeError):
            p.run_coupled(r, 0, 8, 4)
        assert p.steps_done == 0


def test_insitu_run_small():
    """The in-situ application end to end on a small box: timings, growing
    magnetic energy, finite positive spectra with a peak per window and observer."""
    from paper_1003_1140_gb300 import insitu
    res, spectra = insitu.run(n=32, ppc=2, steps=120, tracked=512, windows=2, n_omega=64,
                              pic_only_steps=20, chunk=40)
    assert res["pic_ms_per_step"] > 0 and res["coupled_ms_per_step"] > 0
    assert res["diagnostic_updates"] == 512 * 120 * 6 * 64
    assert res["magnetic_energy"][-1][1] > res["magnetic_energy"][0][1]
    assert len(res["peak_omega"]) == 2 and len(res["peak_omega"][0]) == 6
    for S in spectra:
        assert np.isfinite(S).all() and (S >= 0).all() and S.max() > 0
