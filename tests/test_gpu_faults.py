"""Failure detection through the RAD_FAULT test hooks: every failure is made on
the host (an allocation reported failed, a graph capture reported failed, a
lost step hand-over) or by a bounded device wait that nothing ends (the
accumulation kernel's producer in block 0 waits on a barrier no one arrives
on).  No GPU is faulted or hung: the wait expires after its poll limit, the
kernel raises the device error word and returns, the host reports
RAD_ETIMEOUT, and after rad_reset the same context gives the oracle's result."""
import time

import numpy as np
import pytest

import oracle
import trajgen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RAD_EINVAL, RAD_ENOMEM, RAD_ESTEP, RAD_ETIMEOUT = -1, -2, -4, -6


def _rad():
    import paper_1003_1140_gb300 as R
    return R


def relL2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def small():
    """21 electrons (gamma 3), 97 calls, 3 directions, 2 grids, 3 windows."""
    w = trajgen.Workload("faults", [(21, -1.0, 1.0, 3.0)], 97, 0.05,
                         np.array([[0.0, 1.0, 0.0], [1.0, 0.0, 0.0], [0.6, 0.0, 0.8]]),
                         [trajgen.log_grid(0.1, 100.0, 70), np.linspace(0.5, 10.0, 33)],
                         [(0, 96, 1, 0), (10, 60, 1, 1), (40, 41, 1, 0)], b_rms=0.3)
    X, U = w.trajectory_numpy()
    ref = oracle.spectra(X, U, w.dt, w.dirs, w.grids, w.windows,
                         [(s[0], s[1]) for s in w.species], coherent=False, box_L=w.L)
    return w, X, U, ref


# fixed kernel build: no autotuning launches before the hooked ones
FP32_OPTS = {"variant": 1, "anchor_K": 16, "freq_per_lane": 8}


def _ctx(w, precision, options=None):
    R = _rad()
    return R.Radiation(w.dirs, w.grids, w.dt, [(s[0], s[1], s[2]) for s in w.species],
                       w.windows, precision=precision, box_L=w.L, options=options)


def _check(got, ref, tol):
    for g, e in zip(got, ref):
        for d in range(e.shape[0]):
            assert relL2(g[d], e[d]) <= tol, (d, relL2(g[d], e[d]))


def test_allocation_failure_is_reported_and_cleaned_up(small, monkeypatch):
    R = _rad()
    w, X, U, ref = small
    monkeypatch.setenv("RAD_FAULT", "alloc")
    for _ in range(3):    # the partial allocations are released each time
        with pytest.raises(R.RadError) as ei:
            _ctx(w, R.RAD_FP64)
        assert ei.value.code == RAD_ENOMEM
    monkeypatch.setenv("RAD_FAULT", "no-such-hook")
    with pytest.raises(R.RadError) as ei:
        _ctx(w, R.RAD_FP64)
    assert ei.value.code == RAD_EINVAL
    monkeypatch.delenv("RAD_FAULT")
    with _ctx(w, R.RAD_FP64) as r:
        r.accumulate_steps(0, X, U)
        _check(r.finalize(), ref, 1e-10)


def test_graph_capture_failure_falls_back_to_direct_launches(small, monkeypatch):
    """use_graph with the capture reported failed: every step still runs (direct
    launches), rad_get_options shows use_graph = 0, the spectrum is the oracle's."""
    R = _rad()
    w, X, U, ref = small
    Xd = torch.as_tensor(X, device="cuda")
    Ud = torch.as_tensor(U, device="cuda")
    monkeypatch.setenv("RAD_FAULT", "graph")
    r = _ctx(w, R.RAD_FP32_SPLIT, dict(FP32_OPTS, use_graph=1))
    monkeypatch.delenv("RAD_FAULT")
    with r:
        assert r.options()["use_graph"] == 1
        for s in range(X.shape[0]):
            r.accumulate(s, Xd[s], Ud[s])
        assert r.options()["use_graph"] == 0
        got = r.finalize()
    with _ctx(w, R.RAD_FP32_SPLIT, dict(FP32_OPTS, use_graph=1)) as r:
        for s in range(X.shape[0]):
            r.accumulate(s, Xd[s], Ud[s])
        assert r.options()["use_graph"] == 1
        graphed = r.finalize()
    for g, e in zip(got, graphed):
        np.testing.assert_allclose(g, e, rtol=1e-9, atol=1e-300)
    _check(got, ref, 1e-4)


@pytest.mark.parametrize("precision", [0, 1])
def test_lost_step_is_detected_and_can_be_resent(small, monkeypatch, precision):
    """The hand-over of step 37 is lost once: the next call is refused with
    RAD_ESTEP, and resending step 37 restores the oracle's spectrum."""
    R = _rad()
    w, X, U, ref = small
    monkeypatch.setenv("RAD_FAULT", "step:37")
    r = _ctx(w, precision, FP32_OPTS if precision == R.RAD_FP32_SPLIT else None)
    monkeypatch.delenv("RAD_FAULT")
    with r:
        r.accumulate_steps(0, X[:37], U[:37])
        r.accumulate(37, X[37], U[37])          # lost
        with pytest.raises(R.RadError) as ei:
            r.accumulate(38, X[38], U[38])
        assert ei.value.code == RAD_ESTEP
        r.accumulate(37, X[37], U[37])          # sent again
        r.accumulate_steps(38, X[38:], U[38:])
        _check(r.finalize(), ref, 1e-10 if precision == R.RAD_FP64 else 1e-4)


@pytest.mark.parametrize("precision", [0, 1])
def test_expired_device_wait_is_reported_and_recoverable(small, monkeypatch, precision):
    """A producer wait that nothing ends expires after its poll limit: the kernel
    returns, rad_finalize reports RAD_ETIMEOUT, the CUDA context stays usable,
    and after rad_reset the same context reproduces the oracle."""
    R = _rad()
    w, X, U, ref = small
    Xd = torch.as_tensor(X, device="cuda")
    Ud = torch.as_tensor(U, device="cuda")
    monkeypatch.setenv("RAD_FAULT", "stall")
    r = _ctx(w, precision, FP32_OPTS if precision == R.RAD_FP32_SPLIT else None)
    monkeypatch.delenv("RAD_FAULT")
    with r:
        t0 = time.perf_counter()
        r.accumulate_steps(0, Xd, Ud)
        with pytest.raises(R.RadError) as ei:
            r.finalize()
        waited = time.perf_counter() - t0
        assert ei.value.code == RAD_ETIMEOUT
        assert "expired" in str(ei.value)
        print(f"bounded wait expired after {waited:.2f} s")
        assert waited < 10.0         # the poll limit is about a second
        # the device is fine: an unrelated kernel runs and synchronises
        z = torch.arange(1000, device="cuda", dtype=torch.float64).sum().item()
        assert z == 999 * 1000 / 2
        r.reset()
        r.accumulate_steps(0, Xd, Ud)
        _check(r.finalize(), ref, 1e-10 if precision == R.RAD_FP64 else 1e-4)
