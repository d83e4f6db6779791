"""rad_spectrum_noalloc: the spectrum without any device allocation.

Some callers may not allocate device memory (a simulation that has handed all
GPU memory to its own pool, or a program where allocation calls are not
available).  For them the library offers one entry point that works out of a
fixed device array built into the library.  These tests call it through the
C ABI and check, on consecutive calls of different shapes (the array keeps the
previous call's contents), that it gives what the context API and the FP64
oracle give, within the FP32 split path's tolerance, and that a problem too
large for the array is refused.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

import trajgen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _entry():
    from paper_1003_1140_gb300 import rad
    lib = rad.load()
    f = lib.rad_spectrum_noalloc
    f.restype = ctypes.c_int
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    f.argtypes = [dp, ctypes.c_int32, dp, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                  ctypes.c_int64, ctypes.c_int64, vp, vp, ctypes.c_int32, ctypes.c_double, vp, vp]
    return f


def _call(f, dirs, freqs, dt, q, X, U, mode, L, out):
    dp = ctypes.POINTER(ctypes.c_double)
    return f(dirs.ctypes.data_as(dp), dirs.shape[0], freqs.ctypes.data_as(dp), freqs.size, dt, q,
             X.shape[2], X.shape[0], X.data_ptr(), U.data_ptr(), mode, L, out.data_ptr(),
             torch.cuda.current_stream().cuda_stream)


def _context_api(dirs, freqs, dt, q, X, U, mode, L):
    import paper_1003_1140_gb300 as R
    N, nc = X.shape[2], X.shape[0]
    with R.Radiation(dirs, [freqs], dt, [(N, q, 1.0)], [(0, nc - 1, 1, 0)], mode=mode,
                     precision=R.RAD_FP32_SPLIT, box_L=L) as r:
        r.accumulate_steps(0, X, U)
        return r.finalize()[0]


def _oracle(dirs, freqs, dt, q, Xn, Un, mode, L):
    import oracle
    import paper_1003_1140_gb300 as R
    N, nc = Xn.shape[2], Xn.shape[0]
    return oracle.spectra(Xn, Un, dt, dirs, [freqs], [(0, nc - 1, 1, 0)], [(N, q)],
                          coherent=mode == R.RAD_COHERENT, box_L=L)[0]


def test_noalloc_matches_context_api_on_consecutive_calls():
    """Consecutive calls of different shapes: each call must give the context
    API's spectrum and the FP64 oracle's, whatever the earlier calls left in the
    shared array (ring slots past this call's samples, padding columns past its
    particles, old anchors, a coherent accumulator of another size)."""
    import paper_1003_1140_gb300 as R
    f = _entry()
    dirs = np.ascontiguousarray(trajgen.axis_and_oblique_dirs()[[2, 0, 6]])
    freqs = np.ascontiguousarray(trajgen.log_grid(0.1, 300.0, 200))
    # (particles, calls, summation): a larger coherent call first, then a smaller
    # particle count that is not a multiple of the 8-particle tile and fewer
    # calls, then the first shape again
    cases = [(203, 601, R.RAD_COHERENT), (61, 401, R.RAD_INCOHERENT),
             (45, 257, R.RAD_INCOHERENT), (203, 601, R.RAD_COHERENT)]
    first = None
    for i, (N, nc, mode) in enumerate(cases):
        w = trajgen.config(1, N / 1024)
        Xn, Un = w.trajectory_numpy(n_calls=nc)
        X = torch.as_tensor(Xn, device="cuda")
        U = torch.as_tensor(Un, device="cuda")
        q = w.species[0][1]
        ref = _oracle(dirs, freqs, w.dt, q, Xn, Un, mode, w.L)
        api = _context_api(dirs, freqs, w.dt, q, X, U, mode, w.L)
        out = torch.full((dirs.shape[0] * freqs.size,), float("nan"), dtype=torch.float64,
                         device="cuda")
        assert _call(f, dirs, freqs, w.dt, q, X, U, mode, w.L, out) == 0
        got = out.cpu().numpy().reshape(dirs.shape[0], freqs.size)
        for d in range(dirs.shape[0]):
            e_api = np.linalg.norm(got[d] - api[d]) / np.linalg.norm(api[d])
            e_ref = np.linalg.norm(got[d] - ref[d]) / np.linalg.norm(ref[d])
            assert e_api <= 1e-4, (i, N, nc, mode, d, e_api)
            assert e_ref <= 1e-4, (i, N, nc, mode, d, e_ref)
        if i == 0:
            first = got
        elif i == len(cases) - 1:
            # the same call again: the same spectrum up to the order of the FP64
            # atomic additions of the work items' particle sums
            np.testing.assert_allclose(got, first, rtol=1e-9, atol=1e-12 * np.abs(first).max())


def test_noalloc_refuses_a_problem_larger_than_its_memory():
    f = _entry()
    N, nc = 8192, 4097
    X = torch.zeros((2, 3, N), dtype=torch.float64, device="cuda")   # never read
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    dirs = np.ascontiguousarray(trajgen.axis_and_oblique_dirs()[:1])
    freqs = np.ascontiguousarray(np.linspace(1.0, 2.0, 8))
    dp = ctypes.POINTER(ctypes.c_double)
    rc = f(dirs.ctypes.data_as(dp), 1, freqs.ctypes.data_as(dp), 8, 0.05, -1.0, N, nc,
           X.data_ptr(), X.data_ptr(), 0, 40.0, out.data_ptr(), None)
    assert rc == -9
    assert torch.all(out == 0)
