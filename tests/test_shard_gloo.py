"""Multi-rank particle sharding (CPU, gloo, world size 2): each rank computes its
shard's partial sums with the FP64 oracle, the ranks all-reduce them, and the
spectrum of the union equals the oracle's spectrum of all particles."""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    import trajgen
    w = trajgen.config(1, 9 / 1024)
    X, U = w.trajectory_numpy(n_calls=121)
    dirs = np.array([[0.0, 1.0, 0.0], [0.6, 0.0, 0.8]])
    om = np.array([0.3, 3.0, 30.0])
    return w, X, U, dirs, om


def _basis(n):
    """An orthonormal pair (e1, e2) normal to the unit vector n (any such pair: the
    coherent spectrum |A|^2 = |A.e1|^2 + |A.e2|^2 because A is normal to n)."""
    a = np.eye(3)[int(np.argmin(np.abs(n)))]
    e1 = np.cross(n, a)
    e1 /= np.linalg.norm(e1)
    return e1, np.cross(n, e1)


def _partial(X, U, w, dirs, om, first, n, coherent, layout="vector"):
    """A shard's unscaled particle sums: incoherent sum_j |A_j|^2 per bin; coherent
    sum_j A_j per bin as its 3 complex components ("vector", 6 numbers) or, as
    rad_partial_sums lays it out, as Re, Im of A.e1 and A.e2 ("basis", 4 numbers)."""
    import oracle
    r, b, bd = oracle.samples(X[:, :, first:first + n], U[:, :, first:first + n], w.dt, w.L)
    if not coherent:
        S = oracle.window_spectrum(r, b, bd, -np.ones(n), w.dt, dirs, om, 0, 120)
        return (S * 4 * math.pi ** 2).reshape(-1)
    width = 6 if layout == "vector" else 4
    out = np.zeros((len(dirs) * len(om), width))
    for d, nv in enumerate(dirs):
        e1, e2 = _basis(np.asarray(nv) / np.linalg.norm(nv))
        for j in range(n):
            A = oracle.amplitude(r, b, bd, j, 0, 120, w.dt, -1.0, nv, om)   # [nf, 3]
            if layout == "vector":
                part = np.concatenate([A.real, A.imag], 1)
            else:
                a1, a2 = A @ e1, A @ e2
                part = np.stack([a1.real, a1.imag, a2.real, a2.imag], 1)
            out[d * len(om):(d + 1) * len(om)] += part
    return out


def _worker(rank, world, port, coherent, layout, result_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1003_1140_gb300 import shard
    w, X, U, dirs, om = _case()
    first, n = shard.shard(X.shape[2], rank, world)
    part = _partial(X, U, w, dirs, om, first, n, coherent, layout)
    S = shard.allreduce_spectrum(part, coherent)
    if rank == 0:
        result_q.put(S)
    dist.destroy_process_group()


@pytest.mark.parametrize("coherent,layout", [(False, "vector"), (True, "vector"),
                                             (True, "basis")])
def test_two_rank_shards_reduce_to_the_full_spectrum(coherent, layout):
    import multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, coherent, layout, q))
             for r in range(2)]
    for p in procs:
        p.start()
    S = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w, X, U, dirs, om = _case()
    ref = oracle.spectra(X, U, w.dt, dirs, [om], [(0, 120, 1, 0)], [(X.shape[2], -1.0)],
                         coherent=coherent, box_L=w.L)[0].reshape(-1)
    np.testing.assert_allclose(S, ref, rtol=1e-11)


def test_shard_ranges_cover_and_balance():
    from paper_1003_1140_gb300 import shard
    for count in (0, 1, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            rs = [shard.shard(count, r, world) for r in range(world)]
            assert rs[0][0] == 0
            assert sum(n for _, n in rs) == count
            for (f0, n0), (f1, _) in zip(rs, rs[1:]):
                assert f0 + n0 == f1
            assert max(n for _, n in rs) - min(n for _, n in rs) <= 1


# ---------------------------------------------------------------------------
# failure detection between ranks, on the host (no GPU is involved)
# ---------------------------------------------------------------------------
def _failure_worker(rank, world, port, store_port, mode, result_q):
    """mode "ok": both ranks check in and reduce; "fail": rank 1 raises before it
    checks in (its shard failed); "leave": rank 1 exits right after joining and
    rank 0 reduces without a store (only the process-group timeout can end it)."""
    import datetime
    import time as _time
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    store = dist.TCPStore("127.0.0.1", store_port, world, is_master=(rank == 0),
                          timeout=datetime.timedelta(seconds=30), wait_for_workers=False)
    from paper_1003_1140_gb300 import shard
    part = np.full(6, float(rank + 1))
    if rank == 1 and mode == "leave":
        os._exit(0)                                  # gone between steps, nothing in flight
    if rank == 1 and mode == "fail":
        raise RuntimeError("shard 1 failed")         # never checks in
    t0 = _time.monotonic()
    try:
        if mode == "leave":
            S = shard.allreduce_spectrum(part, False)
        else:
            S = shard.allreduce_spectrum(part, False, store=store, tag="window-0", timeout_s=2.0)
        out = ("ok", S.tolist(), _time.monotonic() - t0)
    except Exception as e:                           # noqa: BLE001 -- reported to the test
        out = ("raised", str(e), _time.monotonic() - t0)
    if rank == 0:
        result_q.put(out)
        result_q.close()
        result_q.join_thread()                       # flush before the hard exit
    if mode == "ok":
        dist.destroy_process_group()
    os._exit(0)


def _run_failure_case(mode):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port, store_port = _free_port(), _free_port()
    procs = [ctx.Process(target=_failure_worker, args=(r, 2, port, store_port, mode, q))
             for r in range(2)]
    for p in procs:
        p.start()
    try:
        return q.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()                              # this test's own child, by handle
                p.join(timeout=10)


def test_check_in_then_reduce():
    kind, S, _ = _run_failure_case("ok")
    assert kind == "ok"
    np.testing.assert_allclose(S, 3.0 / (4 * math.pi ** 2))  # 1 + 2 over both ranks


def test_a_rank_that_failed_is_named_before_the_reduction():
    kind, msg, waited = _run_failure_case("fail")
    assert kind == "raised" and "[1]" in msg and "window-0" in msg
    assert waited < 10.0


def test_a_reduction_whose_peer_left_ends_with_an_error():
    kind, msg, waited = _run_failure_case("leave")
    assert kind == "raised"
    assert waited < 60.0
