"""GPU pusher of the synthetic-trajectory generator (builds trajgen/push.cu).

Input generation only: it makes the leapfrog states of a ``Workload`` on the
GPU (FP32 Boris steps in the workload's mode field) for sizes the NumPy
pusher cannot handle.  Uses torch for device memory.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libtrajgen.so")
SRC = os.path.join(HERE, "push.cu")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                           "-Xcompiler", "-fPIC", "-shared", SRC, "-o", tmp])
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            lib.tg_push.restype = ctypes.c_int
            lib.tg_push.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                    ctypes.c_double, vp, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                                    vp, vp, vp]
            _lib = lib
    return _lib


class GpuPusher:
    """Holds a workload's particle state on the GPU and emits calls on demand."""

    def __init__(self, workload, first: int = 0, count: int | None = None, device="cuda"):
        import torch
        self.torch = torch
        x0, u0, qm = workload.initial_state(first, count)
        f = workload.field()
        t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device).contiguous()
        self.xs, self.us, self.qm = t(x0), t(u0), t(qm)
        self.ky, self.kz, self.psi, self.amp = t(f.ky), t(f.kz), t(f.psi), t(f.amp)
        self.N = x0.shape[1]
        self.L = workload.L
        self.dt = workload.dt
        self.device = device

    def push(self, n_calls: int, X=None, U=None):
        """Fill (or allocate) X, U [n_calls, 3, N] with the next n_calls states."""
        torch = self.torch
        if X is None:
            X = torch.empty((n_calls, 3, self.N), dtype=torch.float64, device=self.device)
            U = torch.empty_like(X)
        st = torch.cuda.current_stream().cuda_stream
        rc = _load().tg_push(self.N, n_calls, self.L, self.dt, self.qm.data_ptr(),
                             self.ky.numel(), self.ky.data_ptr(), self.kz.data_ptr(),
                             self.psi.data_ptr(), self.amp.data_ptr(), self.xs.data_ptr(),
                             self.us.data_ptr(), X.data_ptr(), U.data_ptr(), st)
        if rc != 0:
            raise RuntimeError(f"tg_push failed ({rc})")
        return X, U


def trajectory_gpu(workload, first: int = 0, count: int | None = None, n_calls=None):
    """Whole trajectory X, U [n_calls, 3, N] as CUDA tensors."""
    p = GpuPusher(workload, first, count)
    return p.push(workload.n_calls if n_calls is None else n_calls)
