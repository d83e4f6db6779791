"""ctypes binding of include/rad_mlp.h (argument marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import rad as _rad

RAD_MLP_OK = 0
EXPORTED = ("rad_mlp_init", "rad_mlp_set_layer", "rad_mlp_get_layer", "rad_mlp_forward",
            "rad_mlp_gradients", "rad_mlp_adam", "rad_mlp_train_step", "rad_mlp_gemm",
            "rad_mlp_check",
            "rad_mlp_set_transform", "rad_mlp_predict",
            "rad_mlp_last_error", "rad_mlp_destroy")


def _lib():
    lib = _rad.load()
    if not getattr(lib, "_mlp_bound", False):
        vp = ctypes.c_void_p
        lib.rad_mlp_init.restype = ctypes.c_int
        lib.rad_mlp_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.c_int32, ctypes.c_int32, vp]
        lib.rad_mlp_set_layer.restype = ctypes.c_int
        lib.rad_mlp_set_layer.argtypes = [vp, ctypes.c_int32, vp, vp]
        lib.rad_mlp_get_layer.restype = ctypes.c_int
        lib.rad_mlp_get_layer.argtypes = [vp, ctypes.c_int32, vp, vp, vp, vp]
        lib.rad_mlp_forward.restype = ctypes.c_int
        lib.rad_mlp_forward.argtypes = [vp, ctypes.c_int32, vp, vp]
        lib.rad_mlp_gradients.restype = ctypes.c_int
        lib.rad_mlp_gradients.argtypes = [vp, ctypes.c_int32, vp, vp,
                                          ctypes.POINTER(ctypes.c_double)]
        lib.rad_mlp_adam.restype = ctypes.c_int
        lib.rad_mlp_adam.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float]
        lib.rad_mlp_train_step.restype = ctypes.c_int
        lib.rad_mlp_train_step.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.c_float,
                                           ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                           ctypes.POINTER(ctypes.c_double)]
        lib.rad_mlp_gemm.restype = ctypes.c_int
        lib.rad_mlp_gemm.argtypes = [ctypes.c_int32] * 5 + [vp, vp, vp]
        lib.rad_mlp_set_transform.restype = ctypes.c_int
        lib.rad_mlp_set_transform.argtypes = [vp, vp, vp, vp, vp, ctypes.c_float]
        lib.rad_mlp_predict.restype = ctypes.c_int
        lib.rad_mlp_predict.argtypes = [vp, ctypes.c_int32, vp, vp]
        lib.rad_mlp_check.restype = ctypes.c_int
        lib.rad_mlp_check.argtypes = []
        lib.rad_mlp_last_error.restype = ctypes.c_char_p
        lib.rad_mlp_last_error.argtypes = []
        lib.rad_mlp_destroy.restype = None
        lib.rad_mlp_destroy.argtypes = [vp]
        lib._mlp_bound = True
    return lib


def _p(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float32 and a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


class MLP:
    """A ReLU MLP whose every step runs in the library's kernels."""

    def __init__(self, widths, max_batch, stream=None):
        self._lib = _lib()
        self.widths = [int(w) for w in widths]
        self.h = ctypes.c_void_p()
        arr = (ctypes.c_int32 * len(widths))(*self.widths)
        st = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        rc = self._lib.rad_mlp_init(ctypes.byref(self.h), arr, len(widths) - 1, int(max_batch), st)
        if rc != RAD_MLP_OK:
            self.h = None
            raise RuntimeError(f"rad_mlp_init failed ({rc})")

    def _chk(self, rc, what):
        if rc != RAD_MLP_OK:
            raise RuntimeError(f"{what} failed ({rc}): {last_error()}")

    @property
    def n_layers(self):
        return len(self.widths) - 1

    def set_layer(self, l, W, b):
        self._chk(self._lib.rad_mlp_set_layer(self.h, l, _p(W), _p(b)), "rad_mlp_set_layer")

    def get_layer(self, l, grads=False):
        o, i = self.widths[l + 1], self.widths[l]
        W = np.empty((o, i), np.float32)
        b = np.empty(o, np.float32)
        dW = np.empty((o, i), np.float32) if grads else None
        db = np.empty(o, np.float32) if grads else None
        self._chk(self._lib.rad_mlp_get_layer(self.h, l, _p(W), _p(b), _p(dW), _p(db)),
                  "rad_mlp_get_layer")
        return (W, b, dW, db) if grads else (W, b)

    def init_params(self, seed=0):
        """He-initialised weights, zero biases (FP32 master copies)."""
        rng = np.random.default_rng(seed)
        for l in range(self.n_layers):
            o, i = self.widths[l + 1], self.widths[l]
            W = (rng.standard_normal((o, i)) * np.sqrt(2.0 / i)).astype(np.float32)
            self.set_layer(l, W, np.zeros(o, np.float32))

    def forward(self, x, y=None):
        if y is None:
            y = np.empty((x.shape[0], self.widths[-1]), np.float32)
        self._chk(self._lib.rad_mlp_forward(self.h, x.shape[0], _p(x), _p(y)), "rad_mlp_forward")
        return y

    def set_transform(self, in_mu, in_sd, out_mu, out_sd, floor):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (in_mu, in_sd, out_mu, out_sd)]
        self._chk(self._lib.rad_mlp_set_transform(self.h, *[_p(a) for a in arrs], float(floor)),
                  "rad_mlp_set_transform")

    def predict(self, x, y=None):
        """Physical-unit prediction (transforms on the device)."""
        if y is None:
            y = np.empty((x.shape[0], self.widths[-1]), np.float32)
        self._chk(self._lib.rad_mlp_predict(self.h, x.shape[0], _p(x), _p(y)), "rad_mlp_predict")
        return y

    def gradients(self, x, t):
        loss = ctypes.c_double()
        self._chk(self._lib.rad_mlp_gradients(self.h, x.shape[0], _p(x), _p(t), ctypes.byref(loss)),
                  "rad_mlp_gradients")
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self._chk(self._lib.rad_mlp_adam(self.h, lr, beta1, beta2, eps), "rad_mlp_adam")

    def train_step(self, x, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        """Gradients and Adam in one call (rad_mlp_train_step)."""
        loss = ctypes.c_double()
        self._chk(self._lib.rad_mlp_train_step(self.h, x.shape[0], _p(x), _p(t), lr, beta1, beta2,
                                               eps, ctypes.byref(loss)), "rad_mlp_train_step")
        return loss.value

    def close(self):
        if getattr(self, "h", None):
            self._lib.rad_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gemm(A, B, M, N, K, a_kcontig, b_kcontig, C):
    """C (FP32, device) = op(A) op(B) on the tensor cores; A, B BF16 device tensors
    (M, N multiples of 128, K of 64).  Enqueued on the default stream."""
    rc = _lib().rad_mlp_gemm(1 if a_kcontig else 0, 1 if b_kcontig else 0, M, N, K,
                             A.data_ptr(), B.data_ptr(), C.data_ptr())
    if rc != RAD_MLP_OK:
        raise RuntimeError(f"rad_mlp_gemm failed ({rc}): {last_error()}")
    return C


def check():
    """Waits for the device; raises if a GEMM block's bounded wait expired."""
    rc = _lib().rad_mlp_check()
    if rc != RAD_MLP_OK:
        raise RuntimeError(f"rad_mlp_check failed ({rc}): {last_error()}")


def last_error():
    return _lib().rad_mlp_last_error().decode(errors="replace")
