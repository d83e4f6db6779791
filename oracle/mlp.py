"""FP64 CPU reference of the surrogate network -- TEST INFRASTRUCTURE ONLY.

Plain NumPy forward, backward and Adam of the ReLU MLP the surrogate uses,
with the rounding points the device library documents (include/rad_mlp.h):
operands are rounded to BF16 where they enter a product, every product and
sum is then carried out in FP64.  Used by the tests to check the tensor-core
kernels' gradients and updates; never imported by the library.

Parity status: pinned by tests/test_mlp_oracle.py (finite differences of the
FP64 network without BF16 rounding, and a closed-form single-layer case).
"""
from __future__ import annotations

import numpy as np


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    if nan.any():
        out[nan] = np.nan
    return out


def forward(Ws, bs, x, round_bf16=True):
    """Returns (y, hs, zs): hs[l] the inputs of layer l (after rounding), zs[l] the
    pre-activations z_{l+1}."""
    rnd = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    h = rnd(x)
    hs, zs = [h], []
    L = len(Ws)
    for l in range(L):
        z = h @ rnd(Ws[l]).T + np.asarray(bs[l], dtype=np.float64)
        zs.append(z)
        if l < L - 1:
            h = rnd(np.maximum(z, 0.0))
            hs.append(h)
    return zs[-1], hs, zs


def gradients(Ws, bs, x, t, round_bf16=True):
    """MSE loss and its gradients dW, db for every layer."""
    rnd = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    y, hs, zs = forward(Ws, bs, x, round_bf16)
    B, N = y.shape
    diff = y - t
    loss = float(np.mean(diff ** 2))
    g = 2.0 * diff / (B * N)
    if round_bf16:
        g = g.astype(np.float32).astype(np.float64)
    L = len(Ws)
    dW, db = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        gr = rnd(g)
        dW[l] = gr.T @ hs[l]
        db[l] = g.sum(0)
        if l > 0:
            gp = (gr @ rnd(Ws[l])) * (zs[l - 1] > 0)
            if round_bf16:
                gp = gp.astype(np.float32).astype(np.float64)
            g = gp
    return loss, dW, db


def adam(w, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (returns new w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
