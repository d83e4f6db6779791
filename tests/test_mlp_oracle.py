"""Pins for the FP64 MLP reference (oracle/mlp.py), CPU only."""
import numpy as np

from oracle import mlp


def test_bf16_rounding_ties_to_even():
    # BF16 keeps 8 significant bits: the spacing just above 1 is 2^-7
    x = np.array([1.0, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -8,
                  1.0 + 2 ** -7 + 2 ** -8, -2.5, 0.0], dtype=np.float32)
    r = mlp.bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # below half-way: down
    assert r[2] == 1.0 + 2 ** -7            # above half-way: up
    assert r[3] == 1.0                      # half-way, 1.0 has the even last bit: down
    assert r[4] == 1.0 + 2 ** -6            # half-way, 1 + 2^-6 is the even neighbour: up
    assert r[5] == -2.5 and r[6] == 0.0


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    widths = [5, 7, 6, 4]
    Ws = [rng.normal(size=(widths[l + 1], widths[l])) for l in range(3)]
    bs = [rng.normal(size=widths[l + 1]) * 0.1 for l in range(3)]
    x = rng.normal(size=(9, 5))
    t = rng.normal(size=(9, 4))
    loss, dW, db = mlp.gradients(Ws, bs, x, t, round_bf16=False)
    eps = 1e-6
    for l in range(3):
        for (i, j) in [(0, 0), (1, 2), (widths[l + 1] - 1, widths[l] - 1)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][i, j] += eps
            Wm[l][i, j] -= eps
            fd = (mlp.gradients(Wp, bs, x, t, False)[0] - mlp.gradients(Wm, bs, x, t, False)[0]) / (2 * eps)
            assert abs(fd - dW[l][i, j]) <= 1e-6 * max(1.0, abs(fd))
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][1] += eps
        bm[l][1] -= eps
        fd = (mlp.gradients(Ws, bp, x, t, False)[0] - mlp.gradients(Ws, bm, x, t, False)[0]) / (2 * eps)
        assert abs(fd - db[l][1]) <= 1e-6 * max(1.0, abs(fd))


def test_single_linear_layer_closed_form():
    rng = np.random.default_rng(1)
    W = rng.normal(size=(3, 4))
    b = rng.normal(size=3)
    x = rng.normal(size=(6, 4))
    t = rng.normal(size=(6, 3))
    loss, dW, db = mlp.gradients([W], [b], x, t, round_bf16=False)
    r = x @ W.T + b - t
    np.testing.assert_allclose(loss, (r ** 2).mean())
    np.testing.assert_allclose(dW[0], 2.0 / r.size * r.T @ x)
    np.testing.assert_allclose(db[0], 2.0 / r.size * r.sum(0))


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3])
    w, m, v = mlp.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.1, eps=0.0)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> w = -lr sign(g)
    np.testing.assert_allclose(w, -0.1 * np.sign(g), rtol=1e-12)
