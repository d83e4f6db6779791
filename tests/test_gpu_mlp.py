"""The surrogate network's tensor-core kernels against the FP64 MLP reference,
and a small end-to-end surrogate trained and judged on the GPU."""
import math

import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _bf16_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda").to(torch.bfloat16)


@pytest.mark.parametrize("ak,bk", [(True, True), (True, False), (False, True), (False, False)])
def test_gemm_layouts(ak, bk):
    from paper_1003_1140_gb300 import mlp
    rng = np.random.default_rng(2)
    M, N, K = 256, 384, 192
    A = ref.bf16(rng.normal(size=(M, K)))          # op(A) [M][K]
    B = ref.bf16(rng.normal(size=(N, K)))          # op(B)^T [N][K]
    Ad = _bf16_dev(A if ak else A.T.copy())
    Bd = _bf16_dev(B if bk else B.T.copy())
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    mlp.gemm(Ad, Bd, M, N, K, ak, bk, C)
    mlp.check()
    exp = A @ B.T
    got = C.cpu().numpy()
    assert np.abs(got - exp).max() <= 1e-4 * np.abs(exp).max()


@pytest.mark.parametrize("ak,bk", [(True, False), (False, True)])
def test_gemm_split_k(ak, bk):
    """Two output tiles over K = 64 x 331: the product splits K into 82 slices
    of 4 or 5 tiles (ragged), reduced in a fixed order."""
    from paper_1003_1140_gb300 import mlp
    rng = np.random.default_rng(5)
    M, N, K = 128, 256, 64 * 331
    A = ref.bf16(rng.normal(size=(M, K)))
    B = ref.bf16(rng.normal(size=(N, K)))
    Ad = _bf16_dev(A if ak else A.T.copy())
    Bd = _bf16_dev(B if bk else B.T.copy())
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    mlp.gemm(Ad, Bd, M, N, K, ak, bk, C)
    C2 = torch.empty_like(C)
    mlp.gemm(Ad, Bd, M, N, K, ak, bk, C2)
    mlp.check()
    exp = A @ B.T
    got = C.cpu().numpy()
    # FP32 accumulation of 10,592 products of unit normals: |error| ~ sqrt(K) 2^-24 max|partial|
    assert np.abs(got - exp).max() <= 1e-4 * np.sqrt(K)
    assert torch.equal(C, C2)            # the slice order is fixed: bitwise repeatable


def test_gradients_split_k_match_reference():
    """A wide output layer (4096) over a 256-wide hidden layer: the input
    gradient G W (M = 128, N = 256, K = 4096) runs split over K."""
    from paper_1003_1140_gb300 import mlp
    rng = np.random.default_rng(6)
    widths = [128, 256, 4096]
    net = mlp.MLP(widths, 100)
    Ws = [(rng.normal(size=(widths[l + 1], widths[l])) / np.sqrt(widths[l])).astype(np.float32)
          for l in range(2)]
    bs = [(rng.normal(size=widths[l + 1]) * 0.1).astype(np.float32) for l in range(2)]
    for l in range(2):
        net.set_layer(l, Ws[l], bs[l])
    x = rng.normal(size=(100, widths[0])).astype(np.float32)
    t = rng.normal(size=(100, widths[-1])).astype(np.float32)
    loss = net.gradients(x, t)
    loss_ref, dW_ref, db_ref = ref.gradients([w.astype(np.float64) for w in Ws], bs, x, t)
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    for l in range(2):
        W, b, dW, db = net.get_layer(l, grads=True)
        assert np.linalg.norm(dW - dW_ref[l]) <= 2e-3 * np.linalg.norm(dW_ref[l]), l
        assert np.linalg.norm(db - db_ref[l]) <= 2e-3 * np.linalg.norm(db_ref[l]), l


def test_gradients_and_adam_match_reference():
    from paper_1003_1140_gb300 import mlp
    rng = np.random.default_rng(3)
    widths = [256, 128, 256, 384]
    net = mlp.MLP(widths, 200)
    Ws = [(rng.normal(size=(widths[l + 1], widths[l])) / np.sqrt(widths[l])).astype(np.float32)
          for l in range(3)]
    bs = [(rng.normal(size=widths[l + 1]) * 0.1).astype(np.float32) for l in range(3)]
    for l in range(3):
        net.set_layer(l, Ws[l], bs[l])
    x = rng.normal(size=(150, widths[0])).astype(np.float32)     # a ragged batch (pads to 256)
    t = rng.normal(size=(150, widths[-1])).astype(np.float32)
    y = net.forward(x)
    y_ref = ref.forward([w.astype(np.float64) for w in Ws], bs, x)[0]
    assert np.linalg.norm(y - y_ref) <= 1e-3 * np.linalg.norm(y_ref)
    loss = net.gradients(x, t)
    loss_ref, dW_ref, db_ref = ref.gradients([w.astype(np.float64) for w in Ws], bs, x, t)
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    grads = []
    for l in range(3):
        W, b, dW, db = net.get_layer(l, grads=True)
        assert np.linalg.norm(dW - dW_ref[l]) <= 2e-3 * np.linalg.norm(dW_ref[l]), l
        assert np.linalg.norm(db - db_ref[l]) <= 2e-3 * np.linalg.norm(db_ref[l]), l
        grads.append((dW, db))
    net.adam(1e-2)
    for l in range(3):
        W, b = net.get_layer(l)
        w_exp, _, _ = ref.adam(Ws[l].astype(np.float64), 0.0, 0.0, grads[l][0].astype(np.float64), 1, 1e-2)
        assert np.abs(W - w_exp).max() <= 1e-5
    net.close()


@pytest.mark.parametrize("widths", [[256, 128, 256, 1024], [128, 384]])
def test_train_step_matches_gradients_then_adam(widths):
    """rad_mlp_train_step against rad_mlp_gradients + rad_mlp_adam over three steps
    of ragged batches: every layer's weights and biases and the losses agree."""
    from paper_1003_1140_gb300 import mlp
    rng = np.random.default_rng(9)
    L = len(widths) - 1
    Ws = [(rng.normal(size=(widths[l + 1], widths[l])) / np.sqrt(widths[l])).astype(np.float32)
          for l in range(L)]
    bs = [(rng.normal(size=widths[l + 1]) * 0.1).astype(np.float32) for l in range(L)]
    nets = [mlp.MLP(widths, 200), mlp.MLP(widths, 200)]
    for net in nets:
        for l in range(L):
            net.set_layer(l, Ws[l], bs[l])
    for step, batch in enumerate((150, 200, 37)):
        x = rng.normal(size=(batch, widths[0])).astype(np.float32)
        t = rng.normal(size=(batch, widths[-1])).astype(np.float32)
        la = nets[0].gradients(x, t)
        nets[0].adam(3e-3)
        lb = nets[1].train_step(x, t, 3e-3)
        assert lb == pytest.approx(la, rel=1e-5), step
        for l in range(L):
            Wa, ba = nets[0].get_layer(l)
            Wb, bb = nets[1].get_layer(l)
            np.testing.assert_allclose(Wb, Wa, rtol=1e-5, atol=1e-7, err_msg=f"step {step} W{l}")
            np.testing.assert_allclose(bb, ba, rtol=1e-5, atol=1e-7, err_msg=f"step {step} b{l}")
            assert np.abs(Wb - Ws[l]).max() > 1e-4          # the step did move the weights
    # the forward pass reads the refreshed BF16 W
    xf = rng.normal(size=(64, widths[0])).astype(np.float32)
    np.testing.assert_allclose(nets[1].forward(xf), nets[0].forward(xf), rtol=1e-3, atol=1e-4)
    for net in nets:
        net.close()
    mlp.check()


def test_predict_applies_transforms_on_device():
    """rad_mlp_predict = log10/standardise -> forward -> 10^(z sd + mu), against
    the same three steps composed on the host around the raw forward pass."""
    from paper_1003_1140_gb300 import mlp
    rng = np.random.default_rng(8)
    widths = [256, 128, 384]
    net = mlp.MLP(widths, 64)
    net.init_params(3)
    x = (10.0 ** rng.uniform(-8, 2, size=(50, widths[0]))).astype(np.float32)
    x[:, -6:] = 0.0                                       # padded features: raw zero
    floor = 1e-30
    in_mu = rng.normal(size=widths[0]) - 3.0
    in_sd = rng.uniform(0.5, 2.0, size=widths[0])
    in_mu[-6:], in_sd[-6:] = math.log10(floor), 1.0
    out_mu = rng.normal(size=widths[-1])
    out_sd = rng.uniform(0.1, 0.5, size=widths[-1])
    net.set_transform(in_mu, in_sd, out_mu, out_sd, floor)
    got = net.predict(x)
    xn = ((np.log10(np.maximum(x.astype(np.float64), floor)) - in_mu) / in_sd).astype(np.float32)
    assert np.all(xn[:, -6:] == 0.0)
    z = net.forward(xn).astype(np.float64)
    exp = 10.0 ** (z * out_sd + out_mu)
    # the device takes log10 in FP32: standardised inputs may round to a
    # neighbouring BF16 value, moving log10 y by a small fraction of a percent
    assert np.abs(np.log10(got) - np.log10(exp)).max() <= 2e-3
    net.close()


def test_training_reduces_loss():
    from paper_1003_1140_gb300 import mlp
    rng = np.random.default_rng(4)
    net = mlp.MLP([128, 256, 128], 128)
    net.init_params(0)
    x = torch.as_tensor(rng.normal(size=(128, 128)).astype(np.float32), device="cuda")
    Wt = rng.normal(size=(128, 128)).astype(np.float32) / 11
    t = torch.as_tensor(np.tanh(x.cpu().numpy() @ Wt.T), device="cuda")
    first = net.train_step(x, t, 1e-3)
    for _ in range(300):
        last = net.train_step(x, t, 1e-3)
    assert last < 0.2 * first
    net.close()


def test_small_surrogate_beats_interpolation():
    """Sparse (12 directions x 16 omega, exact) -> dense (48 directions x 256 omega)
    on 64-particle, 400-sample workloads: the trained network's held-out error is
    below that of the method without it (interpolating the sparse set)."""
    from paper_1003_1140_gb300 import surrogate as su
    spec = su.SurrogateSpec(particles=64, n_calls=401, nside=2, n_omega=256, omega_stride=16,
                            hidden=(256, 256, 256))
    tr_d, tr_s = su.generate(spec, range(384))
    te_d, te_s = su.generate(spec, range(100_000, 100_032))
    assert np.all(np.isfinite(tr_d)) and np.all(tr_d > 0)
    s = su.Surrogate(spec, tr_s, tr_d)
    losses = s.train(tr_s, tr_d, epochs=150, lr=1e-3)
    assert losses[-1] < 0.5 * losses[0]
    pred = s.predict(te_s)
    base = su.interpolate_baseline(spec, te_s)
    _, dex_n = su.errors(pred, te_d)
    _, dex_b = su.errors(base, te_d)
    print("held-out rms dex: network", np.median(dex_n), "interpolation", np.median(dex_b))
    assert np.median(dex_n) < np.median(dex_b)
