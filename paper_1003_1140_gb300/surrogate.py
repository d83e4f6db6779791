"""Learned surrogate: dense omega x n spectra from a sparse, exactly computed subset.

The sparse input is a literal subset of the dense grid -- every `stride`-th
frequency at a few directions (one per HEALPix base pixel for the 192-direction
grid) -- computed exactly by the radiation library.  A ReLU MLP (BF16 weights,
FP32 accumulation, trained by the library's own tensor-core kernels) maps the
normalised log10 sparse spectrum to the normalised log10 dense spectrum.  The
full accumulation is both the fallback and the measure of its error: held-out
spectra are compared with it, and with the method without the network (interpolation of
the sparse set in log-frequency and, across directions, from the nearest
sparse direction).

Workload (5 in the workload list): 1024 electrons, 2000 samples, dt 0.05,
192 HEALPix Nside-4 directions, 2048 log omega in [0.1, 1000]; training seeds
vary the field seed, the beam gamma in U[2, 10] and the rms field in
logU[0.03, 0.3].
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

import trajgen

from . import rad as R
from .mlp import MLP


@dataclass
class SurrogateSpec:
    particles: int = 1024
    n_calls: int = 2001
    dt: float = 0.05
    nside: int = 4
    n_omega: int = 2048
    omega_lo: float = 0.1
    omega_hi: float = 1000.0
    omega_stride: int = 32          # sparse frequencies: every 32nd
    hidden: tuple = (512, 512, 512)
    gamma_range: tuple = (2.0, 10.0)
    brms_range: tuple = (0.03, 0.3)
    dirs_subset: int | None = None  # keep only the first n dense directions (tests)

    def dense_dirs(self):
        d = trajgen.healpix_centres(self.nside)
        return d if self.dirs_subset is None else d[: self.dirs_subset]

    def sparse_dir_index(self):
        """One dense direction per HEALPix base pixel: the nearest to each of the
        12 base-pixel centres (restricted to the kept directions)."""
        dense = self.dense_dirs()
        base = trajgen.healpix_centres(1)
        idx = []
        for b in base:
            order = np.argsort(-(dense @ b))
            for i in order:
                if i not in idx:
                    idx.append(int(i))
                    break
        return np.array(sorted(set(idx))[: min(12, len(dense))])

    def omegas(self):
        return trajgen.log_grid(self.omega_lo, self.omega_hi, self.n_omega)

    def sparse_omega_index(self):
        return np.arange(0, self.n_omega, self.omega_stride)


def _workload(spec: SurrogateSpec, seed: int):
    rng = np.random.default_rng(10_000 + seed)
    gamma = rng.uniform(*spec.gamma_range)
    brms = math.exp(rng.uniform(math.log(spec.brms_range[0]), math.log(spec.brms_range[1])))
    w = trajgen.Workload(f"surrogate-seed{seed}", [(spec.particles, -1.0, 1.0, gamma)],
                         spec.n_calls, spec.dt, spec.dense_dirs(), [spec.omegas()],
                         [(0, spec.n_calls - 1, 1, 0)], field_seed=1000 + seed,
                         particle_seed=5000 + seed, b_rms=brms)
    return w


def generate(spec: SurrogateSpec, seeds, with_timing=False):
    """Dense spectra [n, D, F] and sparse inputs [n, Ds, Fs] for the seeds (GPU)."""
    import torch
    from trajgen import gpu as tg
    dense, sparse = [], []
    t_dense = t_sparse = 0.0
    si, fi = spec.sparse_dir_index(), spec.sparse_omega_index()
    for seed in seeds:
        w = _workload(spec, seed)
        X, U = tg.trajectory_gpu(w)
        sp = [(w.species[0][0], w.species[0][1], 1.0)]
        with R.Radiation(w.dirs, w.grids, w.dt, sp, w.windows, precision=R.RAD_FP32_SPLIT,
                         box_L=w.L) as r:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r.accumulate_steps(0, X, U)
            S = r.finalize()[0]
            t_dense += time.perf_counter() - t0
        with R.Radiation(w.dirs[si], [w.grids[0][fi]], w.dt, sp, w.windows,
                         precision=R.RAD_FP32_SPLIT, box_L=w.L) as r:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r.accumulate_steps(0, X, U)
            Ss = r.finalize()[0]
            t_sparse += time.perf_counter() - t0
        dense.append(S.astype(np.float32))
        sparse.append(Ss.astype(np.float32))
        del X, U
    out = (np.stack(dense), np.stack(sparse))
    if with_timing:
        return out + (t_dense / len(seeds), t_sparse / len(seeds))
    return out


FLOOR = 1e-30


def _pad128(n):
    return (n + 127) // 128 * 128


class Normaliser:
    """log10, then per-feature standardisation fitted on the training set."""

    def __init__(self, data):
        lg = np.log10(np.maximum(data.reshape(len(data), -1), FLOOR))
        self.mu = lg.mean(0)
        self.sd = lg.std(0) + 1e-3

    def forward(self, data):
        lg = np.log10(np.maximum(data.reshape(len(data), -1), FLOOR))
        return ((lg - self.mu) / self.sd).astype(np.float32)

    def inverse(self, z):
        return 10.0 ** (z.astype(np.float64) * self.sd + self.mu)


class Surrogate:
    def __init__(self, spec: SurrogateSpec, train_sparse, train_dense, seed=0):
        self.spec = spec
        self.nx = Normaliser(train_sparse)
        self.ny = Normaliser(train_dense)
        self.in_dim = train_sparse[0].size
        self.out_dim = train_dense[0].size
        self.in_pad = _pad128(self.in_dim)
        self.out_pad = _pad128(self.out_dim)
        self.dense_shape = train_dense.shape[1:]
        self.batch = 128
        self.net = MLP([self.in_pad, *spec.hidden, self.out_pad], self.batch)
        self.net.init_params(seed)
        # the same transforms on the device for prediction; padded input
        # features (raw 0 -> log10 floor) map to 0 as in training
        lf = math.log10(FLOOR)
        in_mu = np.full(self.in_pad, lf)
        in_sd = np.ones(self.in_pad)
        in_mu[: self.in_dim], in_sd[: self.in_dim] = self.nx.mu, self.nx.sd
        out_mu = np.zeros(self.out_pad)
        out_sd = np.ones(self.out_pad)
        out_mu[: self.out_dim], out_sd[: self.out_dim] = self.ny.mu, self.ny.sd
        self.net.set_transform(in_mu, in_sd, out_mu, out_sd, FLOOR)

    def _x(self, sparse):
        x = np.zeros((len(sparse), self.in_pad), np.float32)
        x[:, : self.in_dim] = self.nx.forward(sparse)
        return x

    def _y(self, dense):
        y = np.zeros((len(dense), self.out_pad), np.float32)
        y[:, : self.out_dim] = self.ny.forward(dense)
        return y

    def train(self, sparse, dense, epochs=100, lr=1e-3, lr_final=1e-5, seed=0, log=None):
        import torch
        X = torch.as_tensor(self._x(sparse), device="cuda")
        Y = torch.as_tensor(self._y(dense), device="cuda")
        n = len(X)
        rng = np.random.default_rng(seed)
        steps_per_epoch = max(1, math.ceil(n / self.batch))
        total = epochs * steps_per_epoch
        k = 0
        losses = []
        for ep in range(epochs):
            perm = torch.as_tensor(rng.permutation(n), device="cuda")
            el = 0.0
            for s in range(steps_per_epoch):
                idx = perm[s * self.batch:(s + 1) * self.batch]
                xb = X.index_select(0, idx).contiguous()
                yb = Y.index_select(0, idx).contiguous()
                cur = lr * (lr_final / lr) ** (k / max(1, total - 1))   # exponential decay
                el += self.net.train_step(xb, yb, cur)
                k += 1
            losses.append(el / steps_per_epoch)
            if log and (ep % 10 == 0 or ep == epochs - 1):
                log(f"epoch {ep} loss {losses[-1]:.5f}")
        return losses

    def predict(self, sparse):
        """Dense spectra from raw sparse spectra: log/standardise, the network and
        the inverse transform all run on the device (rad_mlp_predict)."""
        import torch
        raw = np.zeros((len(sparse), self.in_pad), np.float32)
        raw[:, : self.in_dim] = sparse.reshape(len(sparse), -1)
        X = torch.as_tensor(raw, device="cuda")
        Y = torch.empty((len(sparse), self.out_pad), dtype=torch.float32, device="cuda")
        for s in range(0, len(X), self.batch):
            self.net.predict(X[s:s + self.batch], Y[s:s + self.batch])
        return Y[:, : self.out_dim].cpu().numpy().astype(np.float64).reshape(
            (len(sparse),) + self.dense_shape)


def interpolate_baseline(spec: SurrogateSpec, sparse):
    """The method without the network: log-log interpolation in omega of each
    sparse direction, and the nearest sparse direction for every dense one."""
    dense_dirs = spec.dense_dirs()
    si = spec.sparse_dir_index()
    lw_dense = np.log(spec.omegas())
    lw_sparse = lw_dense[spec.sparse_omega_index()]
    nearest = np.argmax(dense_dirs @ dense_dirs[si].T, axis=1)
    out = np.empty((len(sparse), len(dense_dirs), len(lw_dense)))
    for i, S in enumerate(sparse):
        lg = np.log10(np.maximum(S, FLOOR))
        per_sparse = np.stack([np.interp(lw_dense, lw_sparse, lg[d]) for d in range(len(si))])
        out[i] = 10.0 ** per_sparse[nearest]
    return out


def errors(pred, true):
    """Per-spectrum relative L2 errors, in linear and in log10 space."""
    lin = np.linalg.norm((pred - true).reshape(len(true), -1), axis=1) / \
        np.linalg.norm(true.reshape(len(true), -1), axis=1)
    lg = np.log10(np.maximum(pred, FLOOR)) - np.log10(np.maximum(true, FLOOR))
    rms_dex = np.sqrt((lg.reshape(len(true), -1) ** 2).mean(1))
    return lin, rms_dex


def gemm_bench(batch=128, reps=20):
    """Tensor-core throughput of the network's three GEMM shapes at the workload's
    size, with the operands laid out as the training step holds them (all
    K-contiguous): forward X W^T, input gradient G (W^T)^T and weight gradient
    G^T H of the 512 x 393,216 output layer; then one whole training step
    (forward, backward, Adam) of the surrogate network.  CUDA-event timed."""
    import torch
    from . import mlp as M
    K, N = 512, 393216
    res = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    shapes = {"forward": (batch, N, K), "input_grad": (batch, K, N), "weight_grad": (N, K, batch)}
    for name, (m, n, k) in shapes.items():
        A = torch.randn((m, k), device="cuda").to(torch.bfloat16)
        B = torch.randn((n, k), device="cuda").to(torch.bfloat16)
        C = torch.empty((m, n), dtype=torch.float32, device="cuda")
        for _ in range(3):
            M.gemm(A, B, m, n, k, True, True, C)
        M.check()
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(reps):
            M.gemm(A, B, m, n, k, True, True, C)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"M": m, "N": n, "K": k, "ms": ms, "tflops": 2.0 * m * n * k / (ms * 1e-3) / 1e12}
        del A, B, C
    M.check()
    widths = [768, 512, 512, 512, N]
    net = M.MLP(widths, batch)
    net.init_params(0)
    x = torch.randn((batch, widths[0]), device="cuda")
    t = torch.randn((batch, widths[-1]), device="cuda")
    flop = sum(2.0 * batch * widths[l] * widths[l + 1] for l in range(len(widths) - 1))

    def two_calls(x, t, lr):
        net.gradients(x, t)
        net.adam(lr)

    # one call per step, then the same step as gradients + Adam in two calls
    for name, fn in (("train_step", net.train_step), ("train_step_two_calls", two_calls)):
        for _ in range(3):
            fn(x, t, 1e-4)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(reps):
            fn(x, t, 1e-4)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"batch": batch, "ms": ms,
                     "gemm_tflops": (3 * flop - 2.0 * batch * widths[0] * widths[1]) / (ms * 1e-3) / 1e12}
    net.close()
    return res


def main(argv=None):
    """Train and judge the surrogate; prints one JSON line."""
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--particles", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=None)
    ap.add_argument("--gemm-bench", action="store_true")
    ap.add_argument("--train-steps", type=int, default=0,
                    help="only run this many training steps of the workload's network on "
                         "random device data (profiling)")
    a = ap.parse_args(argv)
    if a.train_steps:
        from . import mlp as M
        net = M.MLP([768, 512, 512, 512, 393216], 128)
        net.init_params(0)
        x = torch.randn((128, 768), device="cuda")
        t = torch.randn((128, 393216), device="cuda")
        for _ in range(a.train_steps):
            net.train_step(x, t, 1e-4)
        torch.cuda.synchronize()
        M.check()
        net.close()
        return None
    if a.gemm_bench:
        import json
        line = json.dumps(gemm_bench())
        print(line, flush=True)
        return line
    spec = SurrogateSpec(particles=a.particles)
    t0 = time.perf_counter()
    tr_dense, tr_sparse = generate(spec, range(a.train))
    te_dense, te_sparse, t_dense, t_sparse = generate(spec, range(100_000, 100_000 + a.test),
                                                      with_timing=True)
    t_gen = time.perf_counter() - t0
    sur = Surrogate(spec, tr_sparse, tr_dense)
    t0 = time.perf_counter()
    losses = sur.train(tr_sparse, tr_dense, epochs=a.epochs, lr=a.lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    t0 = time.perf_counter()
    pred = sur.predict(te_sparse)
    torch.cuda.synchronize()
    t_pred = (time.perf_counter() - t0) / a.test
    # tensor-core throughput of the network's GEMMs at this size (batch 128)
    xb = torch.zeros((128, sur.in_pad), dtype=torch.float32, device="cuda")
    yb = torch.zeros((128, sur.out_pad), dtype=torch.float32, device="cuda")
    for _ in range(3):
        sur.net.gradients(xb, yb)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 20
    for _ in range(reps):
        sur.net.gradients(xb, yb)
    e1.record()
    torch.cuda.synchronize()
    widths = sur.net.widths
    flop = sum(2.0 * 128 * widths[l] * widths[l + 1] for l in range(len(widths) - 1))
    flop_train = 3 * flop - 2.0 * 128 * widths[0] * widths[1]   # no input gradient
    tflops = flop_train * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
    base = interpolate_baseline(spec, te_sparse)
    lin_n, dex_n = errors(pred, te_dense)
    lin_b, dex_b = errors(base, te_dense)
    res = {"train": a.train, "test": a.test, "epochs": a.epochs, "final_loss": losses[-1],
           "held_out_rel_l2_median": float(np.median(lin_n)),
           "held_out_rms_dex_median": float(np.median(dex_n)),
           "interp_rel_l2_median": float(np.median(lin_b)),
           "interp_rms_dex_median": float(np.median(dex_b)),
           "dense_exact_s_per_spectrum": t_dense, "sparse_exact_s_per_spectrum": t_sparse,
           "network_s_per_spectrum_batched": t_pred,
           "speedup_vs_dense": t_dense / (t_sparse + t_pred),
           "generation_s": t_gen, "training_s": t_train,
           "train_step_gemm_tflops_incl_elementwise": tflops}
    line = json.dumps(res)
    print(line, flush=True)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(line + "\n")
    return res


if __name__ == "__main__":
    main()
