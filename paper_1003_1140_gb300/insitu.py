"""In-situ radiation from a live two-stream PIC (Sec. 2.1 setup, Sec. 2.2
diagnostic): the GPU PIC hands a contiguous subset of its electrons to the
radiation context every step from device memory, over consecutive windows of
steps, and the run reports what that costs next to the PIC alone and what the
spectra look like (peak frequency per observer and window).

    python -m paper_1003_1140_gb300.insitu [--n 256] [--steps 1200] ...

prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

import trajgen

from . import rad as R
from .pic import Pic


def run(n=256, d=0.1, dt=0.05, ppc=4, gamma=3.0, mass_ratio=64.0, tracked=16384, steps=1200,
        windows=3, n_omega=512, omega=(0.1, 1000.0), precision=R.RAD_FP32_SPLIT, seed=31,
        pic_only_steps=100, chunk=100):
    import torch
    ts = trajgen.TwoStream(n=n, d=d, dt=dt, ppc=ppc, gamma=gamma, u_th=1e-3,
                           mass_ratio=mass_ratio, axis=0, seed=seed)
    dirs = trajgen.paper_observers(axis=(1.0, 0.0, 0.0), perp=(0.0, 0.0, 1.0))
    grid = trajgen.log_grid(omega[0], omega[1], n_omega)
    wins = [(k * steps // windows, (k + 1) * steps // windows, 1, 0) for k in range(windows)]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {"grid": n, "particles": ts.n_particles, "tracked": tracked, "steps": steps,
           "dt": dt, "gamma": gamma, "mass_ratio": mass_ratio, "directions": len(dirs),
           "omegas": n_omega, "windows": [list(w[:2]) for w in wins]}

    # the PIC alone
    with Pic.two_stream(ts) as p:
        p.step(5)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        p.step(pic_only_steps)
        e1.record()
        torch.cuda.synchronize()
        out["pic_ms_per_step"] = e0.elapsed_time(e1) / pic_only_steps

    # the same run with the diagnostic in situ
    eb = []
    with Pic.two_stream(ts) as p, \
            R.Radiation(dirs, [grid], dt, [(tracked, -1.0, 1.0)], wins, precision=precision,
                        box_L=ts.L) as r:
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            p.run_coupled(r, 0, tracked, k)
            done += k
            E, B = p.fields()
            eb.append((done * dt, 0.5 * float(np.sum(B * B)) * d * d))
        e1.record()
        spectra = r.finalize()
        torch.cuda.synchronize()
        total_ms = e0.elapsed_time(e1)
        updates = r.updates()
    out["coupled_ms_per_step"] = total_ms / steps
    out["diagnostic_updates"] = int(updates)
    out["in_situ_overhead_ms_per_step"] = out["coupled_ms_per_step"] - out["pic_ms_per_step"]
    # the time the run spent beyond the PIC's own steps (diagnostic ingest,
    # accumulation and finalize, plus one field read-back per chunk)
    extra_s = max(1e-9, (total_ms - out["pic_ms_per_step"] * steps) * 1e-3)
    out["diagnostic_updates_per_s_in_situ"] = updates / extra_s
    out["magnetic_energy"] = [[round(t, 3), e] for t, e in eb]
    peaks = []
    for S in spectra:
        peaks.append([float(grid[int(np.argmax(S[di]))]) for di in range(len(dirs))])
    out["peak_omega"] = peaks                       # [window][observer]
    out["observer_angles_deg"] = [round(math.degrees(math.acos(max(-1.0, min(1.0, v[0])))), 1)
                                  for v in dirs]
    return out, spectra


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--ppc", type=int, default=4)
    ap.add_argument("--steps", type=int, default=1200)
    ap.add_argument("--tracked", type=int, default=16384)
    ap.add_argument("--omegas", type=int, default=512)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    res, spectra = run(n=a.n, ppc=a.ppc, steps=a.steps, tracked=a.tracked, n_omega=a.omegas,
                       precision=R.RAD_FP64 if a.fp64 else R.RAD_FP32_SPLIT)
    line = json.dumps(res)
    print(line, flush=True)
    if a.out:
        np.save(a.out, np.stack(spectra))
    return res


if __name__ == "__main__":
    main()
