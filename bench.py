#!/usr/bin/env python
"""Throughput of the in-situ radiation-spectrum hot path on GB300.

One step = one whole pass of the hot path over one batch of synthetic input:
reset, ingest of every PIC call of the window (leapfrog states already
resident in HBM), the FP32 split-phase accumulation of the Lienard-Wiechert
far-field amplitude for every particle x sample x direction x frequency, the
window-close particle reduction and the finalize, through the C ABI.

Workload: the precision workload -- 1,048,576 electrons in two gamma = 10
beams in a 64-mode static field, 4096 samples, 8 observer directions, 1024
log-spaced omega in [0.1, 1000].  Its FP64 trajectory (206 GB) is resident in
HBM; the whole-window ring for every particle at once (192 GB) does not fit
beside it, so one context sized for a shard of the particles takes the shards
one after another (rad_next_shard) and sums them into one spectrum.  The
metric is particle.sample.omega.direction updates per second; the FP32 split
path's error against the FP64 GPU path is measured per direction on 65,536 of
the particles.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

N > 1 runs under torchrun, one rank per GPU, each on its own 1,048,576
particles (weak scaling); the ranks' partial sums are added by one NCCL
all-reduce inside the step (the only exchange of the method) and the
spectrum is formed from the total; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "G particle·step·ω·n updates/s, FP32 split vs FP64 GPU at ≤1e-4 rel L2"

# DRAM bytes (read + write) of one accumulation launch from an ncu capture of this
# workload scaled to 4096 particles (same samples, directions and omegas), valid while
# the code (comments aside) of the kernel and of its work-list builder is the code that
# was captured; traffic scales with the particle count.
TRAFFIC_CAPTURE = {"sources_sha256": "cadabcb64484e3e00e449b1f01f7142ba83ff5aac4b20d3cd0e4aa48eb6da180",
                   "bytes_per_launch": 699.964416e6, "particles": 4096}
UNIT = "G updates/s"
# phase budget (rad per update) of the accuracy side-run: the upper decade of the
# precision workload's grid (dt 0.05, w <= 1000) takes anchor blocks of 8 samples
PHASE_BUDGET = 2.1e-5
WORKLOAD = 3
# device memory kept free beside the resident trajectory and one shard's ring
MEM_MARGIN = 12 << 30


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--shards", type=int, default=0,
                    help="particle shards per step (0: the fewest that fit in device memory)")
    ap.add_argument("--fp64-particles", type=int, default=65536)
    ap.add_argument("--e2e-particles", type=int, default=65536)
    ap.add_argument("--cpu-particles", type=int, default=None)
    ap.add_argument("--cpu-1core-particles", type=int, default=18)
    ap.add_argument("--particles", type=int, default=None,
                    help="scale the workload to this many particles (profiling cases)")
    ap.add_argument("--variant", type=int, default=None)
    ap.add_argument("--anchor-K", type=int, default=None)
    ap.add_argument("--freq-per-lane", type=int, default=None)
    ap.add_argument("--blocks-per-sm", type=int, default=None)
    ap.add_argument("--poly-per-lane", type=int, default=None)
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def workload_name(w):
    (cnt, _, _, gamma), = w.species
    return (f"precision: {cnt} e- gamma {gamma:g} two-beam, {w.windows[0][1] - w.windows[0][0]} "
            f"samples, {len(w.dirs)} dirs, {len(w.grids[0])} log omega "
            f"[{w.grids[0][0]:g}, {w.grids[0][-1]:g}]")


def workload_config(w, extra=None):
    cfg = {"workload": workload_name(w), "particles": w.n_total,
           "samples": w.windows[0][1] - w.windows[0][0], "directions": len(w.dirs),
           "omegas": len(w.grids[0]), "dt": w.dt, "gamma": w.species[0][3],
           "path": "FP32 split-phase (float-float anchor)", "mode": "incoherent",
           "l2": "inputs larger than L2 (FP64 trajectory resident in HBM)"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------
# CPU oracle sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(n_particles: int):
    """Time the FP64 CPU oracle on the first n_particles of the workload."""
    import oracle
    import trajgen
    w = trajgen.config(WORKLOAD)
    X, U = w.trajectory_numpy(0, n_particles)
    sp = [(n_particles, w.species[0][1])]
    t0 = time.perf_counter()
    oracle.spectra(X, U, w.dt, w.dirs, w.grids, w.windows, sp, box_L=w.L)
    el = time.perf_counter() - t0
    s0, s1 = w.windows[0][0], w.windows[0][1]
    upd = n_particles * (s1 - s0) * len(w.dirs) * len(w.grids[0])
    return upd, el, oracle.num_threads(), w


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    # a bounded sample per step (about 6 s on 16 cores), so that the whole
    # --steps K --warmup W run ends within a few minutes
    npart = args.cpu_particles or 144
    vals = []
    for i in range(args.warmup + args.steps):
        upd, el, cores, w = oracle_sample(npart)
        if i >= args.warmup:
            vals.append((upd, el))
    upd = sum(v[0] for v in vals)
    el = sum(v[1] for v in vals)
    value = upd / el / 1e9
    sample = (f"{npart} of {w.n_total} particles, all samples/directions/omegas "
              f"({vals[0][0]:.3e} updates per step)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, {"path": "FP64 CPU oracle (C, libm, OpenMP)",
                                          "l2": "not applicable: CPU oracle on host memory"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


_C_TOKENS = re.compile(r'"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'|//[^\n]*|/\*.*?\*/', re.S)


def code_only(src: str) -> str:
    """C/C++/CUDA source with its comments removed and whitespace runs collapsed:
    the text the compiler acts on, so that editing a comment does not void a capture."""
    return " ".join(_C_TOKENS.sub(lambda m: " " if m.group(0)[0] == "/" else m.group(0),
                                  src).split())


def traffic_sources_hash() -> str:
    """SHA-256 over the code (not the comments) of the accumulation kernel and of
    the host library that builds its work list and launches it."""
    import hashlib
    h = hashlib.sha256()
    for f in ("paper_1003_1140_gb300/csrc/rad_accum32.cuh", "paper_1003_1140_gb300/csrc/rad_api.cu"):
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()


def captured_traffic(n_particles: int):
    """DRAM bytes per accumulation launch from the ncu capture, or None if there is
    none or the code of the kernel or of its work-list builder changed since."""
    if not TRAFFIC_CAPTURE or traffic_sources_hash() != TRAFFIC_CAPTURE["sources_sha256"]:
        return None
    return TRAFFIC_CAPTURE["bytes_per_launch"] * n_particles / TRAFFIC_CAPTURE["particles"]


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200",
                                       "-i", str(gpu_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for ln in fh:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2])
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def ring_bytes_per_particle(samples: int, K: int = 8) -> int:
    """Device bytes of one particle's whole-window ring (40 B per sample, the ring's
    64-sample margin) and anchor ring (24 B per K samples)."""
    slots = (samples + 31) // 32 * 32 + 64
    return slots * 40 + (slots // K) * 24


def choose_shards(n_total: int, n_calls: int, samples: int, free_bytes: int) -> int:
    """The fewest power-of-two particle shards whose ring fits beside the resident
    FP64 trajectory (48 bytes per particle and call) with MEM_MARGIN to spare."""
    inputs = n_total * n_calls * 48
    shards = 1
    while shards < n_total:
        per = -(-n_total // shards)
        if inputs + per * ring_bytes_per_particle(samples) + MEM_MARGIN <= free_bytes:
            return shards
        shards *= 2
    return shards


def batched_subrange(args, R, tg, trajgen, torch):
    """The batched workload (electrons and ions, 192 HEALPix directions, three omega
    grids, five uneven windows) through its in-situ path: one rad_accumulate per PIC
    step replayed as CUDA graphs, autotuned persistent launch at each window close.
    Timed on the step sub-range 0..1536, which closes the electrons' [1024, 1536)
    window on the 512-omega grid (the ingest of every window's samples so far is
    inside the timed region; only the closed window's updates are counted)."""
    w4 = trajgen.config(4)
    if args.particles:
        w4 = trajgen.config(4, args.particles / trajgen.config(WORKLOAD).n_total)
    s_end = 1536
    X4, U4 = tg.trajectory_gpu(w4, n_calls=s_end + 1)
    sp4 = [(s[0], s[1], s[2]) for s in w4.species]
    ctx4 = R.Radiation(w4.dirs, w4.grids, w4.dt, sp4, w4.windows, precision=R.RAD_FP32_SPLIT,
                       box_L=w4.L, options={"use_graph": 1})
    st = torch.cuda.current_stream()
    closed = [i for i, (s0, s1, _, _) in enumerate(w4.windows) if s1 <= s_end]
    upd = sum(sum(c for i2, (c, _, _, _) in enumerate(w4.species) if (w4.windows[i][2] >> i2) & 1)
              * (w4.windows[i][1] - w4.windows[i][0]) * len(w4.dirs)
              * len(w4.grids[w4.windows[i][3]]) for i in closed)
    ms = []
    for rep in range(2):          # the first pass tunes and captures the graphs
        ctx4.reset()
        t_before = ctx4.timing()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for s in range(s_end + 1):
            ctx4.accumulate(s, X4[s], U4[s])
        e1.record(st)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        t_after = ctx4.timing()
    opts = ctx4.options()
    ctx4.close()
    del X4, U4
    torch.cuda.empty_cache()
    return {"value": upd / (ms[-1] * 1e-3) / 1e9, "unit": UNIT,
            "workload": f"batched: {w4.species[0][0]} e- + {w4.species[1][0]} ions (m = 16, "
                        f"q = +1), {len(w4.dirs)} HEALPix Nside-4 dirs, grids "
                        f"{'/'.join(str(len(g)) for g in w4.grids)}, windows {w4.windows}",
            "timed": f"steps 0..{s_end}, one rad_accumulate per step with use_graph; "
                     f"closes windows {closed}",
            "updates": upd, "ms": ms[-1], "first_pass_ms": ms[0],
            "accum_launches": t_after["accum_launches"] - t_before["accum_launches"],
            "step_calls": s_end + 1, "options": opts}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    import trajgen
    from trajgen import gpu as tg
    import paper_1003_1140_gb300 as R
    from paper_1003_1140_gb300 import roofline

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    w = trajgen.config(WORKLOAD)
    if args.particles:
        w = trajgen.config(WORKLOAD, args.particles / w.n_total)
    N = w.n_total
    samples = w.windows[0][1] - w.windows[0][0]
    free, _ = torch.cuda.mem_get_info()
    P = args.shards or choose_shards(N, w.n_calls, samples, free)
    n = -(-N // P)                                  # particles per shard
    # weak scaling: rank r owns particles [r N, (r + 1) N) of the generator; its
    # shards are consecutive blocks of them, each a contiguous [calls][3][n] slab
    Xs, Us = [], []
    for b in range(P):
        cnt = min(n, N - b * n)
        X, U = tg.trajectory_gpu(w, first=rank * N + b * n, count=cnt)
        if cnt < n:
            # a short last shard is padded with particles at rest, which radiate
            # exactly nothing (uniform motion: betadot = 0)
            Xp = torch.full((X.shape[0], 3, n), 1.0, dtype=torch.float64, device="cuda")
            Up = torch.zeros_like(Xp)
            Xp[:, :, :cnt] = X
            Up[:, :, :cnt] = U
            X, U = Xp, Up
        Xs.append(X)
        Us.append(U)
    torch.cuda.synchronize()
    q, mass = w.species[0][1], w.species[0][2]
    opts = {}
    if args.variant is not None:
        opts["variant"] = args.variant
    if args.anchor_K is not None:
        opts["anchor_K"] = args.anchor_K
    if args.freq_per_lane is not None:
        opts["freq_per_lane"] = args.freq_per_lane
    if args.blocks_per_sm is not None:
        opts["blocks_per_sm"] = args.blocks_per_sm
    if args.poly_per_lane is not None:
        opts["poly_per_lane"] = args.poly_per_lane
    ctx = R.Radiation(w.dirs, w.grids, w.dt, [(n, q, mass)], w.windows,
                      precision=R.RAD_FP32_SPLIT, box_L=w.L, options=opts or None)
    nbins = ctx.spectrum_size()
    out = torch.empty(nbins, dtype=torch.float64, device="cuda")
    sums = torch.empty(nbins, dtype=torch.float64, device="cuda")
    upd_shard = ctx.updates()
    upd = w.updates()                 # the padding particles of a short shard are not counted

    def step():
        ctx.reset()
        for b in range(P):
            if b:
                ctx.next_shard()
            ctx.accumulate_steps(0, Xs[b], Us[b])
        if world == 1:
            ctx.finalize(out)
        else:
            # the method's one exchange: the ranks' particle sums are added, then
            # the spectrum of all ranks' particles is formed from the total
            ctx.partial_sums(sums)
            dist.all_reduce(sums, op=dist.ReduceOp.SUM)
            R.spectrum_from_sums(sums, R.RAD_INCOHERENT, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t_before = ctx.timing()
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    t_after = ctx.timing()
    acc_ms = t_after["accum_ms"] - t_before["accum_ms"]
    acc_n = t_after["accum_launches"] - t_before["accum_launches"]
    ing_n = t_after["ingest_launches"] - t_before["ingest_launches"]
    # + one finalize (or spectrum-from-sums) kernel per step
    launches = int(acc_n + ing_n + args.steps)
    ms_step = ms / args.steps
    value = world * upd / (ms_step * 1e-3) / 1e9
    opts_used = ctx.options()
    S_full = out.cpu().numpy().reshape(len(w.dirs), -1)
    ctx.close()
    del ctx

    # roofline of the dominant kernel (the window accumulation, one launch per
    # shard), measured live with CUDA events on the context's stream
    sm_mhz = clocks["sm_mhz"] if clocks else None
    rl = roofline.accum32_roofline(upd_shard, acc_ms / max(acc_n, 1),
                                   torch.cuda.get_device_properties(local).multi_processor_count,
                                   sm_mhz, opts_used)
    rl["traffic"] = captured_traffic(n)

    # the particle sample for the FP64 comparison and the end-to-end run: the
    # first particles of shard 0
    keep = max(args.e2e_particles if not args.no_e2e else 0,
               args.fp64_particles if not args.no_fp64 else 0)
    keep = min(keep, n)
    Xk = Xs[0][:, :, :keep].contiguous() if keep else None
    Uk = Us[0][:, :, :keep].contiguous() if keep else None
    del Xs, Us, X, U
    torch.cuda.empty_cache()

    # end to end through the public API with host buffers (pinned), H2D/D2H inside
    e2e = None
    if not args.no_e2e and keep:
        ne = min(args.e2e_particles, keep)
        Xd = Xk[:, :, :ne].contiguous()
        Ud = Uk[:, :, :ne].contiguous()
        ce = R.Radiation(w.dirs, w.grids, w.dt, [(ne, q, mass)], w.windows,
                         precision=R.RAD_FP32_SPLIT, box_L=w.L, options=opts or None)
        upd_e = ce.updates()
        oute = torch.empty(ce.spectrum_size(), dtype=torch.float64, device="cuda")
        host_mem = "pinned"
        try:
            Xh = torch.empty(Xd.shape, dtype=torch.float64, pin_memory=True)
            Uh = torch.empty(Ud.shape, dtype=torch.float64, pin_memory=True)
        except RuntimeError:
            # many ranks on one node may not be able to lock this much each
            host_mem = "pageable"
            Xh = torch.empty(Xd.shape, dtype=torch.float64)
            Uh = torch.empty(Ud.shape, dtype=torch.float64)
        Xh.copy_(Xd)
        Uh.copy_(Ud)
        outh = np.empty(ce.spectrum_size())
        ke = max(1, args.steps)

        # the same sample from device memory, for the exposed-copy figure
        def step_dev():
            ce.reset()
            ce.accumulate_steps(0, Xd, Ud)
            ce.finalize(oute)

        step_dev()
        torch.cuda.synchronize()
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(st)
        for _ in range(ke):
            step_dev()
        d1.record(st)
        torch.cuda.synchronize()
        dev_ms = d0.elapsed_time(d1) / ke

        # the host-to-device link on its own: one copy of the sample's x, on a
        # side stream, timed with CUDA events on that stream
        cs = torch.cuda.Stream()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        h2d_ms = []
        for _ in range(3):
            with torch.cuda.stream(cs):
                c0.record(cs)
                Xd.copy_(Xh, non_blocking=True)
                c1.record(cs)
            torch.cuda.synchronize()
            h2d_ms.append(c0.elapsed_time(c1))
        h2d_gbs = Xh.numel() * 8 / (min(h2d_ms) * 1e-3) / 1e9

        def step_e2e():
            ce.reset()
            ce.accumulate_steps(0, Xh, Uh)
            ce.finalize(outh)

        for _ in range(2):
            step_e2e()
        torch.cuda.synchronize()
        barrier()
        times = []
        for _ in range(ke):
            t0 = time.perf_counter()
            step_e2e()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        el = sum(times) / ke
        if world > 1:
            t = torch.tensor([el], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": world * upd_e / el / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(Xh.numel() * 8 + Uh.numel() * 8),
               "d2h_bytes_per_step": int(outh.size * 8), "host_memory": host_mem,
               "sample": f"first {ne} particles of the workload, all samples/directions/omegas "
                         f"({upd_e:.3e} updates per step; per-particle work as in the "
                         f"device-resident step)",
               "steps": ke, "ms_per_step": 1e3 * el,
               "step_ms_min_median_max": [1e3 * min(times), 1e3 * statistics.median(times),
                                          1e3 * max(times)],
               "device_ms_per_step_same_sample": dev_ms,
               "exposed_copy_ms_per_step": 1e3 * el - dev_ms,
               "h2d_gbs_measured": h2d_gbs}
        ce.close()
        del Xh, Uh, Xd, Ud, ce

    # FP64 GPU path on a particle sample, and the FP32 split error against it
    fp64 = rel = perbin = None
    n64 = 0
    fp32_kernel_rate = upd_shard / (acc_ms / max(acc_n, 1) * 1e-3) / 1e9 if acc_n else None
    if not args.no_fp64 and keep:
        n64 = min(args.fp64_particles, keep)
        X64 = Xk[:, :, :n64].contiguous()
        U64 = Uk[:, :, :n64].contiguous()
        c64 = R.Radiation(w.dirs, w.grids, w.dt, [(n64, q, mass)], w.windows,
                          precision=R.RAD_FP64, box_L=w.L)
        c64.accumulate_steps(0, X64, U64)
        S64 = c64.finalize()[0]
        t64 = c64.timing()
        upd64 = c64.updates()
        c64.close()
        c32 = R.Radiation(w.dirs, w.grids, w.dt, [(n64, q, mass)], w.windows,
                          precision=R.RAD_FP32_SPLIT, box_L=w.L, options=opts or None)
        c32.accumulate_steps(0, X64, U64)
        S32 = c32.finalize()[0]
        t32 = c32.timing()
        c32.close()
        rel = np.linalg.norm(S32 - S64, axis=1) / np.linalg.norm(S64, axis=1)
        # single bins of the upper decade, where the FP32 offset phase is least accurate
        hi = w.grids[0] >= 100.0
        perbin = {"upper_decade_worst_bin_vs_fp64": float((np.abs(S32 - S64) / S64)[:, hi].max()),
                  "sample": f"first {n64} particles, omega >= 100",
                  "kernel_rate": upd64 / (t32["accum_ms"] * 1e-3) / 1e9}
        # the same sample under a phase budget: the frequency tile of the upper
        # decade anchored every 8 samples, the lower tiles every 32
        cb = R.Radiation(w.dirs, w.grids, w.dt, [(n64, q, mass)], w.windows,
                         precision=R.RAD_FP32_SPLIT, box_L=w.L,
                         options={"phase_budget": PHASE_BUDGET})
        cb.accumulate_steps(0, X64, U64)
        Sb = cb.finalize()[0]
        tb = cb.timing()
        ob = cb.options()
        cb.close()
        perbin["with_phase_budget"] = {
            "budget_rad": PHASE_BUDGET, "ring_anchor_K": ob["anchor_K"],
            "upper_decade_worst_bin_vs_fp64": float((np.abs(Sb - S64) / S64)[:, hi].max()),
            "rel_l2_max": float((np.linalg.norm(Sb - S64, axis=1) / np.linalg.norm(S64, axis=1)).max()),
            "kernel_rate": upd64 / (tb["accum_ms"] * 1e-3) / 1e9}
        # and with the precise phase (float-float offsets, reduced to one turn)
        cp = R.Radiation(w.dirs, w.grids, w.dt, [(n64, q, mass)], w.windows,
                         precision=R.RAD_FP32_SPLIT, box_L=w.L,
                         options={"variant": R.RAD_VARIANT_PRECISE})
        cp.accumulate_steps(0, X64, U64)
        Sp = cp.finalize()[0]
        tp = cp.timing()
        cp.close()
        perbin["precise_phase"] = {
            "upper_decade_worst_bin_vs_fp64": float((np.abs(Sp - S64) / S64)[:, hi].max()),
            "worst_bin_vs_fp64": float((np.abs(Sp - S64) / S64).max()),
            "rel_l2_max": float((np.linalg.norm(Sp - S64, axis=1) / np.linalg.norm(S64, axis=1)).max()),
            "kernel_rate": upd64 / (tp["accum_ms"] * 1e-3) / 1e9}
        # the precise phase only where the phase budget needs it (the upper decade)
        cq = R.Radiation(w.dirs, w.grids, w.dt, [(n64, q, mass)], w.windows,
                         precision=R.RAD_FP32_SPLIT, box_L=w.L,
                         options={"variant": R.RAD_VARIANT_PRECISE, "phase_budget": PHASE_BUDGET})
        cq.accumulate_steps(0, X64, U64)
        Sq = cq.finalize()[0]
        tq = cq.timing()
        cq.close()
        perbin["precise_phase_with_budget"] = {
            "budget_rad": PHASE_BUDGET,
            "upper_decade_worst_bin_vs_fp64": float((np.abs(Sq - S64) / S64)[:, hi].max()),
            "rel_l2_max": float((np.linalg.norm(Sq - S64, axis=1) / np.linalg.norm(S64, axis=1)).max()),
            "kernel_rate": upd64 / (tq["accum_ms"] * 1e-3) / 1e9}
        fp64_rate = upd64 / (t64["accum_ms"] * 1e-3) / 1e9
        fp64 = {"value": fp64_rate, "unit": UNIT,
                "sample": f"first {n64} particles, same samples/dirs/omegas"}
    del Xk, Uk

    batched = None
    if not args.no_batched:
        batched = batched_subrange(args, R, tg, trajgen, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        ncpu = args.cpu_particles or 288
        cupd, cel, cores, _ = oracle_sample(ncpu)
        cpu = {"value": cupd / cel / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {ncpu} particles of the workload, all {samples} "
                         f"samples x {len(w.dirs)} dirs x {len(w.grids[0])} omega "
                         f"({cupd:.3e} updates, {cel:.1f} s)"}
        if args.cpu_1core_particles > 0:
            # the same oracle on one core (a smaller bounded sample)
            oracle.set_num_threads(1)
            try:
                c1upd, c1el, _, _ = oracle_sample(args.cpu_1core_particles)
            finally:
                oracle.set_num_threads(cores)
            cpu["one_core"] = {"value": c1upd / c1el / 1e9, "unit": UNIT, "cores": 1,
                               "sample": f"first {args.cpu_1core_particles} particles "
                                         f"({c1upd:.3e} updates, {c1el:.1f} s)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": workload_config(w, {"options": opts_used, "shards_per_step": P,
                                              "particles_per_shard": n,
                                              "parallelism": f"particle shards x{world}"
                                              + (", NCCL all-reduce of the partial sums"
                                                 if world > 1 else "")}),
                "clocks": clocks, "gpu_launches": launches, "roofline": rl,
                "e2e": e2e, "cpu_baseline": cpu, "fp64_gpu": fp64, "batched_workload": batched,
                "fp32_vs_fp64_rel_l2": None if rel is None else
                {"max": float(rel.max()), "per_direction": [float(v) for v in rel],
                 "particles": n64},
                "fp32_vs_fp64_per_bin": perbin,
                "fp32_kernel_speedup_vs_fp64_gpu": (fp32_kernel_rate / fp64["value"]
                                                    if fp64 and fp32_kernel_rate else None),
                "spectrum_finite": bool(np.all(np.isfinite(S_full)) and np.all(S_full >= 0))}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
