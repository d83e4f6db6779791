"""Particle sharding across processes or GPUs, with one host-side exchange.

Incoherent spectra of disjoint particle sets add; coherent amplitudes add
before the modulus is taken (Sec. 2.2's sum over j).  Each rank runs the
radiation library on its own particles, exports the unscaled FP64 particle
sums (``Radiation.partial_sums``), and the ranks sum those; the spectrum of
the union is formed once from the total.  No collective is needed on the
data path -- only this final reduction.
"""
from __future__ import annotations

import math
import time

import numpy as np

PREF = 1.0 / (4.0 * math.pi ** 2)


def shard(count: int, rank: int, world: int):
    """[first, first + n) of `count` items owned by `rank` of `world` (balanced)."""
    base, extra = divmod(int(count), int(world))
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def spectrum_from_sums(total, coherent: bool):
    """Spectrum from summed partials: [n] (incoherent) or [n, c] (coherent)."""
    total = np.asarray(total, dtype=np.float64)
    if coherent:
        return PREF * (total.reshape(total.shape[0], -1) ** 2).sum(1)
    return PREF * total.reshape(-1)


def combine(partials, coherent: bool):
    """Spectrum of the union of shards from each shard's partial sums."""
    total = np.sum([np.asarray(p, dtype=np.float64) for p in partials], axis=0)
    return spectrum_from_sums(total, coherent)


def check_in(store, rank: int, tag: str) -> None:
    """Record in a key-value store (a torch.distributed Store) that this rank's
    shard is done for `tag` (a window, a batch of steps)."""
    store.set(f"{tag}/done/{int(rank)}", "1")


def missing_ranks(store, world: int, tag: str, timeout_s: float) -> list:
    """Ranks that have not checked in for `tag` within timeout_s seconds (empty
    when every rank has).  Polls the store; never enters a collective."""
    deadline = time.monotonic() + float(timeout_s)
    missing = list(range(int(world)))
    while True:
        missing = [r for r in missing if not store.check([f"{tag}/done/{r}"])]
        if not missing or time.monotonic() >= deadline:
            return missing
        time.sleep(0.02)


def allreduce_spectrum(partial, coherent: bool, group=None, store=None, tag: str = "",
                       timeout_s: float = 30.0):
    """Sum the partials over the torch.distributed group (gloo or nccl) and return
    the spectrum of all ranks' particles on every rank.

    With a store, every rank first checks in for `tag` and waits (up to
    timeout_s) for the others: a rank that failed or left before finishing its
    shard is reported as a RuntimeError naming it, before any rank enters the
    collective, instead of leaving the others blocked in it."""
    import torch
    import torch.distributed as dist
    if store is not None:
        world = dist.get_world_size(group)
        check_in(store, dist.get_rank(group), tag)
        missing = missing_ranks(store, world, tag, timeout_s)
        if missing:
            raise RuntimeError(f"ranks {missing} did not finish their shard of {tag!r} "
                               f"within {timeout_s:g} s")
    t = torch.as_tensor(np.ascontiguousarray(partial, dtype=np.float64))
    if dist.is_initialized() and dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return spectrum_from_sums(t.cpu().numpy(), coherent)
