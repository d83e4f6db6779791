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


def allreduce_spectrum(partial, coherent: bool, group=None):
    """Sum the partials over the torch.distributed group (gloo or nccl) and return
    the spectrum of all ranks' particles on every rank."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.ascontiguousarray(partial, dtype=np.float64))
    if dist.is_initialized() and dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return spectrum_from_sums(t.cpu().numpy(), coherent)
