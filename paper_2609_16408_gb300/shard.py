"""Multi-GPU sharding of the probe-points (one process per GPU).

The (coarse point, frequency) pairs are independent Lanczos runs (Section 4 of the paper:
no communication inside the grid-point loop), so they are partitioned across ranks with no
collective on the data path.  The only exchange is one gather of the coarse energy-density
array (N_w x P doubles) before the interpolation and E_c sum, the counterpart of the
paper's single gather per frequency.
"""
from __future__ import annotations

import numpy as np


def probe_point_shard(P: int, nw: int, rank: int, world: int):
    """Contiguous, balanced block of the frequency-major probe-point list for one rank.

    Returns (probe indices into the coarse list, frequency indices), both int arrays."""
    total = P * nw
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    ids = np.arange(start, stop, dtype=np.int64)
    return ids % P, (ids // P).astype(np.int32)


def gather_coarse(d_local, P: int, nw: int, rank: int, world: int, group=None):
    """All-gather the per-rank d values into the full (nw, P) array on every rank.

    d_local: 1-D torch tensor (this rank's shard, in shard order).  With a backend that
    cannot exchange device tensors (gloo) the exchange goes through host memory; the result
    lives where d_local lives."""
    import torch
    import torch.distributed as dist
    counts = [len(probe_point_shard(P, nw, r, world)[0]) for r in range(world)]
    mx = max(counts)
    via_host = d_local.is_cuda and dist.get_backend(group) != "nccl"
    dev = torch.device("cpu") if via_host else d_local.device
    buf = torch.zeros(mx, dtype=d_local.dtype, device=dev)
    buf[: d_local.numel()] = d_local.to(dev)
    outs = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    full = torch.cat([o[:c] for o, c in zip(outs, counts)])
    return full.reshape(nw, P).to(d_local.device)


def energy_density_sharded(ctx, P: int, nw: int, nd: int, rank: int, world: int, device,
                           group=None):
    """E_c on `world` GPUs: each rank runs its shard of probe-points through the C ABI,
    the coarse array is gathered, and every rank interpolates and sums (the result is
    identical on all ranks).  Returns (d_coarse (nw, P), E_c)."""
    import torch

    from . import rpa_interpolate, rpa_probe_density, rpa_probe_indices
    sel, fq = probe_point_shard(P, nw, rank, world)
    idx = torch.from_numpy(rpa_probe_indices(ctx)).to(device)
    pr = idx[torch.from_numpy(sel).to(device)]
    out = rpa_probe_density(ctx, pr, torch.from_numpy(fq).to(device))
    dco = gather_coarse(out["d"], P, nw, rank, world, group)
    _, ec = rpa_interpolate(ctx, dco, nd)
    return dco, ec
