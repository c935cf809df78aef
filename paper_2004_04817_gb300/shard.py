"""Sharding of the volume-side sums over the volume points, one process per
GPU (torch.distributed).

The volume displacement of Eq. 6 at point v depends on v alone, so the N_v
points are split into contiguous per-rank ranges with the support set S and
its weights W replicated on every rank: no data exchange.  The adjoint
dJ/dd_c = Phi_cc^-1 sum_v phi(v, c) dJ/dd_v is linear in the per-point terms,
so every rank computes it over its own range and one all-reduce (sum) of the
N_c x 3 FP64 result combines them (Sec. 2: Phi_cc is the same on every
rank).  The greedy itself does not shard usefully (one argmax and one
Cholesky append per iteration); it runs on each rank alike.

The compute calls default to the library's (``deform_volume``, ``adjoint``);
``compute`` lets a caller substitute another implementation of the same
signature.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import rbf


def shard_range(n, rank, world):
    """Contiguous range [lo, hi) of rank ``rank`` among ``world``: sizes differ
    by at most one, the first n % world ranks take the extra point."""
    n, rank, world = int(n), int(rank), int(world)
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def _world(group):
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def deform_volume_sharded(xv_local, xb, sel_idx, w, *, radius, eval_prec=rbf.PREC_F32X2,
                          group=None, gather=False, compute=None):
    """Eq. 6 on this rank's points ``xv_local``.  With ``gather`` the ranks'
    results are concatenated in rank order on every rank (all-gather; ranges
    from ``shard_range`` make that the original point order)."""
    fn = compute or (lambda *a, **k: rbf.deform_volume(*a, **k))
    dv = fn(xv_local, xb, sel_idx, w, radius=radius, eval_prec=eval_prec)
    rank, world = _world(group)
    if not gather or world == 1:
        return dv
    n = torch.tensor([dv.shape[0]], dtype=torch.int64, device=dv.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    mx = int(max(int(s.item()) for s in sizes))
    pad = torch.zeros((mx, 3), dtype=dv.dtype, device=dv.device)
    pad[:dv.shape[0]] = dv
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:int(s.item())] for p, s in zip(parts, sizes)], dim=0)


def adjoint_sharded(xv_local, xb, sel_idx, gv_local, *, radius, eval_prec=rbf.PREC_F32X2,
                    group=None, compute=None):
    """dJ/dd_c over all ranks' points: this rank's adjoint over its own points,
    summed over the ranks by one all-reduce of N_c x 3 FP64 values."""
    fn = compute or (lambda *a, **k: rbf.adjoint(*a, **k)[0])
    g = fn(xv_local, xb, sel_idx, gv_local, radius=radius, eval_prec=eval_prec)
    rank, world = _world(group)
    if world > 1:
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return g
