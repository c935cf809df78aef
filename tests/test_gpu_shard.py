"""The sharded volume-side path with the library's kernels on one GPU: the
shards of a 4-way split are computed one after another (no process waits on
another) and combined as the ranks would combine them (concatenation of the
volume shards, sum of the adjoint shards), against one call over all points
and against the oracle's FP64 gradient."""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import synth
from paper_2004_04817_gb300.shard import adjoint_sharded, deform_volume_sharded, shard_range

pytestmark = pytest.mark.gpu


def _cuda(a, t=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")


def test_four_shards_match_one_call():
    c = synth.wing_small(n_vol=20_001)
    R = c["radius"]
    xb, db = _cuda(c["xb"]), _cuda(c["db"])
    g = P.greedy_select(xb, db, radius=R, tol=c["tol_rel"], tol_mode=1, m=5,
                        eval_prec=P.PREC_F32X2, weights=True)
    xv = _cuda(c["xv"])
    gv = _cuda(synth.random_field(len(c["xv"]), seed=5, sigma=0.01))
    world = 4
    parts, gsum = [], None
    for r in range(world):
        lo, hi = shard_range(len(c["xv"]), r, world)
        parts.append(deform_volume_sharded(xv[lo:hi].contiguous(), xb, g["idx"], g["w"],
                                           radius=R))
        gr = adjoint_sharded(xv[lo:hi].contiguous(), xb, g["idx"], gv[lo:hi].contiguous(),
                             radius=R)
        gsum = gr if gsum is None else gsum + gr
    full = P.deform_volume(xv, xb, g["idx"], g["w"], radius=R, eval_prec=P.PREC_F32X2)
    assert torch.equal(torch.cat(parts), full)        # per-point sums: identical bits
    gfull, _ = P.adjoint(xv, xb, g["idx"], gv, radius=R)
    ref, st = oracle.adjoint(c["xv"], c["xb"], g["idx"].cpu().numpy(), R, gv.cpu().numpy())
    scale = np.abs(ref).max()
    assert np.abs(gsum.cpu().numpy() - ref).max() <= 1e-8 * scale
    assert np.abs(gsum.cpu().numpy() - gfull.cpu().numpy()).max() <= 1e-8 * scale
