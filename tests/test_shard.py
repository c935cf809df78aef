"""The sharded volume-side path on CPU ranks (gloo, world size 2): point
ranges, the gathered volume sum and the all-reduced adjoint.  The per-rank
compute is the FP64 oracle here (the library needs a GPU; the GPU run of
the same host path is tests/test_gpu_shard.py), so the check is of the
sharding and the collective, against the oracle on all points at once."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n,world", [(0, 3), (1, 2), (10, 3), (1001, 4), (7, 7)])
def test_shard_ranges_cover_without_overlap(n, world):
    sys.path.insert(0, ROOT)
    from paper_2004_04817_gb300.shard import shard_range
    rs = [shard_range(n, r, world) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == n
    assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
    sizes = [hi - lo for lo, hi in rs]
    assert max(sizes) - min(sizes) <= 1


def _oracle_volume(xv, xb, S, w, radius, eval_prec):
    import oracle
    return torch.from_numpy(oracle.rbf_sum(xv.numpy(), xb.numpy(), S.numpy(), w.numpy(), radius))


def _oracle_adjoint(xv, xb, S, gv, radius, eval_prec):
    import oracle
    g, st = oracle.adjoint(xv.numpy(), xb.numpy(), S.numpy(), radius, gv.numpy())
    assert st == 0
    return torch.from_numpy(g)


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2004_04817_gb300 import synth
    from paper_2004_04817_gb300.shard import shard_range, deform_volume_sharded, adjoint_sharded
    import oracle
    c = synth.tiny_wing(n_span=6, n_chord=30, n_vol=999, radius=1.0)
    estar = oracle.tolerance(c["db"], 2e-3)
    r = oracle.greedy(c["xb"], c["db"], 1.0, estar, m=3, seed=2, history=False)
    S = torch.from_numpy(r["idx"].astype(np.int32))
    W, _, _ = oracle.solve_weights(c["xb"], c["db"], r["idx"], 1.0)
    lo, hi = shard_range(len(c["xv"]), rank, world)
    xv = torch.from_numpy(np.ascontiguousarray(c["xv"][lo:hi]))
    xb = torch.from_numpy(c["xb"])
    dv = deform_volume_sharded(xv, xb, S, torch.from_numpy(W), radius=1.0, gather=True,
                               compute=lambda a, b, s, w, radius, eval_prec:
                               _oracle_volume(a, b, s, w, radius, eval_prec))
    gv_all = synth.random_field(len(c["xv"]), seed=5, sigma=0.01)
    gv = torch.from_numpy(np.ascontiguousarray(gv_all[lo:hi]))
    g = adjoint_sharded(xv, xb, S, gv, radius=1.0,
                        compute=lambda a, b, s, q, radius, eval_prec:
                        _oracle_adjoint(a, b, s, q, radius, eval_prec))
    full_dv = oracle.rbf_sum(c["xv"], c["xb"], r["idx"], W, 1.0)
    full_g, _ = oracle.adjoint(c["xv"], c["xb"], r["idx"], 1.0, gv_all)
    out[rank] = (float(np.abs(dv.numpy() - full_dv).max()),
                 float(np.abs(g.numpy() - full_g).max() / np.abs(full_g).max()),
                 int(dv.shape[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_volume_and_adjoint():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=180)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        for r in range(world):
            dv_err, g_rel, n = out[r]
            assert n == 999
            assert dv_err == 0.0          # per-point sums: the same arithmetic per point
            assert g_rel <= 1e-12         # a sum of per-rank adjoints: rounding only
