"""rbf_deform_volume_noalloc: the volume sum for callers that cannot allocate
device memory, such as a solver plug-in whose host application owns all
device memory, or a time-critical loop that cannot take the implicit
synchronisation of an allocation.  Its scratch is a fixed array that belongs
to the library, so it needs no workspace from the caller.

Called through the C ABI and compared with rbf_deform_volume (FP32) and with
the FP64 oracle at the FP32 rounding bound, on consecutive calls with
different support sets, so a stale scratch table from an earlier call would
show up in a later one.  Support sets of more than one shared-memory tile
(2,048 centres) up to the array's limit of 8,192 centres are covered.  This
file is collected last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import rbf, synth

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
MAX_CENTRES = 8192


def _entry():
    L = P.lib()
    f = L.rbf_deform_volume_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                  C.POINTER(rbf.Params), C.c_void_p, C.c_void_p]
    return f


def _call(f, xv, xb, idx, w, radius):
    dv = torch.full((xv.shape[0], 3), float("nan"), dtype=torch.float64, device="cuda")
    p = rbf.make_params(radius, eval_prec=P.PREC_F32)
    st = f(xv.data_ptr(), xv.shape[0], xb.data_ptr(), idx.data_ptr(), idx.numel(),
           w.data_ptr(), C.byref(p), dv.data_ptr(),
           C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, dv


def _dev(a, t=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")


def _check(c_xv, c_xb, S, W, radius, a, ref, sample):
    """a: noalloc result; ref: rbf_deform_volume FP32 result (both host)."""
    assert np.all(np.isfinite(a))
    X = max(np.abs(c_xv).max(), np.abs(c_xb).max()) / radius
    # same FP32 arithmetic as the workspace entry point: agreement well inside
    # the FP32 rounding bound of the sum
    assert np.abs(a - ref).max() <= U32 * 16 * X * np.abs(W).sum()
    # the FP64 oracle with the same weights, at the FP32 rounding bound
    o = oracle.rbf_sum(c_xv[sample], c_xb, S, W, radius)
    Phi = oracle.phi(np.linalg.norm(c_xv[sample][:, None] - c_xb[S][None], axis=-1) / radius)
    bound = U32 * (64 * (Phi @ np.abs(W).sum(1)) + 16 * X * np.abs(W).sum())
    err = np.abs(a[sample] - o).max(axis=1)
    assert np.all(err <= bound), (err / bound).max()


def test_noalloc_volume_matches_workspace_entry_point_twice():
    f = _entry()
    c = synth.wing_small(n_vol=30_000)
    xb, db, xv = _dev(c["xb"]), _dev(c["db"]), _dev(c["xv"])
    sample = np.sort(np.random.default_rng(3).choice(len(c["xv"]), 2000, replace=False))
    for tol_rel, m in ((1e-3, 1), (3e-4, 5)):        # two support sets of different size
        g = P.greedy_select(xb, db, radius=c["radius"], tol=tol_rel, tol_mode=1, m=m,
                            eval_prec=P.PREC_F64)
        w, _ = P.solve_weights(xb, db, g["idx"], radius=c["radius"])
        st, dv = _call(f, xv, xb, g["idx"], w, c["radius"])
        assert st == 0
        ref = P.deform_volume(xv, xb, g["idx"], w, radius=c["radius"], eval_prec=P.PREC_F32)
        torch.cuda.synchronize()
        _check(c["xv"], c["xb"], g["idx"].cpu().numpy(), w.cpu().numpy(), c["radius"],
               dv.cpu().numpy(), ref.cpu().numpy(), sample)


def test_noalloc_volume_several_tiles_up_to_the_limit():
    """Support sets of 8,192 (the limit), 2,049 and 5,000 centres in a row:
    several shared-memory tiles and a ragged last tile.  The centres are
    random distinct nodes of the 50,000-node wing with random weights (the
    sum needs no solve)."""
    f = _entry()
    c = synth.wing_gcb(n_vol=20_000)
    xb, xv = _dev(c["xb"]), _dev(c["xv"])
    rng = np.random.default_rng(21)
    sample = np.sort(rng.choice(len(c["xv"]), 1000, replace=False))
    for nc in (MAX_CENTRES, 2049, 5000):
        S = np.sort(rng.choice(len(c["xb"]), nc, replace=False)).astype(np.int32)
        W = rng.normal(0.0, 0.01, (nc, 3))
        idx, w = _dev(S, torch.int32), _dev(W)
        st, dv = _call(f, xv, xb, idx, w, c["radius"])
        assert st == 0
        ref = P.deform_volume(xv, xb, idx, w, radius=c["radius"], eval_prec=P.PREC_F32)
        torch.cuda.synchronize()
        _check(c["xv"], c["xb"], S, W, c["radius"], dv.cpu().numpy(), ref.cpu().numpy(),
               sample)


def test_noalloc_empty_calls():
    """nv = 0 does the per-device set-up only; nc = 0 gives zero displacements."""
    f = _entry()
    xv = torch.ones((5, 3), dtype=torch.float64, device="cuda")
    xb = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    idx = torch.zeros(0, dtype=torch.int32, device="cuda")
    w = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    st, _ = _call(f, xv[:0], xb, idx, w, 2.0)
    assert st == 0
    st, dv = _call(f, xv, xb, idx, w, 2.0)
    assert st == 0 and torch.count_nonzero(dv).item() == 0


def test_noalloc_rejects_too_many_centres():
    f = _entry()
    xv = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    xb = torch.zeros((9000, 3), dtype=torch.float64, device="cuda")
    idx = torch.arange(9000, dtype=torch.int32, device="cuda")
    w = torch.zeros((9000, 3), dtype=torch.float64, device="cuda")
    st, _ = _call(f, xv, xb, idx, w, 2.0)
    assert st == 1
