"""rbf_deform_volume_noalloc: the volume sum for callers that cannot allocate
device memory (its scratch is a fixed array reserved by the library).

Called through the C ABI and compared with rbf_deform_volume (FP32) on two
consecutive calls with different support sets, so a stale scratch table from
the first call would show up in the second.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import rbf, synth

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


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


def test_noalloc_volume_matches_workspace_entry_point_twice():
    f = _entry()
    c = synth.wing_small(n_vol=30_000)
    dev = lambda a, t=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=t,
                                                      device="cuda")
    xb, db, xv = dev(c["xb"]), dev(c["db"]), dev(c["xv"])
    for tol_rel, m in ((1e-3, 1), (3e-4, 5)):        # two support sets of different size
        g = P.greedy_select(xb, db, radius=c["radius"], tol=tol_rel, tol_mode=1, m=m,
                            eval_prec=P.PREC_F64)
        w, _ = P.solve_weights(xb, db, g["idx"], radius=c["radius"])
        st, dv = _call(f, xv, xb, g["idx"], w, c["radius"])
        assert st == 0
        ref = P.deform_volume(xv, xb, g["idx"], w, radius=c["radius"], eval_prec=P.PREC_F32)
        torch.cuda.synchronize()
        a, b = dv.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        # same FP32 arithmetic: agreement far inside the FP32 rounding bound
        W = w.cpu().numpy()
        X = max(np.abs(c["xv"]).max(), np.abs(c["xb"]).max()) / c["radius"]
        assert np.abs(a - b).max() <= U32 * 16 * X * np.abs(W).sum()


def test_noalloc_rejects_too_many_centres():
    f = _entry()
    xv = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    xb = torch.zeros((9000, 3), dtype=torch.float64, device="cuda")
    idx = torch.arange(9000, dtype=torch.int32, device="cuda")
    w = torch.zeros((9000, 3), dtype=torch.float64, device="cuda")
    st, _ = _call(f, xv, xb, idx, w, 2.0)
    assert st == 1
