"""Volume points read from, and displacements written to, pinned host memory
by the kernels themselves (rbf_deform_volume accepts host memory the device
reaches at the same address): the results must be bit-identical to the
device-resident call in every precision, and memory the device cannot reach
must be refused before any device work."""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import rbf, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [P.PREC_F32, P.PREC_F32X2, P.PREC_F64])
def test_pinned_host_points_and_output_match_device_call(prec):
    c = synth.wing_small(n_vol=50_001)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    xb, db, xv = dev(c["xb"]), dev(c["db"]), dev(c["xv"])
    g = P.greedy_select(xb, db, radius=c["radius"], tol=c["tol_rel"], tol_mode=1, m=5,
                        eval_prec=P.PREC_F32X2, weights=True)
    ref = P.deform_volume(xv, xb, g["idx"], g["w"], radius=c["radius"], eval_prec=prec)
    hx = torch.from_numpy(np.ascontiguousarray(c["xv"])).pin_memory()
    hout = torch.full((len(c["xv"]), 3), float("nan"), dtype=torch.float64).pin_memory()
    P.deform_volume(hx, xb, g["idx"], g["w"], radius=c["radius"], eval_prec=prec, out=hout)
    torch.cuda.synchronize()
    assert torch.equal(hout, ref.cpu())
    # host points, device output
    d2 = P.deform_volume(hx, xb, g["idx"], g["w"], radius=c["radius"], eval_prec=prec)
    assert torch.equal(d2, ref)


def test_pageable_host_memory_is_refused():
    c = synth.wing_small(n_vol=1000)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    xb, db = dev(c["xb"]), dev(c["db"])
    g = P.greedy_select(xb, db, radius=c["radius"], tol=c["tol_rel"], tol_mode=1, m=5,
                        eval_prec=P.PREC_F64, weights=True)
    hx = np.ascontiguousarray(c["xv"])                  # ordinary (pageable) host memory
    out = torch.empty((len(hx), 3), dtype=torch.float64, device="cuda")
    L = P.lib()
    p = rbf.make_params(c["radius"], eval_prec=P.PREC_F32X2)
    ws = torch.empty(L.rbf_volume_workspace_bytes(len(hx), g["nc"], C.byref(p)),
                     dtype=torch.uint8, device="cuda")
    st = L.rbf_deform_volume(C.c_void_p(hx.ctypes.data), len(hx), C.c_void_p(xb.data_ptr()),
                             C.c_void_p(g["idx"].data_ptr()), g["nc"],
                             C.c_void_p(g["w"].data_ptr()), C.byref(p),
                             C.c_void_p(out.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(),
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1
    with pytest.raises(TypeError):
        P.deform_volume(torch.from_numpy(hx), xb, g["idx"], g["w"], radius=c["radius"])
