"""CPU checks of the C-ABI library: it loads without a GPU, exports every
entry point include/rbfgcb.h declares, validates arguments on the host, and
its host-side partition matches the oracle's."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import rbf

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "rbfgcb.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("rbf_greedy_select", "rbf_solve_weights", "rbf_deform_volume"):
        assert want in names


def test_library_exports_every_declared_symbol():
    L = P.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_status_strings_and_version():
    for code, name in rbf.STATUS.items():
        assert P.status_string(code).startswith(name)
    assert b"sm_103a" in P.lib().rbf_version()


def test_workspace_queries_validate_arguments():
    L = P.lib()
    p = rbf.make_params(2.0, 1e-3, 1, 64, m=1, nc_max=100)
    assert L.rbf_greedy_workspace_bytes(2000, C.byref(p)) > 0
    for bad in (rbf.make_params(0.0, 1e-3, 1, 64, m=1, nc_max=100),       # radius
                rbf.make_params(2.0, 1e-3, 1, 64, m=0, nc_max=100),        # m
                rbf.make_params(2.0, 1e-3, 1, 64, m=3000, nc_max=100),     # m > nb
                rbf.make_params(2.0, 1e-3, 1, 16, m=1, nc_max=100),        # precision
                rbf.make_params(2.0, -1.0, 1, 64, m=1, nc_max=100),        # tolerance
                rbf.make_params(2.0, 1e-3, 1, 64, m=1, nc_max=2)):         # capacity
        assert L.rbf_greedy_workspace_bytes(2000, C.byref(bad)) == 0
    assert L.rbf_solve_workspace_bytes(0) == 0
    assert L.rbf_solve_workspace_bytes(500) > 8 * 500 * 500


def test_calls_reject_bad_arguments_before_touching_a_device():
    L = P.lib()
    p = rbf.make_params(2.0, 1e-3, 1, 64, m=1, nc_max=100)
    nc = C.c_int64(0)
    # null inputs
    st = L.rbf_greedy_select(None, None, 2000, C.byref(p), None, None, None, None, 0,
                             C.byref(nc), None, None, None, 0, None)
    assert st == 1
    bad = rbf.make_params(-1.0, eval_prec=32)
    st = L.rbf_deform_volume(C.c_void_p(16), 10, C.c_void_p(16), C.c_void_p(16), 5,
                             C.c_void_p(16), C.byref(bad), C.c_void_p(16), None, 0, None)
    assert st == 1


@pytest.mark.parametrize("nb,m,seed", [(1, 1, 0), (10, 3, 7), (2000, 13, 1), (50000, 161, 1),
                                       (999, 999, 12345)])
def test_partition_matches_oracle_bit_exact(nb, m, seed):
    assert np.array_equal(P.group_of(nb, m, seed), oracle.groups(nb, m, seed))


def test_partition_rejects_bad_sizes():
    with pytest.raises(P.RBFError):
        P.group_of(10, 11, 0)


def test_newer_entry_points_reject_bad_arguments_before_touching_a_device():
    L = P.lib()
    E_ARG, E_WS = 1, 5
    fake = C.c_void_p(256)   # never dereferenced: every call below fails its checks first
    # culled volume plans
    p32 = rbf.make_params(0.25, eval_prec=32, nc_max=100)
    assert L.rbf_volume_plan_workspace_bytes(1000, C.byref(p32)) > 0
    for bad in (rbf.make_params(0.25, eval_prec=64, nc_max=100),     # precision
                rbf.make_params(0.25, eval_prec=32, nc_max=0)):      # capacity
        assert L.rbf_volume_plan_workspace_bytes(1000, C.byref(bad)) == 0
    assert L.rbf_volume_plan_workspace_bytes(0, C.byref(p32)) == 0
    h = C.c_void_p()
    assert L.rbf_volume_plan_create(None, 1000, C.byref(p32), fake, 1 << 20, None,
                                    C.byref(h)) == E_ARG
    bad_r = rbf.make_params(-1.0, eval_prec=32, nc_max=100)
    assert L.rbf_volume_plan_create(fake, 1000, C.byref(bad_r), fake, 1 << 20, None,
                                    C.byref(h)) == E_ARG
    assert L.rbf_volume_plan_create(fake, 1000, C.byref(p32), None, 0, None,
                                    C.byref(h)) == E_WS
    assert L.rbf_volume_plan_run(None, fake, fake, 10, fake, fake, None, None) == E_ARG
    # support-set KL divergence
    assert L.rbf_support_kl_workspace_bytes(0) == 0
    kl = C.c_double(0.0)
    assert L.rbf_support_kl(fake, 0, fake, 3, fake, 3, C.byref(kl), fake, 1 << 20,
                            None) == E_ARG
    assert L.rbf_support_kl(fake, 100, fake, 0, fake, 3, C.byref(kl), fake, 1 << 20,
                            None) == E_ARG
    assert L.rbf_support_kl(fake, 100, fake, 3, fake, 3, C.byref(kl), None, 0, None) == E_WS
    assert L.rbf_nearest_support(fake, 100, fake, 0, fake, None) == E_ARG
    # factor objects and the factored adjoint
    assert L.rbf_factor_workspace_bytes(0) == 0
    assert L.rbf_factor_workspace_bytes(300) > 8 * 300 * 300
    pf = rbf.make_params(2.0)
    assert L.rbf_factor_create(fake, 1000, fake, 300, C.byref(pf), fake, 1 << 30, None,
                               None) == E_ARG
    assert L.rbf_factor_create(fake, 1000, fake, 300, C.byref(pf), None, 0, None,
                               C.byref(h)) == E_WS
    res = C.c_double(0.0)
    assert L.rbf_factor_solve(None, fake, 2, fake, C.byref(res), None) == E_ARG
    pa = rbf.make_params(2.0, eval_prec=48)
    assert L.rbf_deform_volume_adjoint_factored(fake, 10, fake, None, C.byref(pa), fake,
                                                C.byref(res), fake, 1 << 20, None) == E_ARG
    # peak selection: peaks in 1..16, separation finite and >= 0, then the
    # usual greedy checks (all before any device work)
    pg = rbf.make_params(2.0, tol=1e-3, m=4, nc_max=50)
    nc_out = C.c_int64(0)
    for peaks, sep in ((0, 0.1), (17, 0.1), (4, -0.5), (4, float("nan")), (4, float("inf"))):
        assert L.rbf_greedy_select_peaks(fake, fake, 1000, C.byref(pg), peaks, sep, fake, None,
                                         None, C.byref(nc_out), None, fake, 1 << 30,
                                         None) == E_ARG
    assert L.rbf_greedy_select_peaks(None, fake, 1000, C.byref(pg), 4, 0.1, fake, None, None,
                                     C.byref(nc_out), None, fake, 1 << 30, None) == E_ARG
    assert L.rbf_greedy_select_peaks(fake, fake, 1000, C.byref(pg), 4, 0.1, fake, None, None,
                                     C.byref(nc_out), None, None, 0, None) == E_WS
    # latency microbenchmarks
    assert L.rbf_measure_latency(99, 0, C.byref(res), None) == E_ARG
    assert L.rbf_measure_latency(1, 64, None, None) == E_ARG


def test_noalloc_entry_point_rejects_bad_arguments_before_touching_a_device():
    """rbf_deform_volume_noalloc checks its arguments before any CUDA call, so
    every rejection below runs without a GPU (the dummy addresses are never
    dereferenced)."""
    L = P.lib()
    f = L.rbf_deform_volume_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                  C.POINTER(rbf.Params), C.c_void_p, C.c_void_p]
    E_ARG = 1
    fake = C.c_void_p(256)
    ok = rbf.make_params(2.0, eval_prec=P.PREC_F32)
    cap = 8192                                   # RBF_NOALLOC_MAX_CENTRES
    assert f"#define RBF_NOALLOC_MAX_CENTRES {cap}" in open(HEADER).read()
    # more centres than the fixed scratch array holds
    assert f(fake, 10, fake, fake, cap + 1, fake, C.byref(ok), fake, None) == E_ARG
    # only the FP32 sum is offered
    for prec in (P.PREC_F64, P.PREC_F32X2, 16):
        bad = rbf.make_params(2.0, eval_prec=prec)
        assert f(fake, 10, fake, fake, 5, fake, C.byref(bad), fake, None) == E_ARG
    # radius must be positive and finite
    for r in (0.0, -1.0, float("nan")):
        bad = rbf.make_params(r, eval_prec=P.PREC_F32)
        assert f(fake, 10, fake, fake, 5, fake, C.byref(bad), fake, None) == E_ARG
    # null parameters and null arrays
    assert f(fake, 10, fake, fake, 5, fake, None, fake, None) == E_ARG
    assert f(None, 10, fake, fake, 5, fake, C.byref(ok), fake, None) == E_ARG
    assert f(fake, 10, None, fake, 5, fake, C.byref(ok), fake, None) == E_ARG
    assert f(fake, 10, fake, None, 5, fake, C.byref(ok), fake, None) == E_ARG
    assert f(fake, 10, fake, fake, 5, None, C.byref(ok), fake, None) == E_ARG
    assert f(fake, 10, fake, fake, 5, fake, C.byref(ok), None, None) == E_ARG
    # negative sizes
    assert f(fake, -1, fake, fake, 5, fake, C.byref(ok), fake, None) == E_ARG
    assert f(fake, 10, fake, fake, -1, fake, C.byref(ok), fake, None) == E_ARG
