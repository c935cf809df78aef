"""GPU parity of the support-set KL divergence (Sec. 4.1) and of the
nearest-support distances it is built on, against the FP64 oracle.

At full size (the 50,000-node wing, N_c fixed to the plain greedy's count as
in Sec. 4.1) it also checks the paper's qualitative finding (Table 4): the
GCB support sets lie much closer to the plain greedy's set than random sets
of the same size do.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_nearest_support_matches_oracle_ragged():
    xb = synth.random_cloud(5003, seed=12)
    for nc in (1, 37, 2049, 2500):        # one and several shared-memory chunks
        S = np.sort(np.random.default_rng(nc).choice(len(xb), nc, replace=False)).astype(np.int32)
        d = P.nearest_support(_dev(xb), _dev(S, torch.int32)).cpu().numpy()
        ref = oracle.nearest_support(xb, S)
        assert np.allclose(d, ref, rtol=1e-14, atol=0)
        assert np.all(d[S] == 0.0)


def test_kl_small_cases():
    xb = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0], [3.0, 0, 0]])
    s0, s3 = _dev(np.array([0], np.int32), torch.int32), _dev(np.array([3], np.int32), torch.int32)
    assert P.support_kl(_dev(xb), s0, s3) == pytest.approx(np.log(2.0), rel=1e-14)
    xr = synth.random_cloud(3000, seed=4)
    rng = np.random.default_rng(8)
    S1 = np.sort(rng.choice(3000, 120, replace=False)).astype(np.int32)
    S2 = np.sort(rng.choice(3000, 90, replace=False)).astype(np.int32)
    d_x = _dev(xr)
    assert P.support_kl(d_x, _dev(S1, torch.int32), _dev(S1, torch.int32)) == 0.0
    kl = P.support_kl(d_x, _dev(S1, torch.int32), _dev(S2, torch.int32))
    assert kl == pytest.approx(oracle.support_kl(xr, S1, S2), rel=1e-12)


def test_kl_full_size_gcb_closer_than_random():
    c = synth.wing_gcb(n_vol=0)
    xb, db = _dev(c["xb"]), _dev(c["db"])
    estar = oracle.tolerance(c["db"], c["tol_rel"])
    plain = P.greedy_select(xb, db, radius=c["radius"], tol=estar, tol_mode=0, m=1, seed=1,
                            eval_prec=P.PREC_F32X2)
    nc = plain["nc"]
    nb = len(c["xb"])
    S1 = plain["idx"]
    rows = []
    for factor in (1.0, 1.5, 2.0):
        m = int(round(factor * nb / nc))
        # N_c fixed to the plain greedy's count (tolerance 0, capacity N_c)
        g = P.greedy_select(xb, db, radius=c["radius"], tol=0.0, tol_mode=0, m=m, seed=1,
                            nc_max=nc, eval_prec=P.PREC_F32X2)
        assert g["status"] == P.rbf.E_NC_MAX and g["nc"] == nc
        kl = P.support_kl(xb, S1, g["idx"])
        ref = oracle.support_kl(c["xb"], S1.cpu().numpy(), g["idx"].cpu().numpy())
        assert kl == pytest.approx(ref, rel=1e-12)
        rows.append(("m=%d" % m, kl))
    rng = np.random.default_rng(1)
    rand = []
    for r in range(2):
        S2 = np.sort(rng.choice(nb, nc, replace=False)).astype(np.int32)
        kl = P.support_kl(xb, S1, _dev(S2, torch.int32))
        assert kl == pytest.approx(oracle.support_kl(c["xb"], S1.cpu().numpy(), S2), rel=1e-12)
        rand.append(kl)
        rows.append(("random-%d" % (r + 1), kl))
    print("\nKL(plain || S), N_c = %d: " % nc + ", ".join("%s %.3f" % t for t in rows))
    assert max(k for _, k in rows[:3]) < 0.5 * min(rand)
