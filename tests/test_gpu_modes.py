"""GPU parity for the comparison modes and second workloads of the paper's
Sec. 4: the fixed-N_c mode (tolerance 0, capacity N_c, as Sec. 4.1 fixes N_c
to compare m) and the Sec. 4.1 bending-twisting deformation (Eqs. 7-8, radius
7, absolute tolerance 1e-6) on the 2,000-node wing.  Every GPU decision is
checked by the oracle's follow mode (ties within 1e-6 relative accepted and
counted); with no divergence the sequences must be identical.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import synth
from _follow import check_follow

pytestmark = pytest.mark.gpu
TIE = 1e-6


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _follow(c, r, estar, m, ncmax=None):
    return oracle.greedy(c["xb"], c["db"], c["radius"], estar, m=m, seed=1, ncmax=ncmax,
                         follow=(r["idx"].cpu().numpy(), r["iter"].cpu().numpy()),
                         tie_rel=TIE, history=False)


@pytest.mark.parametrize("m", [1, 7, 40])
def test_fixed_nc_mode_follows_oracle(m):
    c = synth.wing_small(n_vol=0)
    n_fix = 150
    r = P.greedy_select(_cuda(c["xb"]), _cuda(c["db"]), radius=c["radius"], tol=0.0, tol_mode=0,
                        m=m, seed=1, nc_max=n_fix, eval_prec=P.PREC_F32X2)
    assert r["status"] == P.rbf.E_NC_MAX and r["nc"] == n_fix
    f = _follow(c, r, 0.0, m, ncmax=n_fix)
    assert f["status"] == oracle.E_NC_MAX and f["nc"] == n_fix
    check_follow(f, f"fixed N_c m={m}")
    assert f["stats"]["iterations"] == r["stats"]["iterations"]
    if f["stats"]["n_div"] == 0:
        o = oracle.greedy(c["xb"], c["db"], c["radius"], 0.0, m=m, seed=1, ncmax=n_fix,
                          history=False)
        assert r["idx"].cpu().numpy().tolist() == o["idx"].tolist()


@pytest.mark.parametrize("prec,m", [(P.PREC_F64, 1), (P.PREC_F32X2, 1), (P.PREC_F32X2, 7)])
def test_paper_mode_eq7_8_follows_oracle(prec, m):
    c = synth.wing_paper_mode_case(n_vol=2000)
    estar = c["tol_abs"]
    xb, db = _cuda(c["xb"]), _cuda(c["db"])
    r = P.greedy_select(xb, db, radius=c["radius"], tol=estar, tol_mode=0, m=m, seed=1,
                        eval_prec=prec, weights=True)
    assert r["status"] == 0
    f = _follow(c, r, estar, m)
    check_follow(f, f"Eqs. 7-8 prec {prec} m={m}")
    assert r["stats"]["final_max"] <= estar
    S = r["idx"].cpu().numpy()
    # weights and volume displacements against the oracle's solve for the set
    Wo, st, _ = oracle.solve_weights(c["xb"], c["db"], S, c["radius"])
    assert st == 0
    dmax = np.abs(c["db"]).max()
    ref = oracle.rbf_sum(c["xv"], c["xb"], S, Wo, c["radius"])
    dv = P.deform_volume(_cuda(c["xv"]), xb, r["idx"], r["w"], radius=c["radius"],
                         eval_prec=P.PREC_F32X2).cpu().numpy()
    assert np.abs(dv - ref).max() <= 1e-5 * dmax
    print(f"\nEqs. 7-8 mode, prec {prec}, m {m}: N_c {r['nc']}, iterations "
          f"{r['stats']['iterations']}, tie divergences {f['stats']['n_div']}")


@pytest.mark.parametrize("prec,m", [(P.PREC_F64, 1), (P.PREC_F32X2, 1), (P.PREC_F32X2, 2),
                                    (P.PREC_F32, 2)])
def test_paper_mode_eq10_follows_oracle(prec, m):
    """Sec. 4.2's deformation (Eq. 10: sinusoidal spanwise bending of the whole
    assembly) with the paper's radius 5 and absolute tolerance 2e-6, on a
    coarse copy of the wing-body-nacelle-pylon assembly (581 nodes): at these
    settings the greedy keeps almost every node, so the whole run is replayed
    by the oracle's follow mode."""
    c = synth.wbnp_paper_mode_case(n_vol=0, density=0.002)
    estar = c["tol_abs"]
    xb, db = _cuda(c["xb"]), _cuda(c["db"])
    r = P.greedy_select(xb, db, radius=c["radius"], tol=estar, tol_mode=0, m=m, seed=1,
                        eval_prec=prec, weights=True)
    assert r["status"] == 0
    f = _follow(c, r, estar, m)
    check_follow(f, f"Eq. 10 prec {prec} m={m}")
    assert f["nc"] == r["nc"]
    assert f["stats"]["iterations"] == r["stats"]["iterations"]
    assert r["stats"]["final_max"] <= estar
    S = r["idx"].cpu().numpy()
    Wo, st, _ = oracle.solve_weights(c["xb"], c["db"], S, c["radius"])
    assert st == 0
    dmax = np.abs(c["db"]).max()
    assert r["stats"]["max_resid"] <= 1e-10 * dmax
    print(f"\nEq. 10 mode, prec {prec}, m {m}: N_b {len(c['xb'])}, N_c {r['nc']}, "
          f"iterations {r['stats']['iterations']}")
