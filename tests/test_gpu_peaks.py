"""GPU parity of the peak-selection variant (several separated error peaks
appended per iteration, the prior art cited in Sec. 1) with the oracle's
orc_greedy_peaks: identical node sequences, iteration numbers and iteration
counts, in FP64 and in double-float (whose selection is certified from the
error bounds or re-scored in FP64)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import synth

pytestmark = pytest.mark.gpu


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec", [P.PREC_F64, P.PREC_F32X2])
@pytest.mark.parametrize("m,peaks,sep", [(1, 3, 0.3), (3, 4, 0.25), (5, 2, 0.0), (7, 16, 0.1)])
def test_peaks_match_oracle_tiny(prec, m, peaks, sep):
    c = synth.tiny_wing(n_span=5, n_chord=24, radius=1.0)
    estar = oracle.tolerance(c["db"], 3e-3)
    r = P.greedy_select_peaks(_cuda(c["xb"]), _cuda(c["db"]), radius=c["radius"], tol=estar,
                              tol_mode=0, m=m, peaks=peaks, separation=sep, eval_prec=prec)
    o = oracle.greedy_peaks(c["xb"], c["db"], c["radius"], estar, m=m, peaks=peaks, sep=sep)
    assert r["status"] == 0 and o["status"] == oracle.OK
    assert r["idx"].cpu().numpy().tolist() == o["idx"].tolist()
    assert r["iter"].cpu().numpy().tolist() == o["iter"].tolist()
    assert r["stats"]["iterations"] == o["iterations"]


def test_one_peak_is_greedy_select():
    c = synth.wing_small(n_vol=0)
    estar = oracle.tolerance(c["db"], c["tol_rel"])
    xb, db = _cuda(c["xb"]), _cuda(c["db"])
    a = P.greedy_select(xb, db, radius=c["radius"], tol=estar, tol_mode=0, m=7,
                        eval_prec=P.PREC_F32X2)
    b = P.greedy_select_peaks(xb, db, radius=c["radius"], tol=estar, tol_mode=0, m=7, peaks=1,
                              separation=0.0, eval_prec=P.PREC_F32X2)
    assert a["idx"].cpu().numpy().tolist() == b["idx"].cpu().numpy().tolist()
    assert a["stats"]["iterations"] == b["stats"]["iterations"]


@pytest.mark.parametrize("m,peaks", [(1, 4), (40, 4)])
def test_peaks_wing_2000(m, peaks):
    c = synth.wing_small(n_vol=2000)
    estar = oracle.tolerance(c["db"], c["tol_rel"])
    sep = 0.25 * c["radius"]
    xb, db = _cuda(c["xb"]), _cuda(c["db"])
    r = P.greedy_select_peaks(xb, db, radius=c["radius"], tol=estar, tol_mode=0, m=m,
                              peaks=peaks, separation=sep, eval_prec=P.PREC_F32X2, weights=True)
    o = oracle.greedy_peaks(c["xb"], c["db"], c["radius"], estar, m=m, peaks=peaks, sep=sep)
    assert r["status"] == 0 and o["status"] == oracle.OK
    assert r["idx"].cpu().numpy().tolist() == o["idx"].tolist()
    assert r["iter"].cpu().numpy().tolist() == o["iter"].tolist()
    S = o["idx"]
    # several nodes per iteration, pairwise separated
    it = o["iter"][3:]
    assert len(np.unique(it)) < len(it)
    for k in np.unique(it):
        nodes = S[3:][it == k]
        for i in range(len(nodes)):
            for j in range(i):
                assert np.linalg.norm(c["xb"][nodes[i]] - c["xb"][nodes[j]]) >= sep
    # the selected set reproduces the prescribed displacement within E*
    Wo, st, _ = oracle.solve_weights(c["xb"], c["db"], S, c["radius"])
    F = oracle.rbf_sum(c["xb"], c["xb"], S, Wo, c["radius"])
    assert np.linalg.norm(c["db"] - F, axis=1).max() <= estar * (1 + 1e-6)
    dmax = np.abs(c["db"]).max()
    assert np.abs(r["w"].cpu().numpy() - Wo).max() <= 1e-5 * dmax


@pytest.mark.parametrize("prec", [P.PREC_F64, P.PREC_F32X2, P.PREC_F32])
@pytest.mark.parametrize("m,ctas", [(1, 0), (2, 0), (1, 1)])
def test_peaks_grid_split(prec, m, ctas):
    # 10,000 nodes: groups above 2,048 positions are split over the grid (one
    # record exchange per round); on one CTA each thread owns 39 positions,
    # more than its 32 exclusion bits
    c = synth.wing_case(80, 125, 0, vol_seed=0, radius=2.0, tol_rel=1e-4)
    estar = oracle.tolerance(c["db"], c["tol_rel"])
    sep = 0.2 * c["radius"]
    r = P.greedy_select_peaks(_cuda(c["xb"]), _cuda(c["db"]), radius=c["radius"], tol=estar,
                              tol_mode=0, m=m, peaks=6, separation=sep, eval_prec=prec, ctas=ctas)
    o = oracle.greedy_peaks(c["xb"], c["db"], c["radius"], estar, m=m, peaks=6, sep=sep)
    assert r["status"] == 0 and o["status"] == oracle.OK
    assert r["idx"].cpu().numpy().tolist() == o["idx"].tolist()
    assert r["iter"].cpu().numpy().tolist() == o["iter"].tolist()
    assert r["stats"]["iterations"] == o["iterations"]
    if ctas:
        assert r["stats"]["ctas"] == ctas


@pytest.mark.parametrize("prec", [P.PREC_F64, P.PREC_F32X2])
def test_peaks_capacity_truncates_the_last_block(prec):
    # 3 seeds + blocks of 4: the capacity 10 cuts the second block to 3 nodes
    c = synth.tiny_wing(n_span=5, n_chord=24, radius=1.0)
    estar = oracle.tolerance(c["db"], 1e-5)
    r = P.greedy_select_peaks(_cuda(c["xb"]), _cuda(c["db"]), radius=c["radius"], tol=estar,
                              tol_mode=0, m=1, peaks=4, separation=0.1, nc_max=10,
                              eval_prec=prec)
    o = oracle.greedy_peaks(c["xb"], c["db"], c["radius"], estar, m=1, ncmax=10, peaks=4,
                            sep=0.1)
    assert r["status"] == P.rbf.E_NC_MAX and o["status"] == oracle.E_NC_MAX
    assert r["idx"].cpu().numpy().tolist() == o["idx"].tolist()
    assert r["iter"].cpu().numpy().tolist() == o["iter"].tolist()


@pytest.mark.parametrize("case", ["in_s", "same_block"])
def test_peaks_coincident_nodes_not_spd(case):
    # in_s: node 7 is appended first and its twin 49 later (the block's first
    # pivot fails); same_block: both twins are peaks of one iteration, so the
    # block's pivot fails after its first node
    rng = np.random.default_rng(1 if case == "in_s" else 4)
    xb = rng.random((50, 3))
    xb[49] = xb[7]                       # a coincident pair with different displacements
    db = rng.standard_normal((50, 3)) * 0.1
    if case == "same_block":
        db[7], db[49], db[0] = (0.6, 0, 0), (-0.6, 0, 0), (2.0, 0, 0)
    o = oracle.greedy_peaks(xb, db, 1.5, 1e-9, m=1, peaks=8, sep=0.0)
    idx, it = o["idx"].tolist(), o["iter"].tolist()
    assert o["status"] == oracle.E_NOT_SPD
    assert (it[idx.index(7)] == it[idx.index(49)]) == (case == "same_block")
    with pytest.raises(P.RBFError) as e:
        P.greedy_select_peaks(_cuda(xb), _cuda(db), radius=1.5, tol=1e-9, tol_mode=0, m=1,
                              peaks=8, separation=0.0, eval_prec=P.PREC_F64)
    assert e.value.status == 2
