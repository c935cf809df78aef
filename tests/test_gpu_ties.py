"""GPU argmax on near-ties and exact ties (Alg. 1: largest error, lowest node
index among equal errors), against the oracle with no tie allowance.

The near-tie line (synth.line_near_tie) has one free node whose error
exceeds all the others by the relative amount 2^-35: far above FP64 rounding,
so both sides decide it the same way, but below the resolution of a key that
keeps only 28 mantissa bits.  The picks after it are exact ties.  Every
evaluation precision must reproduce the oracle's sequence exactly: the
screened ones cannot separate the candidates from their bounds and decide in
the FP64 re-score.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import synth

pytestmark = pytest.mark.gpu
NC = 8


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def line():
    c = synth.line_near_tie()
    c["estar"] = 0.5 * c["t"]
    o = oracle.greedy(c["xb"], c["db"], c["radius"], c["estar"], m=1, seed=1, ncmax=NC,
                      history=False)
    assert o["status"] == oracle.E_NC_MAX and o["idx"][3] == c["near"]
    c["o"] = o
    return c


@pytest.mark.parametrize("prec", [P.PREC_F64, P.PREC_F32, P.PREC_F32X2])
@pytest.mark.parametrize("ctas", [0, 1])
def test_greedy_near_tie_and_exact_ties(line, prec, ctas):
    c = line
    r = P.greedy_select(_cuda(c["xb"]), _cuda(c["db"]), radius=c["radius"], tol=c["estar"],
                        tol_mode=0, m=1, nc_max=NC, eval_prec=prec, ctas=ctas)
    torch.cuda.synchronize()
    assert r["status"] == P.E_NC_MAX
    assert r["idx"].cpu().numpy().tolist() == c["o"]["idx"].tolist()
    assert r["iter"].cpu().numpy().tolist() == c["o"]["iter"].tolist()


@pytest.mark.parametrize("prec", [P.PREC_F64, P.PREC_F32X2])
@pytest.mark.parametrize("peaks,sep", [(1, 0.0), (4, 0.0), (4, 3.0)])
def test_peaks_near_tie_and_exact_ties(line, prec, peaks, sep):
    c = line
    r = P.greedy_select_peaks(_cuda(c["xb"]), _cuda(c["db"]), radius=c["radius"],
                              tol=c["estar"], tol_mode=0, m=1, peaks=peaks, separation=sep,
                              nc_max=NC, eval_prec=prec)
    torch.cuda.synchronize()
    o = oracle.greedy_peaks(c["xb"], c["db"], c["radius"], c["estar"], m=1, ncmax=NC,
                            peaks=peaks, sep=sep)
    assert r["status"] == P.E_NC_MAX and o["status"] == oracle.E_NC_MAX
    assert r["idx"].cpu().numpy().tolist() == o["idx"].tolist()
    assert r["iter"].cpu().numpy().tolist() == o["iter"].tolist()


def test_batched_near_tie_and_exact_ties(line):
    c = line
    xb, db = _cuda(c["xb"]), _cuda(c["db"])
    probs = [dict(xb=xb, db=db, radius=c["radius"], tol=c["estar"], tol_mode=0, m=1, seed=1,
                  nc_max=NC) for _ in range(3)]
    gb = P.GreedyBatch(probs)
    gb.run()
    res = gb.results()
    torch.cuda.synchronize()
    for i in range(3):
        assert res[i]["status"] == P.E_NC_MAX
        assert gb.idx[i][:res[i]["nc"]].cpu().numpy().tolist() == c["o"]["idx"].tolist(), i
