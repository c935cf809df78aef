"""GPU parity at the benchmark's full sizes (GCB wing: N_b = 50,000 boundary
nodes, N_v = 2,000,000 volume points), in the configuration bench.py times.

The oracle follows the GPU's whole selection sequence (every decision checked
in FP64, ties within 1e-6 relative accepted and counted); volume
displacements are compared on a seeded sample of points the oracle computes
one by one.
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


@pytest.fixture(scope="module")
def case():
    c = synth.wing_gcb(n_vol=2_000_000)
    dev = lambda a, t=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=t,
                                                      device="cuda")
    c["d_xb"], c["d_db"], c["d_xv"] = dev(c["xb"]), dev(c["db"]), dev(c["xv"])
    c["estar"] = oracle.tolerance(c["db"], c["tol_rel"])
    plain = P.greedy_select(c["d_xb"], c["d_db"], radius=c["radius"], tol=c["estar"],
                            tol_mode=0, m=1, seed=1, eval_prec=P.PREC_F32X2)
    c["plain"] = plain
    c["m"] = int(round(1.5 * len(c["xb"]) / plain["nc"]))
    return c


def _follow(c, r, m):
    return oracle.greedy(c["xb"], c["db"], c["radius"], c["estar"], m=m, seed=1,
                         follow=(r["idx"].cpu().numpy(), r["iter"].cpu().numpy()),
                         tie_rel=TIE, history=False)


def test_plain_greedy_full_size_certified(case):
    f = _follow(case, case["plain"], 1)
    check_follow(f, "plain greedy, 50,000 nodes")
    assert case["plain"]["stats"]["final_max"] <= case["estar"]


@pytest.mark.parametrize("factor", [1.0, 1.5, 2.0])
def test_gcb_greedy_full_size_certified(case, factor):
    m = int(round(factor * len(case["xb"]) / case["plain"]["nc"]))
    r = P.greedy_select(case["d_xb"], case["d_db"], radius=case["radius"], tol=case["estar"],
                        tol_mode=0, m=m, seed=1, eval_prec=P.PREC_F32X2)
    f = _follow(case, r, m)
    check_follow(f, f"GCB m={m}, 50,000 nodes")
    assert r["stats"]["final_max"] <= case["estar"]
    # GCB evaluates far fewer pairs than the plain greedy (Sec. 3)
    assert r["stats"]["pairs_ff"] * 5 < case["plain"]["stats"]["pairs_ff"]


def test_weights_and_volume_full_size(case):
    c = case
    r = P.greedy_select(c["d_xb"], c["d_db"], radius=c["radius"], tol=c["estar"], tol_mode=0,
                        m=c["m"], seed=1, eval_prec=P.PREC_F32X2, weights=True)
    S = r["idx"].cpu().numpy()
    w, res = P.solve_weights(c["d_xb"], c["d_db"], r["idx"], radius=c["radius"])
    Wo, st, _ = oracle.solve_weights(c["xb"], c["db"], S, c["radius"])
    dmax = np.abs(c["db"]).max()
    assert np.abs(w.cpu().numpy() - Wo).max() <= 1e-5 * dmax
    assert res <= 1e-10 * dmax
    assert np.abs(r["w"].cpu().numpy() - Wo).max() <= 1e-5 * dmax
    assert r["stats"]["max_resid"] <= 1e-10 * dmax
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(len(c["xv"]), 4000, replace=False))
    ref = oracle.rbf_sum(c["xv"][sample], c["xb"], S, Wo, c["radius"])
    dv = P.deform_volume(c["d_xv"], c["d_xb"], r["idx"], w, radius=c["radius"],
                         eval_prec=P.PREC_F32X2).cpu().numpy()[sample]
    assert np.abs(dv - ref).max() <= 1e-5 * dmax
    # the FP32 kernel: error stated against its rounding bound
    dv32 = P.deform_volume(c["d_xv"], c["d_xb"], r["idx"], w, radius=c["radius"],
                           eval_prec=P.PREC_F32).cpu().numpy()[sample]
    R = c["radius"]
    Phi = oracle.phi(np.linalg.norm(c["xv"][sample][:, None] - c["xb"][S][None], axis=-1) / R)
    X = max(np.abs(c["xv"]).max(), np.abs(c["xb"]).max()) / R
    bound = 2.0 ** -24 * (64 * (Phi @ np.abs(Wo).sum(1)) + 16 * X * np.abs(Wo).sum())
    err32 = np.abs(dv32 - ref).max(axis=1)
    assert np.all(err32 <= bound), (err32 / bound).max()
    print(f"\nFP32 volume error: max {err32.max():.3e} = {err32.max() / dmax:.3e} of max|dr|")
