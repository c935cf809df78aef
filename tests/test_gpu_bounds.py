"""The certified error bounds of the screened evaluation (FP32 and
double-float modes of the greedy), checked node by node.

Alg. 1's argmax and its E > E* test are taken on screened errors E~ with a
bound beta derived term by term in the library's sources: |E~ - E| <= beta,
E the exact error with the evaluation table's weights.  After a run every
node outside S was last evaluated with the final weights, so the library's
record of (E~, beta) is compared here with the oracle's FP64 errors for those
weights, on every node.  The derivation assumes the two hardware
approximations it uses (sqrt.approx.f32 and rsqrtf) are within 2^-22
relative; that is measured on every normal float in [2^-126, 4).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import synth

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53


@pytest.mark.parametrize("which", [P.rbf.APPROX_SQRT, P.rbf.APPROX_RSQRT])
def test_hardware_approximations_within_the_bound_constant(which):
    r = P.measure_approx_error(which)
    print(f"\napproximation {which}: max relative error {r:.4e} = 2^{np.log2(r):.2f}")
    assert 0.0 < r <= 2.0 ** -22


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("prec", [P.PREC_F32X2, P.PREC_F32])
@pytest.mark.parametrize("m,ctas", [(5, 0), (1, 0), (1, 1)])
def test_screened_errors_within_certified_bounds(prec, m, ctas):
    """(m, ctas) = (1, 1): one CTA of 256 lanes for 2,000 nodes, so every lane
    sums over all N_c centres (the longest accumulation chains)."""
    c = synth.wing_small(n_vol=0)
    R = c["radius"]
    xb, db = _cuda(c["xb"]), _cuda(c["db"])
    r = P.greedy_select(xb, db, radius=R, tol=c["tol_rel"], tol_mode=1, m=m, seed=1,
                        eval_prec=prec, ctas=ctas, screen=True)
    assert r["status"] == 0
    S = r["idx"].cpu().numpy()
    sc = r["screen"]
    err = sc["err"].cpu().numpy()
    bnd = sc["bound"].cpu().numpy().astype(np.float64)
    W = sc["w_eval"].cpu().numpy()
    free = np.setdiff1d(np.arange(len(c["xb"])), S)
    F = oracle.rbf_sum(c["xb"][free], c["xb"], S, W, R)
    E = np.linalg.norm(c["db"][free] - F, axis=1)
    # the oracle's own FP64 rounding, bounded from the same sums
    Phi = oracle.phi(np.linalg.norm(c["xb"][free][:, None] - c["xb"][S][None], axis=-1) / R)
    sb = Phi @ np.abs(W).sum(1)
    slack = U64 * ((len(S) + 20) * sb + 4 * np.abs(c["db"][free]).sum(1) + 4 * E)
    b = bnd[free]
    screened = b > 0
    dev = np.abs(err[free] - E)
    assert np.all(dev[screened] <= b[screened] + slack[screened]), \
        (dev[screened] / b[screened]).max()
    ratio = (dev[screened] / b[screened]).max() if screened.any() else 0.0
    print(f"\nprec {prec}, m {m}, ctas {ctas}: N_c {r['nc']}, {screened.sum()} screened "
          f"nodes, {(~screened).sum()} re-scored in FP64, largest |E~ - E| / beta "
          f"{ratio:.3e}, median beta / E* {np.median(b[screened]) / r['stats']['estar']:.2e}")
    # the certified final maximum bounds every screened node's exact error
    # (re-scored nodes were evaluated in FP64 with the FP64 weights, not with
    # the table's rounded ones)
    if screened.any():
        assert r["stats"]["final_max"] >= (E - slack)[screened].max()
