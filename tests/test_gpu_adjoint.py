"""GPU parity of the adjoint (dJ/dd_c = Phi_cc^-1 Phi_vc^T dJ/dd_v) with the
oracle's FP64 gradient, central finite differences of the quadratic
objective J = sum_v 1/2 |d_v - t_v|^2, and the autograd wrapper."""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import synth

pytestmark = pytest.mark.gpu


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _case(n_vol=20_000):
    c = synth.wing_small(n_vol=n_vol)
    estar = oracle.tolerance(c["db"], c["tol_rel"])
    o = oracle.greedy(c["xb"], c["db"], c["radius"], estar, m=1, seed=1, history=False)
    t = synth.random_field(len(c["xv"]), seed=5, sigma=0.01)
    return c, o["idx"].astype(np.int32), t


def _gv(c, S, t):
    W, _, _ = oracle.solve_weights(c["xb"], c["db"], S, c["radius"])
    dv = oracle.rbf_sum(c["xv"], c["xb"], S, W, c["radius"])
    return dv - t


@pytest.mark.parametrize("prec", [P.PREC_F32X2, P.PREC_F32])
def test_adjoint_matches_oracle_gradient(prec):
    c, S, t = _case()
    gv = _gv(c, S, t)
    ref, st = oracle.adjoint(c["xv"], c["xb"], S, c["radius"], gv)
    g, res = P.adjoint(cuda(c["xv"]), cuda(c["xb"]), cuda(S, torch.int32), cuda(gv),
                       radius=c["radius"], eval_prec=prec)
    err = np.abs(g.cpu().numpy() - ref).max() / np.abs(ref).max()
    # double-float sums: at the FP64 level; FP32 sums: stated, amplified by
    # the conditioning of Phi_cc
    assert err <= (1e-8 if prec == P.PREC_F32X2 else 1e-1), err


def test_adjoint_central_differences():
    """Configuration 5's check on a reduced volume (N_v = 20,000): J is
    quadratic in the boundary displacements, so central differences of the
    oracle's FP64 objective (h = 1e-6) are exact up to rounding.  200 random
    support components (seed 6) of the GPU's autograd gradient are compared
    with them, and 10 components of non-support nodes, on which J does not
    depend, must come back exactly 0."""
    c, S, t = _case(n_vol=20_000)
    R = c["radius"]
    xv, xb, Sd = cuda(c["xv"]), cuda(c["xb"]), cuda(S, torch.int32)
    tt = cuda(t)

    def J(db_full):
        W, st, _ = oracle.solve_weights(c["xb"], db_full, S, R)
        assert st == 0
        dv = oracle.rbf_sum(c["xv"], c["xb"], S, W, R)
        return 0.5 * float(((dv - t) ** 2).sum())

    # the full N_b x 3 displacement field is the leaf: the support rows are
    # gathered from it, so its gradient is 0 on every other node
    db_full = cuda(c["db"]).requires_grad_(True)
    dv = P.deform(db_full.index_select(0, Sd.long()), xv, xb, Sd, radius=R,
                  eval_prec=P.PREC_F32X2)
    (0.5 * ((dv - tt) ** 2).sum()).backward()
    g = db_full.grad.cpu().numpy()
    rng = np.random.default_rng(6)
    h = 1e-6
    sup = rng.choice(3 * len(S), 200, replace=False)
    comps = [(int(S[k // 3]), int(k % 3)) for k in sup]
    free = np.setdiff1d(np.arange(len(c["xb"])), S)
    comps_free = [(int(n), int(rng.integers(0, 3))) for n in rng.choice(free, 10, replace=False)]
    scale = np.abs(g).max()
    worst = 0.0
    for node, ax in comps + comps_free:
        dp, dm = c["db"].copy(), c["db"].copy()
        dp[node, ax] += h
        dm[node, ax] -= h
        fd = (J(dp) - J(dm)) / (2 * h)
        if (node, ax) in comps_free:
            assert fd == 0.0 and g[node, ax] == 0.0, (node, ax, fd, g[node, ax])
        else:
            worst = max(worst, abs(fd - g[node, ax]) / scale)
            assert abs(fd - g[node, ax]) <= 1e-5 * scale, (node, ax, fd, g[node, ax])
    print(f"\ncentral differences, 200 support components: worst |fd - g| / max|g| {worst:.2e}")


def test_autograd_matches_adjoint_entry_point():
    c, S, t = _case(n_vol=8_000)
    xv, xb, Sd = cuda(c["xv"]), cuda(c["xb"]), cuda(S, torch.int32)
    d0 = cuda(c["db"][S]).requires_grad_(True)
    dv = P.deform(d0, xv, xb, Sd, radius=c["radius"])
    gv = torch.randn_like(dv)
    dv.backward(gv)
    g2, _ = P.adjoint(xv, xb, Sd, gv.contiguous(), radius=c["radius"])
    assert torch.allclose(d0.grad, g2, rtol=0, atol=1e-12 * float(g2.abs().max()))


def test_adjoint_full_size():
    """Support set of the GCB wing (N_b = 50,000, m = 1.5 N_b/N_c) and its
    2,000,000 volume points; t_v Gaussian (sigma 0.01, seed 5)."""
    c = synth.wing_gcb(n_vol=2_000_000)
    estar = oracle.tolerance(c["db"], c["tol_rel"])
    xb, db = cuda(c["xb"]), cuda(c["db"])
    plain = P.greedy_select(xb, db, radius=c["radius"], tol=estar, tol_mode=0, m=1,
                            eval_prec=P.PREC_F32X2)
    m = int(round(1.5 * len(c["xb"]) / plain["nc"]))
    r = P.greedy_select(xb, db, radius=c["radius"], tol=estar, tol_mode=0, m=m,
                        eval_prec=P.PREC_F32X2, weights=True)
    S = r["idx"].cpu().numpy()
    xv = cuda(c["xv"])
    t = synth.random_field(len(c["xv"]), seed=5, sigma=0.01)
    dv = P.deform_volume(xv, xb, r["idx"], r["w"], radius=c["radius"], eval_prec=P.PREC_F32X2)
    gv = dv - cuda(t)
    g, _ = P.adjoint(xv, xb, r["idx"], gv.contiguous(), radius=c["radius"])
    ref, st = oracle.adjoint(c["xv"], c["xb"], S, c["radius"], gv.cpu().numpy())
    err = np.abs(g.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 1e-7, err


# ---------------------------------------------------------------- factor ----
def test_factor_solves_match_oracle_and_fresh_solves():
    c, S, _ = _case(n_vol=0)
    xb, dS = cuda(c["xb"]), cuda(S, torch.int32)
    f = P.Factor(xb, dS, radius=c["radius"])
    # the prescribed displacements: the oracle's weights
    Wo, st, _ = oracle.solve_weights(c["xb"], c["db"], S, c["radius"])
    assert st == oracle.OK
    w, res = f.solve(cuda(c["db"][S]))
    assert np.abs(w.cpu().numpy() - Wo).max() <= 1e-9 * np.abs(Wo).max()
    assert res <= 1e-12
    # several right-hand sides through the same factor: residual of
    # Phi_SS X = B in FP64, and agreement with a fresh factorisation
    rng = np.random.default_rng(3)
    Phi = oracle.phi(np.linalg.norm(c["xb"][S][:, None] - c["xb"][S][None], axis=-1) / c["radius"])
    for _ in range(3):
        B = rng.standard_normal((len(S), 3))
        x, res = f.solve(cuda(B))
        xh = x.cpu().numpy()
        assert np.abs(Phi @ xh - B).max() <= 1e-10 * np.abs(B).max()
        x2, _ = P.solve_system(xb, dS, cuda(B), radius=c["radius"])
        assert np.abs(xh - x2.cpu().numpy()).max() <= 1e-9 * np.abs(xh).max()


@pytest.mark.parametrize("prec", [P.PREC_F32X2, P.PREC_F32])
def test_factored_adjoint_matches_unfactored_and_oracle(prec):
    c, S, t = _case()
    gv = _gv(c, S, t)
    xb, dS, xv = cuda(c["xb"]), cuda(S, torch.int32), cuda(c["xv"])
    f = P.Factor(xb, dS, radius=c["radius"])
    g1, _ = P.adjoint(xv, xb, dS, cuda(gv), radius=c["radius"], eval_prec=prec)
    g2, res = P.adjoint_factored(xv, cuda(gv), f, eval_prec=prec)
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    assert np.abs(g1 - g2).max() <= 1e-9 * np.abs(g1).max()
    ref, st = oracle.adjoint(c["xv"], c["xb"], S, c["radius"], gv)
    tol = 1e-8 if prec == P.PREC_F32X2 else 1e-1   # as the unfactored adjoint
    assert np.abs(g2 - ref).max() <= tol * np.abs(ref).max()


def test_deform_autograd_with_factor():
    c, S, t = _case()
    xb, dS, xv = cuda(c["xb"]), cuda(S, torch.int32), cuda(c["xv"])
    f = P.Factor(xb, dS, radius=c["radius"])
    tt = cuda(t)
    grads = []
    for fac in (None, f):
        dc = cuda(c["db"][S]).requires_grad_(True)
        dv = P.deform(dc, xv, xb, dS, radius=c["radius"], factor=fac)
        J = 0.5 * ((dv - tt) ** 2).sum()
        J.backward()
        grads.append(dc.grad.cpu().numpy())
    assert np.abs(grads[0] - grads[1]).max() <= 1e-9 * np.abs(grads[0]).max()
