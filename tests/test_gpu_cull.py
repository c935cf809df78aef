"""GPU parity of the culled volume sum (rbf_volume_plan_*): Eq. 6 with the
pairs farther apart than R skipped (the Wendland C2 basis is zero there,
Sec. 2).

The culled double-float sum keeps the standard double-float split of the
coordinates, the unculled kernel the grid split of its exact-difference
distances, so the two agree to the double-float rounding (2^-38 sum |w|,
far inside the FP64 oracle check below); the culled FP32 sum may differ
from the unculled FP32 kernel only by the phi values the latter gives at
d >= R (below 1e-28).  Both are compared with the FP64
oracle on seeded samples, at a radius where culling removes most pairs and
at one where it removes none.
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


@pytest.fixture(scope="module")
def wing():
    c = synth.wing_case(32, 250, 300_000, vol_seed=4, vol_kind="log", radius=0.25)
    rng = np.random.default_rng(21)
    c["d_xb"], c["d_xv"] = _dev(c["xb"]), _dev(c["xv"])
    c["rng"] = rng
    return c


def _support(c, nc, seed):
    rng = np.random.default_rng(seed)
    S = np.sort(rng.choice(len(c["xb"]), nc, replace=False)).astype(np.int32)
    W = synth.random_field(nc, seed + 1, sigma=0.1)
    return S, W


def _check(c, plan, S, W, R, prec, sample=3000):
    d_S, d_W = _dev(S, torch.int32), _dev(W)
    dv, pairs = plan.run(c["d_xb"], d_S, d_W, count=True)
    ref_gpu = P.deform_volume(c["d_xv"], c["d_xb"], d_S, d_W, radius=R, eval_prec=prec)
    dv_h, ref_h = dv.cpu().numpy(), ref_gpu.cpu().numpy()
    if prec == P.PREC_F32X2:
        assert np.abs(dv_h - ref_h).max() <= 2.0 ** -38 * np.abs(W).sum(), \
            np.abs(dv_h - ref_h).max()
    else:
        assert np.abs(dv_h - ref_h).max() <= 1e-24 * np.abs(W).sum()
    rng = np.random.default_rng(len(S))
    smp = np.sort(rng.choice(len(c["xv"]), min(sample, len(c["xv"])), replace=False))
    ref = oracle.rbf_sum(c["xv"][smp], c["xb"], S, W, R)
    err = np.abs(dv_h[smp] - ref).max(axis=1)
    if prec == P.PREC_F32X2:
        assert err.max() <= 1e-12 * max(1.0, np.abs(W).sum())
    else:
        Phi = oracle.phi(np.linalg.norm(c["xv"][smp][:, None] - c["xb"][S][None], axis=-1) / R)
        X = max(np.abs(c["xv"]).max(), np.abs(c["xb"]).max()) / R
        bound = 2.0 ** -24 * (64 * (Phi @ np.abs(W).sum(1)) + 16 * X * np.abs(W).sum()) + 1e-30
        assert np.all(err <= bound), (err / bound).max()
    return pairs


@pytest.mark.parametrize("prec", [P.PREC_F32X2, P.PREC_F32])
def test_cull_small_radius_matches_unculled_and_oracle(wing, prec):
    R = 0.25
    plan = P.VolumePlan(wing["d_xv"], radius=R, eval_prec=prec, nc_max=4096)
    S, W = _support(wing, 600, 31)
    pairs = _check(wing, plan, S, W, R, prec)
    total = len(wing["xv"]) * len(S)
    assert 0 < pairs < 0.5 * total, (pairs, total)
    # the exact count of pairs at distance < R is a lower bound of the visited pairs
    print(f"\nprec {prec}: visited {pairs / total:.3f} of {total} pairs, plan {plan.info()}")


@pytest.mark.parametrize("prec", [P.PREC_F32X2, P.PREC_F32])
def test_cull_large_radius_visits_every_pair(wing, prec):
    R = 2.0
    plan = P.VolumePlan(wing["d_xv"], radius=R, eval_prec=prec, nc_max=512)
    S, W = _support(wing, 300, 41)
    pairs = _check(wing, plan, S, W, R, prec)
    assert pairs == len(wing["xv"]) * len(S)


@pytest.mark.parametrize("prec", [P.PREC_F32X2, P.PREC_F32])
def test_cull_many_centres_chunks_and_reuse(wing, prec):
    # more centres than one shared-memory chunk (1024 double-float, 2048 FP32)
    R = 0.25
    plan = P.VolumePlan(wing["d_xv"], radius=R, eval_prec=prec, nc_max=2600)
    S, W = _support(wing, 2600, 51)
    _check(wing, plan, S, W, R, prec, sample=1500)
    # the same plan with another support set
    S2, W2 = _support(wing, 77, 61)
    _check(wing, plan, S2, W2, R, prec, sample=1500)


@pytest.mark.parametrize("prec", [P.PREC_F32X2, P.PREC_F32])
@pytest.mark.parametrize("nv", [1, 513, 1537])
def test_cull_ragged_and_far_points(wing, prec, nv):
    R = 0.25
    xv = wing["xv"][:nv].copy()
    xv[: max(1, nv // 3)] += 10.0          # points beyond R of every centre
    S, W = _support(wing, 150, 71)
    plan = P.VolumePlan(_dev(xv), radius=R, eval_prec=prec, nc_max=150)
    dv = plan.run(wing["d_xb"], _dev(S, torch.int32), _dev(W)).cpu().numpy()
    ref = oracle.rbf_sum(xv, wing["xb"], S, W, R)
    tol = 1e-12 if prec == P.PREC_F32X2 else 1e-4
    assert np.abs(dv - ref).max() <= tol * max(1.0, np.abs(W).sum())
    assert np.all(dv[: max(1, nv // 3)] == 0.0)


def test_cull_empty_support_and_bad_args(wing):
    plan = P.VolumePlan(wing["d_xv"][:1000].contiguous(), radius=0.25, eval_prec=P.PREC_F32,
                        nc_max=8)
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    dv = plan.run(wing["d_xb"], empty, torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert torch.count_nonzero(dv).item() == 0
    S, W = _support(wing, 9, 81)
    with pytest.raises(P.RBFError):
        plan.run(wing["d_xb"], _dev(S, torch.int32), _dev(W))   # nc > nc_max
