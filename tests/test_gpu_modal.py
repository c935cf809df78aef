"""GPU parity of the tensor-core modal path D = Phi_vc W (tcgen05, BF16 or
FP16 inputs, FP32 accumulation) against FP64, at the error bounds its input
rounding allows: BF16 |err| <= 2^-7 (Phi |W|), BF16x3 |err| <= 2^-18 (Phi |W|),
FP16x2 |err| <= 2^-20 (Phi |W|) + 2^-24 sum_j |W_j| (phi below the FP16 normal
range keeps an absolute precision of 2^-25) elementwise."""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_04817_gb300 as P
from paper_2004_04817_gb300 import synth

pytestmark = pytest.mark.gpu


def cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _ref(xv, xc, W, R):
    D = np.linalg.norm(xv[:, None, :] - xc[None], axis=-1) / R
    Phi = oracle.phi(D)
    return Phi @ W, Phi @ np.abs(W)


def _bound(mode, scale, bnd, W):
    if mode == P.MODAL_F16X2:
        return 2.0 ** -20 * bnd + 2.0 ** -24 * np.abs(W).sum(axis=0)[None, :] + 1e-6
    return scale * bnd + 1e-6


@pytest.mark.parametrize("n_out", [16, 96])
@pytest.mark.parametrize("mode,scale", [(P.MODAL_BF16, 2.0 ** -7), (P.MODAL_BF16X3, 2.0 ** -18),
                                        (P.MODAL_F16X2, None)])
def test_modal_small_against_fp64(n_out, mode, scale):
    rng = np.random.default_rng(3)
    xb = rng.random((200, 3))
    S = np.sort(rng.choice(200, 70, replace=False)).astype(np.int32)   # 2 K-tiles, padded
    W = rng.standard_normal((70, n_out))
    xv = rng.random((1000, 3)) * 1.2 - 0.1                              # ragged M tile
    R = 0.8
    ref, bnd = _ref(xv, xb[S], W, R)
    d = P.deform_modal(cuda(xv), cuda(xb), cuda(S, torch.int32), cuda(W), radius=R, mode=mode)
    err = np.abs(d.cpu().numpy().astype(np.float64) - ref)
    assert np.all(np.isfinite(err))
    lim = _bound(mode, scale, bnd, W)
    assert np.all(err <= lim), (err / lim).max()


@pytest.mark.parametrize("wmag", [1e-3, 1.0, 1e5])
def test_modal_f16x2_column_scaling(wmag):
    # weights far outside the FP16 range (1e5 x N(0, 1)) and far below it:
    # each column is scaled by a power of two before the FP16 split
    rng = np.random.default_rng(9)
    xb = rng.random((200, 3))
    S = np.sort(rng.choice(200, 70, replace=False)).astype(np.int32)
    W = rng.standard_normal((70, 48)) * wmag * np.logspace(0, 3, 48)[None, :]
    xv = rng.random((3000, 3)) * 1.2 - 0.1
    ref, bnd = _ref(xv, xb[S], W, 0.8)
    d = P.deform_modal(cuda(xv), cuda(xb), cuda(S, torch.int32), cuda(W), radius=0.8,
                       mode=P.MODAL_F16X2)
    err = np.abs(d.cpu().numpy().astype(np.float64) - ref)
    assert np.all(np.isfinite(err))
    lim = 2.0 ** -20 * bnd + 2.0 ** -24 * np.abs(W).sum(axis=0)[None, :] + 1e-30
    assert np.all(err <= lim), (err / lim).max()


@pytest.mark.parametrize("mode,scale,n_out", [(P.MODAL_BF16, 2.0 ** -7, 48),
                                               (P.MODAL_BF16, 2.0 ** -7, 256),
                                               (P.MODAL_BF16X3, 2.0 ** -18, 48),
                                               (P.MODAL_BF16X3, 2.0 ** -18, 160),
                                               (P.MODAL_F16X2, None, 48),
                                               (P.MODAL_F16X2, None, 256)])
def test_modal_many_tiles_and_wide_outputs(mode, scale, n_out):
    # 40,000 points: 313 M tiles, two or three per CTA; n_out = 48 ends in a
    # 16-column tail of the second column group, 160 and 256 wrap the column
    # groups (BF16x3 buffers for 256 columns exceed shared memory: below)
    rng = np.random.default_rng(5)
    xb = rng.random((300, 3))
    S = np.sort(rng.choice(300, 150, replace=False)).astype(np.int32)   # 3 K-tiles, padded
    W = rng.standard_normal((150, n_out))
    xv = rng.random((40_000, 3)) * 1.2 - 0.1
    R = 0.6
    ref, bnd = _ref(xv, xb[S], W, R)
    d = P.deform_modal(cuda(xv), cuda(xb), cuda(S, torch.int32), cuda(W), radius=R, mode=mode)
    err = np.abs(d.cpu().numpy().astype(np.float64) - ref)
    assert np.all(np.isfinite(err))
    lim = _bound(mode, scale, bnd, W)
    assert np.all(err <= lim), (err / lim).max()


def test_modal_rejects_buffers_beyond_shared_memory():
    # BF16x3 with 256 columns: two A and two W buffers of three splits each
    # (96 KB + 192 KB) do not fit in one CTA's shared memory
    rng = np.random.default_rng(6)
    xb = rng.random((300, 3))
    S = np.arange(150, dtype=np.int32)
    with pytest.raises(P.RBFError) as e:
        P.deform_modal(cuda(rng.random((100, 3))), cuda(xb), cuda(S, torch.int32),
                       cuda(rng.standard_normal((150, 256))), radius=0.6, mode=P.MODAL_BF16X3)
    assert e.value.status == 1


def test_modal_sinusoidal_modes_full_support():
    """32 sinusoidal bending modes dz_q = 0.05 sin((2q-1) pi y / (2b)) on the
    GCB support set of the N_b = 50,000 wing; W (N_c x 96) from the FP64
    solve; sampled volume points compared with FP64 sums."""
    c = synth.wing_gcb(n_vol=200_000)
    xb, db = cuda(c["xb"]), cuda(c["db"])
    estar = oracle.tolerance(c["db"], c["tol_rel"])
    r = P.greedy_select(xb, db, radius=2.0, tol=estar, tol_mode=0, m=241, seed=1,
                        eval_prec=P.PREC_F32X2)
    S = r["idx"].cpu().numpy()
    y = c["xb"][S, 1]
    modes = np.zeros((len(S), 96))
    for q in range(1, 33):
        modes[:, 3 * (q - 1) + 2] = 0.05 * np.sin((2 * q - 1) * np.pi * y / 2.0)
    W = np.zeros_like(modes)
    for q in range(32):
        x, res = P.solve_system(xb, r["idx"], cuda(modes[:, 3 * q:3 * q + 3]), radius=2.0)
        W[:, 3 * q:3 * q + 3] = x.cpu().numpy()
    xv = c["xv"]
    sample = np.random.default_rng(8).choice(len(xv), 2000, replace=False)
    ref, bnd = _ref(xv[sample], c["xb"][S], W, 2.0)
    for mode, scale in ((P.MODAL_BF16, 2.0 ** -7), (P.MODAL_BF16X3, 2.0 ** -18),
                        (P.MODAL_F16X2, None)):
        d = P.deform_modal(cuda(xv), xb, r["idx"], cuda(W), radius=2.0, mode=mode)
        got = d.cpu().numpy()[sample].astype(np.float64)
        err = np.abs(got - ref)
        lim = _bound(mode, scale, bnd, W)
        assert np.all(err <= lim), (mode, (err / lim).max())


# ---- many fields in double-float (the accurate path for heavily cancelling
# weights): FP64-level results, bound 2^-40 sum_j |w_j phi_vj| (the derived
# double-float error is about 2^-44 of that sum) ----
@pytest.mark.parametrize("n_out", [3, 24, 96, 150])
def test_volume_fields_against_fp64(n_out):
    rng = np.random.default_rng(5)
    xb = rng.random((3000, 3))
    S = np.sort(rng.choice(3000, 1100, replace=False)).astype(np.int32)   # 35 tiles, ragged
    W = rng.standard_normal((1100, n_out)) * np.logspace(0, 4, n_out)[None, :]
    xv = rng.random((1500, 3)) * 1.2 - 0.1                               # ragged point tile
    R = 0.8
    ref, bnd = _ref(xv, xb[S], W, R)
    d = P.deform_volume_fields(cuda(xv), cuda(xb), cuda(S, torch.int32), cuda(W), radius=R)
    err = np.abs(d.cpu().numpy() - ref)
    lim = 2.0 ** -40 * bnd + 1e-300
    assert np.all(err <= lim), (err / lim).max()
    # each column agrees with the 3-column double-float volume sum
    if n_out >= 3:
        dv = P.deform_volume(cuda(xv), cuda(xb), cuda(S, torch.int32),
                             cuda(np.ascontiguousarray(W[:, :3])), radius=R,
                             eval_prec=P.PREC_F32X2).cpu().numpy()
        assert np.abs(dv - d.cpu().numpy()[:, :3]).max() <= 2.0 ** -39 * bnd[:, :3].max()


def test_volume_fields_sinusoidal_modes_full_support():
    """Configuration 4b with an accurate result: the 32 sinusoidal bending
    modes on the GCB support set of the N_b = 50,000 wing, where every
    FP32-accumulating path (tensor cores, FP32 sums) misses.  The
    double-float fields must match FP64 to 1e-5 of the largest modal
    displacement (and in fact to the double-float bound)."""
    c = synth.wing_gcb(n_vol=200_000)
    xb, db = cuda(c["xb"]), cuda(c["db"])
    estar = oracle.tolerance(c["db"], c["tol_rel"])
    r = P.greedy_select(xb, db, radius=2.0, tol=estar, tol_mode=0, m=241, seed=1,
                        eval_prec=P.PREC_F32X2)
    S = r["idx"].cpu().numpy()
    y = c["xb"][S, 1]
    modes = np.zeros((len(S), 96))
    for q in range(1, 33):
        modes[:, 3 * (q - 1) + 2] = 0.05 * np.sin((2 * q - 1) * np.pi * y / 2.0)
    W = np.zeros_like(modes)
    for q in range(32):
        x, res = P.solve_system(xb, r["idx"], cuda(modes[:, 3 * q:3 * q + 3]), radius=2.0)
        W[:, 3 * q:3 * q + 3] = x.cpu().numpy()
    xv = c["xv"]
    sample = np.random.default_rng(8).choice(len(xv), 2000, replace=False)
    ref, bnd = _ref(xv[sample], c["xb"][S], W, 2.0)
    d = P.deform_volume_fields(cuda(xv), xb, r["idx"], cuda(W), radius=2.0)
    err = np.abs(d.cpu().numpy()[sample] - ref)
    assert err.max() <= 1e-5 * 0.05, err.max()
    assert np.all(err <= 2.0 ** -40 * bnd + 1e-300), (err / (2.0 ** -40 * bnd)).max()
    print(f"\n32 modes, double-float fields: max error {err.max():.3e} "
          f"(largest sum |w phi| {bnd.max():.3e})")
