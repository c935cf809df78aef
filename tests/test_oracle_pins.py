"""Pins for the FP64 CPU oracle: each check ties the oracle to something other
than itself (closed forms, published generator outputs, library routines on
special cases, brute force on tiny inputs, invariants the paper states).

CPU only.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2004_04817_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- Eq. 2 -----
def test_phi_closed_form_values():
    """Eq. 2 at dyadic points (exact hand-worked values)."""
    for eta, val in _load_golden("wendland_c2_values.txt"):
        assert oracle.phi(float(eta)) == float(val)


def test_phi_matches_wendland_integral_construction():
    """Wendland's C2 function is 20 x the integral over [eta, 1] of t (1-t)^3
    (the dimension-walk operator applied to the truncated power (1-t)^3_+).
    This definition shares nothing with the polynomial in the oracle."""
    for eta in np.linspace(0.0, 1.0, 37):
        ref, _ = integrate.quad(lambda t: t * (1.0 - t) ** 3, eta, 1.0,
                                epsabs=1e-15, epsrel=1e-14)
        assert abs(oracle.phi(eta) - 20.0 * ref) < 1e-14


def test_phi_c2_at_both_ends():
    """phi'(0) = 0 (smooth at the centre) and phi, phi', phi'' vanish at 1."""
    h = 1e-4
    f = lambda e: float(oracle.phi(e))
    # phi(eta) = 1 - 10 eta^2 + O(eta^3): no linear term at the centre
    assert abs((f(h) - f(0.0)) / h) < 20 * h
    assert abs((f(1 + h) - f(1 - h)) / (2 * h)) < 1e-10
    d2 = (f(1 + h) - 2 * f(1.0) + f(1 - h)) / h**2
    assert abs(d2) < 1e-6


def test_phi_matrix_is_positive_definite():
    """Wendland C2 is positive definite in 3-D (the paper relies on it to use
    Cholesky), so Phi on distinct points has positive eigenvalues and the
    oracle's Cholesky succeeds with positive pivots."""
    x = synth.random_cloud(60, seed=11)
    for R in (0.3, 1.0, 3.0):
        D = np.linalg.norm(x[:, None] - x[None], axis=-1)
        P = oracle.phi(D / R)
        assert np.linalg.eigvalsh(P).min() > 0
        A = P.copy()
        st = oracle.lib().orc_cholesky(len(x), A.ctypes.data_as(
            __import__("ctypes").POINTER(__import__("ctypes").c_double)))
        assert st == oracle.OK
        Lc = np.tril(A)
        assert np.allclose(Lc, np.linalg.cholesky(P), atol=1e-13)


# ----------------------------------------------------------- partition ------
def test_splitmix64_published_outputs():
    want = [int(r[0]) for r in _load_golden("splitmix64_seed1234567.txt")]
    assert oracle.splitmix64(1234567, 5) == want


@pytest.mark.parametrize("nb,m", [(10, 1), (10, 3), (101, 7), (2000, 13), (50, 50)])
def test_partition_invariants(nb, m):
    """Groups are disjoint, cover all nodes and differ in size by <= 1."""
    perm = oracle.permutation(nb, 5)
    assert sorted(perm.tolist()) == list(range(nb))
    g = oracle.groups(nb, m, 5)
    sizes = np.bincount(g, minlength=m)
    assert sizes.sum() == nb and len(sizes) == m
    assert sizes.max() - sizes.min() <= 1
    assert g.min() >= 0 and g.max() < m


def test_fisher_yates_is_uniform():
    """All 24 permutations of 4 items appear with equal frequency over many
    seeds (a Sattolo-style off-by-one would produce only the 6 cycles)."""
    counts = {}
    n_seeds = 24000
    for s in range(n_seeds):
        p = tuple(oracle.permutation(4, s).tolist())
        counts[p] = counts.get(p, 0) + 1
    assert len(counts) == 24
    exp = n_seeds / 24
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 60.0          # 23 dof: p ~ 5e-5 at 60


def test_partition_matches_fisher_yates_by_hand():
    """Replays the Fisher-Yates shuffle on the published SplitMix64 stream."""
    nb = 5
    vals = [int(r[0]) for r in _load_golden("splitmix64_seed1234567.txt")]
    perm = list(range(nb))
    for step, i in enumerate(range(nb - 1, 0, -1)):
        j = vals[step] % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    assert oracle.permutation(nb, 1234567).tolist() == perm


# ------------------------------------------------------------ seed nodes ----
def test_seed_nodes_brute_force():
    for seed in range(5):
        x = synth.random_cloud(40, seed=seed)
        d = synth.random_field(40, seed=seed + 100)
        n0 = max(range(40), key=lambda j: (np.dot(d[j], d[j]), -j))
        n1 = max(range(40), key=lambda j: (np.sum((x[j] - x[n0]) ** 2), -j))
        n2 = max(range(40), key=lambda j: (min(np.sum((x[j] - x[n0]) ** 2),
                                              np.sum((x[j] - x[n1]) ** 2)), -j))
        assert oracle.seed_nodes(x, d).tolist() == [n0, n1, n2]


# --------------------------------------------------------------- solve ------
def test_single_and_two_node_weights_closed_form():
    x = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])
    d = np.array([[1.0, -2.0, 0.5], [0.25, 0.0, -1.0]])
    W, st, _ = oracle.solve_weights(x, d, [0], 1.0)
    assert st == oracle.OK and np.array_equal(W[0], d[0])     # phi(0) = 1
    p = float(oracle.phi(0.5))                                 # |x1 - x0| = 0.5
    W, st, _ = oracle.solve_weights(x, d, [0, 1], 1.0)
    det = 1.0 - p * p
    w0 = (d[0] - p * d[1]) / det
    w1 = (d[1] - p * d[0]) / det
    assert np.allclose(W, np.stack([w0, w1]), rtol=0, atol=1e-15)


def test_solve_matches_numpy_and_reproduces():
    c = synth.tiny_wing(n_span=6, n_chord=24)
    xb, db = c["xb"], c["db"]
    rng = np.random.default_rng(3)
    S = rng.choice(len(xb), 40, replace=False).astype(np.int32)
    W, st, mp = oracle.solve_weights(xb, db, S, c["radius"])
    assert st == oracle.OK and mp > 0
    P = oracle.phi(np.linalg.norm(xb[S][:, None] - xb[S][None], axis=-1) / c["radius"])
    Wn = np.linalg.solve(P, db[S])
    scale = np.abs(Wn).max()
    assert np.abs(W - Wn).max() <= 1e-6 * scale
    F = oracle.rbf_sum(xb[S], xb, S, W, c["radius"])
    assert np.abs(F - db[S]).max() <= 1e-10 * np.abs(db).max()


def test_duplicate_points_are_not_spd():
    x = np.array([[0.0, 0, 0], [1.0, 0, 0], [1.0, 0, 0]])
    d = np.ones((3, 3))
    _, st, _ = oracle.solve_weights(x, d, [0, 1, 2], 2.0)
    assert st == oracle.E_NOT_SPD


# ------------------------------------------------------- Eq. 1 / Eq. 6 ------
def test_rbf_sum_brute_force_and_compact_support():
    rng = np.random.default_rng(7)
    xb = rng.random((30, 3))
    S = np.arange(0, 30, 2).astype(np.int32)
    W = rng.standard_normal((len(S), 3))
    xq = np.concatenate([rng.random((25, 3)), np.array([[5.0, 5.0, 5.0]])])
    R = 0.7
    F = oracle.rbf_sum(xq, xb, S, W, R)
    ref = np.zeros((len(xq), 3))
    for q in range(len(xq)):
        for t, j in enumerate(S):
            eta = math.dist(xq[q], xb[j]) / R
            if eta < 1:
                ref[q] += W[t] * (1 - eta) ** 4 * (4 * eta + 1)
    assert np.abs(F - ref).max() < 1e-13
    assert np.all(F[-1] == 0.0)            # farther than R from every centre


# -------------------------------------------------------------- greedy ------
def _np_greedy(xb, db, R, Estar, m, seed, ncmax=10**9):
    """Independent brute force of Algorithm 1 (numpy.linalg.solve every step,
    errors at the active group, lowest index on ties, strict E > E*, stop
    after m consecutive iterations without an append)."""
    nb = len(xb)
    grp = oracle.groups(nb, m, seed)
    S = [int(v) for v in oracle.seed_nodes(xb, db)]
    iters = [-1, -1, -1]
    D = np.linalg.norm(xb[:, None] - xb[None], axis=-1)
    Phi = oracle.phi(D / R)
    k = 3
    idle = 0
    while True:
        W = np.linalg.solve(Phi[np.ix_(S, S)], db[S])
        G = np.flatnonzero(grp == (k % m))
        G = np.array([q for q in G if q not in S], dtype=int)
        add = -1
        if len(G):
            E = np.linalg.norm(db[G] - Phi[np.ix_(G, S)] @ W, axis=1)
            t = int(np.argmax(E))               # first occurrence = lowest index
            if E[t] > Estar:
                add = int(G[t])
        if add >= 0:
            assert len(S) < ncmax
            S.append(add)
            iters.append(k)
            idle = 0
        else:
            idle += 1
        if idle >= m:
            Eall = np.linalg.norm(db - Phi[:, S] @ W, axis=1)
            assert Eall.max() <= Estar
            return np.array(S), np.array(iters), Eall.max()
        k += 1


@pytest.mark.parametrize("m", [1, 2, 5, 9])
def test_greedy_matches_brute_force(m):
    c = synth.tiny_wing(n_span=6, n_chord=30, radius=1.0)     # N_b = 180
    xb, db = c["xb"], c["db"]
    Estar = oracle.tolerance(db, 2e-3)
    S, it, gmax = _np_greedy(xb, db, c["radius"], Estar, m, seed=1)
    r = oracle.greedy(xb, db, c["radius"], Estar, m=m, seed=1)
    assert r["status"] == oracle.OK
    assert r["idx"].tolist() == S.tolist()
    assert r["iter"].tolist() == it.tolist()
    assert r["stats"]["final_max"] <= Estar
    assert abs(r["stats"]["final_max"] - gmax) < 1e-12
    # the history's all-node check after every m-th iteration (diagnostic)
    h = r["hist"]
    assert np.all((h[:, 3] < 0) | ((h[:, 0] - 2) % m == 0))


def test_gcb_m1_is_plain_greedy_and_seed_independent():
    """With m = 1 every iteration sees all nodes: the result cannot depend on
    the grouping seed (Sec. 4: GCB with m = 1 is the plain greedy)."""
    c = synth.tiny_wing(n_span=5, n_chord=36, radius=2.0)
    Estar = oracle.tolerance(c["db"], 1e-3)
    a = oracle.greedy(c["xb"], c["db"], 2.0, Estar, m=1, seed=1)
    b = oracle.greedy(c["xb"], c["db"], 2.0, Estar, m=1, seed=987654321)
    assert a["idx"].tolist() == b["idx"].tolist()
    # m = 1: every iteration adds a node except the last one, which finds
    # every error <= E*
    assert a["stats"]["iterations"] == a["nc"] - 3 + 1


def test_greedy_reproduction_and_pair_count():
    c = synth.tiny_wing(n_span=8, n_chord=25, radius=2.0)
    xb, db, R = c["xb"], c["db"], c["radius"]
    Estar = oracle.tolerance(db, 1e-3)
    m = 4
    r = oracle.greedy(xb, db, R, Estar, m=m, seed=3)
    S = r["idx"]
    W, st, _ = oracle.solve_weights(xb, db, S, R)
    F = oracle.rbf_sum(xb, xb, S, W, R)
    assert np.abs(F[S] - db[S]).max() <= 1e-10 * np.abs(db).max()
    assert np.linalg.norm(F - db, axis=1).max() <= Estar
    # Sec. 3 work count: sum over iterations of |G_i| * |S|
    g = np.bincount(oracle.groups(len(xb), m, 3), minlength=m)
    h = r["hist"]
    want = int(sum(g[int(k) % m] * int(n) for k, n in zip(h[:, 0], h[:, 1])))
    assert r["stats"]["pairs_group"] == want


def test_greedy_visits_every_group_once_per_cycle():
    c = synth.tiny_wing(n_span=6, n_chord=30, radius=1.0)
    Estar = oracle.tolerance(c["db"], 1e-3)
    m = 5
    r = oracle.greedy(c["xb"], c["db"], 1.0, Estar, m=m, seed=2)
    ks = r["hist"][:, 0].astype(int)
    assert ks.tolist() == list(range(3, 3 + len(ks)))
    for start in range(0, len(ks) - m + 1):
        assert sorted(ks[start:start + m] % m) == list(range(m))


def test_follow_mode_accepts_own_sequence_and_flags_a_planted_error():
    c = synth.tiny_wing(n_span=6, n_chord=30, radius=1.0)
    xb, db = c["xb"], c["db"]
    Estar = oracle.tolerance(db, 1e-3)
    r = oracle.greedy(xb, db, 1.0, Estar, m=3, seed=4)
    f = oracle.greedy(xb, db, 1.0, Estar, m=3, seed=4, follow=(r["idx"], r["iter"]))
    assert f["stats"]["n_fail"] == 0 and f["stats"]["n_div"] == 0
    assert f["idx"].tolist() == r["idx"].tolist()
    # planted mistake: replace the 6th added node by a node of the same group
    # that is not the maximiser
    bad = r["idx"].copy()
    grp = oracle.groups(len(xb), 3, 4)
    g = grp[bad[5]]
    alt = [q for q in np.flatnonzero(grp == g) if q not in bad][0]
    bad[5] = alt
    f = oracle.greedy(xb, db, 1.0, Estar, m=3, seed=4, follow=(bad, r["iter"]))
    assert f["stats"]["n_fail"] >= 1


def test_nc_max_cap():
    c = synth.tiny_wing(n_span=6, n_chord=30, radius=1.0)
    Estar = oracle.tolerance(c["db"], 1e-5)
    r = oracle.greedy(c["xb"], c["db"], 1.0, Estar, m=1, seed=1, ncmax=10)
    assert r["status"] == oracle.E_NC_MAX and r["nc"] == 10


# ------------------------------------------------------------- adjoint ------
def test_adjoint_matches_central_differences():
    """J(d_c) = sum_v 1/2 |Phi_vc Phi_cc^-1 d_c - t_v|^2 is quadratic, so the
    central difference is exact up to rounding."""
    rng = np.random.default_rng(9)
    xb = rng.random((25, 3))
    S = np.arange(0, 25, 3).astype(np.int32)
    xv = rng.random((60, 3)) * 1.2 - 0.1
    R = 0.8
    dc = rng.standard_normal((len(S), 3)) * 0.1
    t = rng.standard_normal((60, 3)) * 0.01
    Pcc = oracle.phi(np.linalg.norm(xb[S][:, None] - xb[S][None], axis=-1) / R)
    Pvc = oracle.phi(np.linalg.norm(xv[:, None] - xb[S][None], axis=-1) / R)

    def J(d):
        dv = Pvc @ np.linalg.solve(Pcc, d)
        return 0.5 * np.sum((dv - t) ** 2)

    dv = Pvc @ np.linalg.solve(Pcc, dc)
    g, st = oracle.adjoint(xv, xb, S, R, dv - t)
    assert st == oracle.OK
    h = 1e-6
    for a in range(len(S)):
        for comp in range(3):
            e = np.zeros_like(dc)
            e[a, comp] = h
            fd = (J(dc + e) - J(dc - e)) / (2 * h)
            assert abs(fd - g[a, comp]) <= 1e-6 * max(1.0, abs(g).max())


# --------------------------------------------------------------------------
# KL divergence of two support sets (Sec. 4.1)
# --------------------------------------------------------------------------
def test_kl_hand_example_on_a_line():
    # nodes at x = 0, 1, 2, 3; S1 = {0}, S2 = {3}: d1 = (0, 1, 2, 3),
    # d2 = (3, 2, 1, 0).  Node 0 (d1 = 0) and node 3 (d2 = 0) drop out, so
    # KL = 1 log(1/2) + 2 log(2/1) = log 2.
    xb = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0], [3.0, 0, 0]])
    assert np.array_equal(oracle.nearest_support(xb, [0]), [0.0, 1.0, 2.0, 3.0])
    assert oracle.support_kl(xb, [0], [3]) == pytest.approx(math.log(2.0), rel=1e-15)
    # reversed: 2 log(2/1) + 1 log(1/2) = log 2 as well (the line is symmetric)
    assert oracle.support_kl(xb, [3], [0]) == pytest.approx(math.log(2.0), rel=1e-15)


def test_kl_of_a_set_with_itself_is_zero_and_scales_with_length():
    rng = np.random.default_rng(5)
    xb = synth.random_cloud(400, seed=3)
    S1 = np.sort(rng.choice(400, 30, replace=False))
    S2 = np.sort(rng.choice(400, 30, replace=False))
    assert oracle.support_kl(xb, S1, S1) == 0.0
    kl = oracle.support_kl(xb, S1, S2)
    # distances scale with the coordinates, their ratios do not
    assert oracle.support_kl(2.5 * xb, S1, S2) == pytest.approx(2.5 * kl, rel=1e-12)


def test_nearest_support_matches_kdtree():
    from scipy.spatial import cKDTree
    xb = synth.random_cloud(3000, seed=9)
    S = np.sort(np.random.default_rng(2).choice(3000, 70, replace=False))
    d_ref, _ = cKDTree(xb[S]).query(xb)
    assert np.allclose(oracle.nearest_support(xb, S), d_ref, rtol=1e-14, atol=0)


def test_follow_mode_ends_at_the_capacity_of_the_followed_run():
    # N_c^max caps |S| (Alg. 1's loop bound): a run stopped by the capacity,
    # followed by the oracle with the same capacity, ends at the same
    # iteration with the same status and no rejected step
    c = synth.tiny_wing(n_span=6, n_chord=30, radius=1.0)
    for m in (1, 4):
        r = oracle.greedy(c["xb"], c["db"], c["radius"], 0.0, m=m, seed=1, ncmax=40,
                          history=False)
        assert r["status"] == oracle.E_NC_MAX and r["nc"] == 40
        f = oracle.greedy(c["xb"], c["db"], c["radius"], 0.0, m=m, seed=1, ncmax=40,
                          follow=(r["idx"], r["iter"]), history=False)
        assert f["status"] == oracle.E_NC_MAX and f["nc"] == 40
        assert f["stats"]["n_fail"] == 0 and f["stats"]["n_div"] == 0
        assert f["stats"]["iterations"] == r["stats"]["iterations"]


# --------------------------------------------------------------------------
# Peak-selection variant (several separated error peaks per iteration)
# --------------------------------------------------------------------------
def _peaks_reference(xb, db, R, Estar, m, peaks, sep):
    """The peak-selection reading written independently with numpy: dense
    solve per iteration, errors of the active group, separated peaks in
    decreasing error (lowest index on ties).  Partition and seed nodes come
    from the oracle routines pinned above."""
    nb = len(xb)
    grp = oracle.groups(nb, m, 1)
    S = list(oracle.seed_nodes(xb, db))
    it = [-1, -1, -1]
    idle, k = 0, 3
    phi = lambda d: np.where(d < 1.0, (1.0 - d) ** 4 * (4.0 * d + 1.0), 0.0)
    while True:
        A = phi(np.linalg.norm(xb[S][:, None] - xb[S][None], axis=-1) / R)
        W = np.linalg.solve(A, db[S])
        members = np.flatnonzero(grp == k % m)
        members = members[~np.isin(members, S)]
        F = phi(np.linalg.norm(xb[members][:, None] - xb[S][None], axis=-1) / R) @ W
        E = np.linalg.norm(db[members] - F, axis=1)
        order = sorted(range(len(members)), key=lambda t: (-E[t], members[t]))
        taken = []
        for t in order:
            if len(taken) == peaks or not E[t] > Estar:
                break
            if all(np.linalg.norm(xb[members[t]] - xb[u]) >= sep for u in taken):
                taken.append(members[t])
        if not taken:
            idle += 1
            if idle >= m:
                return np.array(S), np.array(it), k - 3 + 1
        else:
            idle = 0
            S += taken
            it += [k] * len(taken)
        k += 1


@pytest.mark.parametrize("m,peaks,sep", [(1, 3, 0.3), (3, 4, 0.25), (5, 2, 0.0)])
def test_peaks_oracle_matches_independent_reference(m, peaks, sep):
    c = synth.tiny_wing(n_span=5, n_chord=24, radius=1.0)
    estar = oracle.tolerance(c["db"], 3e-3)
    r = oracle.greedy_peaks(c["xb"], c["db"], c["radius"], estar, m=m, peaks=peaks, sep=sep)
    S, it, iters = _peaks_reference(c["xb"], c["db"], c["radius"], estar, m, peaks, sep)
    assert r["status"] == oracle.OK
    assert r["idx"].tolist() == S.tolist()
    assert r["iter"].tolist() == it.tolist()
    assert r["iterations"] == iters


def test_peaks_one_is_algorithm_1():
    c = synth.tiny_wing(n_span=6, n_chord=30, radius=1.0)
    estar = oracle.tolerance(c["db"], 2e-3)
    for m in (1, 4):
        a = oracle.greedy(c["xb"], c["db"], c["radius"], estar, m=m, history=False)
        b = oracle.greedy_peaks(c["xb"], c["db"], c["radius"], estar, m=m, peaks=1, sep=0.0)
        assert a["idx"].tolist() == b["idx"].tolist()
        assert a["iter"].tolist() == b["iter"].tolist()
        assert a["stats"]["iterations"] == b["iterations"]


def test_argmax_resolves_a_difference_of_2_pow_35_and_exact_ties_by_index():
    """Alg. 1 picks the node of largest error, the lowest index among equal
    errors.  On the near-tie line the fourth pick is the node whose error is
    t (1 + 2^-35) (every other free node far from the seeds has exactly t);
    the picks after it are exact ties, taken in ascending index, skipping the
    neighbours of each pick (their error drops below t)."""
    c = synth.line_near_tie()
    r = oracle.greedy(c["xb"], c["db"], c["radius"], 0.5 * c["t"], m=1, seed=1, ncmax=8)
    n = len(c["xb"])
    # seeds: largest displacement; farthest from it; farthest from both
    # (nodes 36 and 37 are 26 from the nearer seed: the lower index wins)
    assert r["idx"][:3].tolist() == [c["big"], n - 1, 36]
    assert r["idx"][3] == c["near"]
    assert r["idx"][4:8].tolist() == [0, 2, 4, 6]


# The follow mode's acceptance band.  The comparison rule lets the GPU's
# sequence leave the oracle's only where the two values that decide a step
# (the two largest errors of the active group for the argmax, or the group
# maximum and E* for the E > E* test of Alg. 1) agree to 1e-6 relative, and
# every such step is logged.  On the near-tie line every free node far from
# the seeds keeps exactly its own displacement as its error, so the deciding
# gaps below are set by the displacements alone.  A band read 1000x too wide,
# or too narrow, or with the wrong sign, fails one side of each pair.
BAND = 1e-6


@pytest.mark.parametrize("gap,accepted", [(0.5e-6, True), (0.9e-6, True),
                                          (1.1e-6, False), (2e-6, False)])
def test_follow_band_on_the_argmax(gap, accepted):
    """The followed run appends node 0 (error t) while node `near` has the
    group's largest error t (1 + gap), then `near`, then the exact ties."""
    c = synth.line_near_tie(rel=gap)
    estar = 0.5 * c["t"]
    r = oracle.greedy(c["xb"], c["db"], c["radius"], estar, m=1, seed=1, ncmax=8)
    assert r["idx"].tolist() == [c["big"], 63, 36, c["near"], 0, 2, 4, 6]
    seq = np.array([c["big"], 63, 36, 0, c["near"], 2, 4, 6], dtype=np.int32)
    f = oracle.greedy(c["xb"], c["db"], c["radius"], estar, m=1, seed=1, ncmax=8,
                      follow=(seq, r["iter"]), tie_rel=BAND)
    s = f["stats"]
    assert f["idx"].tolist() == seq.tolist()
    assert s["worst_rel_gap"] == pytest.approx(gap / (1.0 + gap), rel=1e-9)
    if accepted:
        assert (s["n_fail"], s["n_div"]) == (0, 1)
    else:
        assert (s["n_fail"], s["n_div"]) == (1, 0)


@pytest.mark.parametrize("gap,accepted", [(0.5e-6, True), (0.9e-6, True),
                                          (1.1e-6, False), (2e-6, False)])
def test_follow_band_on_a_missing_append(gap, accepted):
    """E* = t (1 - gap): the literal run keeps appending nodes of error t;
    the followed run stops after its fourth node although the group's
    maximum t lies above E* by the relative gap."""
    c = synth.line_near_tie()
    estar = c["t"] * (1.0 - gap)
    r = oracle.greedy(c["xb"], c["db"], c["radius"], estar, m=1, seed=1)
    assert r["nc"] > 8
    f = oracle.greedy(c["xb"], c["db"], c["radius"], estar, m=1, seed=1,
                      follow=(r["idx"][:4], r["iter"][:4]), tie_rel=BAND)
    s = f["stats"]
    assert f["nc"] == 4
    assert s["worst_rel_gap"] == pytest.approx((c["t"] - estar) / estar, rel=1e-6)
    if accepted:
        assert (s["n_fail"], s["n_div"]) == (0, 1)
    else:
        assert (s["n_fail"], s["n_div"]) == (1, 0)


@pytest.mark.parametrize("gap,accepted", [(0.5e-6, True), (0.9e-6, True),
                                          (1.1e-6, False), (2e-6, False)])
def test_follow_band_on_an_append_at_or_below_estar(gap, accepted):
    """E* = t (1 + gap): the literal run appends nothing after the seeds; the
    followed run appends `near` (error t (1 + 2^-35), the group's maximum),
    which lies below E* by about the relative gap."""
    c = synth.line_near_tie()
    estar = c["t"] * (1.0 + gap)
    lit = oracle.greedy(c["xb"], c["db"], c["radius"], estar, m=1, seed=1)
    assert lit["nc"] == 3
    seq = np.array([c["big"], 63, 36, c["near"]], dtype=np.int32)
    f = oracle.greedy(c["xb"], c["db"], c["radius"], estar, m=1, seed=1,
                      follow=(seq, np.array([-1, -1, -1, 3])), tie_rel=BAND)
    s = f["stats"]
    e_near = c["db"][c["near"], 0]
    assert s["worst_rel_gap"] == pytest.approx((estar - e_near) / estar, rel=1e-6)
    if accepted:
        assert (s["n_fail"], s["n_div"]) == (0, 1)
    else:
        assert (s["n_fail"], s["n_div"]) == (1, 0)


@pytest.mark.parametrize("m", [1, 5])
def test_recurrence_cholesky_greedy_selects_the_literal_sequence(m):
    """The fair CPU baseline (Alg. 1 with the recurrence-Cholesky append of
    Sec. 1) must select exactly the nodes, at exactly the iterations, of the
    literal oracle (dense re-solve every iteration), stop at the same
    iteration with the same final maximum to rounding, and give weights that
    reproduce the displacements at the support nodes."""
    for c in (synth.tiny_wing(n_span=6, n_chord=30, radius=1.0),
              synth.tiny_wing(n_span=8, n_chord=25, radius=2.0)):
        estar = oracle.tolerance(c["db"], 2e-3)
        a = oracle.greedy(c["xb"], c["db"], c["radius"], estar, m=m, seed=3, history=False)
        b = oracle.greedy_rc(c["xb"], c["db"], c["radius"], estar, m=m, seed=3)
        assert a["status"] == b["status"] == 0
        assert b["idx"].tolist() == a["idx"].tolist()
        assert b["iter"].tolist() == a["iter"].tolist()
        assert b["iterations"] == a["stats"]["iterations"]
        assert abs(b["final_max"] - a["stats"]["final_max"]) <= 1e-12
        assert b["final_max"] <= estar
        W, st, _ = oracle.solve_weights(c["xb"], c["db"], a["idx"], c["radius"])
        assert np.abs(b["w"] - W).max() <= 1e-9 * np.abs(W).max()
        F = oracle.rbf_sum(c["xb"][b["idx"]], c["xb"], b["idx"], b["w"], c["radius"])
        assert np.abs(F - c["db"][b["idx"]]).max() <= 1e-10 * np.abs(c["db"]).max()


def test_recurrence_cholesky_greedy_reports_a_singular_append():
    """Two coincident boundary nodes make Phi_SS singular (Sec. 2): with
    tolerance 0 the greedy must eventually try to append the duplicate, and
    the RC pivot d^2 = phi(0) - l.l vanishes there."""
    c = synth.tiny_wing(n_span=4, n_chord=12, radius=1.0)
    xb = np.vstack([c["xb"], c["xb"][5:6]])
    db = np.vstack([c["db"], c["db"][5:6] + 1e-3])
    b = oracle.greedy_rc(xb, db, 1.0, 0.0, m=1, seed=1)
    assert b["status"] == oracle.E_NOT_SPD
