"""FP64 CPU oracle for GCB-greedy RBF mesh deformation (test infrastructure).

This package is TEST INFRASTRUCTURE: a plain, slow, obviously correct CPU
restatement of the paper's method (Eqs. 1-6 and Algorithm 1) in double
precision.  Only the test-suite, the smoke check and the benchmark's
CPU-baseline leg use it; the library never does, and the two share no code.

The arithmetic lives in ``rbf_oracle.c`` (plain C, compiled by ``build.py``
with gcc, FMA contraction off so that x86 and Arm give identical bits).  This
module only marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

OK, E_ARG, E_NOT_SPD, E_NC_MAX, E_NOMEM = 0, 1, 2, 3, 5
HIST_COLS = 6


class GreedyStats(C.Structure):
    _fields_ = [
        ("iterations", C.c_int64),
        ("full_checks", C.c_int64),
        ("pairs_group", C.c_int64),
        ("pairs_full", C.c_int64),
        ("final_max", C.c_double),
        ("final_rms", C.c_double),
        ("min_pivot", C.c_double),
        ("n_div", C.c_int64),
        ("n_fail", C.c_int64),
        ("worst_rel_gap", C.c_double),
    ]


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        lp = C.POINTER(C.c_int64)
        L.orc_phi.restype = C.c_double
        L.orc_phi.argtypes = [C.c_double]
        L.orc_splitmix64_next.restype = C.c_uint64
        L.orc_splitmix64_next.argtypes = [C.POINTER(C.c_uint64)]
        L.orc_permutation.argtypes = [C.c_int64, C.c_uint64, ip]
        L.orc_groups.argtypes = [C.c_int64, C.c_int64, C.c_uint64, ip]
        L.orc_seed_nodes.argtypes = [dp, dp, C.c_int64, ip]
        L.orc_cholesky.restype = C.c_int
        L.orc_cholesky.argtypes = [C.c_int64, dp]
        L.orc_solve_weights.restype = C.c_int
        L.orc_solve_weights.argtypes = [dp, dp, ip, C.c_int64, C.c_double, dp, dp]
        L.orc_rbf_sum.argtypes = [dp, C.c_int64, dp, ip, C.c_int64, dp, C.c_double, dp,
                                  C.c_int]
        L.orc_greedy.restype = C.c_int
        L.orc_greedy.argtypes = [dp, dp, C.c_int64, C.c_double, C.c_double, C.c_int64,
                                 C.c_uint64, C.c_int64, ip, lp, C.c_int64, C.c_double,
                                 ip, lp, lp, dp, C.c_int64, lp, C.POINTER(GreedyStats),
                                 C.c_int]
        L.orc_adjoint.restype = C.c_int
        L.orc_adjoint.argtypes = [dp, C.c_int64, dp, ip, C.c_int64, C.c_double, dp, dp,
                                  C.c_int]
        L.orc_num_threads.restype = C.c_int
        L.orc_nearest_support.argtypes = [dp, C.c_int64, ip, C.c_int64, dp, C.c_int]
        L.orc_greedy_peaks.restype = C.c_int
        L.orc_greedy_peaks.argtypes = [dp, dp, C.c_int64, C.c_double, C.c_double, C.c_int64,
                                       C.c_uint64, C.c_int64, C.c_int64, C.c_double, ip,
                                       C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                       C.POINTER(C.c_int64), C.c_int]
        L.orc_greedy_rc.restype = C.c_int
        L.orc_greedy_rc.argtypes = [dp, dp, C.c_int64, C.c_double, C.c_double, C.c_int64,
                                    C.c_uint64, C.c_int64, ip, C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_double), dp, C.c_int]
        L.orc_support_kl.restype = C.c_int
        L.orc_support_kl.argtypes = [dp, C.c_int64, ip, C.c_int64, ip, C.c_int64,
                                     C.POINTER(C.c_double), C.c_int]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(C.POINTER(C.c_int64))


def default_threads():
    return int(os.environ.get("RBF_ORACLE_THREADS", os.cpu_count() or 1))


# --------------------------------------------------------------------------
def phi(eta):
    """Wendland C2 basis (Eq. 2), elementwise."""
    L = lib()
    e = np.asarray(eta, dtype=np.float64)
    return np.vectorize(L.orc_phi, otypes=[np.float64])(e)


def splitmix64(seed, n):
    """First n outputs of the SplitMix64 stream started at ``seed``."""
    L = lib()
    st = C.c_uint64(seed)
    return [L.orc_splitmix64_next(C.byref(st)) for _ in range(n)]


def permutation(nb, seed):
    L = lib()
    perm = np.empty(nb, dtype=np.int32)
    L.orc_permutation(nb, seed, perm.ctypes.data_as(C.POINTER(C.c_int32)))
    return perm


def groups(nb, m, seed):
    """group_of[node] for the random uniform partition into m groups."""
    L = lib()
    g = np.empty(nb, dtype=np.int32)
    L.orc_groups(nb, m, seed, g.ctypes.data_as(C.POINTER(C.c_int32)))
    return g


def seed_nodes(xb, db):
    L = lib()
    xb, px = _d(xb)
    db, pd = _d(db)
    out = np.empty(3, dtype=np.int32)
    L.orc_seed_nodes(px, pd, len(xb), out.ctypes.data_as(C.POINTER(C.c_int32)))
    return out


def solve_weights(xb, db, S, R):
    """W (k, 3) with Phi_SS W = dX_S; returns (W, status, min_pivot)."""
    L = lib()
    xb, px = _d(xb)
    db, pd = _d(db)
    S, ps = _i32(S)
    W = np.zeros((len(S), 3))
    mp = C.c_double(0.0)
    st = L.orc_solve_weights(px, pd, ps, len(S), R, W.ctypes.data_as(C.POINTER(C.c_double)),
                             C.byref(mp))
    return W, st, mp.value


def rbf_sum(xq, xb, S, W, R, threads=None):
    """F at the query points (Eq. 1 / Eq. 6), shape (nq, 3)."""
    L = lib()
    xq, pq = _d(np.asarray(xq).reshape(-1, 3))
    xb, px = _d(xb)
    S, ps = _i32(S)
    W, pw = _d(W)
    out = np.zeros((len(xq), 3))
    L.orc_rbf_sum(pq, len(xq), px, ps, len(S), pw, R,
                  out.ctypes.data_as(C.POINTER(C.c_double)),
                  threads or default_threads())
    return out


def greedy(xb, db, R, Estar, m=1, seed=1, ncmax=None, follow=None, tie_rel=1e-6,
           threads=None, history=True, hist_cap=None):
    """Algorithm 1.  ``follow`` = (idx, iter) of another run to check.

    ``history`` records one row per iteration, with the all-node maximum and
    RMS error after every m-th iteration (extra all-node evaluations that do
    not change the selection).  Returns dict(status, idx, iter, nc, hist,
    stats).
    """
    L = lib()
    xb, px = _d(xb)
    db, pd = _d(db)
    nb = len(xb)
    ncmax = int(ncmax or nb)
    if follow is not None:
        fidx, pfi = _i32(follow[0])
        fit, pft = _i64(follow[1])
        fn = len(fidx)
    else:
        fidx, pfi = _i32(np.zeros(1))
        fit, pft = _i64(np.zeros(1))
        fn = -1
    out_idx = np.zeros(ncmax, dtype=np.int32)
    out_it = np.zeros(ncmax, dtype=np.int64)
    nc = C.c_int64(0)
    hist_cap = int(hist_cap or (4 * nb + 16)) if history else 0
    hist = np.zeros((max(hist_cap, 1), HIST_COLS))
    nh = C.c_int64(0)
    stats = GreedyStats()
    st = L.orc_greedy(px, pd, nb, float(R), float(Estar), int(m), int(seed), ncmax,
                      pfi, pft, fn, float(tie_rel),
                      out_idx.ctypes.data_as(C.POINTER(C.c_int32)),
                      out_it.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(nc),
                      hist.ctypes.data_as(C.POINTER(C.c_double)) if history else None,
                      hist_cap, C.byref(nh),
                      C.byref(stats), threads or default_threads())
    n = nc.value
    return dict(status=st, idx=out_idx[:n].copy(), iter=out_it[:n].copy(), nc=n,
                hist=hist[:min(nh.value, hist_cap)].copy() if history else None,
                stats={f: getattr(stats, f) for f, _ in GreedyStats._fields_})


def adjoint(xv, xb, S, R, gv, threads=None):
    """dJ/dd_c = Phi_cc^{-1} Phi_vc^T gv (support components), shape (k, 3)."""
    L = lib()
    xv, pv = _d(np.asarray(xv).reshape(-1, 3))
    xb, px = _d(xb)
    S, ps = _i32(S)
    gv, pg = _d(np.asarray(gv).reshape(-1, 3))
    gc = np.zeros((len(S), 3))
    st = L.orc_adjoint(pv, len(xv), px, ps, len(S), float(R), pg,
                       gc.ctypes.data_as(C.POINTER(C.c_double)), threads or default_threads())
    return gc, st


def greedy_peaks(xb, db, R, Estar, m=1, seed=1, ncmax=None, peaks=1, sep=0.0, threads=None):
    """Peak-selection variant: up to ``peaks`` separated nodes (at least ``sep``
    apart) appended per iteration.  Returns dict(status, idx, iter, nc,
    iterations)."""
    L = lib()
    xb, px = _d(xb)
    db, pd = _d(db)
    nb = len(xb)
    ncmax = int(ncmax or nb)
    out_idx = np.zeros(ncmax, dtype=np.int32)
    out_it = np.zeros(ncmax, dtype=np.int64)
    nc = C.c_int64(0)
    its = C.c_int64(0)
    st = L.orc_greedy_peaks(px, pd, nb, float(R), float(Estar), int(m), int(seed), ncmax,
                            int(peaks), float(sep), out_idx.ctypes.data_as(C.POINTER(C.c_int32)),
                            out_it.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(nc),
                            C.byref(its), threads or default_threads())
    n = nc.value
    return dict(status=st, idx=out_idx[:n].copy(), iter=out_it[:n].copy(), nc=n,
                iterations=its.value)


def greedy_rc(xb, db, R, Estar, m=1, seed=1, ncmax=None, threads=None):
    """Algorithm 1 with the recurrence-Cholesky append of Sec. 1 (the paper's
    own CPU procedure; the fair CPU baseline).  Returns dict(status, idx,
    iter, nc, iterations, final_max, w) with w the final weights (nc x 3)."""
    L = lib()
    xb, px = _d(xb)
    db, pd = _d(db)
    nb = len(xb)
    ncmax = int(ncmax or nb)
    out_idx = np.zeros(ncmax, dtype=np.int32)
    out_it = np.zeros(ncmax, dtype=np.int64)
    nc = C.c_int64(0)
    its = C.c_int64(0)
    fmax = C.c_double(0.0)
    w = np.zeros((ncmax, 3))
    st = L.orc_greedy_rc(px, pd, nb, float(R), float(Estar), int(m), int(seed), ncmax,
                         out_idx.ctypes.data_as(C.POINTER(C.c_int32)),
                         out_it.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(nc),
                         C.byref(its), C.byref(fmax), w.ctypes.data_as(C.POINTER(C.c_double)),
                         threads or default_threads())
    n = nc.value
    return dict(status=st, idx=out_idx[:n].copy(), iter=out_it[:n].copy(), nc=n,
                iterations=its.value, final_max=fmax.value, w=w[:n].copy())


def nearest_support(xb, S, threads=None):
    """d_i = min over j in S of |r_i - r_j| for every boundary node (Sec. 4.1)."""
    L = lib()
    xb, px = _d(xb)
    S, ps = _i32(S)
    d = np.empty(len(xb))
    L.orc_nearest_support(px, len(xb), ps, len(S), d.ctypes.data_as(C.POINTER(C.c_double)),
                          threads or default_threads())
    return d


def support_kl(xb, S1, S2, threads=None):
    """KL(S1 || S2) = sum_i d1_i log(d1_i / d2_i) (Sec. 4.1), terms with a zero
    distance left out."""
    L = lib()
    xb, px = _d(xb)
    S1, p1 = _i32(S1)
    S2, p2 = _i32(S2)
    kl = C.c_double(0.0)
    st = L.orc_support_kl(px, len(xb), p1, len(S1), p2, len(S2), C.byref(kl),
                          threads or default_threads())
    if st != 0:
        raise MemoryError("orc_support_kl")
    return kl.value


def tolerance(db, tol_rel):
    """E* = tol * max_j |dr_j|_2 (tolerance relative to the largest displacement)."""
    return float(tol_rel) * float(np.max(np.linalg.norm(np.asarray(db), axis=1)))
