"""ctypes binding of librbfgcb.so: argument marshalling only.

Every function takes and returns torch tensors on the current CUDA device and
forwards raw device pointers, sizes and the current stream to the C ABI of
``include/rbfgcb.h``.  Workspaces are torch allocations sized by the
library's own *_workspace_bytes queries.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

PREC_F32 = 32
PREC_F32X2 = 48
PREC_F64 = 64
HIST_COLS = 6
STATUS = {0: "RBF_OK", 1: "RBF_E_ARG", 2: "RBF_E_NOT_SPD", 3: "RBF_E_NC_MAX",
          4: "RBF_E_NONFINITE", 5: "RBF_E_WORKSPACE", 6: "RBF_E_TIMEOUT", 7: "RBF_E_CUDA"}
E_NC_MAX = 3


class RBFError(RuntimeError):
    def __init__(self, status, where):
        self.status = int(status)
        super().__init__(f"{where}: {status_string(status)}")


class Params(C.Structure):
    _fields_ = [
        ("radius", C.c_double),
        ("tol", C.c_double),
        ("tol_mode", C.c_int32),
        ("eval_prec", C.c_int32),
        ("m", C.c_int64),
        ("seed", C.c_uint64),
        ("nc_max", C.c_int64),
        ("refine_steps", C.c_int32),
        ("flags", C.c_int32),
        ("ctas", C.c_int32),
        ("reserved", C.c_int32),
    ]


class GreedyStats(C.Structure):
    _fields_ = [
        ("iterations", C.c_int64),
        ("nc", C.c_int64),
        ("full_checks", C.c_int64),
        ("pairs_f32", C.c_int64),
        ("pairs_f64", C.c_int64),
        ("pairs_ff", C.c_int64),
        ("rescored", C.c_int64),
        ("estar", C.c_double),
        ("final_max", C.c_double),
        ("final_rms", C.c_double),
        ("min_pivot", C.c_double),
        ("max_resid", C.c_double),
        ("phase_ns", C.c_int64 * 12),
        ("barriers", C.c_int64),
        ("ctas", C.c_int64),
    ]


class GreedyProblem(C.Structure):
    _fields_ = [
        ("d_xb", C.c_void_p),
        ("d_db", C.c_void_p),
        ("nb", C.c_int64),
        ("params", Params),
        ("d_sel_idx", C.c_void_p),
        ("d_w", C.c_void_p),
        ("d_sel_iter", C.c_void_p),
    ]


class VolumeProblem(C.Structure):
    _fields_ = [
        ("d_xv", C.c_void_p),
        ("nv", C.c_int64),
        ("d_xb", C.c_void_p),
        ("d_sel_idx", C.c_void_p),
        ("d_w", C.c_void_p),
        ("d_nc", C.c_void_p),
        ("nc_max", C.c_int64),
        ("radius", C.c_double),
        ("d_dv", C.c_void_p),
    ]


_lib = None
_vp = C.c_void_p


def lib():
    """Load librbfgcb.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or os.environ.get("RBF_REBUILD"):
            path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER(Params)
        L.rbf_greedy_workspace_bytes.restype = C.c_size_t
        L.rbf_greedy_workspace_bytes.argtypes = [C.c_int64, P]
        L.rbf_greedy_select.restype = C.c_int
        L.rbf_greedy_select.argtypes = [_vp, _vp, C.c_int64, P, _vp, _vp, _vp, _vp, C.c_int64,
                                        C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                        C.POINTER(GreedyStats), _vp, C.c_size_t, _vp]
        L.rbf_greedy_select_peaks.restype = C.c_int
        L.rbf_greedy_select_peaks.argtypes = [_vp, _vp, C.c_int64, P, C.c_int, C.c_double, _vp,
                                              _vp, _vp, C.POINTER(C.c_int64),
                                              C.POINTER(GreedyStats), _vp, C.c_size_t, _vp]
        L.rbf_solve_workspace_bytes.restype = C.c_size_t
        L.rbf_solve_workspace_bytes.argtypes = [C.c_int64]
        L.rbf_solve_weights.restype = C.c_int
        L.rbf_solve_weights.argtypes = [_vp, _vp, C.c_int64, _vp, C.c_int64, P, _vp,
                                        C.POINTER(C.c_double), _vp, C.c_size_t, _vp]
        L.rbf_volume_workspace_bytes.restype = C.c_size_t
        L.rbf_volume_workspace_bytes.argtypes = [C.c_int64, C.c_int64, P]
        L.rbf_deform_volume.restype = C.c_int
        L.rbf_deform_volume.argtypes = [_vp, C.c_int64, _vp, _vp, C.c_int64, _vp, P, _vp, _vp,
                                        C.c_size_t, _vp]
        L.rbf_measure_fma_peak.restype = C.c_int
        L.rbf_measure_fma_peak.argtypes = [C.c_int, C.POINTER(C.c_double), _vp]
        L.rbf_last_device_status.restype = C.c_int
        L.rbf_status_string.restype = C.c_char_p
        L.rbf_status_string.argtypes = [C.c_int]
        L.rbf_version.restype = C.c_char_p
        L.rbf_solve_system.restype = C.c_int
        L.rbf_solve_system.argtypes = [_vp, C.c_int64, _vp, C.c_int64, _vp, P, _vp,
                                       C.POINTER(C.c_double), _vp, C.c_size_t, _vp]
        L.rbf_adjoint_workspace_bytes.restype = C.c_size_t
        L.rbf_adjoint_workspace_bytes.argtypes = [C.c_int64, C.c_int64]
        L.rbf_deform_volume_adjoint.restype = C.c_int
        L.rbf_deform_volume_adjoint.argtypes = [_vp, C.c_int64, _vp, C.c_int64, _vp, C.c_int64,
                                                _vp, P, _vp, C.POINTER(C.c_double), _vp,
                                                C.c_size_t, _vp]
        PP = C.POINTER(GreedyProblem)
        L.rbf_greedy_batch_workspace_bytes.restype = C.c_size_t
        L.rbf_greedy_batch_workspace_bytes.argtypes = [PP, C.c_int]
        L.rbf_greedy_batch_create.restype = C.c_int
        L.rbf_greedy_batch_create.argtypes = [PP, C.c_int, _vp, C.c_size_t, _vp,
                                              C.POINTER(C.c_void_p)]
        L.rbf_greedy_batch_run.restype = C.c_int
        L.rbf_greedy_batch_run.argtypes = [_vp, _vp]
        L.rbf_greedy_batch_nc_device.restype = C.c_void_p
        L.rbf_greedy_batch_nc_device.argtypes = [_vp]
        L.rbf_greedy_batch_results.restype = C.c_int
        L.rbf_greedy_batch_results.argtypes = [_vp, C.POINTER(C.c_int32),
                                               C.POINTER(GreedyStats), _vp]
        L.rbf_greedy_batch_destroy.restype = None
        L.rbf_greedy_batch_destroy.argtypes = [_vp]
        VP = C.POINTER(VolumeProblem)
        L.rbf_volume_batch_workspace_bytes.restype = C.c_size_t
        L.rbf_volume_batch_workspace_bytes.argtypes = [VP, C.c_int, C.c_int]
        L.rbf_volume_batch_create.restype = C.c_int
        L.rbf_volume_batch_create.argtypes = [VP, C.c_int, C.c_int, _vp, C.c_size_t, _vp,
                                              C.POINTER(C.c_void_p)]
        L.rbf_volume_batch_run.restype = C.c_int
        L.rbf_volume_batch_run.argtypes = [_vp, _vp]
        L.rbf_volume_batch_info.restype = C.c_int
        L.rbf_volume_batch_info.argtypes = [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                            C.POINTER(C.c_float)]
        L.rbf_volume_batch_destroy.restype = None
        L.rbf_volume_batch_destroy.argtypes = [_vp]
        L.rbf_modal_workspace_bytes.restype = C.c_size_t
        L.rbf_modal_workspace_bytes.argtypes = [C.c_int64, C.c_int64, C.c_int, C.c_int]
        L.rbf_deform_modal.restype = C.c_int
        L.rbf_deform_modal.argtypes = [_vp, C.c_int64, _vp, _vp, C.c_int64, _vp, C.c_int, P,
                                       C.c_int, _vp, _vp, C.c_size_t, _vp]
        L.rbf_modal_check.restype = C.c_int
        L.rbf_modal_check.argtypes = [_vp, _vp]
        L.rbf_group_of.restype = C.c_int
        L.rbf_group_of.argtypes = [C.c_int64, C.c_int64, C.c_uint64, C.POINTER(C.c_int32)]
        L.rbf_volume_plan_workspace_bytes.restype = C.c_size_t
        L.rbf_volume_plan_workspace_bytes.argtypes = [C.c_int64, P]
        L.rbf_volume_plan_create.restype = C.c_int
        L.rbf_volume_plan_create.argtypes = [_vp, C.c_int64, P, _vp, C.c_size_t, _vp,
                                             C.POINTER(C.c_void_p)]
        L.rbf_volume_plan_run.restype = C.c_int
        L.rbf_volume_plan_run.argtypes = [_vp, _vp, _vp, C.c_int64, _vp, _vp, _vp, _vp]
        L.rbf_volume_plan_info.restype = C.c_int
        L.rbf_volume_plan_info.argtypes = [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int64),
                                           C.POINTER(C.c_int64)]
        L.rbf_nearest_support.restype = C.c_int
        L.rbf_nearest_support.argtypes = [_vp, C.c_int64, _vp, C.c_int64, _vp, _vp]
        L.rbf_support_kl_workspace_bytes.restype = C.c_size_t
        L.rbf_support_kl_workspace_bytes.argtypes = [C.c_int64]
        L.rbf_support_kl.restype = C.c_int
        L.rbf_support_kl.argtypes = [_vp, C.c_int64, _vp, C.c_int64, _vp, C.c_int64,
                                     C.POINTER(C.c_double), _vp, C.c_size_t, _vp]
        L.rbf_volume_fields_workspace_bytes.restype = C.c_size_t
        L.rbf_volume_fields_workspace_bytes.argtypes = [C.c_int64, C.c_int64, C.c_int]
        L.rbf_deform_volume_fields.restype = C.c_int
        L.rbf_deform_volume_fields.argtypes = [_vp, C.c_int64, _vp, _vp, C.c_int64, _vp, C.c_int,
                                               P, _vp, _vp, C.c_size_t, _vp]
        L.rbf_greedy_screen_errors.restype = C.c_int
        L.rbf_greedy_screen_errors.argtypes = [_vp, C.c_size_t, C.c_int64, P, C.c_int64, _vp,
                                               _vp, _vp, _vp]
        L.rbf_measure_approx_error.restype = C.c_int
        L.rbf_measure_approx_error.argtypes = [C.c_int, C.POINTER(C.c_double), _vp]
        L.rbf_measure_latency.restype = C.c_int
        L.rbf_measure_latency.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), _vp]
        L.rbf_factor_workspace_bytes.restype = C.c_size_t
        L.rbf_factor_workspace_bytes.argtypes = [C.c_int64]
        L.rbf_factor_create.restype = C.c_int
        L.rbf_factor_create.argtypes = [_vp, C.c_int64, _vp, C.c_int64, P, _vp, C.c_size_t, _vp,
                                        C.POINTER(C.c_void_p)]
        L.rbf_factor_solve.restype = C.c_int
        L.rbf_factor_solve.argtypes = [_vp, _vp, C.c_int, _vp, C.POINTER(C.c_double), _vp]
        L.rbf_factor_destroy.restype = None
        L.rbf_factor_destroy.argtypes = [_vp]
        L.rbf_deform_volume_adjoint_factored.restype = C.c_int
        L.rbf_deform_volume_adjoint_factored.argtypes = [_vp, C.c_int64, _vp, _vp, P, _vp,
                                                         C.POINTER(C.c_double), _vp, C.c_size_t,
                                                         _vp]
        L.rbf_volume_plan_destroy.restype = None
        L.rbf_volume_plan_destroy.argtypes = [_vp]
        _lib = L
    return _lib


def status_string(s):
    return lib().rbf_status_string(int(s)).decode()


def _check(st, where, allow=()):
    if st != 0 and st not in allow:
        raise RBFError(st, where)
    return st


def _dev(t, dtype, name, shape2=None, host_ok=False):
    if not isinstance(t, torch.Tensor) or not (t.is_cuda or (host_ok and t.is_pinned())):
        raise TypeError(f"{name} must be a CUDA tensor" +
                        (" or a pinned host tensor" if host_ok else ""))
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape2 is not None and (t.dim() != 2 or t.shape[1] != shape2):
        raise ValueError(f"{name} must have shape (n, {shape2})")
    return t


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


FLAG_HISTORY_FULL = 1


def make_params(radius, tol=0.0, tol_mode=1, eval_prec=PREC_F64, m=1, seed=1, nc_max=0,
                refine_steps=2, flags=0, ctas=0):
    return Params(float(radius), float(tol), int(tol_mode), int(eval_prec), int(m), int(seed),
                  int(nc_max), int(refine_steps), int(flags), int(ctas), 0)


def greedy_select(xb, db, *, radius, tol, tol_mode=1, m=1, seed=1, nc_max=None,
                  eval_prec=PREC_F64, hist_cap=0, history_full=False, weights=False,
                  refine_steps=2, ctas=0, stream=None, workspace=None, screen=False):
    """GCB greedy (m = 1: plain greedy).  Returns a dict with ``idx`` (int32
    CUDA tensor, selection order), ``iter`` (int64), ``nc``, ``hist`` (CUDA
    (n, 6) or None), ``stats`` (dict) and ``status`` (0 or RBF_E_NC_MAX).
    ``history_full`` adds FP64 all-node maxima to the history after every
    m-th iteration (diagnostic).  ``weights`` also returns ``w``, the refined
    FP64 weights of the selected set.  ``screen`` (FP32 and double-float
    modes) also returns ``screen``: the final screened error and certified
    bound of every node (``err``, ``bound``, node order) and the evaluation
    table's weights ``w_eval`` (rbf_greedy_screen_errors)."""
    L = lib()
    _dev(xb, torch.float64, "xb", 3)
    _dev(db, torch.float64, "db", 3)
    nb = xb.shape[0]
    if db.shape[0] != nb:
        raise ValueError("xb and db must have the same number of rows")
    nc_max = int(nc_max or min(nb, 4096))
    p = make_params(radius, tol, tol_mode, eval_prec, m, seed, nc_max, refine_steps,
                    flags=FLAG_HISTORY_FULL if history_full else 0, ctas=ctas)
    need = L.rbf_greedy_workspace_bytes(nb, C.byref(p))
    if need == 0:
        raise RBFError(1, "rbf_greedy_workspace_bytes")
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        _workspace(need, xb.device)
    idx = torch.empty(nc_max, dtype=torch.int32, device=xb.device)
    it = torch.empty(nc_max, dtype=torch.int64, device=xb.device)
    w = torch.empty((nc_max, 3), dtype=torch.float64, device=xb.device) if weights else None
    hist = torch.empty((hist_cap, HIST_COLS), dtype=torch.float64, device=xb.device) \
        if hist_cap else None
    nc = C.c_int64(0)
    nh = C.c_int64(0)
    stats = GreedyStats()
    st = L.rbf_greedy_select(_ptr(xb), _ptr(db), nb, C.byref(p), _ptr(idx), _ptr(it),
                             _ptr(w), _ptr(hist), int(hist_cap), C.byref(nc), C.byref(nh),
                             C.byref(stats), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "rbf_greedy_select", allow=(E_NC_MAX,))
    n = nc.value
    scr = None
    if screen and st == 0:
        err = torch.empty(nb, dtype=torch.float64, device=xb.device)
        bnd = torch.empty(nb, dtype=torch.float32, device=xb.device)
        wev = torch.empty((max(n, 1), 3), dtype=torch.float64, device=xb.device)
        _check(L.rbf_greedy_screen_errors(_ptr(ws), ws.numel(), nb, C.byref(p), n, _ptr(err),
                                          _ptr(bnd), _ptr(wev), _stream(stream)),
               "rbf_greedy_screen_errors")
        scr = dict(err=err, bound=bnd, w_eval=wev[:n])
    return dict(idx=idx[:n], iter=it[:n], nc=n, status=st, screen=scr,
                w=w[:n] if w is not None else None,
                hist=hist[:min(nh.value, hist_cap)] if hist is not None else None,
                n_hist=nh.value,
                stats={f: (list(getattr(stats, f)) if f == "phase_ns" else getattr(stats, f))
                       for f, _ in GreedyStats._fields_})


def greedy_select_peaks(xb, db, *, radius, tol, peaks, separation, tol_mode=1, m=1, seed=1,
                        nc_max=None, eval_prec=PREC_F64, weights=False, refine_steps=2, ctas=0,
                        stream=None, workspace=None):
    """Peak-selection variant of greedy_select: up to ``peaks`` nodes of the
    active group, at least ``separation`` apart, appended per iteration.
    Returns a dict like greedy_select (no history)."""
    L = lib()
    _dev(xb, torch.float64, "xb", 3)
    _dev(db, torch.float64, "db", 3)
    nb = xb.shape[0]
    nc_max = int(nc_max or min(nb, 4096))
    p = make_params(radius, tol, tol_mode, eval_prec, m, seed, nc_max, refine_steps, ctas=ctas)
    need = L.rbf_greedy_workspace_bytes(nb, C.byref(p))
    if need == 0:
        raise RBFError(1, "rbf_greedy_workspace_bytes")
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        _workspace(need, xb.device)
    idx = torch.empty(nc_max, dtype=torch.int32, device=xb.device)
    it = torch.empty(nc_max, dtype=torch.int64, device=xb.device)
    w = torch.empty((nc_max, 3), dtype=torch.float64, device=xb.device) if weights else None
    nc = C.c_int64(0)
    stats = GreedyStats()
    st = L.rbf_greedy_select_peaks(_ptr(xb), _ptr(db), nb, C.byref(p), int(peaks),
                                   float(separation), _ptr(idx), _ptr(it), _ptr(w), C.byref(nc),
                                   C.byref(stats), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "rbf_greedy_select_peaks", allow=(E_NC_MAX,))
    n = nc.value
    return dict(idx=idx[:n], iter=it[:n], nc=n, status=st, w=w[:n] if w is not None else None,
                stats={f: (list(getattr(stats, f)) if f == "phase_ns" else getattr(stats, f))
                       for f, _ in GreedyStats._fields_})


def solve_weights(xb, db, sel_idx, *, radius, refine_steps=2, stream=None, workspace=None):
    """FP64 weights (nc, 3) of the support set; returns (w, max_residual)."""
    L = lib()
    _dev(xb, torch.float64, "xb", 3)
    _dev(db, torch.float64, "db", 3)
    _dev(sel_idx, torch.int32, "sel_idx")
    nc = sel_idx.numel()
    p = make_params(radius, refine_steps=refine_steps)
    need = L.rbf_solve_workspace_bytes(nc)
    if need == 0:
        raise RBFError(1, "rbf_solve_workspace_bytes")
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        _workspace(need, xb.device)
    w = torch.empty((nc, 3), dtype=torch.float64, device=xb.device)
    res = C.c_double(0.0)
    st = L.rbf_solve_weights(_ptr(xb), _ptr(db), xb.shape[0], _ptr(sel_idx), nc, C.byref(p),
                             _ptr(w), C.byref(res), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "rbf_solve_weights")
    return w, res.value


def solve_system(xb, sel_idx, rhs, *, radius, refine_steps=2, stream=None, workspace=None):
    """X (nc, 3) with Phi_SS X = rhs (FP64 factor + refinement); returns
    (X, max_residual)."""
    L = lib()
    _dev(xb, torch.float64, "xb", 3)
    _dev(sel_idx, torch.int32, "sel_idx")
    _dev(rhs, torch.float64, "rhs", 3)
    nc = sel_idx.numel()
    if rhs.shape[0] != nc:
        raise ValueError("rhs must have one row per support node")
    p = make_params(radius, refine_steps=refine_steps)
    need = L.rbf_solve_workspace_bytes(nc)
    if need == 0:
        raise RBFError(1, "rbf_solve_workspace_bytes")
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        _workspace(need, xb.device)
    x = torch.empty((nc, 3), dtype=torch.float64, device=xb.device)
    res = C.c_double(0.0)
    st = L.rbf_solve_system(_ptr(xb), xb.shape[0], _ptr(sel_idx), nc, _ptr(rhs), C.byref(p),
                            _ptr(x), C.byref(res), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "rbf_solve_system")
    return x, res.value


def adjoint(xv, xb, sel_idx, gv, *, radius, eval_prec=PREC_F32X2, refine_steps=2,
            stream=None, workspace=None):
    """dJ/dd_c = Phi_cc^-1 Phi_vc^T dJ/dd_v (nc, 3); returns (grad, residual)."""
    L = lib()
    _dev(xv, torch.float64, "xv", 3)
    _dev(xb, torch.float64, "xb", 3)
    _dev(sel_idx, torch.int32, "sel_idx")
    _dev(gv, torch.float64, "gv", 3)
    nv, nc = xv.shape[0], sel_idx.numel()
    if gv.shape[0] != nv:
        raise ValueError("gv must have one row per volume point")
    p = make_params(radius, eval_prec=eval_prec, refine_steps=refine_steps)
    need = L.rbf_adjoint_workspace_bytes(nv, nc)
    if need == 0:
        raise RBFError(1, "rbf_adjoint_workspace_bytes")
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        _workspace(need, xv.device)
    gc = torch.empty((nc, 3), dtype=torch.float64, device=xv.device)
    res = C.c_double(0.0)
    st = L.rbf_deform_volume_adjoint(_ptr(xv), nv, _ptr(xb), xb.shape[0], _ptr(sel_idx), nc,
                                     _ptr(gv), C.byref(p), _ptr(gc), C.byref(res), _ptr(ws),
                                     ws.numel(), _stream(stream))
    _check(st, "rbf_deform_volume_adjoint")
    return gc, res.value


class Factor:
    """Phi_SS factorised once for a support set (``rbf_factor_*``): ``solve``
    then costs Z^T Z B plus FP64 refinement instead of a new factorisation.
    ``xb`` and ``sel_idx`` must stay alive and unchanged while it is used."""

    def __init__(self, xb, sel_idx, *, radius, stream=None):
        L = lib()
        _dev(xb, torch.float64, "xb", 3)
        _dev(sel_idx, torch.int32, "sel_idx")
        self.xb, self.sel_idx = xb, sel_idx
        self.nc = sel_idx.numel()
        self.radius = float(radius)
        need = L.rbf_factor_workspace_bytes(self.nc)
        if need == 0:
            raise RBFError(1, "rbf_factor_workspace_bytes")
        self.ws = _workspace(need, xb.device)
        p = make_params(radius)
        h = C.c_void_p()
        _check(L.rbf_factor_create(_ptr(xb), xb.shape[0], _ptr(sel_idx), self.nc, C.byref(p),
                                   _ptr(self.ws), self.ws.numel(), _stream(stream), C.byref(h)),
               "rbf_factor_create")
        self.handle = h

    def solve(self, rhs, *, refine_steps=2, stream=None):
        """X with Phi_SS X = rhs (nc, 3); returns (X, max residual)."""
        _dev(rhs, torch.float64, "rhs", 3)
        x = torch.empty_like(rhs)
        res = C.c_double(0.0)
        _check(lib().rbf_factor_solve(self.handle, _ptr(rhs), int(refine_steps), _ptr(x),
                                      C.byref(res), _stream(stream)), "rbf_factor_solve")
        return x, res.value

    def __del__(self):
        if getattr(self, "handle", None):
            lib().rbf_factor_destroy(self.handle)
            self.handle = None


def adjoint_factored(xv, gv, factor, *, eval_prec=PREC_F32X2, refine_steps=2, stream=None,
                     workspace=None):
    """``adjoint`` with the support system of ``factor`` (no refactorisation)."""
    L = lib()
    _dev(xv, torch.float64, "xv", 3)
    _dev(gv, torch.float64, "gv", 3)
    nv, nc = xv.shape[0], factor.nc
    p = make_params(factor.radius, eval_prec=eval_prec, refine_steps=refine_steps)
    need = L.rbf_adjoint_workspace_bytes(nv, nc)
    if need == 0:
        raise RBFError(1, "rbf_adjoint_workspace_bytes")
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        _workspace(need, xv.device)
    gc = torch.empty((nc, 3), dtype=torch.float64, device=xv.device)
    res = C.c_double(0.0)
    _check(L.rbf_deform_volume_adjoint_factored(_ptr(xv), nv, _ptr(gv), factor.handle,
                                                C.byref(p), _ptr(gc), C.byref(res), _ptr(ws),
                                                ws.numel(), _stream(stream)),
           "rbf_deform_volume_adjoint_factored")
    return gc, res.value


class RBFDeform(torch.autograd.Function):
    """d_v = Phi_vc Phi_cc^-1 d_c as a differentiable map of the support
    displacements d_c (nc, 3); the backward pass is the adjoint kernel.  With
    a ``Factor`` of the support set both passes reuse its factorisation."""

    @staticmethod
    def forward(ctx, dc, xv, xb, sel_idx, radius, eval_prec, factor):
        rhs = dc.detach().contiguous()
        if factor is not None:
            w, _ = factor.solve(rhs)
        else:
            w, _ = solve_system(xb, sel_idx, rhs, radius=radius)
        dv = deform_volume(xv, xb, sel_idx, w, radius=radius, eval_prec=eval_prec)
        ctx.save_for_backward(xv, xb, sel_idx)
        ctx.radius = radius
        ctx.eval_prec = eval_prec
        ctx.factor = factor
        return dv

    @staticmethod
    def backward(ctx, gv):
        xv, xb, sel_idx = ctx.saved_tensors
        prec = PREC_F32 if ctx.eval_prec == PREC_F32 else PREC_F32X2
        if ctx.factor is not None:
            gc, _ = adjoint_factored(xv, gv.contiguous(), ctx.factor, eval_prec=prec)
        else:
            gc, _ = adjoint(xv, xb, sel_idx, gv.contiguous(), radius=ctx.radius, eval_prec=prec)
        return gc, None, None, None, None, None, None


def deform(dc, xv, xb, sel_idx, *, radius, eval_prec=PREC_F32X2, factor=None):
    """Differentiable volume deformation (see RBFDeform)."""
    return RBFDeform.apply(dc, xv, xb, sel_idx, float(radius), int(eval_prec), factor)


def deform_volume(xv, xb, sel_idx, w, *, radius, eval_prec=PREC_F32, stream=None,
                  workspace=None, out=None):
    """Volume displacements (nv, 3) FP64 by Eq. 6 in FP32, double-float or
    FP64 pairs.  ``xv`` and ``out`` may be pinned host tensors: the kernels
    then read the points from, and write the displacements to, host memory
    directly (each once), with no copy through the copy engines."""
    L = lib()
    _dev(xv, torch.float64, "xv", 3, host_ok=True)
    _dev(xb, torch.float64, "xb", 3)
    _dev(sel_idx, torch.int32, "sel_idx")
    _dev(w, torch.float64, "w", 3)
    nv, nc = xv.shape[0], sel_idx.numel()
    p = make_params(radius, eval_prec=eval_prec)
    need = L.rbf_volume_workspace_bytes(nv, nc, C.byref(p))
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        _workspace(need, xb.device)
    dv = out if out is not None else torch.empty((nv, 3), dtype=torch.float64, device=xb.device)
    _dev(dv, torch.float64, "out", 3, host_ok=True)
    st = L.rbf_deform_volume(_ptr(xv), nv, _ptr(xb), _ptr(sel_idx), nc, _ptr(w), C.byref(p),
                             _ptr(dv), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "rbf_deform_volume")
    return dv


def deform_volume_fields(xv, xb, sel_idx, w, *, radius, stream=None, workspace=None, out=None):
    """Eq. 6 for every column of ``w`` (nc x n_out FP64) on one support set,
    double-float (FP64-level accuracy): (nv, n_out) FP64."""
    L = lib()
    _dev(xv, torch.float64, "xv", 3)
    _dev(xb, torch.float64, "xb", 3)
    _dev(sel_idx, torch.int32, "sel_idx")
    if w.device.type != "cuda" or w.dtype != torch.float64 or w.dim() != 2 or \
            not w.is_contiguous() or w.shape[0] != sel_idx.numel():
        raise ValueError("w must be a contiguous CUDA float64 (nc, n_out) tensor")
    nv, nc, n_out = xv.shape[0], sel_idx.numel(), w.shape[1]
    need = L.rbf_volume_fields_workspace_bytes(nv, nc, n_out)
    if need == 0:
        raise RBFError(1, "rbf_volume_fields_workspace_bytes")
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        _workspace(need, xv.device)
    d = out if out is not None else torch.empty((nv, n_out), dtype=torch.float64,
                                                device=xv.device)
    p = make_params(radius, eval_prec=PREC_F32X2)
    st = L.rbf_deform_volume_fields(_ptr(xv), nv, _ptr(xb), _ptr(sel_idx), nc, _ptr(w), n_out,
                                    C.byref(p), _ptr(d), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "rbf_deform_volume_fields")
    return d


def group_of(nb, m, seed):
    """The partition the greedy uses: group index of every node (host)."""
    import numpy as np
    g = np.empty(int(nb), dtype=np.int32)
    _check(lib().rbf_group_of(int(nb), int(m), int(seed),
                              g.ctypes.data_as(C.POINTER(C.c_int32))), "rbf_group_of")
    return g


MODAL_BF16 = 1
MODAL_F16X2 = 2
MODAL_BF16X3 = 3


def deform_modal(xv, xb, sel_idx, W, *, radius, mode=MODAL_BF16X3, stream=None,
                 workspace=None, out=None, check=True):
    """D = Phi_vc W on the tensor cores for many displacement fields at once:
    W is FP64 (nc, n_out), the result FP32 (nv, n_out)."""
    L = lib()
    _dev(xv, torch.float64, "xv", 3)
    _dev(xb, torch.float64, "xb", 3)
    _dev(sel_idx, torch.int32, "sel_idx")
    _dev(W, torch.float64, "W")
    nv, nc, n_out = xv.shape[0], sel_idx.numel(), W.shape[1]
    need = L.rbf_modal_workspace_bytes(nv, nc, n_out, mode)
    if need == 0:
        raise RBFError(1, "rbf_modal_workspace_bytes")
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        _workspace(need, xv.device)
    d = out if out is not None else torch.empty((nv, n_out), dtype=torch.float32,
                                                device=xv.device)
    p = make_params(radius)
    st = L.rbf_deform_modal(_ptr(xv), nv, _ptr(xb), _ptr(sel_idx), nc, _ptr(W), n_out,
                            C.byref(p), int(mode), _ptr(d), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "rbf_deform_modal")
    if check:
        _check(L.rbf_modal_check(_ptr(ws), _stream(stream)), "rbf_deform_modal (device)")
    return d


def nearest_support(xb, sel_idx, *, stream=None):
    """d_i = min over j in S of |r_i - r_j| for every boundary node (Sec. 4.1),
    CUDA FP64 (nb,)."""
    _dev(xb, torch.float64, "xb", 3)
    _dev(sel_idx, torch.int32, "sel_idx")
    d = torch.empty(xb.shape[0], dtype=torch.float64, device=xb.device)
    _check(lib().rbf_nearest_support(_ptr(xb), xb.shape[0], _ptr(sel_idx), sel_idx.numel(),
                                     _ptr(d), _stream(stream)), "rbf_nearest_support")
    return d


def support_kl(xb, sel1, sel2, *, stream=None, workspace=None):
    """KL(S1 || S2) = sum_i d1_i log(d1_i / d2_i) over the boundary nodes
    (Sec. 4.1), terms with a zero distance left out."""
    L = lib()
    _dev(xb, torch.float64, "xb", 3)
    _dev(sel1, torch.int32, "sel1")
    _dev(sel2, torch.int32, "sel2")
    nb = xb.shape[0]
    need = L.rbf_support_kl_workspace_bytes(nb)
    ws = workspace if workspace is not None and workspace.numel() >= need else \
        _workspace(need, xb.device)
    kl = C.c_double(0.0)
    _check(L.rbf_support_kl(_ptr(xb), nb, _ptr(sel1), sel1.numel(), _ptr(sel2), sel2.numel(),
                            C.byref(kl), _ptr(ws), ws.numel(), _stream(stream)),
           "rbf_support_kl")
    return kl.value


LAT_GRID_BARRIER, LAT_FP64_WARP, LAT_FP32_WARP = 1, 2, 3


def measure_latency(what, param=0, stream=None):
    """Nanoseconds per grid barrier among `param` CTAs (LAT_GRID_BARRIER) or
    per FMA instruction of a lone warp (LAT_FP64_WARP, LAT_FP32_WARP)."""
    ns = C.c_double(0.0)
    _check(lib().rbf_measure_latency(int(what), int(param), C.byref(ns), _stream(stream)),
           "rbf_measure_latency")
    return ns.value


APPROX_SQRT, APPROX_RSQRT = 1, 2


def measure_approx_error(which, stream=None):
    """Largest relative error of sqrt.approx.f32 (APPROX_SQRT) or rsqrtf
    (APPROX_RSQRT) over every normal float in [2^-126, 4)."""
    r = C.c_double(0.0)
    _check(lib().rbf_measure_approx_error(int(which), C.byref(r), _stream(stream)),
           "rbf_measure_approx_error")
    return r.value


def measure_fma_peak(prec=32, stream=None):
    """Measured vector FMA peak of this GPU in FLOP/s (an FMA counts 2)."""
    f = C.c_double(0.0)
    _check(lib().rbf_measure_fma_peak(int(prec), C.byref(f), _stream(stream)),
           "rbf_measure_fma_peak")
    return f.value


class GreedyBatch:
    """Many independent greedy problems in one cooperative launch.

    ``problems``: list of dicts with ``xb``, ``db`` (CUDA FP64 (n, 3)),
    ``radius``, ``tol``, ``tol_mode``, ``m``, ``seed``, ``nc_max``.  Outputs
    per problem: ``idx[i]`` (int32, nc_max), ``iter[i]`` (int64, the iteration that
    appended each node), ``w[i]`` (FP64 (nc_max, 3)) and
    the device array ``nc`` (int64, B).  ``run()`` only enqueues (it can be
    captured in a CUDA graph); ``results()`` synchronises.
    """

    def __init__(self, problems, *, eval_prec=PREC_F32X2, refine_steps=2, stream=None):
        L = lib()
        self.B = len(problems)
        dev = problems[0]["xb"].device
        self.problems = problems
        self.idx, self.w, self.iter = [], [], []
        arr = (GreedyProblem * self.B)()
        for i, q in enumerate(problems):
            _dev(q["xb"], torch.float64, "xb", 3)
            _dev(q["db"], torch.float64, "db", 3)
            ncm = int(q.get("nc_max") or min(q["xb"].shape[0], 4096))
            self.idx.append(torch.empty(ncm, dtype=torch.int32, device=dev))
            self.w.append(torch.empty((ncm, 3), dtype=torch.float64, device=dev))
            self.iter.append(torch.empty(ncm, dtype=torch.int64, device=dev))
            arr[i].d_xb = q["xb"].data_ptr()
            arr[i].d_db = q["db"].data_ptr()
            arr[i].nb = q["xb"].shape[0]
            arr[i].params = make_params(q["radius"], q["tol"], q.get("tol_mode", 1), eval_prec,
                                        q.get("m", 1), q.get("seed", 1), ncm, refine_steps)
            arr[i].d_sel_idx = self.idx[i].data_ptr()
            arr[i].d_w = self.w[i].data_ptr()
            arr[i].d_sel_iter = self.iter[i].data_ptr()
        self._arr = arr
        need = L.rbf_greedy_batch_workspace_bytes(arr, self.B)
        if need == 0:
            raise RBFError(1, "rbf_greedy_batch_workspace_bytes")
        self.ws = _workspace(need, dev)
        h = C.c_void_p()
        _check(L.rbf_greedy_batch_create(arr, self.B, _ptr(self.ws), self.ws.numel(),
                                         _stream(stream), C.byref(h)), "rbf_greedy_batch_create")
        self.handle = h
        ncp = L.rbf_greedy_batch_nc_device(h)
        self.nc_ptr = ncp

    def run(self, stream=None):
        _check(lib().rbf_greedy_batch_run(self.handle, _stream(stream)), "rbf_greedy_batch_run")

    def results(self, stream=None):
        st = (C.c_int32 * self.B)()
        stats = (GreedyStats * self.B)()
        lib().rbf_greedy_batch_results(self.handle, st, stats, _stream(stream))
        out = []
        for i in range(self.B):
            d = {f: (list(getattr(stats[i], f)) if f == "phase_ns" else getattr(stats[i], f))
                 for f, _ in GreedyStats._fields_}
            d["status"] = st[i]
            out.append(d)
        return out

    def __del__(self):
        if getattr(self, "handle", None):
            lib().rbf_greedy_batch_destroy(self.handle)
            self.handle = None


class VolumeBatch:
    """Batched double-float volume sums reading |S| on the device.

    ``problems``: list of dicts with ``xv`` (CUDA FP64 (nv, 3)), ``xb``,
    ``idx`` (int32 (nc_max,)), ``w`` (FP64 (nc_max, 3)), ``nc_ptr`` (device
    address of an int64 count), ``radius``.  Outputs ``dv[i]``.  Creating the
    batch runs the kernels to choose the tile shape (autotuning).
    """

    def __init__(self, problems, *, stream=None):
        L = lib()
        self.B = len(problems)
        dev = problems[0]["xv"].device
        self.dv = []
        arr = (VolumeProblem * self.B)()
        for i, q in enumerate(problems):
            _dev(q["xv"], torch.float64, "xv", 3)
            self.dv.append(torch.empty_like(q["xv"]))
            arr[i].d_xv = q["xv"].data_ptr()
            arr[i].nv = q["xv"].shape[0]
            arr[i].d_xb = q["xb"].data_ptr()
            arr[i].d_sel_idx = q["idx"].data_ptr()
            arr[i].d_w = q["w"].data_ptr()
            arr[i].d_nc = q["nc_ptr"]
            arr[i].nc_max = q["idx"].numel()
            arr[i].radius = float(q["radius"])
            arr[i].d_dv = self.dv[i].data_ptr()
        self._arr = arr
        self.problems = problems
        need = L.rbf_volume_batch_workspace_bytes(arr, self.B, PREC_F32X2)
        if need == 0:
            raise RBFError(1, "rbf_volume_batch_workspace_bytes")
        self.ws = _workspace(need, dev)
        h = C.c_void_p()
        _check(L.rbf_volume_batch_create(arr, self.B, PREC_F32X2, _ptr(self.ws), self.ws.numel(),
                                         _stream(stream), C.byref(h)), "rbf_volume_batch_create")
        self.handle = h

    def run(self, stream=None):
        _check(lib().rbf_volume_batch_run(self.handle, _stream(stream)), "rbf_volume_batch_run")

    def info(self):
        t, pp = C.c_int(0), C.c_int(0)
        ms = (C.c_float * 4)()
        lib().rbf_volume_batch_info(self.handle, C.byref(t), C.byref(pp), ms)
        return {"threads": t.value, "points_per_thread": pp.value, "candidate_ms": list(ms)}

    def __del__(self):
        if getattr(self, "handle", None):
            lib().rbf_volume_batch_destroy(self.handle)
            self.handle = None


class VolumePlan:
    """Volume sums with compact-support culling (``rbf_volume_plan_*``).

    The plan sorts the volume points ``xv`` (CUDA FP64 (nv, 3)) once for the
    given radius and precision (PREC_F32 or PREC_F32X2); ``run`` then
    evaluates Eq. 6 for any support set of at most ``nc_max`` centres,
    skipping pairs farther apart than the radius.  ``run(..., count=True)``
    also returns the number of pairs evaluated.
    """

    def __init__(self, xv, *, radius, eval_prec=PREC_F32X2, nc_max=4096, stream=None):
        L = lib()
        _dev(xv, torch.float64, "xv", 3)
        self.nv = xv.shape[0]
        self.device = xv.device
        self.p = make_params(radius, eval_prec=eval_prec, nc_max=nc_max)
        need = L.rbf_volume_plan_workspace_bytes(self.nv, C.byref(self.p))
        if need == 0:
            raise RBFError(1, "rbf_volume_plan_workspace_bytes")
        self.ws = _workspace(need, xv.device)
        h = C.c_void_p()
        _check(L.rbf_volume_plan_create(_ptr(xv), self.nv, C.byref(self.p), _ptr(self.ws),
                                        self.ws.numel(), _stream(stream), C.byref(h)),
               "rbf_volume_plan_create")
        self.handle = h
        self._count = torch.zeros(1, dtype=torch.int64, device=xv.device)

    def run(self, xb, sel_idx, w, *, out=None, count=False, stream=None):
        _dev(xb, torch.float64, "xb", 3)
        _dev(sel_idx, torch.int32, "sel_idx")
        nc = sel_idx.numel()
        if nc:
            _dev(w, torch.float64, "w", 3)
        dv = out if out is not None else torch.empty((self.nv, 3), dtype=torch.float64,
                                                     device=self.device)
        if count:
            self._count.zero_()
        _check(lib().rbf_volume_plan_run(self.handle, _ptr(xb), _ptr(sel_idx), nc,
                                         _ptr(w) if nc else None, _ptr(dv),
                                         _ptr(self._count) if count else None, _stream(stream)),
               "rbf_volume_plan_run")
        return (dv, int(self._count.item())) if count else dv

    def info(self):
        b, t, n = C.c_int(0), C.c_int64(0), C.c_int64(0)
        lib().rbf_volume_plan_info(self.handle, C.byref(b), C.byref(t), C.byref(n))
        return {"bits_per_axis": b.value, "points_per_tile": t.value, "tiles": n.value}

    def __del__(self):
        if getattr(self, "handle", None):
            lib().rbf_volume_plan_destroy(self.handle)
            self.handle = None
