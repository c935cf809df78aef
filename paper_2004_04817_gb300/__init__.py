"""GB300 (sm_103a) RBF mesh deformation with GCB greedy support selection.

The compute runs in ``librbfgcb.so`` (hand-written CUDA behind a C ABI, see
``include/rbfgcb.h``); this package only marshals torch CUDA tensors to it.
Importing the package does not load the library: the first call does, and it
raises if the library or a CUDA device is missing (there is no CPU path).
"""
from .rbf import (  # noqa: F401
    RBFError,
    Params,
    GreedyStats,
    lib,
    greedy_select,
    greedy_select_peaks,
    solve_weights,
    deform_volume,
    deform_volume_fields,
    solve_system,
    adjoint,
    adjoint_factored,
    Factor,
    deform,
    deform_modal,
    MODAL_BF16,
    MODAL_BF16X3,
    MODAL_F16X2,
    RBFDeform,
    GreedyBatch,
    VolumeBatch,
    VolumePlan,
    measure_approx_error,
    measure_fma_peak,
    measure_latency,
    nearest_support,
    support_kl,
    group_of,
    status_string,
    STATUS,
    E_NC_MAX,
    PREC_F32,
    PREC_F32X2,
    PREC_F64,
    HIST_COLS,
)
