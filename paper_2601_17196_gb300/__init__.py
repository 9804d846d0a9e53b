"""GB300 (sm_103a) solver library for entropic Partial Optimal Transport.

Accelerated Sinkhorn for POT (ASPOT, arXiv 2601.17196) and the feasible
Sinkhorn baseline, with rounding to a feasible plan of mass ``s``.  The
compute runs in the CUDA library ``lib/libaspot.so`` (C-ABI declared in
``include/aspot.h``); this package only marshals arguments (torch supplies
device memory and streams).  There is no CPU fallback: if the library is not
built, every call raises.
"""
from .binding import (  # noqa: F401
    DeviceProblem,
    PotError,
    Plan,
    SolveResult,
    aspot_solve,
    aspot_solve_batched,
    aspot_state_export,
    AspotState,
    sinkhorn_pot_solve,
    pot_round,
    pot_objective,
    pot_marginals,
    pot_cost_max,
    pot_plan_dense,
    workspace_bytes,
    marginals_workspace_bytes,
    pass_kernel,
    lib,
    exported_symbols,
    FLAG_STOP_RAW_EPS,
    FLAG_NO_SMOOTH,
    FLAG_TRACE,
    FLAG_NO_STOP,
    FLAG_FORCE_SIMT,
    FLAG_PROFILE,
    FLAG_WARM_CHECK,
    FLAG_AUTOTUNE,
    FLAG_STAGED,
    autotune_set,
    autotune_lookup,
    autotune_clear,
    autotune_save,
    autotune_load,
    COST_DENSE_F32,
    COST_SQEUCLID_BF16,
    COST_SQEUCLID_F16,
    COST_SQEUCLID_F32,
    BLOCK_CYCLIC,
    BLOCK_GREEDY,
)
