"""ctypes loader for ``libsch.so`` (the CUDA library; see include/sch.h).

The library must have been built in-tree (``paper_2402_06927_gb300/build.py``
or ``__graft_entry__.build()``).  There is no fallback: if the shared object
is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as ct
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsch.so")

SCH_MAX_K = 64
PF_RESAMPLE_STATIC_BYTES = 16 * 1024 * 1024

SCH_OK = 0
ERRORS = {
    -1: "SCH_ERR_ARG", -2: "SCH_ERR_CUDA", -3: "SCH_ERR_NOCONVERGE", -4: "SCH_ERR_NONFINITE",
    -5: "SCH_ERR_WORKSPACE", -6: "SCH_ERR_UNSUPPORTED",
}
SCH_DEV_NOCONVERGE = 1
SCH_DEV_NONFINITE = 2
SCH_F64 = 0
SCH_F32 = 1
SCH_SOLVER_AUTO, SCH_SOLVER_LI, SCH_SOLVER_EA = 0, 1, 2

TAG_PRIOR_DW, TAG_PCN, TAG_PCN_ACCEPT, TAG_RESAMPLE, TAG_TRUTH, TAG_OBS, TAG_INIT, TAG_NUDGE = range(1, 9)
TAG_MALA, TAG_MALA_ACCEPT = 9, 10


class SchParams(ct.Structure):
    _fields_ = [
        ("L", ct.c_double), ("n", ct.c_int32), ("alpha", ct.c_double), ("mu", ct.c_double),
        ("dt", ct.c_double), ("K", ct.c_int32), ("amps", ct.c_double * (SCH_MAX_K // 2)),
        ("M", ct.c_int32), ("sigma", ct.c_double), ("tol", ct.c_double), ("max_iter", ct.c_int32),
        ("dtype", ct.c_int32), ("solver", ct.c_int32), ("layout", ct.c_int32),
        ("noise", ct.c_int32), ("kappa", ct.c_double), ("eta", ct.c_double), ("matern_k", ct.c_int32),
    ]


NN_FP32, NN_BF16 = 0, 1


class NNShape(ct.Structure):
    _fields_ = [("n", ct.c_int32), ("K", ct.c_int32), ("Ns", ct.c_int32), ("C", ct.c_int32),
                ("M", ct.c_int32), ("sigma", ct.c_float), ("precision", ct.c_int32)]


P = ct.c_void_p
I = ct.c_int
U64 = ct.c_uint64
D = ct.c_double
SZ = ct.c_size_t
DP = ct.POINTER(ct.c_double)

# name -> argument types (all return int)
SIGNATURES = {
    "sch_create": [ct.POINTER(SchParams), ct.POINTER(P)],
    "sch_destroy": [P],
    "sch_layout": [P],
    "sch_noise_dim": [P],
    "sch_noise_form": [P],
    "sch_prior_exp1": [P, I, U64, I, P, P, P],
    "sch_u_from_m": [P, I, P, P, P],
    "sch_m_from_u": [P, I, P, P, P],
    "sch_draw_increments": [P, I, I, U64, U64, U64, I, P, P],
    "sch_ensemble_step": [P, I, I, P, P, P, P, P, P, P, P, P, P, P],
    "sch_loglik": [P, I, P, P, P, P, I, P, P, P],
    "pf_temper": [I, P, P, D, D, P, P, P],
    "pf_temper_halving": [I, P, P, D, D, P, P, P],
    "sch_synth_obs": [P, P, U64, U64, P, P],
    "pf_diagnostics": [P, I, P, P, P, P, P],
    "pf_resample": [I, P, U64, U64, P, I, P, P, P, SZ, P],
    "pf_gather_rows": [I, P, P, P, SZ, P],
    "pf_temper_dev": [I, P, P, P, D, I, P, P, P],
    "pf_resample_gated": [I, P, U64, U64, P, P, P],
    "pf_resample_static": [I, P, U64, U64, P, I, P, P, P],
    "pf_jitter": [P, I, I, I, D, D, U64, U64, P, P, P, P, P, P, P, P, P, P, P, P],
    "pf_jitter_dev": [P, I, I, I, P, D, U64, U64, P, P, P, P, P, P, P, P, P, P, P, P],
    "sch_set_jitter_workspace": [P, P, SZ],
    "pf_mala_propose": [P, I, I, D, D, U64, U64, I, P, P, P, P, P],
    "pf_mala_accept": [P, I, I, D, D, U64, U64, I, P, P, P, P, P, P, P, P, P],
    "pf_gated_stages": [P, I, I, I, I, D, I, D, I, U64, U64, P, P, P, P, P, P, P, P, P, P, P, P],
    "sch_prior_sample": [P, I, P, U64, D, P, P, P],
    "sch_adjoint_window": [P, I, I, I, P, P, P, P, P, P, P, P, P, P, P, SZ, P],
    "pf_nudge": [P, I, I, I, I, D, I, U64, U64, P, P, P, P, P, P, P, P, SZ, P],
    "nn_forward": [P, I, P, P, P, I, P, P, SZ, P],
    "nn_backward": [P, I, P, P, P, I, P, P, P, P, SZ, P],
    "nn_adam_step": [SZ, P, P, P, P, I, ct.c_float, ct.c_float, ct.c_float, ct.c_float, P],
}
RESTYPES = {"pf_resample_workspace_bytes": (SZ, [I, SZ]),
            "sch_adjoint_workspace_bytes": (SZ, [P, I, I, I]),
            "pf_nudge_workspace_bytes": (SZ, [P, I, I, I]),
            "sch_jitter_workspace_bytes": (SZ, [P, I, I]),
            "nn_param_count": (SZ, [P]),
            "nn_workspace_bytes": (SZ, [P, I])}

_LIB = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libsch.so not found at {LIB_PATH}: build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ct.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ct.c_int
        for name, (res, args) in RESTYPES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _LIB = L
    return _LIB


def check(rc: int, what: str) -> None:
    if rc != SCH_OK:
        raise RuntimeError(f"{what} failed: {ERRORS.get(rc, rc)}")
