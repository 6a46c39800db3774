"""ctypes view of the C ABI in include/ipanema.h (structs, enums, prototypes).

Loading fails loudly when libipanema.so has not been built: there is no CPU
fallback.  Build it with ``python -c "import __graft_entry__ as g; g.build()"``
or ``python paper_1706_01420_gb300/build.py``.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_size_t, c_uint64, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libipanema.so")

IPA_OK, IPA_ERR_ARG, IPA_ERR_OOM, IPA_ERR_CUDA, IPA_ERR_TIMEOUT, IPA_ERR_BUSY, IPA_PENDING = 0, -1, -2, -3, -4, -5, 1
IPA_MODEL_TIME1D, IPA_MODEL_ANGTIME4D, IPA_MODEL_TAGGED1D, IPA_MODEL_PHIS = 1, 2, 3, 4
IPA_GAMMA, IPA_SIGMA, IPA_MU, IPA_FB, IPA_A0SQ, IPA_APESQ, IPA_DPA, IPA_DPE, IPA_FS, IPA_DS = range(10)
IPA_DG, IPA_DM, IPA_PHIS, IPA_OMEGA = 4, 5, 6, 7
IPA_PHIS_DG, IPA_PHIS_DM, IPA_PHIS_PHIS, IPA_PHIS_OMEGA, IPA_PHIS_CSP, IPA_PHIS_QNORM = 10, 11, 12, 13, 14, 15
IPA_NPAR_1D, IPA_NPAR_4D, IPA_NPAR_TAGGED, IPA_NPAR_PHIS, IPA_MAX_PAR = 4, 10, 8, 16, 32
IPA_NOALLOC_MAX_EVENTS = 8388608
IPA_SHARD_EVENTS = 16384
IPA_FAULT_ALLOC, IPA_FAULT_SUBMIT, IPA_FAULT_ADMIT = 1, 2, 4
IPA_MATH_EXP, IPA_MATH_LOG, IPA_MATH_SIN, IPA_MATH_COS, IPA_MATH_ERFCX, IPA_MATH_RCP = range(6)
IPA_FIT_CONVERGED, IPA_FIT_MAXITER, IPA_FIT_AT_LIMIT, IPA_FIT_BAD_PDF, IPA_FIT_EMPTY = range(5)
(IPA_MINOS_OK, IPA_MINOS_MAXROUNDS, IPA_MINOS_AT_LIMIT, IPA_MINOS_FIT_FAILED, IPA_MINOS_NEW_MINIMUM,
 IPA_MINOS_NOT_SCANNED) = range(6)
STATUS_NAMES = {0: "IPA_OK", -1: "IPA_ERR_ARG", -2: "IPA_ERR_OOM", -3: "IPA_ERR_CUDA",
                -4: "IPA_ERR_TIMEOUT", -5: "IPA_ERR_BUSY", 1: "IPA_PENDING"}


class ipa_model(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("n_par", c_int32), ("t_lo", c_double), ("t_hi", c_double)]


class ipa_events(ctypes.Structure):
    _fields_ = [("n", c_int64), ("t", c_void_p), ("ck", c_void_p), ("cl", c_void_p),
                ("phi", c_void_p), ("w", c_void_p), ("fk", c_void_p), ("fk_stride", c_int64), ("q", c_void_p)]


class ipa_event_buffers(ctypes.Structure):
    _fields_ = [("capacity", c_int64), ("t", c_void_p), ("ck", c_void_p), ("cl", c_void_p),
                ("phi", c_void_p), ("q", c_void_p)]


class ipa_param(ctypes.Structure):
    _fields_ = [("value", c_double), ("lo", c_double), ("hi", c_double), ("step", c_double),
                ("fixed", c_int32), ("_pad", c_int32)]


class ipa_joint(ctypes.Structure):
    _fields_ = [("n_cat", c_int32), ("n_joint", c_int32), ("map", c_void_p), ("value", c_void_p)]


class ipa_launch_config(ctypes.Structure):
    _fields_ = [("warps_per_block", c_int32), ("warps_per_sm", c_int32), ("tiles_per_take", c_int32),
                ("ms", ctypes.c_float)]


# name -> (restype, argtypes); every function declared in include/ipanema.h
PROTOTYPES = {
    "ipa_model_init": (c_int32, [POINTER(ipa_model), c_int32, c_double, c_double]),
    "ipa_nll": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_void_p, c_void_p]),
    "ipa_nll_grad": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_void_p, c_void_p]),
    "ipa_nll_grad_host": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_void_p, c_void_p]),
    "ipa_nll_grad_segmented": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_int32,
                                         c_void_p, c_void_p, c_void_p]),
    "ipa_angular_basis": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_int64, c_void_p]),
    "ipa_toygen": (c_int32, [POINTER(ipa_model), c_void_p, c_uint64, c_int32, c_void_p, c_void_p,
                             c_void_p, POINTER(ipa_event_buffers), c_void_p]),
    "ipa_fit_batch": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_int32,
                                POINTER(ipa_param), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_int32, c_double, c_void_p]),
    "ipa_nll_grad_joint": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_int32, POINTER(ipa_joint),
                                     c_void_p, c_void_p, c_void_p]),
    "ipa_fit_joint": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_int32, POINTER(ipa_joint),
                                POINTER(ipa_param), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_int32, c_double, c_void_p]),
    "ipa_hesse_joint": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_int32, POINTER(ipa_joint),
                                  POINTER(ipa_param), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ipa_hesse": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_int32, POINTER(ipa_param),
                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ipa_minos": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_int32, POINTER(ipa_param),
                            c_void_p, c_void_p, c_void_p, POINTER(c_int32), c_double, c_double, c_int32, c_int32,
                            c_double, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ipa_minos_joint": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_int32, POINTER(ipa_joint),
                                  POINTER(ipa_param), c_void_p, c_void_p, c_void_p, POINTER(c_int32), c_double,
                                  c_double, c_int32, c_int32, c_double, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ipa_binned_generate": (c_int32, [c_void_p, c_int64, c_uint64, c_int32, c_int32, c_int32, c_void_p, c_void_p]),
    "ipa_binned_smear": (c_int32, [c_void_p, c_int64, c_double, c_double, c_void_p, c_void_p]),
    "ipa_cls": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_int32, c_uint64, c_void_p, c_void_p, c_void_p,
                          c_void_p]),
    "ipa_nll_grad_noalloc": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_void_p, c_void_p]),
    "ipa_server_create": (c_int32, [POINTER(ipa_model), c_size_t, c_int32, c_int32, c_double,
                                    POINTER(c_void_p)]),
    "ipa_serve_submit": (c_int32, [c_void_p, POINTER(ipa_events), POINTER(ipa_param), POINTER(c_uint64)]),
    "ipa_serve_poll": (c_int32, [c_void_p, c_uint64, POINTER(c_double), POINTER(c_double), POINTER(c_double),
                                 POINTER(c_int32)]),
    "ipa_server_destroy": (c_int32, [c_void_p]),
    "ipa_reserve": (c_int32, [c_int64, c_int32]),
    "ipa_fit_state_bytes": (c_uint64, [c_int32, c_int32]),
    "ipa_fit_begin": (c_int32, [POINTER(ipa_model), POINTER(ipa_param), c_int32, c_void_p, c_int32, c_double,
                                c_void_p, c_void_p]),
    "ipa_fit_advance": (c_int32, [POINTER(ipa_model), c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ipa_fit_end": (c_int32, [POINTER(ipa_model), c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_void_p, c_void_p]),
    "ipa_shard_width": (c_int32, [POINTER(ipa_model), POINTER(c_int32)]),
    "ipa_nll_grad_shard": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_void_p, c_void_p,
                                     c_void_p]),
    "ipa_nll_grad_combine": (c_int32, [POINTER(ipa_model), c_void_p, c_void_p, c_int64, c_int32, c_void_p,
                                       c_void_p]),
    "ipa_scratch_bytes": (c_int32, [POINTER(c_uint64)]),
    "ipa_fault_inject": (ctypes.c_uint32, [ctypes.c_uint32]),
    "ipa_autotune": (c_int32, [POINTER(ipa_model), POINTER(ipa_events), c_void_p, c_int32, c_void_p, c_int32,
                               POINTER(ipa_launch_config), c_void_p]),
    "ipa_launch_config_get": (c_int32, [POINTER(ipa_model), c_int64, c_int32, c_int32, c_int32,
                                        POINTER(ipa_launch_config)]),
    "ipa_launch_config_set": (c_int32, [POINTER(ipa_model), c_int64, c_int32, c_int32, c_int32,
                                        POINTER(ipa_launch_config)]),
    "ipa_calibrate_fp64": (c_int32, [POINTER(c_double), c_void_p]),
    "ipa_math_eval": (c_int32, [c_int32, c_void_p, c_void_p, c_int64, c_void_p]),
    "ipa_faddeeva": (c_int32, [c_void_p, c_void_p, c_int64, c_void_p]),
    "ipa_last_error": (c_char_p, []),
    "ipa_version": (c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libipanema.so and attach the prototypes (cached)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(paper_1706_01420_gb300/build.py); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
