"""ctypes declarations of libfst.so (the C ABI in include/fst.h).

Loading fails loudly when the library has not been built: there is no CPU
fallback behind this binding.
"""
from __future__ import annotations

import ctypes
import os
import threading

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfst.so")

FST_OK = 0
STATUS_NAMES = {
    0: "FST_OK", -1: "FST_ERR_INVALID_ARG", -2: "FST_ERR_TOPOLOGY", -3: "FST_ERR_INERTIA",
    -4: "FST_ERR_UNSUPPORTED", -5: "FST_ERR_CUDA", -6: "FST_ERR_NO_MEMORY", -7: "FST_ERR_DEVICE_CHECK",
}
MAX_BODIES = 64
MAX_LINKS = 16
VARIANTS = {"auto": 0, "generic": 1, "specialized": 2, "level": 3, "mixed": 4, "path": 5, "pathwarp": 6, "pinned": 7,
            "level2": 8, "levellean": 9}
SPEC_KINDS = ("fk", "jacobian", "rnea", "crba", "aba", "eval", "fk_vjp", "rnea_vjp", "aba_vjp", "loss_grad",
              "eval_mixed", "rnea_store", "rnea_vjp_stored", "rnea_derivatives", "aba_derivatives")

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
c_float_p = ctypes.POINTER(ctypes.c_float)


class BodyDesc(ctypes.Structure):
    """fst_body_desc: one row of the body table."""
    _fields_ = [
        ("parent", c_int32),
        ("type", c_int32),
        ("axis", c_double * 3),
        ("T_joint", c_double * 12),
        ("T_link", c_double * 12),
        ("mass", c_double),
        ("com", c_double * 3),
        ("I_com", c_double * 6),
    ]


class FstError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class EvalIO(ctypes.Structure):
    """fst_eval_io: inputs and requested outputs of one fused evaluation."""
    _fields_ = [
        ("q", c_void_p), ("qd", c_void_p), ("qdd", c_void_p), ("tau", c_void_p),
        ("poses", c_void_p), ("J", c_void_p), ("links", ctypes.POINTER(c_int32)), ("n_links", c_int32),
        ("tau_out", c_void_p), ("M", c_void_p), ("qdd_out", c_void_p),
        ("tau_bar", c_void_p), ("q_bar", c_void_p), ("qd_bar", c_void_p), ("qdd_bar", c_void_p),
        ("flags", ctypes.c_uint32),
    ]


EVAL_ONE_SWEEP = 1     # FST_EVAL_ONE_SWEEP
EVAL_PACKED = 2        # FST_EVAL_PACKED


class MultiIO(ctypes.Structure):
    """fst_multi_io: one tree's inputs and requested outputs in a mixed batch."""
    _fields_ = [("B", c_int64), ("q", c_void_p), ("qd", c_void_p), ("qdd", c_void_p), ("tau", c_void_p),
                ("poses", c_void_p), ("tau_out", c_void_p), ("M", c_void_p), ("qdd_out", c_void_p)]


# (name, restype, argtypes); pointers to device memory travel as c_void_p
_SIGS = {
    "fst_model_create": (c_int32, [ctypes.POINTER(BodyDesc), c_int32, ctypes.POINTER(c_double), ctypes.POINTER(c_void_p)]),
    "fst_model_destroy": (c_int32, [c_void_p]),
    "fst_model_info": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                 ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
    "fst_model_specialize": (c_int32, [c_void_p, ctypes.c_uint32]),
    "fst_model_specialized": (c_int32, [c_void_p, ctypes.POINTER(ctypes.c_uint32)]),
    "fst_model_set_launch": (c_int32, [c_void_p, ctypes.c_uint32, c_int32, c_int32]),
    "fst_set_smem_carveout": (c_int32, [c_int32]),
    "fst_model_theta": (c_int32, [c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "fst_fk": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "fst_jacobian": (c_int32, [c_void_p, c_int64, c_void_p, ctypes.POINTER(c_int32), c_int32, c_void_p, c_void_p]),
    "fst_rnea": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "fst_crba": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "fst_aba": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "fst_eval": (c_int32, [c_void_p, c_int64, ctypes.POINTER(EvalIO), c_void_p, c_void_p]),
    "fst_adjoint_scratch_bytes": (c_int32, [c_void_p, c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "fst_fk_vjp": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "fst_rnea_vjp": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_size_t, c_void_p]),
    "fst_rnea_tape_bytes": (c_int32, [c_void_p, c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "fst_rnea_store": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 ctypes.c_size_t, c_void_p]),
    "fst_rnea_vjp_stored": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_size_t,
                                      c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_size_t,
                                      c_void_p]),
    "fst_model_set_sm_roles": (c_int32, [c_void_p, ctypes.POINTER(c_int32), c_int32]),
    "fst_jacobian_vjp": (c_int32, [c_void_p, c_int64, c_void_p, ctypes.POINTER(c_int32), c_int32, c_void_p, c_void_p,
                                   c_void_p]),
    "fst_crba_vjp": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                               ctypes.c_size_t, c_void_p]),
    "fst_rnea_derivatives": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p]),
    "fst_aba_derivatives": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_void_p]),
    "fst_aba_vjp": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_size_t, c_void_p]),
    "fst_rnea_loss_grad": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, ctypes.c_size_t, c_void_p]),
    "fst_rnea_vjp_noalloc": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_void_p, c_void_p]),
    "fst_multi_create": (c_int32, [ctypes.POINTER(c_void_p), c_int32, ctypes.POINTER(c_void_p)]),
    "fst_multi_destroy": (c_int32, [c_void_p]),
    "fst_multi_eval": (c_int32, [c_void_p, ctypes.POINTER(MultiIO), c_void_p]),
    "fst_multi_set_launch": (c_int32, [c_void_p, c_int32, c_int32]),
    "fst_packed_layout": (c_int32, [c_void_p, ctypes.POINTER(c_int32), c_int32, ctypes.POINTER(c_int32),
                                    ctypes.POINTER(c_int32), ctypes.POINTER(c_int32)]),
    "fst_fp32_probe": (c_int32, [c_int32, c_int32, c_void_p, ctypes.c_size_t, ctypes.POINTER(c_double), c_void_p]),
    "fst_sm_ids": (c_int32, [ctypes.POINTER(c_int32), c_int32, ctypes.POINTER(c_int32)]),
    "fst_device_can_access": (c_int32, [c_void_p, ctypes.POINTER(c_int32)]),
    "fst_sm_partition_create": (c_int32, [c_int32, ctypes.POINTER(c_int32), c_int32, ctypes.POINTER(c_void_p)]),
    "fst_sm_partition_info": (c_int32, [c_void_p, c_int32, ctypes.POINTER(c_void_p), ctypes.POINTER(c_int32)]),
    "fst_sm_partition_destroy": (c_int32, [c_void_p]),
    "fst_last_error": (ctypes.c_char_p, []),
    "fst_version": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def exported_names():
    return list(_SIGS)


def lib():
    """The loaded library (ImportError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing: build it with `python -m paper_2605_31481_gb300.build` "
                    "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int):
    if status != FST_OK:
        raise FstError(status, lib().fst_last_error().decode(errors="replace"))
