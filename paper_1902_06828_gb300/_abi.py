"""ctypes declarations of include/te_ksg.h (argument marshalling only).

The shared library is built in-tree by paper_1902_06828_gb300.build; loading
fails loudly when it is missing.  There is no fallback of any kind.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

TE_OK, TE_EINVAL, TE_ENOMEM, TE_ECUDA, TE_ETIMEOUT, TE_ECANCELLED, TE_EBUSY, TE_EINTERNAL = (
    0, -1, -2, -3, -4, -5, -6, -7)
STATUS_NAMES = {0: "TE_OK", -1: "TE_EINVAL", -2: "TE_ENOMEM", -3: "TE_ECUDA", -4: "TE_ETIMEOUT",
                -5: "TE_ECANCELLED", -6: "TE_EBUSY", -7: "TE_EINTERNAL"}
TE_MAX_DIMS = 32
TE_MAX_K = 16


class TeVar(C.Structure):
    _fields_ = [("proc", C.c_int32), ("lag", C.c_int32)]


class KsgParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("theiler", C.c_int32), ("max_lag", C.c_int32),
                ("n_surr", C.c_int32), ("seed", C.c_uint64), ("stream_tag", C.c_uint64)]


class CmiJob(C.Structure):
    _fields_ = [("data", C.c_void_p), ("x", C.POINTER(TeVar)), ("y", C.POINTER(TeVar)),
                ("z", C.POINTER(TeVar)), ("dx", C.c_int32), ("dy", C.c_int32),
                ("dz", C.c_int32), ("params", KsgParams)]


class InferParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("theiler", C.c_int32), ("max_lag_target", C.c_int32),
                ("max_lag_sources", C.c_int32), ("n_surr", C.c_int32),
                ("alpha_max", C.c_double), ("alpha_min", C.c_double),
                ("alpha_omnibus", C.c_double), ("alpha_seq", C.c_double),
                ("seq_test", C.c_int32), ("fdr", C.c_int32), ("alpha_fdr", C.c_double),
                ("seed", C.c_uint64), ("targets", C.POINTER(C.c_int32)),
                ("n_targets", C.c_int32), ("indep_surr", C.c_int32), ("surr_mode", C.c_int32),
                ("estimator", C.c_int32)]


class TargetResult(C.Structure):
    _fields_ = [("target", C.c_int32), ("n_sel_target", C.c_int32),
                ("sel_target", C.POINTER(TeVar)), ("n_sel_sources", C.c_int32),
                ("sel_sources", C.POINTER(TeVar)), ("omnibus_cmi", C.c_double),
                ("omnibus_p", C.c_double), ("omnibus_tested", C.c_int32),
                ("significant", C.c_int32), ("n_estimates", C.c_uint64)]


class NetworkResult(C.Structure):
    _fields_ = [("n_proc", C.c_int32), ("n_targets", C.c_int32),
                ("targets", C.POINTER(TargetResult)), ("adjacency", C.POINTER(C.c_uint8)),
                ("min_lag", C.POINTER(C.c_int32)), ("n_estimates", C.c_uint64),
                ("seconds", C.c_double), ("theiler", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("estimates", C.c_uint64), ("launches", C.c_uint64), ("pair_evals", C.c_uint64),
                ("kernel_ms", C.c_double), ("ksg_launches", C.c_uint64),
                ("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64),
                ("pair_evals_bruteforce", C.c_uint64), ("ksg_ops", C.c_uint64)]


class ServeConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_inflight", C.c_int32),
                ("max_batch_jobs", C.c_int32)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("cancelled", C.c_uint64),
                ("batches", C.c_uint64), ("in_use_bytes", C.c_size_t), ("peak_bytes", C.c_size_t),
                ("pending", C.c_uint64)]


# te_ctx_set_option options (include/te_ksg.h)
OPTIONS = {"ksg_tile": 1, "ksg_members_per_lane": 2, "persistent": 3, "graph": 4, "ksg_order": 5}

# every symbol include/te_ksg.h declares: name -> (restype, argtypes)
_P = C.c_void_p
_I32 = C.c_int32
# te_trace_fn(user, target, stage, iter, vars, n_vars, n_cand, n_surr, keys)
TRACE_FN = C.CFUNCTYPE(None, _P, _I32, _I32, _I32, C.POINTER(TeVar), _I32, _I32, _I32,
                       C.POINTER(C.c_int64))
SIGNATURES = {
    "te_ctx_create": (C.c_int, [C.c_int, C.POINTER(_P)]),
    "te_ctx_set_stream": (C.c_int, [_P, _P]),
    "te_ctx_destroy": (None, [_P]),
    "te_last_error": (C.c_char_p, [_P]),
    "te_data_create": (C.c_int, [_P, _P, _I32, _I32, C.c_int, C.POINTER(_P)]),
    "te_data_destroy": (None, [_P]),
    "cmi_ksg": (C.c_int, [_P, _P, C.POINTER(TeVar), _I32, C.POINTER(TeVar), _I32,
                          C.POINTER(TeVar), _I32, C.POINTER(KsgParams), _P, _P]),
    "cmi_ksg_debug": (C.c_int, [_P, _P, C.POINTER(TeVar), _I32, C.POINTER(TeVar), _I32,
                                C.POINTER(TeVar), _I32, C.POINTER(KsgParams), _I32, _P, _P, _P,
                                _P]),
    "cmi_ksg_batch": (C.c_int, [_P, C.POINTER(CmiJob), _I32, _P, _P]),
    "cmi_gauss": (C.c_int, [_P, _P, C.POINTER(TeVar), _I32, C.POINTER(TeVar), _I32,
                            C.POINTER(TeVar), _I32, C.POINTER(KsgParams), _P, _P]),
    "te_network_infer": (C.c_int, [_P, _P, C.POINTER(InferParams),
                                   C.POINTER(C.POINTER(NetworkResult))]),
    "te_network_result_free": (None, [C.POINTER(NetworkResult)]),
    "te_ctx_set_trace": (C.c_int, [_P, TRACE_FN, _P]),
    "te_ctx_set_option": (C.c_int, [_P, _I32, C.c_int64]),
    "te_autocorr_decay": (C.c_int, [_P, _P, _I32, C.POINTER(C.c_int32)]),
    "te_alu_peak": (C.c_int, [_P, _I32, C.POINTER(C.c_double)]),
    "te_data_create_trials": (C.c_int, [_P, _P, _I32, _I32, _I32, _I32, C.c_int, _P]),
    "te_get_stats": (C.c_int, [_P, C.POINTER(Stats)]),
    "te_serve_start": (C.c_int, [_P, C.POINTER(ServeConfig)]),
    "te_serve_submit": (C.c_int, [_P, C.POINTER(CmiJob), C.POINTER(C.c_uint64)]),
    "te_serve_poll": (C.c_int, [_P, C.c_uint64, _I32, _P, _P]),
    "te_serve_cancel": (C.c_int, [_P, C.c_uint64]),
    "te_serve_stop": (C.c_int, [_P]),
    "te_serve_get_stats": (C.c_int, [_P, C.POINTER(ServeStats)]),
    "cmi_ksg_static": (C.c_int, [_P, _I32, _I32, C.POINTER(TeVar), _I32, C.POINTER(TeVar), _I32,
                                 C.POINTER(TeVar), _I32, C.POINTER(KsgParams), _P, _P, _P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libte_ksg.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and _build.stale():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libte_ksg.so is not built ({path}); run "
                           "python -c 'import __graft_entry__ as g; g.build()'")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
