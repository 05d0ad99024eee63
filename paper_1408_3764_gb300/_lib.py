"""ctypes binding of the C ABI in include/gcmc.h (argument marshalling only).

Loads ``_build/libgcmc_gb300.so`` (building it with nvcc when missing).  There
is no fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

MAX_SPECIES = 8

GCMC_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CELL_OVERFLOW", 3: "CAPACITY", 4: "NONFINITE",
                5: "TIMEOUT", 6: "CUDA", 7: "STATE"}

FP64 = 0
FP32 = 1


class Params(C.Structure):
    _fields_ = [("L", C.c_double), ("rc", C.c_double), ("n_species", C.c_int32),
                ("precision", C.c_int32), ("eps", C.POINTER(C.c_double)),
                ("sigma", C.POINTER(C.c_double)), ("max_particles", C.c_int64),
                ("cell_capacity", C.c_int32), ("reserved", C.c_int32)]


MIX_VIRIAL = 1


class MoveMix(C.Structure):
    _fields_ = [("p_disp", C.c_double), ("p_ins", C.c_double), ("p_del", C.c_double),
                ("max_disp", C.c_double), ("beta", C.c_double),
                ("log_z", C.c_double * MAX_SPECIES), ("flags", C.c_int32), ("reserved", C.c_int32)]


class MoveStats(C.Structure):
    _fields_ = [("attempted", C.c_int64 * 3), ("accepted", C.c_int64 * 3), ("flagged", C.c_int64),
                ("moves_done", C.c_int64), ("energy", C.c_double), ("sum_energy", C.c_double),
                ("sum_n", C.c_double), ("n", C.c_int64 * MAX_SPECIES), ("virial", C.c_double),
                ("sum_virial", C.c_double), ("chain_ms", C.c_double)]


class Geometry(C.Structure):
    _fields_ = [("T", C.c_int64), ("n_cells", C.c_int64), ("cell_capacity", C.c_int64),
                ("max_particles", C.c_int64), ("cutoff_grid2", C.c_uint64), ("h", C.c_double)]


TRACE_BYTES = 32
CHAIN_CONFIGS = 4
NOALLOC_MAX_CELLS = 131072


class ProbeResult(C.Structure):
    _fields_ = [("l2_hop_ns", C.c_double), ("sync_round_ns", C.c_double), ("philox_ns", C.c_double),
                ("log_ns", C.c_double), ("floor_ns", C.c_double), ("working_set_bytes", C.c_int64)]

class PipePeaks(C.Structure):
    _fields_ = [("fp32_tflops", C.c_double), ("fp64_tflops", C.c_double), ("mufu_gops", C.c_double),
                ("sms", C.c_int32), ("reserved", C.c_int32)]


# every symbol include/gcmc.h declares, with (restype, argtypes)
_vp = C.c_void_p
SIGNATURES = {
    "gcmc_create": (C.c_int, [C.POINTER(Params), _vp, C.POINTER(_vp)]),
    "gcmc_destroy": (C.c_int, [_vp]),
    "gcmc_build_cells": (C.c_int, [_vp, _vp, _vp, C.c_int64]),
    "gcmc_cell_list": (C.c_int, [_vp, _vp, _vp, _vp]),
    "gcmc_export_positions": (C.c_int, [_vp, _vp, _vp, _vp]),
    "gcmc_trial_energy": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, _vp, _vp]),
    "gcmc_run_moves": (C.c_int, [_vp, C.c_uint64, C.c_uint64, C.c_int64, C.POINTER(MoveMix),
                                 C.POINTER(MoveStats), _vp]),
    "gcmc_check_state": (C.c_int, [_vp]),
    "gcmc_set_wait_limit": (C.c_int, [_vp, C.c_uint64, C.c_int64]),
    "gcmc_build_microcells": (C.c_int, [_vp, C.c_double, C.c_int32]),
    "gcmc_microcells": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "gcmc_run_moves_micro": (C.c_int, [_vp, C.c_uint64, C.c_uint64, C.c_int64, C.POINTER(MoveMix),
                                       C.POINTER(MoveStats), _vp]),
    "gcmc_total_energy": (C.c_int, [_vp, C.POINTER(C.c_double)]),
    "gcmc_total_energy_noalloc": (C.c_int, [_vp, _vp]),
    "gcmc_energy_grad": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "gcmc_counts": (C.c_int, [_vp, _vp]),
    "gcmc_get_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "gcmc_set_state": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_double]),
    "gcmc_get_geometry": (C.c_int, [_vp, C.POINTER(Geometry)]),
    "gcmc_kernel_launches": (C.c_int, [_vp, _vp]),
    "gcmc_chain_counters": (C.c_int, [_vp, _vp, _vp]),
    "gcmc_chain_profile": (C.c_int, [_vp, _vp]),
    "gcmc_set_chain_profile": (C.c_int, [_vp, C.c_int32]),
    "gcmc_set_chain_config": (C.c_int, [_vp, C.c_int32]),
    "gcmc_get_chain_config": (C.c_int, [_vp, _vp]),
    "gcmc_batch_create": (C.c_int, [_vp, C.c_int32, C.POINTER(_vp)]),
    "gcmc_batch_destroy": (C.c_int, [_vp]),
    "gcmc_batch_run_moves": (C.c_int, [_vp, _vp, C.c_uint64, C.c_int64, _vp, _vp]),
    "gcmc_batch_set_traces": (C.c_int, [_vp, _vp]),
    "gcmc_batch_prepare": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "gcmc_batch_energy_grad": (C.c_int, [_vp, _vp, _vp, _vp]),
    "gcmc_batch_export_positions": (C.c_int, [_vp, _vp, _vp, _vp]),
    "gcmc_batch_config": (C.c_int, [_vp, C.c_int32, _vp, _vp]),
    "gcmc_batch_launches": (C.c_int, [_vp, _vp]),
    "gcmc_batch_device_ms": (C.c_int, [_vp, C.POINTER(C.c_double)]),
    "gcmc_batch_last_error": (C.c_char_p, [_vp]),
    "gcmc_last_error": (C.c_char_p, [_vp]),
    "gcmc_version": (C.c_char_p, []),
    "gcmc_probe_latency": (C.c_int, [_vp, C.c_int64, C.POINTER(ProbeResult)]),
    "gcmc_probe_pipes": (C.c_int, [_vp, C.POINTER(PipePeaks)]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Returns the loaded library; raises when it cannot be built or loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("GB300 CUDA library missing: %s" % path)
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class GcmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


def check(status: int, ctx=None, what: str = ""):
    if status != GCMC_OK:
        msg = ""
        if ctx:
            msg = load().gcmc_last_error(ctx).decode(errors="replace")
        raise GcmcError(status, (what + " " + msg).strip())
