"""ctypes declarations of the C ABI in include/flare_gb.h.

Argument marshalling only: every computation happens in libflare_gb.so.
Importing this module loads the library and raises if it is missing; there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libflare_gb.so")

FLR_OK = 0
FLR_EINVAL = 1
FLR_ENOMEM = 2
FLR_ECUDA = 3
FLR_ENBR_OVERFLOW = 4
FLR_ETIMEOUT = 5
FLR_EBUDGET = 6
FLR_EDEVICE = 7
FLR_ENOMODEL = 8

PREC = {"fp32": 0, "tf32": 1, "bf16x3": 2}
VAR_MODE = {"auto": 0, "direct": 1, "factored": 2}

TOT_ENERGY = 0
TOT_VIRIAL = 1
TOT_MAX_SIGMA = 10
TOT_N_ISOLATED = 11
TOT_KINETIC = 12
TOT_N_REBUILDS = 13
TOT_N_VAR_FP64 = 14
NTOTALS = 24
TOT_N_UNCERTAIN = 15
TOT_N_CN = 16
TOT_THERMOSTAT = 17

EXPORTED = [
    "flr_last_error", "flr_version", "flr_create", "flr_destroy", "flr_descriptor_dims",
    "flr_set_precision", "flr_set_model", "flr_nbrlist_create", "flr_nbrlist_destroy",
    "flr_nbrlist_view", "flr_build_neighbors", "flr_compute_descriptors",
    "flr_energy_forces_uncertainty", "flr_md_step", "flr_sync", "flr_launch_count",
    "flr_profile_enable", "flr_profile_read", "flr_build_neighbors_noalloc",
    "flr_build_neighbors_batch", "flr_energy_forces_uncertainty_batch", "flr_energy_backward",
    "flr_bytes_per_atom", "flr_server_create", "flr_server_submit", "flr_server_poll", "flr_server_stats_read",
    "flr_server_destroy", "flr_set_variance_mode", "flr_map_sgp", "flr_fp32_fma_peak", "flr_set_option",
    "flr_md_step_host", "flr_host_join",
]

KERNEL_CLASSES = ["descriptor", "qform", "force", "finalize", "drift", "rebuild", "fused"]
OPT_FUSED_ONE_SPECIES = 1
OPT_OVERLAP_TWO_SPECIES = 2
REBUILD_KERNELS = 13   # FLR_REBUILD_KERNELS


class Params(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int32), ("n_max", ctypes.c_int32), ("l_max", ctypes.c_int32),
                ("max_nbr", ctypes.c_int32), ("r_cut", ctypes.c_double), ("skin", ctypes.c_double),
                ("precision", ctypes.c_int32), ("compaction", ctypes.c_int32)]


class System(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("pos", ctypes.c_void_p), ("species", ctypes.c_void_p),
                ("cell", ctypes.c_double * 9), ("pbc", ctypes.c_int32 * 3)]


class Batch(ctypes.Structure):
    _fields_ = [("n_structs", ctypes.c_int32), ("n_atoms", ctypes.c_int32), ("pos", ctypes.c_void_p),
                ("species", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("cells", ctypes.c_void_p),
                ("pbc", ctypes.c_void_p)]


class Outputs(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_void_p), ("forces", ctypes.c_void_p), ("variance", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("totals", ctypes.c_void_p)]


class MDState(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p),
                ("species", ctypes.c_void_p), ("cell", ctypes.c_double * 9), ("pbc", ctypes.c_int32 * 3),
                ("masses", ctypes.c_double * 8), ("dt", ctypes.c_double), ("rebuild_every", ctypes.c_int32),
                ("forces_valid", ctypes.c_int32), ("step", ctypes.c_int64), ("temperature", ctypes.c_double),
                ("tau", ctypes.c_double), ("xi", ctypes.c_double), ("eta", ctypes.c_double),
                ("sigma_stop", ctypes.c_double), ("halted", ctypes.c_int32), ("cn_species", ctypes.c_int32),
                ("cn_cutoff", ctypes.c_double)]


class HostState(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("energy", ctypes.c_void_p),
                ("forces", ctypes.c_void_p), ("variance", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("totals", ctypes.c_void_p)]


class ServerParams(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch_structs", ctypes.c_int32),
                ("max_batch_atoms", ctypes.c_int32), ("reserve_atoms", ctypes.c_int64),
                ("reserve_structs", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("pos", ctypes.c_void_p), ("species", ctypes.c_void_p),
                ("cell", ctypes.c_double * 9), ("pbc", ctypes.c_int32 * 3), ("energy", ctypes.c_void_p),
                ("forces", ctypes.c_void_p), ("variance", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("totals", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("batch_structs", ctypes.c_int32),
                ("batch_atoms", ctypes.c_int64), ("t_submit_ns", ctypes.c_int64), ("t_start_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64), ("slot", ctypes.c_int32), ("gpu_start_ms", ctypes.c_float),
                ("gpu_built_ms", ctypes.c_float), ("gpu_eval_start_ms", ctypes.c_float),
                ("gpu_eval_end_ms", ctypes.c_float), ("gpu_done_ms", ctypes.c_float)]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_int64), ("batches", ctypes.c_int64), ("atoms", ctypes.c_int64),
                ("max_batch_atoms_seen", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("reserved_bytes", ctypes.c_int64), ("bytes_per_atom", ctypes.c_int64),
                ("last_error", ctypes.c_char * 256), ("batches_overlapped", ctypes.c_int64),
                ("grow_events", ctypes.c_int64), ("grow_ms", ctypes.c_double), ("pack_ms", ctypes.c_double),
                ("enqueue_ms", ctypes.c_double), ("finish_ms", ctypes.c_double)]


class FlareError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"flare_gb error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libflare_gb.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing; run paper_2204_12573_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        sig = {
            "flr_last_error": (ctypes.c_char_p, []),
            "flr_version": (ctypes.c_char_p, []),
            "flr_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(P)]),
            "flr_destroy": (ctypes.c_int, [P]),
            "flr_descriptor_dims": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
            "flr_set_precision": (ctypes.c_int, [P, ctypes.c_int32]),
            "flr_set_option": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32]),
            "flr_set_variance_mode": (ctypes.c_int, [P, ctypes.c_int32]),
            "flr_set_model": (ctypes.c_int, [P, ctypes.c_int32, P, P]),
            "flr_map_sgp": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, P, P, P, ctypes.c_double, P, P, P]),
            "flr_nbrlist_create": (ctypes.c_int, [P, ctypes.c_int32, ctypes.POINTER(P)]),
            "flr_nbrlist_destroy": (ctypes.c_int, [P]),
            "flr_nbrlist_view": (ctypes.c_int, [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                                ctypes.POINTER(ctypes.c_int32)]),
            "flr_build_neighbors": (ctypes.c_int, [P, ctypes.POINTER(System), P, P]),
            "flr_compute_descriptors": (ctypes.c_int, [P, ctypes.POINTER(System), P, P, P, P]),
            "flr_energy_forces_uncertainty": (ctypes.c_int, [P, ctypes.POINTER(System), P, ctypes.POINTER(Outputs), P]),
            "flr_md_step": (ctypes.c_int, [P, ctypes.POINTER(MDState), P, ctypes.c_int32, ctypes.POINTER(Outputs), P]),
            "flr_md_step_host": (ctypes.c_int, [P, ctypes.POINTER(MDState), P, ctypes.c_int32,
                                                ctypes.POINTER(Outputs), ctypes.POINTER(HostState), P]),
            "flr_host_join": (ctypes.c_int, [P, P]),
            "flr_sync": (ctypes.c_int, [P, P]),
            "flr_launch_count": (ctypes.c_int64, [P]),
            "flr_profile_enable": (ctypes.c_int, [P, ctypes.c_int32]),
            "flr_build_neighbors_noalloc": (ctypes.c_int, [ctypes.POINTER(System), ctypes.c_double, ctypes.c_int32,
                                                           P, P, P]),
            "flr_build_neighbors_batch": (ctypes.c_int, [P, ctypes.POINTER(Batch), P, P]),
            "flr_energy_forces_uncertainty_batch": (ctypes.c_int, [P, ctypes.POINTER(Batch), P,
                                                                   ctypes.POINTER(Outputs), P]),
            "flr_energy_backward": (ctypes.c_int, [P, ctypes.POINTER(Batch), P, P, P, P, P]),
            "flr_bytes_per_atom": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64)]),
            "flr_server_create": (ctypes.c_int, [P, ctypes.POINTER(ServerParams), ctypes.POINTER(P)]),
            "flr_server_submit": (ctypes.c_int, [P, ctypes.POINTER(Request)]),
            "flr_server_poll": (ctypes.c_int, [P, ctypes.POINTER(Completion), ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_int32), ctypes.c_double]),
            "flr_server_stats_read": (ctypes.c_int, [P, ctypes.POINTER(ServerStats)]),
            "flr_server_destroy": (ctypes.c_int, [P]),
            "flr_profile_read": (ctypes.c_int, [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_int64)]),
            "flr_fp32_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != FLR_OK:
        raise FlareError(code, lib().flr_last_error().decode())
