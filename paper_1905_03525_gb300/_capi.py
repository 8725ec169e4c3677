"""ctypes binding of librmat (include/rmat.h).  Argument marshalling only:
every step of generation runs in the library's CUDA kernels.  The library
must have been built (``python -m paper_1905_03525_gb300.build``); there is no
fallback of any kind when it is missing."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librmat.so")

RMAT_OK = 0
RMAT_ERR_INVALID_ARGUMENT = 1
RMAT_ERR_OUT_OF_MEMORY = 2
RMAT_ERR_CUDA = 3
RMAT_ERR_TIMEOUT = 4
RMAT_ERR_UNSUPPORTED = 5
RMAT_UNDIRECTED = 1

STATUS_NAMES = {0: "RMAT_OK", 1: "RMAT_ERR_INVALID_ARGUMENT", 2: "RMAT_ERR_OUT_OF_MEMORY",
                3: "RMAT_ERR_CUDA", 4: "RMAT_ERR_TIMEOUT", 5: "RMAT_ERR_UNSUPPORTED"}


class RmatError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class TableInfo(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("groups", ctypes.c_int), ("entries", ctypes.c_int),
                ("bits", ctypes.c_int), ("max_len", ctypes.c_int), ("index_bytes", ctypes.c_int),
                ("flags", ctypes.c_uint), ("device_image_bytes", ctypes.c_uint64), ("n0", ctypes.c_int)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("chunk_edges", ctypes.c_uint64),
                ("step_edges", ctypes.c_uint64), ("max_active", ctypes.c_int), ("wait_timeout_s", ctypes.c_double),
                ("gpu_build_min_bound", ctypes.c_uint64)]


class Request(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double), ("d", ctypes.c_double),
                ("k", ctypes.c_int), ("m", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("table_bound", ctypes.c_uint64), ("flags", ctypes.c_uint),
                ("scramble", ctypes.c_int), ("scramble_seed", ctypes.c_uint64)]


class RequestStatus(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("state", ctypes.c_int), ("edges_done", ctypes.c_uint64),
                ("checksum", ctypes.c_uint64), ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("error", ctypes.c_int), ("table_bound", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("edges", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("active", ctypes.c_uint64), ("memory_used", ctypes.c_uint64), ("clock_s", ctypes.c_double)]


CHUNK_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                            ctypes.c_void_p)


class LaunchConfig(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("tile_edges", ctypes.c_int)]


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) for every function of include/rmat.h
_vp, _u64, _i32, _u32, _dbl = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint, ctypes.c_double
_st = ctypes.c_int
SIGNATURES = [
    ("rmat_build_table", _st, [_dbl, _dbl, _dbl, _dbl, _i32, _u64, _vp]),
    ("rmat_build_table_fixed", _st, [_dbl, _dbl, _dbl, _dbl, _i32, _i32, _vp]),
    ("rmat_build_table_levels", _st, [_vp, _i32, _i32, _u32, _vp]),
    ("rmat_table_set_flags", _st, [_vp, _u32]),
    ("rmat_table_set_scramble", _st, [_vp, _i32, _u64]),
    ("rmat_build_table_gpu", _st, [_dbl, _dbl, _dbl, _dbl, _i32, _u64, _vp, _vp]),
    ("rmat_build_table_kron", _st, [_vp, _i32, _i32, _u64, _vp]),
    ("rmat_build_table_kron_fixed", _st, [_vp, _i32, _i32, _i32, _vp]),
    ("rmat_batch_add_tile", _st, [_vp, _vp, _u64, _u64, _u64, _i32, _u64, _u64, _vp]),
    ("rmat_partition_create", _st, [_vp, _i32, _u64, _u64, _u64, _u64, _vp]),
    ("rmat_partition_info", _st, [_vp, _vp, _vp]),
    ("rmat_partition_tiles", _st, [_vp, _vp, _vp, _vp, _vp]),
    ("rmat_generate_partition", _st, [_vp, _vp, _vp]),
    ("rmat_free_partition", None, [_vp]),
    ("rmat_dedup_edges", _st, [_vp, _u64, _i32, _vp, _vp]),
    ("rmat_dedup_release", _st, []),
    ("rmat_selftest_bounded_wait", _st, [_u32]),
    ("rmat_table_info", _st, [_vp, _vp]),
    ("rmat_table_group_info", _st, [_vp, _i32, _vp, _vp, _vp]),
    ("rmat_table_export", _st, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("rmat_table_upload", _st, [_vp]),
    ("rmat_free_table", None, [_vp]),
    ("rmat_generate", _st, [_vp, _u64, _u64, _u64, _vp, _vp]),
    ("rmat_generate_host", _st, [_vp, _u64, _u64, _u64, _vp, _vp]),
    ("rmat_generate_naive", _st, [_vp, _i32, _u32, _u64, _u64, _u64, _vp, _vp]),
    ("rmat_set_launch_config", _st, [_vp, _vp]),
    ("rmat_get_launch_config", _st, [_vp, _vp]),
    ("rmat_batch_create", _st, [_vp]),
    ("rmat_batch_add", _st, [_vp, _vp, _u64, _u64, _u64, _vp]),
    ("rmat_batch_prepare", _st, [_vp, _vp]),
    ("rmat_batch_launch", _st, [_vp, _vp]),
    ("rmat_batch_size", _st, [_vp, _vp, _vp]),
    ("rmat_batch_free", None, [_vp]),
    ("rmat_server_create", _st, [_vp, _vp]),
    ("rmat_server_set_chunk_callback", _st, [_vp, _vp, _vp]),
    ("rmat_server_submit", _st, [_vp, _vp, _vp]),
    ("rmat_server_status", _st, [_vp, _u64, _vp]),
    ("rmat_server_wait", _st, [_vp, _u64, _dbl, _vp]),
    ("rmat_server_drain", _st, [_vp, _dbl]),
    ("rmat_server_stats", _st, [_vp, _vp]),
    ("rmat_server_destroy", None, [_vp]),
    ("rmat_generate_batch_noalloc", _st, [_vp, _vp, _vp, _vp, _vp, ctypes.c_uint32, _vp]),
    ("rmat_check_device_errors", _st, []),
    ("rmat_version", ctypes.c_char_p, []),
    ("rmat_last_error", ctypes.c_char_p, []),
]


def lib() -> ctypes.CDLL:
    """Load librmat.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"librmat.so is not built ({LIB_PATH}); run "
                                  "`python -m paper_1905_03525_gb300.build` (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int) -> None:
    if status != RMAT_OK:
        msg = lib().rmat_last_error()
        raise RmatError(status, msg.decode() if msg else "")
