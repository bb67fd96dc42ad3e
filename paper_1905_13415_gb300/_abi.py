"""ctypes mirror of include/parparaw.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

MAX_STATES = 8
MAX_GROUPS = 16
MAX_SYMBOLS = 16
MAX_COLUMNS = 64
MAX_STRING_COLUMNS = 16

OK = 0
E_ARG, E_NOMEM, E_CUDA, E_INVALID_INPUT, E_UNTERMINATED = -1, -2, -3, -4, -5
E_CAPACITY, E_TIMEOUT, E_BAD_TABLE, E_UNSUPPORTED = -6, -7, -8, -9

STRING, INT32, INT64, FLOAT64, TIMESTAMP_S, DATE_D, TIMESTAMP_CLF, SKIP = range(8)
TYPE_NAMES = {"string": STRING, "int32": INT32, "int64": INT64, "float64": FLOAT64,
              "timestamp": TIMESTAMP_S, "date": DATE_D, "timestamp_clf": TIMESTAMP_CLF, "skip": SKIP}

OPT_TILE_CONFIG, OPT_TIMEOUT_MS, OPT_GRID_LIMIT, OPT_PARTIAL_INPUT, OPT_FIRST_ITEM, OPT_SKIP_RECORDS = 1, 2, 3, 4, 5, 6
OPT_UTF16LE = 7

EXPORTED = ["parparaw_create", "parparaw_destroy", "parparaw_set_option", "parparaw_get_info",
            "parparaw_parse", "parparaw_parse_batch", "parparaw_set_kernel_events",
            "parparaw_status_string", "parparaw_parse_noalloc", "parparaw_batch_create",
            "parparaw_batch_launch", "parparaw_batch_destroy", "parparaw_infer",
            "parparaw_skip_rows_scratch_bytes", "parparaw_skip_rows", "parparaw_stream_create",
            "parparaw_stream_parse", "parparaw_stream_destroy"]

NOALLOC_SCRATCH_BYTES = 32 << 20


class pp_dfa(ctypes.Structure):
    _fields_ = [("num_states", ctypes.c_uint32), ("num_groups", ctypes.c_uint32),
                ("transitions", ctypes.c_void_p), ("emit", ctypes.c_void_p),
                ("start_state", ctypes.c_uint8), ("invalid_state", ctypes.c_uint8),
                ("accept_mask", ctypes.c_uint32)]


class pp_symbol_groups(ctypes.Structure):
    _fields_ = [("num_symbols", ctypes.c_uint32), ("symbols", ctypes.c_void_p),
                ("groups", ctypes.c_void_p), ("catch_all", ctypes.c_uint8)]


class pp_schema(ctypes.Structure):
    _fields_ = [("num_columns", ctypes.c_uint32), ("types", ctypes.c_void_p)]


class pp_column(ctypes.Structure):
    _fields_ = [("values", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("validity", ctypes.c_void_p), ("values_cap", ctypes.c_uint64)]


class pp_parse_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("final_state", ctypes.c_int32),
                ("rows", ctypes.c_int64), ("n_rejected", ctypes.c_int64),
                ("first_invalid_offset", ctypes.c_int64), ("consumed", ctypes.c_int64),
                ("values_bytes_needed", ctypes.c_int64 * MAX_COLUMNS)]


class pp_columns(ctypes.Structure):
    _fields_ = [("num_columns", ctypes.c_uint32), ("rows_cap", ctypes.c_uint64),
                ("cols", pp_column * MAX_COLUMNS), ("row_valid", ctypes.c_void_p),
                ("result", ctypes.c_void_p)]


class pp_batch_item(ctypes.Structure):
    _fields_ = [("parser", ctypes.c_void_p), ("input", ctypes.c_void_p), ("len", ctypes.c_uint64),
                ("out", ctypes.POINTER(pp_columns))]


class pp_parser_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("num_states", "num_groups", "num_symbols", "num_columns", "num_string_columns",
                 "catch_all_idempotent", "tile_bytes", "threads_per_block")]


RESULT_BYTES = ctypes.sizeof(pp_parse_result)


class pp_host_partition(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("row0", ctypes.c_int64), ("input_offset", ctypes.c_uint64),
                ("input_bytes", ctypes.c_uint64), ("cols", pp_column * MAX_COLUMNS), ("row_valid", ctypes.c_void_p),
                ("h2d_ms", ctypes.c_float), ("parse_ms", ctypes.c_float), ("d2h_ms", ctypes.c_float)]


class pp_stream_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("num_partitions", ctypes.c_uint32), ("rows", ctypes.c_int64),
                ("n_rejected", ctypes.c_int64), ("first_invalid_offset", ctypes.c_int64),
                ("arena_bytes", ctypes.c_uint64)]

INFER_MAX_FIELDS = 256
TYPE_NONE = 0xFF


class pp_inference(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("min_fields", ctypes.c_uint32), ("max_fields", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("records", ctypes.c_int64), ("first_invalid_offset", ctypes.c_int64),
                ("type", ctypes.c_uint8 * 64)]


INFERENCE_BYTES = ctypes.sizeof(pp_inference)

_lib = None


def library_path() -> str:
    """The in-tree library; PARPARAW_LIBRARY may name a profiling build of it."""
    return os.environ.get("PARPARAW_LIBRARY") or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                                "libparparaw.so")


def load():
    """Loads the in-tree CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1905_13415_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    L.parparaw_create.argtypes = [ctypes.POINTER(pp_dfa), ctypes.POINTER(pp_symbol_groups),
                                  ctypes.POINTER(pp_schema), ctypes.POINTER(vp)]
    L.parparaw_create.restype = ctypes.c_int
    L.parparaw_destroy.argtypes = [vp]
    L.parparaw_destroy.restype = None
    L.parparaw_set_option.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
    L.parparaw_set_option.restype = ctypes.c_int
    L.parparaw_get_info.argtypes = [vp, ctypes.POINTER(pp_parser_info)]
    L.parparaw_get_info.restype = ctypes.c_int
    L.parparaw_parse.argtypes = [vp, vp, ctypes.c_uint64, ctypes.POINTER(pp_columns), vp]
    L.parparaw_parse.restype = ctypes.c_int
    L.parparaw_batch_create.argtypes = [ctypes.POINTER(pp_batch_item), ctypes.c_uint64, ctypes.POINTER(vp)]
    L.parparaw_batch_create.restype = ctypes.c_int
    L.parparaw_batch_launch.argtypes = [vp, vp]
    L.parparaw_batch_launch.restype = ctypes.c_int
    L.parparaw_batch_destroy.argtypes = [vp]
    L.parparaw_batch_destroy.restype = None
    L.parparaw_parse_noalloc.argtypes = [vp, vp, ctypes.c_uint64, ctypes.POINTER(pp_columns), vp]
    L.parparaw_parse_noalloc.restype = ctypes.c_int
    L.parparaw_parse_batch.argtypes = [ctypes.POINTER(pp_batch_item), ctypes.c_uint64, vp]
    L.parparaw_parse_batch.restype = ctypes.c_int
    L.parparaw_set_kernel_events.argtypes = [vp, vp, vp]
    L.parparaw_set_kernel_events.restype = ctypes.c_int
    L.parparaw_infer.argtypes = [vp, vp, ctypes.c_uint64, vp, vp]
    L.parparaw_infer.restype = ctypes.c_int
    L.parparaw_skip_rows_scratch_bytes.argtypes = [ctypes.c_uint64]
    L.parparaw_skip_rows_scratch_bytes.restype = ctypes.c_uint64
    L.parparaw_skip_rows.argtypes = [vp, ctypes.c_uint64, vp, ctypes.c_uint64, ctypes.c_uint8, vp, vp, vp,
                                     ctypes.c_uint64, vp]
    L.parparaw_skip_rows.restype = ctypes.c_int
    L.parparaw_stream_create.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(vp)]
    L.parparaw_stream_create.restype = ctypes.c_int
    L.parparaw_stream_parse.argtypes = [vp, vp, ctypes.c_uint64, vp, ctypes.c_uint64,
                                        ctypes.POINTER(pp_host_partition), ctypes.c_uint64,
                                        ctypes.POINTER(pp_stream_result)]
    L.parparaw_stream_parse.restype = ctypes.c_int
    L.parparaw_stream_destroy.argtypes = [vp]
    L.parparaw_stream_destroy.restype = None
    L.parparaw_status_string.argtypes = [ctypes.c_int]
    L.parparaw_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


def status_string(code: int) -> str:
    return load().parparaw_status_string(code).decode()
