"""ParPaRaw ORACLE -- test infrastructure only.

A plain sequential CPU parser (``ppo.c``) plus this ctypes wrapper.  It
restates what the ParPaRaw method computes (Stehle & Jacobsen, Sec. 3): the
DFA-driven parse of delimiter-separated bytes into Arrow-like columns, the
per-chunk state-transition vectors and their composite (Sec. 3.1), and the
type conversion of field values (Sec. 3.3).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import this package.  It
shares no code with the CUDA path and imports nothing from it.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build import build as _build, library_path

MAX_STATES = 8
MAX_GROUPS = 16
MAX_COLUMNS = 64
NO_STATE = 0xFF

DATA, FIELD, RECORD, CONTROL = 0, 1, 2, 3
STRING, INT32, INT64, FLOAT64, TIMESTAMP_S, DATE_D, TIMESTAMP_CLF, SKIP = range(8)
OK, E_INVALID_INPUT, E_UNTERMINATED = 0, -4, -5
CONV_OK, CONV_EMPTY, CONV_FAIL = 0, 1, 2


class _Format(ctypes.Structure):
    _fields_ = [
        ("num_states", ctypes.c_uint32),
        ("num_groups", ctypes.c_uint32),
        ("next", (ctypes.c_uint8 * MAX_STATES) * MAX_GROUPS),
        ("emit", (ctypes.c_uint8 * MAX_STATES) * MAX_GROUPS),
        ("group_of", ctypes.c_uint8 * 256),
        ("start_state", ctypes.c_uint8),
        ("invalid_state", ctypes.c_uint8),
        ("accept_mask", ctypes.c_uint32),
        ("catch_all", ctypes.c_uint8),
        ("unit", ctypes.c_uint8),
    ]


class _Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("final_state", ctypes.c_int32),
        ("rows", ctypes.c_int64),
        ("n_rejected", ctypes.c_int64),
        ("first_invalid_offset", ctypes.c_int64),
        ("num_columns", ctypes.c_uint32),
        ("types", ctypes.c_uint32 * MAX_COLUMNS),
        ("values", ctypes.c_void_p * MAX_COLUMNS),
        ("offsets", ctypes.POINTER(ctypes.c_int64) * MAX_COLUMNS),
        ("validity", ctypes.POINTER(ctypes.c_uint8) * MAX_COLUMNS),
        ("bytes_total", ctypes.c_int64 * MAX_COLUMNS),
        ("row_valid", ctypes.POINTER(ctypes.c_uint8)),
    ]


class _Inference(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("min_fields", ctypes.c_uint32),
        ("max_fields", ctypes.c_uint32),
        ("records", ctypes.c_int64),
        ("first_invalid_offset", ctypes.c_int64),
        ("type", ctypes.c_uint8 * MAX_COLUMNS),
    ]


NO_TYPE = 0xFF
INFER_MAX_FIELDS = 256

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            _build()
        L = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        L.ppo_format_init.argtypes = [ctypes.POINTER(_Format), ctypes.c_uint32, ctypes.c_uint32,
                                      u8p, u8p, ctypes.c_uint32, u8p, u8p, ctypes.c_uint8,
                                      ctypes.c_uint8, ctypes.c_uint8, ctypes.c_uint32]
        L.ppo_format_init.restype = ctypes.c_int
        L.ppo_state_vector.argtypes = [ctypes.POINTER(_Format), ctypes.c_void_p, ctypes.c_size_t, u8p]
        L.ppo_state_vector_at.argtypes = [ctypes.POINTER(_Format), ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_size_t, ctypes.c_size_t, u8p]
        L.ppo_format_set_utf16le.argtypes = [ctypes.POINTER(_Format)]
        L.ppo_format_set_utf16le.restype = None
        L.ppo_compose.argtypes = [ctypes.c_uint32, u8p, u8p, u8p]
        L.ppo_trace.argtypes = [ctypes.POINTER(_Format), ctypes.c_void_p, ctypes.c_size_t,
                                ctypes.c_void_p, ctypes.c_void_p]
        L.ppo_parse.argtypes = [ctypes.POINTER(_Format), ctypes.POINTER(ctypes.c_uint32),
                                ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t,
                                ctypes.POINTER(_Result)]
        L.ppo_parse.restype = ctypes.c_int
        L.ppo_parse_skip.argtypes = [ctypes.POINTER(_Format), ctypes.POINTER(ctypes.c_uint32),
                                     ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64,
                                     ctypes.POINTER(_Result)]
        L.ppo_parse_skip.restype = ctypes.c_int
        L.ppo_free.argtypes = [ctypes.POINTER(_Result)]
        L.ppo_convert.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
        L.ppo_convert.restype = ctypes.c_int
        L.ppo_infer.argtypes = [ctypes.POINTER(_Format), ctypes.c_void_p, ctypes.c_size_t,
                                ctypes.POINTER(_Inference)]
        L.ppo_infer.restype = ctypes.c_int
        L.ppo_infer_skip.argtypes = [ctypes.POINTER(_Format), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64,
                                     ctypes.POINTER(_Inference)]
        L.ppo_infer_skip.restype = ctypes.c_int
        L.ppo_skip_rows.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                                    ctypes.c_uint8, ctypes.c_void_p]
        L.ppo_skip_rows.restype = ctypes.c_size_t
        _lib = L
    return _lib


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


@dataclass
class Format:
    """A DFA over symbol groups (Sec. 3.1, Table 1): ``next[g][s]``,
    ``emit[g][s]`` (tag of the symbol read in state s), symbol -> group map."""

    num_states: int
    num_groups: int
    next: np.ndarray           # [G][S] uint8
    emit: np.ndarray           # [G][S] uint8
    symbols: bytes
    groups: list
    catch_all: int
    start_state: int
    invalid_state: int
    accept_mask: int
    utf16le: bool = False  # Sec. 4.2: read UTF-16LE code units (surrogate pairs as one symbol)

    def __post_init__(self):
        self._c = _Format()
        nxt, pn = _u8(np.asarray(self.next).reshape(-1))
        emt, pe = _u8(np.asarray(self.emit).reshape(-1))
        sym, ps = _u8(np.frombuffer(bytes(self.symbols), dtype=np.uint8))
        grp, pg = _u8(np.asarray(self.groups, dtype=np.uint8))
        rc = lib().ppo_format_init(ctypes.byref(self._c), self.num_states, self.num_groups, pn, pe,
                                   len(sym), ps, pg, self.catch_all, self.start_state,
                                   self.invalid_state, self.accept_mask)
        if rc != 0:
            raise ValueError("malformed DFA tables")
        if self.utf16le:
            lib().ppo_format_set_utf16le(ctypes.byref(self._c))

    def as_utf16le(self) -> "Format":
        """The same DFA reading UTF-16LE code units (Sec. 4.2)."""
        return Format(self.num_states, self.num_groups, self.next, self.emit, self.symbols, self.groups,
                      self.catch_all, self.start_state, self.invalid_state, self.accept_mask, True)

    def group_of(self, b: int) -> int:
        return int(self._c.group_of[b])


def _tables(S, G, rows):
    nxt = np.zeros((G, S), np.uint8)
    emt = np.zeros((G, S), np.uint8)
    for g, row in enumerate(rows):
        for s, (n, t) in enumerate(row):
            nxt[g, s], emt[g, s] = n, t
    return nxt, emt


# RFC-4180 CSV: the six states and four symbol groups of Table 1, plus a
# carriage-return group (a reading: CR is a control symbol outside quotes
# and data inside them, and never changes the state).
EOR, ENC, FLD, EOF_, ESC, INV = range(6)
_D, _F, _R, _C = DATA, FIELD, RECORD, CONTROL


def csv6() -> Format:
    rows = [
        # group 0: '\n'
        [(EOR, _R), (ENC, _D), (EOR, _R), (EOR, _R), (EOR, _R), (INV, _C)],
        # group 1: '"'
        [(ENC, _C), (ESC, _C), (INV, _C), (ENC, _C), (ENC, _D), (INV, _C)],
        # group 2: ','
        [(EOF_, _F), (ENC, _D), (EOF_, _F), (EOF_, _F), (EOF_, _F), (INV, _C)],
        # group 3: '\r'
        [(EOR, _C), (ENC, _D), (FLD, _C), (EOF_, _C), (ESC, _C), (INV, _C)],
        # group 4: catch-all
        [(FLD, _D), (ENC, _D), (FLD, _D), (FLD, _D), (INV, _C), (INV, _C)],
    ]
    nxt, emt = _tables(6, 5, rows)
    accept = (1 << EOR) | (1 << FLD) | (1 << EOF_) | (1 << ESC)
    return Format(6, 5, nxt, emt, b"\n\",\r", [0, 1, 2, 3], 4, EOR, INV, accept)


# Space-delimited web-log lines (Common Log Format style): brackets and
# double quotes enclose fields that may contain spaces.
L_EOR, L_EOF, L_FLD, L_QUO, L_QCL, L_BRK, L_BCL, L_INV = range(8)


def log8() -> Format:
    I = (L_INV, _C)

    def row_for(state):
        # returns [(next, tag)] for groups '\n', ' ', '"', '[', ']', catch-all
        if state in (L_EOR, L_EOF):
            return [(L_EOR, _R), (L_EOF, _F), (L_QUO, _C), (L_BRK, _C), I, (L_FLD, _D)]
        if state == L_FLD:
            return [(L_EOR, _R), (L_EOF, _F), I, I, I, (L_FLD, _D)]
        if state == L_QUO:
            return [(L_QUO, _D), (L_QUO, _D), (L_QCL, _C), (L_QUO, _D), (L_QUO, _D), (L_QUO, _D)]
        if state in (L_QCL, L_BCL):
            return [(L_EOR, _R), (L_EOF, _F), I, I, I, I]
        if state == L_BRK:
            return [I, (L_BRK, _D), (L_BRK, _D), (L_BRK, _D), (L_BCL, _C), (L_BRK, _D)]
        return [I] * 6

    per_state = [row_for(s) for s in range(8)]
    rows = [[per_state[s][g] for s in range(8)] for g in range(6)]
    nxt, emt = _tables(8, 6, rows)
    accept = (1 << L_EOR) | (1 << L_EOF) | (1 << L_FLD) | (1 << L_QCL) | (1 << L_BCL)
    return Format(8, 6, nxt, emt, b"\n \"[]", [0, 1, 2, 3, 4], 5, L_EOR, L_INV, accept)


# -------------------------------------------------------------- Sec. 3.1

def state_vector(fmt: Format, chunk: bytes) -> np.ndarray:
    out = np.zeros(MAX_STATES, np.uint8)
    buf = np.frombuffer(bytes(chunk), dtype=np.uint8)
    lib().ppo_state_vector(ctypes.byref(fmt._c), buf.ctypes.data, len(buf),
                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return out[: fmt.num_states].copy()


def state_vector_at(fmt: Format, data: bytes, begin: int, end: int) -> np.ndarray:
    """Vector of the chunk data[begin:end] of a whole input (Sec. 4.2: the
    symbols that start in the chunk)."""
    out = np.zeros(MAX_STATES, np.uint8)
    buf = np.frombuffer(bytes(data), dtype=np.uint8)
    lib().ppo_state_vector_at(ctypes.byref(fmt._c), buf.ctypes.data, len(buf), begin, end,
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return out[: fmt.num_states].copy()


def compose(a, b) -> np.ndarray:
    a, pa = _u8(a)
    b, pb = _u8(b)
    out = np.zeros(len(a), np.uint8)
    lib().ppo_compose(len(a), pa, pb, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return out


def trace(fmt: Format, data: bytes):
    buf = np.frombuffer(bytes(data), dtype=np.uint8)
    tags = np.zeros(len(buf), np.uint8)
    states = np.zeros(len(buf), np.uint8)
    lib().ppo_trace(ctypes.byref(fmt._c), buf.ctypes.data, len(buf), tags.ctypes.data,
                    states.ctypes.data)
    return tags, states


# -------------------------------------------------------------- Sec. 3.3

_NP_TYPE = {INT32: np.int32, DATE_D: np.int32, INT64: np.int64, TIMESTAMP_S: np.int64,
            TIMESTAMP_CLF: np.int64, FLOAT64: np.float64}


def convert(type_: int, text: bytes):
    """(status, value) for one field's data bytes."""
    out = ctypes.c_uint64(0)
    t = bytes(text)
    st = lib().ppo_convert(type_, t, len(t), ctypes.byref(out))
    raw = np.array([out.value], np.uint64)
    if type_ in (INT32, DATE_D):
        v = int(raw.view(np.int32)[0])
    elif type_ == FLOAT64:
        v = float(raw.view(np.float64)[0])
    else:
        v = int(raw.view(np.int64)[0])
    return st, v


@dataclass
class Column:
    type: int
    values: np.ndarray          # uint8 bytes (STRING) or fixed-width values
    offsets: np.ndarray | None  # int64[rows+1] (STRING)
    validity: np.ndarray        # uint8 bitmap, (rows+7)//8 bytes
    bytes_total: int


@dataclass
class ParseResult:
    status: int
    final_state: int
    rows: int
    n_rejected: int
    first_invalid_offset: int
    columns: list
    row_valid: np.ndarray

    def field(self, r: int, c: int):
        col = self.columns[c]
        if col.type == STRING:
            return bytes(col.values[col.offsets[r]: col.offsets[r + 1]])
        return col.values[r].item()

    def valid(self, r: int, c: int) -> bool:
        return bool((self.columns[c].validity[r >> 3] >> (r & 7)) & 1)


def parse(fmt: Format, types, data, skip_records: int = 0) -> ParseResult:
    types_arr = (ctypes.c_uint32 * len(types))(*types)
    buf = np.frombuffer(data, dtype=np.uint8) if not isinstance(data, np.ndarray) else data
    res = _Result()
    rc = lib().ppo_parse_skip(ctypes.byref(fmt._c), types_arr, len(types), buf.ctypes.data, len(buf),
                              skip_records, ctypes.byref(res))
    if rc != 0:
        raise ValueError("bad schema")
    try:
        R = res.rows
        nbits = (R + 7) // 8
        cols = []
        for c, t in enumerate(types):
            validity = np.ctypeslib.as_array(res.validity[c], shape=(max(nbits, 1),))[:nbits].copy()
            if t == STRING:
                offs = np.ctypeslib.as_array(res.offsets[c], shape=(R + 1,)).copy()
                nb = int(res.bytes_total[c])
                if nb > 0:
                    vals = np.ctypeslib.as_array(
                        ctypes.cast(res.values[c], ctypes.POINTER(ctypes.c_uint8)), shape=(nb,)).copy()
                else:
                    vals = np.zeros(0, np.uint8)
                cols.append(Column(t, vals, offs, validity, nb))
            elif t == SKIP:  # a column that is not selected: nothing is kept
                cols.append(Column(t, np.zeros(0, np.uint8), None, np.zeros(0, np.uint8), 0))
            else:
                dt = _NP_TYPE[t]
                width = np.dtype(dt).itemsize
                if R > 0:
                    raw = ctypes.string_at(res.values[c], R * width)
                    vals = np.frombuffer(raw, dtype=dt).copy()
                else:
                    vals = np.zeros(0, dt)
                cols.append(Column(t, vals, None, validity, 0))
        row_valid = np.ctypeslib.as_array(res.row_valid, shape=(max(nbits, 1),))[:nbits].copy()
        return ParseResult(res.status, res.final_state, R, res.n_rejected,
                           res.first_invalid_offset, cols, row_valid)
    finally:
        lib().ppo_free(ctypes.byref(res))


@dataclass
class Inference:
    status: int
    min_fields: int
    max_fields: int
    records: int
    first_invalid_offset: int
    types: list  # per field position: INT32 / INT64 / FLOAT64 / STRING, or NO_TYPE


def infer(fmt: Format, data, skip_records: int = 0) -> Inference:
    """Sec. 4.3: column-count and numeric type inference (see ppo_infer),
    over all but the first ``skip_records`` records."""
    buf = np.frombuffer(data, dtype=np.uint8) if not isinstance(data, np.ndarray) else data
    r = _Inference()
    lib().ppo_infer_skip(ctypes.byref(fmt._c), buf.ctypes.data, len(buf), ctypes.c_uint64(skip_records),
                         ctypes.byref(r))
    return Inference(r.status, r.min_fields, r.max_fields, r.records, r.first_invalid_offset, list(r.type))


def skip_rows(data, rows, terminator: int = 0x0A) -> bytes:
    """Sec. 4.3, skipping rows (see ppo_skip_rows): the input without the
    physical lines listed in ``rows`` (sorted, distinct)."""
    buf = np.frombuffer(bytes(data), dtype=np.uint8)
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.uint64))
    out = np.empty(max(len(buf), 1), np.uint8)
    n = lib().ppo_skip_rows(buf.ctypes.data, len(buf), r.ctypes.data, len(r), terminator, out.ctypes.data)
    return out[:n].tobytes()
