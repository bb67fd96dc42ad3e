"""Seeded synthetic workloads shaped like the paper's evaluation inputs.

The paper (Sec. 5) measures on yelp reviews and NYC taxi trips, which are not
available here; these generators write seeded stand-ins with the published
shape statistics.  The module formats values only and holds no parsing logic,
so both the CUDA path's tests/benchmark and the oracle's tests can use it.

Workloads (each names its DFA and schema by plain names; every side maps the
names onto its own tables):

* ``mixed``  -- RFC-4180 CSV, LF, 8 columns (int32, string, int64, float64,
  timestamp, string, timestamp, string); 30 % of strings quoted, of those
  20 % with ',', 5 % with a line break, 10 % with a doubled quote.
* ``trip``   -- trip-record CSV (NYC-taxi-like, 18 columns), CRLF, no quotes:
  2 timestamps, 4 int32 in [1, 300], 8 float64 with 2 decimals (log-normal,
  mean 15), a one-character flag and 3 short strings.
* ``review`` -- review CSV (yelp-like, 9 columns), LF: 3 ids of 22 characters,
  int32 stars in [1, 5], 3 int32 counts (geometric, p = 0.3), an always
  quoted text of log-normal length (mean 700 B; 40 % with ',', 25 % with line
  breaks, 8 % with doubled quotes), a date.
* ``log``    -- web-log lines (Common Log Format), 7 space-separated fields:
  IPv4, '-', user, [timestamp], "request", int32 status, int64 bytes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

WORKLOADS = {"mixed": 1, "trip": 2, "review": 3, "log": 4}

SCHEMAS = {
    "mixed": ["int32", "string", "int64", "float64", "timestamp", "string", "timestamp", "string"],
    "trip": ["int32", "timestamp", "timestamp", "int32", "float64", "int32", "string", "int32",
             "string", "string"] + ["float64"] * 7 + ["string"],
    "review": ["string", "string", "string", "int32", "int32", "int32", "int32", "string", "date"],
    "log": ["string", "string", "string", "timestamp_clf", "string", "int32", "int64"],
}

DIALECT = {"mixed": "csv", "trip": "csv", "review": "csv", "log": "log"}

BASE_SEED = 190513415


def library_path() -> str:
    return os.path.join(HERE, "libsynth.so")


def build(force: bool = False) -> str:
    out = library_path()
    src = os.path.join(HERE, "synth.c")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-Wall", "-o", tmp, src, "-lm", "-lpthread"])
    os.replace(tmp, out)
    return out


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(library_path()):
            build()
        L = ctypes.CDLL(library_path())
        L.synth_generate.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                     ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
        L.synth_generate.restype = ctypes.c_int64
        L.synth_records.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                                    ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
        L.synth_records.restype = ctypes.c_int
        L.synth_generate_batch.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_uint64, ctypes.c_void_p,
                                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.synth_generate_batch.restype = None
        _lib = L
    return _lib


def generate_into(workload: str, seed: int, target_len: int, ptr: int, cap: int,
                  threads: int | None = None):
    """Write the longest whole-record prefix of length <= target_len at host
    address ``ptr``; returns (length, rows)."""
    rows = ctypes.c_uint64(0)
    n = lib().synth_generate(WORKLOADS[workload], seed, target_len, ptr, cap,
                             threads or min(32, os.cpu_count() or 1), ctypes.byref(rows))
    if n < 0:
        raise ValueError("capacity too small")
    return int(n), int(rows.value)


def generate(workload: str, seed: int, target_len: int, threads: int | None = None) -> np.ndarray:
    buf = np.empty(target_len, np.uint8)
    n, _ = generate_into(workload, seed, target_len, buf.ctypes.data, target_len, threads)
    return buf[:n]


def records(workload: str, seed: int, row0: int, nrows: int):
    """(raw bytes, [[field bytes, ...], ...]) of records [row0, row0 + nrows)."""
    cap = max(4096, nrows * 4096)
    while True:
        raw = np.empty(cap, np.uint8)
        truth = np.empty(cap, np.uint8)
        rl, tl = ctypes.c_uint64(0), ctypes.c_uint64(0)
        rc = lib().synth_records(WORKLOADS[workload], seed, row0, nrows, raw.ctypes.data, cap,
                                 ctypes.byref(rl), truth.ctypes.data, cap, ctypes.byref(tl))
        if rc == 0:
            break
        cap = max(rl.value, tl.value) + 1
    t = bytes(truth[: tl.value])
    recs = [r.split(b"\x1f") for r in t.split(b"\x1e")[:-1]]
    return bytes(raw[: rl.value]), recs


def record_bytes(workload: str, seed: int, row0: int, nrows: int) -> np.ndarray:
    """The raw bytes of records [row0, row0 + nrows) alone (no truth
    returned); they equal that slice of the whole generated input."""
    cap = max(1 << 16, nrows * 2048)
    while True:
        raw = np.empty(cap, np.uint8)
        truth = np.empty(cap, np.uint8)
        rl, tl = ctypes.c_uint64(0), ctypes.c_uint64(0)
        rc = lib().synth_records(WORKLOADS[workload], seed, row0, nrows, raw.ctypes.data, cap,
                                 ctypes.byref(rl), truth.ctypes.data, cap, ctypes.byref(tl))
        if rc == 0:
            return raw[: rl.value]
        cap = max(rl.value, tl.value) + 1


def batch_plan(n: int, total: int, seed: int, lo: int = 1 << 10, hi: int = 64 << 20, sigma: float = 2.0):
    """Sizes and workloads of a batch: log-normal sizes clipped to [lo, hi] and
    rescaled so they sum to about `total`; half CSV ('mixed'), half web logs."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.normal(0.0, sigma, n))
    sizes = sizes / sizes.sum() * total
    for _ in range(20):  # clip, then rescale the unclipped part
        sizes = np.clip(sizes, lo, hi)
        free = (sizes > lo) & (sizes < hi)
        if not free.any():
            break
        fixed = sizes[~free].sum()
        sizes[free] *= max(total - fixed, 0) / max(sizes[free].sum(), 1)
    sizes = np.clip(sizes, lo, hi).astype(np.uint64)
    kinds = ["mixed" if i % 2 == 0 else "log" for i in range(n)]
    seeds = (seed * 1_000_003 + np.arange(n, dtype=np.uint64)).astype(np.uint64)
    return sizes, kinds, seeds


def generate_batch_into(kinds, seeds, targets, ptr: int, threads: int | None = None):
    """Generates every input of a batch at host address ptr, input i at the
    sum of the earlier targets.  Returns (offsets, lengths, rows)."""
    n = len(kinds)
    targets = np.asarray(targets, dtype=np.uint64)
    offsets = np.zeros(n, dtype=np.uint64)
    if n > 1:
        offsets[1:] = np.cumsum(targets)[:-1]
    wl = np.asarray([WORKLOADS[k] for k in kinds], dtype=np.int32)
    seeds = np.asarray(seeds, dtype=np.uint64)
    lens = np.zeros(n, dtype=np.uint64)
    rows = np.zeros(n, dtype=np.uint64)
    lib().synth_generate_batch(wl.ctypes.data, seeds.ctypes.data, targets.ctypes.data, offsets.ctypes.data, n,
                               ptr, lens.ctypes.data, rows.ctypes.data, threads or min(32, os.cpu_count() or 1))
    return offsets, lens, rows
