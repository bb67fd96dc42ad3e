"""Shared helpers for the GPU parity tests: run a parse through the C ABI
and compare it element by element with the oracle."""
from __future__ import annotations

import numpy as np

import oracle as O

OTYPE = {"string": O.STRING, "int32": O.INT32, "int64": O.INT64, "float64": O.FLOAT64,
         "timestamp": O.TIMESTAMP_S, "date": O.DATE_D, "timestamp_clf": O.TIMESTAMP_CLF, "skip": O.SKIP}


def oracle_format(name: str):
    return O.csv6() if name == "csv" else O.log8()


def oracle_parse(dialect: str, schema, raw: bytes, skip_records: int = 0):
    return O.parse(oracle_format(dialect), [OTYPE[t] if isinstance(t, str) else t for t in schema], raw,
                   skip_records=skip_records)


def assert_same(got_host: dict, res, ref, rows_cap: int | None = None, what=""):
    """Every output of the GPU parse equals the oracle's: status, counts,
    offsets, value bytes, fixed-width values, validity and row_valid."""
    assert res.status == ref.status, (what, res, ref.status)
    assert res.rows == ref.rows, (what, res.rows, ref.rows)
    assert res.first_invalid_offset == ref.first_invalid_offset, (what, res.first_invalid_offset,
                                                                  ref.first_invalid_offset)
    assert res.final_state == ref.final_state, (what, res.final_state, ref.final_state)
    rows = ref.rows if rows_cap is None else min(ref.rows, rows_cap)
    if rows_cap is None or ref.rows <= rows_cap:
        assert res.n_rejected == ref.n_rejected, (what, res.n_rejected, ref.n_rejected)
    nb = (rows + 7) // 8
    for c, col in enumerate(ref.columns):
        g = got_host["columns"][c]
        if col.type == O.SKIP:  # not selected: the GPU stores nothing either
            assert g["values"] is None and g["validity"] is None, (what, c)
            continue
        if col.offsets is not None:
            assert res.values_bytes_needed[c] == col.bytes_total, (what, c)
            assert np.array_equal(g["offsets"][: rows + 1], col.offsets[: rows + 1]), (what, c, "offsets")
            end = int(col.offsets[rows])
            assert np.array_equal(g["values"][:end], col.values[:end]), (what, c, "bytes")
        else:
            assert np.array_equal(g["values"][:rows].view(np.uint8), col.values[:rows].view(np.uint8)), \
                (what, c, "values", first_diff(g["values"][:rows], col.values[:rows]))
        assert np.array_equal(g["validity"][:nb], col.validity[:nb]), (what, c, "validity")
    assert np.array_equal(got_host["row_valid"][:nb], ref.row_valid[:nb]), (what, "row_valid")


def first_diff(a, b):
    idx = np.nonzero(a != b)[0]
    return None if len(idx) == 0 else (int(idx[0]), a[idx[0]], b[idx[0]])


def _bits(bm: np.ndarray, r0: int, r1: int) -> np.ndarray:
    """Bits [r0, r1) of an LSB-first bitmap, one uint8 per bit."""
    return np.unpackbits(bm, bitorder="little")[r0:r1]


def assert_rows_equal(out, r0: int, r1: int, ref, what=""):
    """Rows [r0, r1) of a device Output equal, element by element, the
    oracle's parse of exactly those records (string offsets compared relative
    to the first row's; validity and row_valid bit by bit)."""
    import torch

    n = r1 - r0
    assert ref.rows == n, (what, ref.rows, n)
    b0, b1 = r0 // 8, (r1 + 7) // 8
    for c, col in enumerate(ref.columns):
        if col.type == O.SKIP:
            continue
        if col.offsets is not None:
            offs = out.offsets[c][r0: r1 + 1].cpu().numpy()
            assert np.array_equal(offs - offs[0], col.offsets[: n + 1]), (what, c, "offsets")
            vals = out.values[c][int(offs[0]): int(offs[-1])].cpu().numpy()
            assert np.array_equal(vals, col.values[: int(col.offsets[n])]), (what, c, "bytes")
        else:
            got = out.values[c][r0:r1].cpu().numpy()
            assert np.array_equal(got.view(np.uint8), col.values[:n].view(np.uint8)), \
                (what, c, "values", first_diff(got, col.values[:n]))
        vb = out.validity[c][b0:b1].cpu().numpy()
        assert np.array_equal(_bits(vb, r0 - 8 * b0, r1 - 8 * b0), _bits(col.validity, 0, n)), (what, c, "validity")
    rv = out.row_valid[b0:b1].cpu().numpy()
    assert np.array_equal(_bits(rv, r0 - 8 * b0, r1 - 8 * b0), _bits(ref.row_valid, 0, n)), (what, "row_valid")
    torch.cuda.synchronize()
