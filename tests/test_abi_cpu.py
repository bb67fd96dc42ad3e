"""The C-ABI library builds, loads and exports every entry point that
include/parparaw.h declares; create() validates tables on the host (no GPU
needed); the package's format tables agree with the oracle's."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_1905_13415_gb300 import build

    build.build()
    from paper_1905_13415_gb300 import _abi

    return _abi


def declared_entry_points():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            names |= set(re.findall(r"\b(parparaw_\w+)\s*\(", open(os.path.join(inc, f)).read()))
    return names


def test_exports_every_declared_symbol(abi):
    lib = abi.load()
    declared = declared_entry_points()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(abi.EXPORTED)


def test_header_constants_match_binding(abi):
    """The binding's copies of the header's numeric constants cannot drift."""
    text = open(os.path.join(ROOT, "include", "parparaw.h")).read()

    def define(name):
        m = re.search(r"#define\s+" + name + r"\s+\(?(\d+)u?\s*(?:<<\s*(\d+))?\)?", text)
        assert m, name
        return int(m.group(1)) << int(m.group(2) or 0)

    assert define("PP_NOALLOC_SCRATCH_BYTES") == abi.NOALLOC_SCRATCH_BYTES
    assert define("PP_INFER_MAX_FIELDS") == abi.INFER_MAX_FIELDS
    assert define("PP_MAX_COLUMNS") == abi.MAX_COLUMNS
    assert define("PP_MAX_STRING_COLUMNS") == abi.MAX_STRING_COLUMNS


def test_status_strings(abi):
    for code in range(-9, 1):
        assert abi.status_string(code) and abi.status_string(code) != "unknown status"
    assert abi.status_string(-42) == "unknown status"


def _create(abi, fmt, schema):
    from paper_1905_13415_gb300 import Parser

    return Parser(fmt, schema)


def test_create_and_info(abi):
    from paper_1905_13415_gb300 import formats

    p = _create(abi, formats.rfc4180_csv(), ["int32", "string", "float64", "string"])
    info = p.info()
    assert (info.num_states, info.num_groups, info.num_symbols) == (6, 5, 4)
    assert (info.num_columns, info.num_string_columns) == (4, 2)
    assert info.catch_all_idempotent == 1
    assert info.tile_bytes > 0 and info.threads_per_block > 0
    for cfg, tile in [(1, 512), (2, 3072), (3, 28672), (4, 26624)]:
        p.set_option(abi.OPT_TILE_CONFIG, cfg)
        assert p.info().tile_bytes == tile
    p.close()


def test_skip_records_option_bounds(abi):
    from paper_1905_13415_gb300 import ParparawError, formats

    p = _create(abi, formats.rfc4180_csv(), ["int32"])
    for ok in (0, 1, 2**32 - 1):
        p.set_option(abi.OPT_SKIP_RECORDS, ok)
        assert p.skip_records == ok
    for bad in (-1, 2**32):
        with pytest.raises(ParparawError):
            p.set_option(abi.OPT_SKIP_RECORDS, bad)
    assert p.skip_records == 2**32 - 1
    p.close()


def test_create_rejects_bad_tables(abi):
    from paper_1905_13415_gb300 import ParparawError, formats

    good = formats.rfc4180_csv()

    def variant(**kw):
        d = dict(name="x", transitions=good.transitions.copy(), emit=good.emit.copy(), symbols=good.symbols,
                 groups=list(good.groups), catch_all=good.catch_all, start_state=good.start_state,
                 invalid_state=good.invalid_state, accept_states=list(good.accept_states))
        d.update(kw)
        return formats.Format(**d)

    bad_next = good.transitions.copy()
    bad_next[0, 0] = 6
    not_absorbing = good.transitions.copy()
    not_absorbing[1, 5] = 0
    emits_in_inv = good.emit.copy()
    emits_in_inv[4, 5] = 0
    cases = [
        (variant(transitions=bad_next), ["string"], abi.E_BAD_TABLE),
        (variant(transitions=not_absorbing), ["string"], abi.E_BAD_TABLE),
        (variant(emit=emits_in_inv), ["string"], abi.E_BAD_TABLE),
        (variant(symbols=b'\n\n,\r', groups=[0, 1, 2, 3]), ["string"], abi.E_BAD_TABLE),
        (variant(groups=[0, 1, 2, 4]), ["string"], abi.E_BAD_TABLE),
        (variant(start_state=9), ["string"], abi.E_BAD_TABLE),
        (good, [99], abi.E_BAD_TABLE),
        (good, ["string"] * 17, abi.E_UNSUPPORTED),
        (good, ["int32"] * 65, abi.E_UNSUPPORTED),
    ]
    for fmt, schema, code in cases:
        with pytest.raises(ParparawError) as e:
            _create(abi, fmt, schema)
        assert e.value.code == code, (schema, code)


def test_non_idempotent_catch_all_is_flagged(abi):
    from paper_1905_13415_gb300 import formats

    tr = np.array([[0, 0], [1, 0]], np.uint8)  # catch-all toggles between two states
    em = np.zeros((2, 2), np.uint8)
    fmt = formats.Format("toggle", tr, em, b"\n", [0], 1, 0, 0xFF, [0, 1])
    assert _create(abi, fmt, ["string"]).info().catch_all_idempotent == 0


@pytest.mark.parametrize("name", ["csv", "log"])
def test_package_formats_match_oracle_formats(name):
    from paper_1905_13415_gb300 import formats

    f = formats.by_name(name)
    o = O.csv6() if name == "csv" else O.log8()
    assert f.num_states == o.num_states and f.num_groups == o.num_groups
    assert np.array_equal(f.transitions, o.next) and np.array_equal(f.emit, o.emit)
    assert f.start_state == o.start_state and f.invalid_state == o.invalid_state
    assert f.accept_mask == o.accept_mask
    for b in range(256):
        g = f.groups[f.symbols.index(bytes([b]))] if bytes([b]) in f.symbols else f.catch_all
        assert g == o.group_of(b)


def test_parse_rejects_bad_arguments_without_gpu(abi):
    from paper_1905_13415_gb300 import formats

    lib = abi.load()
    p = _create(abi, formats.rfc4180_csv(), ["string"])
    desc = abi.pp_columns()
    desc.num_columns = 2  # schema has one column
    rc = lib.parparaw_parse(p.handle, None, 0, ctypes.byref(desc), None)
    assert rc == abi.E_ARG
    rc = lib.parparaw_parse(None, None, 0, ctypes.byref(desc), None)
    assert rc == abi.E_ARG
    assert lib.parparaw_parse_batch(None, 1, None) == abi.E_ARG
    assert lib.parparaw_parse_batch(None, 0, None) == abi.OK


def test_skip_rows_rejects_bad_arguments_without_gpu(abi):
    lib = abi.load()
    need = lib.parparaw_skip_rows_scratch_bytes(100_000)
    assert need >= 24 * ((100_000 + 16383) // 16384)
    fake = 4096  # never dereferenced: every call below fails its argument checks first
    E = abi.E_ARG
    assert lib.parparaw_skip_rows(fake, 10, None, 0, 10, fake, None, fake, need, None) == E  # no output_len
    assert lib.parparaw_skip_rows(None, 10, None, 0, 10, fake, fake, fake, need, None) == E  # no input
    assert lib.parparaw_skip_rows(fake, 10, None, 3, 10, fake, fake, fake, need, None) == E  # rows missing
    assert lib.parparaw_skip_rows(fake, 100_000, None, 0, 10, fake, fake, fake, need - 1, None) == E  # scratch
    assert lib.parparaw_skip_rows(fake, 10, None, 0, 10, fake, fake, fake + 8, need, None) == E  # misaligned


ABI_STRUCTS = ["pp_dfa", "pp_symbol_groups", "pp_schema", "pp_column", "pp_parse_result", "pp_columns",
               "pp_batch_item", "pp_parser_info", "pp_host_partition", "pp_stream_result", "pp_inference"]


def test_binding_structs_match_the_header(tmp_path):
    """Size and field offsets of every struct the binding mirrors, as the C
    compiler lays them out from include/parparaw.h."""
    import ctypes
    import shutil
    import subprocess

    from paper_1905_13415_gb300 import _abi

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "parparaw.h"', "int main(void) {"]
    for name in ABI_STRUCTS:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(_abi, name)._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for name in ABI_STRUCTS:
        st = getattr(_abi, name)
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert got[(name, field)] == getattr(st, field).offset, (name, field)
