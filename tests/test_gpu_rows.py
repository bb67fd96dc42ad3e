"""Skipping rows (Sec. 4.3) on the GPU against the oracle's pruning pass:
inputs spanning many 16 KiB chunks, random row lists, other terminators,
the edge cases, and a parse of what stays."""
from __future__ import annotations

import random

import numpy as np
import pytest

import oracle as O
import synth
from parity import assert_same, oracle_parse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1905_13415_gb300 as pkg

    return pkg


def _dev(raw: bytes):
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8).to("cuda") if raw else torch.empty(
        0, dtype=torch.uint8, device="cuda")


def _check(pp, raw: bytes, rows, term=b"\n"):
    got = pp.skip_rows(_dev(raw), rows, term).cpu().numpy().tobytes()
    want = O.skip_rows(raw, rows, term[0])
    assert got == want, (len(raw), rows[:10], len(got), len(want))


@pytest.mark.parametrize("raw,rows", [(b"", []), (b"", [0, 3]), (b"a", []), (b"a", [0]), (b"\n\n\n", [1]),
                                      (b"x\ny\nz", [2]), (b"x\ny\nz", [0, 1, 2]), (b"x\ny\n", [5, 9]),
                                      (b"h\n" + b"ab,c\n" * 10, [0])])
def test_edge_cases(pp, raw, rows):
    _check(pp, raw, rows)


def test_random_inputs_and_row_lists(pp):
    rng = random.Random(5)
    g = np.random.default_rng(5)
    for it in range(60):
        n = rng.choice([rng.randint(1, 3000), rng.randint(16000, 70000), rng.randint(100_000, 400_000)])
        density = rng.choice([0.002, 0.03, 0.3])
        b = g.integers(0x20, 0x7F, n, dtype=np.uint8)
        b[g.random(n) < density] = 0x0A
        raw = b.tobytes()
        nl = raw.count(b"\n") + 1
        k = rng.choice([0, 1, rng.randint(1, max(1, nl // 3)), nl])
        rows = sorted(rng.sample(range(nl + 2), min(k, nl + 2)))
        _check(pp, raw, rows)


def test_other_terminator_and_long_input(pp):
    raw, _ = synth.records("trip", 91, 0, 400_000)  # ~44 MB, CRLF lines
    nl = raw.count(b"\n")
    rows = list(range(0, nl, 3)) + [nl + 10]
    _check(pp, raw, rows)
    _check(pp, raw.replace(b"\r\n", b";"), [0, 1, 2, 1000, 1001], b";")


def test_parse_after_skipping_rows(pp):
    # comment lines and a header dropped as rows, then parsed, against the
    # oracle's parse of the oracle's pruned input
    body, _ = synth.records("mixed", 92, 0, 3000)
    raw = b"# exported\n# by a tool\nid,name,value,when,score,flag,text,day\n" + body
    schema = synth.SCHEMAS["mixed"]
    kept = pp.skip_rows(_dev(raw), [0, 1, 2])
    p = pp.Parser(pp.formats.by_name("csv"), schema, tile_config=2)
    out, res = p.parse(kept)
    torch.cuda.synchronize()
    ref = oracle_parse("csv", schema, O.skip_rows(raw, [0, 1, 2]))
    assert ref.rows == 3000
    assert_same(out.to_host(res.rows), res, ref, what="rows 0-2 skipped")


def test_unsorted_rows_are_refused(pp):
    with pytest.raises(pp.ParparawError):
        pp.skip_rows(_dev(b"a\nb\n"), [1, 0])


@pytest.mark.parametrize("offset", [1, 3, 7, 13, 15])
def test_unaligned_input(pp, offset):
    # the input starting anywhere in a 16-byte block, ends ragged
    g = np.random.default_rng(offset)
    b = g.integers(0x20, 0x7F, 50_000 + offset, dtype=np.uint8)
    b[g.random(b.size) < 0.05] = 0x0A
    raw = b.tobytes()
    dev = torch.frombuffer(bytearray(b"\0" * offset + raw), dtype=torch.uint8).to("cuda")[offset:]
    nl = raw.count(b"\n") + 1
    for rows in ([], [0], list(range(0, nl, 7)), [nl - 1], list(range(nl))):
        got = pp.skip_rows(dev, rows).cpu().numpy().tobytes()
        assert got == O.skip_rows(raw, rows), (offset, len(rows))
