"""Column-count and numeric type inference (Sec. 4.3) on the GPU against the
oracle's (ppo_infer): status, records, fewest / most fields per record and
the type of every field position."""
from __future__ import annotations

import random

import numpy as np
import pytest

import oracle as O
import synth

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


def _check(pp, dialect: str, raw: bytes, what: str):
    fmt = O.csv6() if dialect == "csv" else O.log8()
    ref = O.infer(fmt, raw)
    p = pp.Parser(pp.formats.by_name(dialect), ["string"])  # the schema is ignored
    got = p.infer(_dev(raw))
    assert (got.status, got.records, got.min_fields, got.max_fields) == \
        (ref.status, ref.records, ref.min_fields, ref.max_fields), (what, got, ref)
    if ref.status == O.OK:
        assert got.types == ref.types, (what, got.types[:20], ref.types[:20])
    return got


@pytest.mark.parametrize("raw", [b"1,2.5,x\n3,4,y\n", b"1\n2,3\n", b"2147483648,1\n", b"-5,,abc\n",
                                 b"1.5e3,007\n", b"99999999999999999999,1\n", b'"12",""\n', b"a,b", b"",
                                 b'"abc', b'a"b,c\n'])
def test_worked_examples(pp, raw):
    _check(pp, "csv", raw, raw)


@pytest.mark.parametrize("workload,nrows", [("mixed", 20000), ("trip", 20000), ("review", 2000), ("log", 20000)])
def test_generated_workloads(pp, workload, nrows):
    raw, _ = synth.records(workload, 43, 0, nrows)
    got = _check(pp, synth.DIALECT[workload], raw, workload)
    assert got.min_fields == got.max_fields == len(synth.SCHEMAS[workload])


def test_ragged_records_across_tiles(pp):
    # records of 1..80 fields with numbers of every width, long ones crossing
    # tile boundaries, quoted numbers and empty fields
    rng = random.Random(9)
    recs = []
    for i in range(40000):
        n = rng.randint(1, 80)
        f = []
        for c in range(n):
            k = rng.random()
            if k < 0.3:
                f.append(str(rng.randint(-2**31, 2**31 - 1)))
            elif k < 0.4:
                f.append(str(rng.randint(-2**62, 2**62)))
            elif k < 0.55:
                f.append(f"{rng.randint(0, 10**9)}.{rng.randint(0, 99):02d}")
            elif k < 0.65:
                f.append('"' + str(rng.randint(0, 999)) + '"')
            elif k < 0.75:
                f.append("")
            else:
                f.append("".join(rng.choice("abcxyz0123") for _ in range(rng.randint(1, 12))))
        recs.append(",".join(f))
    raw = ("\n".join(recs) + "\n").encode()
    got = _check(pp, "csv", raw, "ragged")
    assert got.min_fields == 1 and got.max_fields == 80


def test_wide_records_and_long_numbers(pp):
    wide = b",".join(b"%d" % i for i in range(500)) + b"\n"
    raw = b"1,2\n" * 3000 + wide + b"9" * 40000 + b",x\n" + b"3,4\n" * 3000
    got = _check(pp, "csv", raw, "wide")
    assert got.max_fields == O.INFER_MAX_FIELDS and got.types[0] == O.STRING
