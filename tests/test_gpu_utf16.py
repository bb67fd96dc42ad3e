"""Variable-length symbols (Sec. 4.2): UTF-16LE inputs on the GPU against the
oracle's UTF-16LE parse, element by element, on tile shapes whose tile and
chunk boundaries fall inside surrogate pairs and between the bytes of code
units; the argument and format checks of the option; the streamed form."""
from __future__ import annotations

import random

import numpy as np
import pytest

import oracle as O
from parity import OTYPE, assert_same

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALPHABET = ["a", "b", "z", "1", " ", "é", "ß", "€", "漢", "字", "😀", "🚀", "𝄞"]


@pytest.fixture(scope="module")
def pp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1905_13415_gb300 as pkg

    return pkg


def csv_text(rng, records, bad=False):
    lines = []
    for _ in range(records):
        def text():
            s = "".join(rng.choice(ALPHABET) for _ in range(rng.randint(0, 40)))
            if rng.random() < 0.4:
                return '"' + s + rng.choice(["", ",", "\n", '""', "\r\n"]) + s[:3] + '"'
            return s
        lines.append(f"{rng.randint(-99, 9999)},{text()},{text()},{rng.randint(0, 999)}.{rng.randint(0, 99):02d}\r\n")
    t = "".join(lines)
    if bad:
        cut = rng.randrange(len(t))
        t = t[:cut] + 'q"' + t[cut:]
    return t


def dev(raw: bytes, offset: int = 0):
    buf = torch.zeros(len(raw) + offset + 16, dtype=torch.uint8)
    if raw:
        buf[offset: offset + len(raw)] = torch.frombuffer(bytearray(raw), dtype=torch.uint8)
    return buf.to("cuda")[offset: offset + len(raw)]


SCHEMA = ["int32", "string", "string", "float64"]


@pytest.mark.parametrize("cfg", [1, 2, 10])
def test_utf16_csv_against_the_oracle(pp, cfg):
    rng = random.Random(cfg)
    ofmt = O.csv6().as_utf16le()
    for it in range(12):
        raw = csv_text(rng, rng.randint(1, 160), bad=(it % 4 == 3)).encode("utf-16-le")
        p = pp.Parser(pp.formats.by_name("csv"), SCHEMA, tile_config=cfg, utf16le=True)
        out, res = p.parse(dev(raw, offset=2 * (it % 3)))
        torch.cuda.synchronize()
        ref = O.parse(ofmt, [OTYPE[t] for t in SCHEMA], raw)
        assert_same(out.to_host(res.rows), res, ref, what=(cfg, it))


def test_utf16_log_against_the_oracle(pp):
    import synth

    raw8, _ = synth.records("log", 77, 0, 300)
    raw = raw8.decode("ascii").replace("GET", "GÉT").replace("HEAD", "HEAD😀").encode("utf-16-le")
    schema = synth.SCHEMAS["log"]
    for cfg in (1, 2, 10):
        p = pp.Parser(pp.formats.by_name("log"), schema, tile_config=cfg, utf16le=True)
        out, res = p.parse(dev(raw))
        ref = O.parse(O.log8().as_utf16le(), [OTYPE[t] for t in schema], raw)
        assert ref.status == 0 and ref.rows == 300
        assert_same(out.to_host(res.rows), res, ref, what=cfg)


def test_utf16_arguments_and_formats(pp):
    from paper_1905_13415_gb300 import _abi

    p = pp.Parser(pp.formats.by_name("csv"), ["string"], utf16le=True)
    raw = "a,b\n".encode("utf-16-le")
    with pytest.raises(pp.ParparawError) as e:  # odd length
        p.parse_into(dev(raw + b"x"), p.allocate(4, 64))
    assert e.value.code == _abi.E_ARG
    with pytest.raises(pp.ParparawError) as e:  # odd address
        p.parse_into(dev(raw, offset=1), p.allocate(4, 64))
    assert e.value.code == _abi.E_ARG
    with pytest.raises(pp.ParparawError) as e:  # no inference for code units
        p.infer(dev(raw))
    assert e.value.code == _abi.E_UNSUPPORTED
    # a catch-all transition that changes the tag after one step cannot read
    # a surrogate pair as two code units
    tr = np.array([[0, 1], [1, 1]], np.uint8)
    em = np.array([[1, 1], [3, 0]], np.uint8)  # catch-all: CONTROL from 0, then DATA
    fmt = pp.formats.Format("odd", tr, em, b",", [0], 1, 0, 0xFF, [0, 1])
    q = pp.Parser(fmt, ["string"])
    with pytest.raises(pp.ParparawError) as e:
        q.set_option(_abi.OPT_UTF16LE, 1)
    assert e.value.code == _abi.E_UNSUPPORTED


def test_utf16_streamed_equals_whole(pp):
    from paper_1905_13415_gb300.stream import StreamParser

    rng = random.Random(5)
    raw = csv_text(rng, 400).encode("utf-16-le")
    p = pp.Parser(pp.formats.by_name("csv"), SCHEMA, tile_config=2, utf16le=True)
    ref = O.parse(O.csv6().as_utf16le(), [OTYPE[t] for t in SCHEMA], raw)
    host = torch.frombuffer(bytearray(raw), dtype=torch.uint8).pin_memory()
    parts = StreamParser(p, partition_bytes=12_000, carry_bytes=12_000).parse(host)
    assert len(parts) > 3 and sum(x.rows for x in parts) == ref.rows
    fields = []
    for x in parts:
        offs = x.columns[1]["offsets"][: x.rows + 1].numpy()
        vals = x.columns[1]["values"].numpy()
        fields += [bytes(vals[offs[i]:offs[i + 1]]) for i in range(x.rows)]
    assert fields == [ref.field(i, 1) for i in range(ref.rows)]
    nums = np.concatenate([x.columns[3]["values"][: x.rows].numpy() for x in parts])
    assert np.array_equal(nums.view(np.uint8), ref.columns[3].values.view(np.uint8))
