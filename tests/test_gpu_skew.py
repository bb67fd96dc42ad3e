"""Skewed inputs (Sec. 5.1 runs one record of 200 MB): records and fields
that span many tiles, a record with far more fields than the schema, and a
tile-sized numeric field.  The whole output is compared with the oracle."""
from __future__ import annotations

import numpy as np
import pytest

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


def _text(n: int, seed: int) -> bytes:
    """n bytes of quoted-field content: words, commas, line breaks, doubled quotes."""
    rng = np.random.default_rng(seed)
    alphabet = np.frombuffer(b"abcdefghij klmnop,qrstu\nvwxyz ", dtype=np.uint8)
    body = alphabet[rng.integers(0, len(alphabet), n)].copy()
    q = rng.choice(n - 1, size=max(1, n // 5000), replace=False)
    body[q] = ord('"')
    out = body.tobytes().replace(b'"', b'""')  # escaped quotes
    return out


def _parse(pp, raw: bytes, schema, cfg=0):
    p = pp.Parser(pp.formats.rfc4180_csv(), schema, tile_config=cfg)
    data = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to("cuda")
    out, res = p.parse(data)
    torch.cuda.synchronize()
    return out.to_host(min(res.rows, out.rows_cap)), res


@pytest.mark.parametrize("cfg", [0, 11, 2])
def test_one_huge_quoted_field(pp, cfg):
    schema = ["int32", "string", "int64"]
    big = _text(64 << 20, 1)
    raw = b"1,a,2\n" * 1000 + b'7,"' + big + b'",9\n' + b"3,b,4\n" * 1000
    ref = oracle_parse("csv", schema, raw)
    assert ref.rows == 2001 and ref.status == 0
    got, res = _parse(pp, raw, schema, cfg)
    assert_same(got, res, ref, what=f"huge field, cfg {cfg}")


def test_record_with_many_fields(pp):
    schema = ["int32", "string", "int32"]
    wide = b",".join(b"%d" % i for i in range(100_000)) + b"\n"
    raw = b"1,x,2\n" * 500 + wide + b"3,y,4\n" * 500 + wide[:-1]  # also a trailing record without \n
    ref = oracle_parse("csv", schema, raw)
    assert ref.rows == 1002 and ref.n_rejected == 2
    got, res = _parse(pp, raw, schema)
    assert_same(got, res, ref, what="many fields")


def test_tile_sized_numeric_field(pp):
    schema = ["int64", "string"]
    raw = b"1,a\n" + b"9" * 40_000 + b",b\n" + b"2,c\n"  # an overlong number: rejected record
    ref = oracle_parse("csv", schema, raw)
    got, res = _parse(pp, raw, schema)
    assert_same(got, res, ref, what="long numeric")
    assert res.n_rejected == 1


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_utf8_text_across_tiles(pp, cfg):
    # Sec. 4.2: multi-byte symbols at chunk boundaries.  With ASCII delimiters a
    # UTF-8 continuation byte (0b10xxxxxx) never matches a symbol, so fields of
    # multi-byte characters cut anywhere by tiles and chunks come out unchanged.
    rng = np.random.default_rng(5)
    words = ["naïve", "Straße", "日本語", "😀", "Ελλάδα", "coöperate", "ça", "€100"]
    recs = []
    for i in range(3000):
        t = " ".join(words[j] for j in rng.integers(0, len(words), rng.integers(1, 30)))
        q = '"' + t.replace('"', '""') + ',"' if i % 3 == 0 else t.replace(",", " ")
        recs.append(f"{i},{q if i % 3 else chr(34) + t + chr(34)},{t.split()[0]}\n")
    raw = "".join(recs).encode("utf-8")
    schema = ["int32", "string", "string"]
    ref = oracle_parse("csv", schema, raw)
    assert ref.rows == 3000 and ref.n_rejected == 0
    got, res = _parse(pp, raw, schema, cfg)
    assert_same(got, res, ref, what=f"utf-8, cfg {cfg}")
    assert bytes(got["columns"][1]["values"]).decode("utf-8")  # whole characters only
