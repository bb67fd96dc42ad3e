"""Selected columns (Sec. 4.3): a PP_SKIP column's fields count for the record
but nothing is converted or stored for it.  GPU against the oracle."""
from __future__ import annotations

import pytest

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


def _skip_every(schema, k, first):
    return ["skip" if (i - first) % k == 0 and i >= first else t for i, t in enumerate(schema)]


@pytest.mark.parametrize("cfg", [0, 1, 2])
@pytest.mark.parametrize("workload,nrows", [("mixed", 3000), ("trip", 3000), ("review", 300), ("log", 3000)])
def test_skipped_columns(pp, workload, nrows, cfg):
    raw, _ = synth.records(workload, 51, 0, nrows)
    schema = _skip_every(synth.SCHEMAS[workload], 3, 1)
    ref = oracle_parse(synth.DIALECT[workload], schema, raw)
    p = pp.Parser(pp.formats.by_name(synth.DIALECT[workload]), schema, tile_config=cfg)
    data = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to("cuda")
    out, res = p.parse(data)
    torch.cuda.synchronize()
    assert_same(out.to_host(res.rows), res, ref, what=f"{workload} cfg {cfg}")


def test_skipped_column_missing_from_short_records(pp):
    schema = ["int32", "string", "skip", "float64", "skip"]
    raw = b"1,a,x,1.5,y\n2,b\n3,c,z\n4,d,w,2.25,v\n5\n" * 700
    ref = oracle_parse("csv", schema, raw)
    assert ref.n_rejected == 3 * 700
    p = pp.Parser(pp.formats.rfc4180_csv(), schema, tile_config=1)
    data = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to("cuda")
    out, res = p.parse(data)
    torch.cuda.synchronize()
    assert_same(out.to_host(res.rows), res, ref, what="short records")
