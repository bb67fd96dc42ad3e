"""DFA formats for the parser (Sec. 3.1; Sec. 4.5, Table 1).

A format is a DFA over symbol groups: ``transitions[g][s]`` is the state after
reading a symbol of group ``g`` in state ``s`` and ``emit[g][s]`` the tag that
symbol receives (data, field delimiter, record delimiter, control).  Symbols
not listed belong to the catch-all group.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TAG_DATA, TAG_FIELD, TAG_RECORD, TAG_CONTROL = 0, 1, 2, 3
NO_STATE = 0xFF


@dataclass
class Format:
    name: str
    transitions: np.ndarray  # uint8 [G][S]
    emit: np.ndarray         # uint8 [G][S]
    symbols: bytes
    groups: list
    catch_all: int
    start_state: int
    invalid_state: int
    accept_states: list = field(default_factory=list)

    @property
    def num_states(self) -> int:
        return int(self.transitions.shape[1])

    @property
    def num_groups(self) -> int:
        return int(self.transitions.shape[0])

    @property
    def accept_mask(self) -> int:
        return sum(1 << s for s in self.accept_states)


def _build(rows):
    G, S = len(rows), len(rows[0])
    tr = np.array([[n for n, _ in r] for r in rows], np.uint8).reshape(G, S)
    em = np.array([[t for _, t in r] for r in rows], np.uint8).reshape(G, S)
    return tr, em


def rfc4180_csv() -> Format:
    """RFC-4180 CSV: the states EOR, ENC, FLD, EOF, ESC, INV and the groups
    '\\n', '"', ',' and catch-all of Table 1, plus a carriage-return group that
    is a control symbol outside quotes and data inside them."""
    EOR, ENC, FLD, EOF, ESC, INV = range(6)
    D, F, R, C = TAG_DATA, TAG_FIELD, TAG_RECORD, TAG_CONTROL
    newline = [(EOR, R), (ENC, D), (EOR, R), (EOR, R), (EOR, R), (INV, C)]
    quote = [(ENC, C), (ESC, C), (INV, C), (ENC, C), (ENC, D), (INV, C)]
    comma = [(EOF, F), (ENC, D), (EOF, F), (EOF, F), (EOF, F), (INV, C)]
    cr = [(EOR, C), (ENC, D), (FLD, C), (EOF, C), (ESC, C), (INV, C)]
    other = [(FLD, D), (ENC, D), (FLD, D), (FLD, D), (INV, C), (INV, C)]
    tr, em = _build([newline, quote, comma, cr, other])
    return Format("csv", tr, em, b'\n",\r', [0, 1, 2, 3], 4, EOR, INV, [EOR, FLD, EOF, ESC])


def web_log() -> Format:
    """Space-separated web-log lines (Common Log Format): '[...]' and '"..."'
    enclose fields that may hold spaces; the enclosing symbols are control
    symbols.  States EOR, EOF (after a separator), FLD, QUO, QCL (after a
    closing quote), BRK, BCL (after ']'), INV."""
    EOR, EOF, FLD, QUO, QCL, BRK, BCL, INV = range(8)
    D, F, R, C = TAG_DATA, TAG_FIELD, TAG_RECORD, TAG_CONTROL
    bad = (INV, C)
    # per state: transitions for '\n', ' ', '"', '[', ']', other
    table = {
        EOR: [(EOR, R), (EOF, F), (QUO, C), (BRK, C), bad, (FLD, D)],
        EOF: [(EOR, R), (EOF, F), (QUO, C), (BRK, C), bad, (FLD, D)],
        FLD: [(EOR, R), (EOF, F), bad, bad, bad, (FLD, D)],
        QUO: [(QUO, D), (QUO, D), (QCL, C), (QUO, D), (QUO, D), (QUO, D)],
        QCL: [(EOR, R), (EOF, F), bad, bad, bad, bad],
        BRK: [bad, (BRK, D), (BRK, D), (BRK, D), (BCL, C), (BRK, D)],
        BCL: [(EOR, R), (EOF, F), bad, bad, bad, bad],
        INV: [bad] * 6,
    }
    rows = [[table[s][g] for s in range(8)] for g in range(6)]
    tr, em = _build(rows)
    return Format("log", tr, em, b'\n "[]', [0, 1, 2, 3, 4], 5, EOR, INV, [EOR, EOF, FLD, QCL, BCL])


def by_name(name: str) -> Format:
    return {"csv": rfc4180_csv, "log": web_log}[name]()
