"""The node-pair table of the Q2 tensor-core epilogue (csrc/fe_pair_table.h):
every pair a <= b of the 27 nodes appears exactly once, and within each group
of 32 lanes the shared-memory banks of the G load (4a + b), the direct K^e
store (20a + b) and the transposed store (20b + a), all mod 32, are distinct."""
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(HERE, "..", "paper_1708_01773_gb300", "csrc", "fe_pair_table.h")


def load_table():
    text = open(HDR).read()
    rows = re.findall(r"\{([^{}]*)\},", text)
    return [[int(v, 16) for v in r.split(",")] for r in rows]


def test_pair_table_covers_every_pair_once():
    table = load_table()
    assert len(table) == 15 and all(len(r) == 32 for r in table)
    seen = [(e >> 8, e & 255) for r in table for e in r if e != 0xFFFF]
    assert sorted(seen) == sorted((a, b) for a in range(27) for b in range(a, 27))


def test_pair_table_groups_are_bank_conflict_free():
    for r in load_table():
        ent = [(e >> 8, e & 255) for e in r if e != 0xFFFF]
        for key in (lambda a, b: 4 * a + b, lambda a, b: 20 * a + b, lambda a, b: 20 * b + a):
            res = [key(a, b) % 32 for a, b in ent]
            assert len(set(res)) == len(res)
