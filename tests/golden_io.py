"""Readers for the text fixtures under tests/golden/ (values printed in the paper)."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line


def int_rows(name):
    """'key: v0 v1 ...' lines -> {key: [ints]}"""
    out = {}
    for line in _lines(name):
        key, vals = line.split(":", 1)
        out[key.strip()] = [int(v) for v in vals.split()]
    return out


def table1():
    rows = []
    for line in _lines("table1_cavity.txt"):
        q, ra, lbm, lpos, ref, rpos = line.split()
        rows.append(dict(quantity=q, Ra=float(ra), lbm=float(lbm), lbm_pos=float(lpos),
                         ref=float(ref), ref_pos=float(rpos)))
    return rows
