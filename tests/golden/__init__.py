"""Parsers for the hand-worked fixtures in this folder (each file cites its passage)."""
import os
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))


def _lines(name):
    with open(os.path.join(HERE, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln


def cdtf_tiny():
    """The CDTF worked example as a dict of exact fractions."""
    d = {"entries": []}
    for ln in _lines("cdtf_tiny.txt"):
        key, val = ln.split(":", 1)
        vals = [Fraction(v) for v in val.split()]
        if key == "entry":
            d["entries"].append(vals)
        else:
            d[key] = vals
    return d


def alg3_cases():
    """List of (name, M, [row nnz per mode], [expected machine per row per mode])."""
    cases, cur = [], None
    for ln in _lines("alg3_greedy.txt"):
        tok = ln.split()
        if tok[0] == "case":
            cur = {"name": tok[1], "modes": [], "expect": []}
            cases.append(cur)
        elif tok[0] == "M":
            cur["M"] = int(tok[1])
        elif tok[0] == "mode":
            cur["modes"].append([int(v) for v in tok[1:]])
        elif tok[0] == "expect":
            cur["expect"].append([int(v) for v in tok[1:]])
    return cases
