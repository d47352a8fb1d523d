"""Readers for the text fixtures in ``tests/golden`` (hand-derived values)."""
import os

import numpy as np

from paper_2208_02995_gb300.inputs import Problem

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _num(tok):
    # tokens are plain numbers or small exact expressions in sqrt2
    return float(eval(tok, {"__builtins__": {}}, {"sqrt2": np.sqrt(2.0)}))


def read(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [_num(v) for v in vals]
    return out


def problem_1d4():
    g = read("emin_1d4.txt")
    Ap = np.array(g["A_rowptr"], dtype=np.int32)
    Pp = np.array(g["P_rowptr"], dtype=np.int32)
    n = len(Ap) - 1
    prob = Problem("golden_1d4", n, int(g["nc"][0]), 1, Ap,
                   np.array(g["A_col"], dtype=np.int32), np.array(g["A_val"]),
                   Pp, np.array(g["P_col"], dtype=np.int32), np.array(g["P0"]),
                   np.ones((n, 1)), np.array(g["Bc"])[:, None], 1, {"kind": "golden"})
    return prob, g
