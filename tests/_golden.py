"""Parsers for the hand-written fixtures under tests/golden/."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def lab_reference_colours():
    out = []
    for r in _rows("lab_reference_colours.txt"):
        out.append((tuple(int(v) for v in r[:3]), tuple(float(v) for v in r[3:6]), float(r[6])))
    return out


def _expr(s):
    # Only arithmetic, numbers and sqrt are allowed in the fixture.
    assert set(s) <= set("0123456789.+-*/() sqrt"), s
    return eval(s, {"__builtins__": {}}, {"sqrt": math.sqrt})


def eq1_examples():
    ex = []
    for r in _rows("eq1_worked_example.txt"):
        if r[0] == "example":
            ex.append({"name": r[1], "W": int(r[2]), "H": int(r[3]), "S": int(r[4]),
                       "m": float(r[5]), "centres": [], "pixels": []})
        elif r[0] == "centre":
            ex[-1]["centres"].append([float(v) for v in r[1:6]] + [0.0])
        elif r[0] == "pixel":
            ex[-1]["pixels"].append({"x": int(r[1]), "y": int(r[2]),
                                     "lab": [float(v) for v in r[3:6]], "label": int(r[6]),
                                     "D_best": _expr(r[7]), "D_second": _expr(r[8])})
    return ex


def connectivity_cases():
    cases, cur, section = [], None, None
    for r in _rows("connectivity_cases.txt"):
        if r[0] == "case":
            cur = {"name": r[1], "W": int(r[2]), "H": int(r[3]), "in": [], "pass1": [], "pass2": []}
            cases.append(cur)
            section = "in"
        elif r[0] in ("pass1", "pass2"):
            section = r[0]
        else:
            cur[section].append([int(v) for v in r])
    for c in cases:
        for k in ("in", "pass1", "pass2"):
            c[k] = np.array(c[k], dtype=np.int32).reshape(c["H"], c["W"])
    return cases
