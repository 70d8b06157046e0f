"""Readers for the hand-derived fixtures in this folder (band membership and ratio-test cases)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _strip(line):
    return line.split("#", 1)[0].strip()


def band_cases():
    """Yields dicts with F (float32[9]), d, q (x, y), points (float32[k,2]) and expected (int[k])."""
    cases, cur = [], None
    with open(os.path.join(HERE, "band_closed_form.txt")) as fh:
        for raw in fh:
            line = _strip(raw)
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = {"name": tok[1], "pts": [], "exp": []}
            elif tok[0] == "F":
                cur["F"] = np.array([float(t) for t in tok[1:10]], np.float32)
            elif tok[0] == "d":
                cur["d"] = float("inf") if tok[1] == "inf" else float(tok[1])
            elif tok[0] == "q":
                cur["q"] = (float(tok[1]), float(tok[2]))
            elif tok[0] == "p":
                cur["pts"].append((float(tok[1]), float(tok[2])))
                cur["exp"].append(int(tok[3]))
            elif tok[0] == "end":
                cur["points"] = np.array(cur.pop("pts"), np.float32).reshape(-1, 2)
                cur["expected"] = np.array(cur.pop("exp"), np.int64)
                cases.append(cur)
    return cases


def _desc(tokens):
    v = np.zeros(128, np.uint8)
    for t in tokens:
        k, val = t.split(":")
        if k == "all":
            v[:] = int(val)
        else:
            v[int(k)] = int(val)
    return v


def ratio_cases():
    """Yields dicts with p, q, expected j, the query descriptor and the B descriptors."""
    cases = []
    with open(os.path.join(HERE, "ratio_cases.txt")) as fh:
        for raw in fh:
            line = _strip(raw)
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                cases.append({"name": tok[1], "p": int(tok[2]), "q": int(tok[3]), "expected": int(tok[4]),
                              "qd": np.zeros(128, np.uint8), "bd": []})
            elif tok[0] == "q_desc":
                cases[-1]["qd"] = _desc(tok[1:])
            elif tok[0] == "b":
                cases[-1]["bd"].append(_desc(tok[1:]))
    for c in cases:
        c["bd"] = np.array(c["bd"], np.uint8).reshape(-1, 128)
    return cases
