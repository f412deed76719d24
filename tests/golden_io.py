"""Readers for the text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def philox_kat():
    out = []
    for tok in _lines("philox4x32_10_kat.txt"):
        vals = [int(x, 16) for x in tok]
        out.append((vals[0:4], vals[4:6], vals[6:10]))
    return out


def hand_step():
    """The N=4, D=2 hand-stepped swarm: dict of params, init, r, and results."""
    g = {"param": {}, "init": {}, "r": {}}
    for tok in _lines("hand_step_n4_d2.txt"):
        kind = tok[0]
        if kind == "param":
            g["param"][tok[1]] = np.float32(tok[2])
        elif kind == "init":
            g["init"][tok[1]] = np.array([np.float32(x) for x in tok[2:]], np.float32)
        elif kind == "r":
            g["r"][int(tok[1])] = np.array([np.float32(x) for x in tok[2:]], np.float32)
        else:
            g.setdefault(kind, {})[tok[1]] = np.array([np.float32(x) for x in tok[2:]], np.float32)
    return g
