"""Readers of the text fixtures in this folder (each file cites its passage)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def pathfinder_example():
    """(program text, inputs) of pathfinder_example.txt; inputs: name -> (cols, tags)."""
    rules, rows = [], {}
    for line in open(os.path.join(HERE, "pathfinder_example.txt")):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        head, rest = line.split(None, 1)
        if head == "rule":
            rules.append(rest)
            continue
        parts = rest.split()
        rows.setdefault(head, []).append(parts)
    inputs = {}
    for name, rs in rows.items():
        if name == "edge":
            cols = (np.array([int(r[0]) for r in rs], np.uint32), np.array([int(r[1]) for r in rs], np.uint32))
            inputs[name] = (cols, np.array([float(r[2]) for r in rs]))
        else:
            inputs[name] = ((np.array([int(r[0]) for r in rs], np.uint32),), None)
    return "\n".join(rules) + "\n", inputs


def provenance_semirings():
    out = {}
    for line in open(os.path.join(HERE, "provenance_semirings.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            name, zero, one, oplus, otimes = line.split()
            out[name] = {"zero": float(zero), "one": float(one), "oplus": oplus, "otimes": otimes}
    return out
