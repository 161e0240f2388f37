"""Readers for the text fixtures under tests/golden (values printed in the paper)."""
from pathlib import Path

import numpy as np

GOLDEN = Path(__file__).resolve().parent / "golden"


def error_table(name):
    """{N: array of 6 errors} from a convergence-table fixture."""
    rows = {}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        rows[int(parts[0])] = np.array([float(p) for p in parts[1:]])
    return rows


def polyphase_example():
    """{('case2'|'case3', k): [(b_index, c_index), ...]}"""
    out = {}
    for line in (GOLDEN / "polyphase_example.txt").read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        out[(parts[0], int(parts[1]))] = [tuple(int(v) for v in p.split(",")) for p in parts[2:]]
    return out
