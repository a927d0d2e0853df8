"""Reader for the hand-worked examples in tests/golden/hand_*.txt.

Each file holds, after `#` comment lines that show the working, the graph (`edges u v w | ...`
in edge-id order), the weighted degrees, the exact scores as fractions and as binary64 bit
patterns, the sorted edge order, and one `nc` line per target: lift | emap | self-mass |
coarse rowptr | coarse col | coarse weights.
"""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILES = ["hand_example.txt", "hand_cycle5_ties.txt"]


def parse(name):
    """(rows, ncs): rows maps a key to the rest of its line; ncs maps n_c to its six lists."""
    rows, ncs = {}, {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("nc "):
                head, rest = line.split(":", 1)
                ncs[int(head.split()[1])] = [[int(x) for x in p.split()]
                                             for p in rest.split("|")]
            else:
                key, rest = line.split(" ", 1)
                rows[key] = rest
    return rows, ncs


def edges(rows):
    """(n, eu, ev, w) of the example; n is one more than the largest endpoint."""
    trip = [t.split() for t in rows["edges"].split("|")]
    eu = np.array([int(t[0]) for t in trip])
    ev = np.array([int(t[1]) for t in trip])
    w = np.array([int(t[2]) for t in trip], dtype=np.int32)
    return int(max(eu.max(), ev.max())) + 1, eu, ev, w


def ints(rows, key):
    return [int(x, 0) for x in rows[key].split()]
