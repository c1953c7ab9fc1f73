"""Loader for the hand-worked fixtures under tests/golden/."""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_hand_example(name="hand_example_3cols_4buckets.json"):
    g = json.load(open(os.path.join(GOLDEN, name)))
    m, n = g["m"], g["n"]
    colptr = [0]
    rows, vals = [], []
    for j in range(n):
        for r, v in g["columns"][str(j)]:
            rows.append(r)
            vals.append(v)
        colptr.append(len(rows))
    g["colptr"] = np.array(colptr, np.int32)
    g["rowidx"] = np.array(rows, np.int32)
    g["val"] = np.array(vals, np.float32)
    return g
