"""Reader for the hand-derived text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _groups(tokens, conv):
    out, cur = [], []
    for t in tokens:
        if t == ";":
            out.append(cur)
            cur = []
        else:
            cur.append(conv(t))
    out.append(cur)
    return out


def load_worked(name):
    d = r = c = None
    points, grids, cells, fields = [], [], [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            if key == "d":
                d = int(rest[0])
            elif key == "r":
                r = float(rest[0])
            elif key == "c":
                c = float(rest[0])
            elif key == "point":
                points.append([float(x) for x in rest])
            elif key == "grid":
                R, s = _groups(rest, float)
                grids.append(np.array(R + s, dtype=np.float64))
            elif key == "cells":
                cells.append(_groups(rest, int))
            else:
                fields[key] = {tuple(p) for p in _groups(rest, int)}
    return {"d": d, "r": r, "c": c, "points": np.array(points, dtype=np.float64),
            "transforms": np.stack(grids), "cells": np.array(cells, dtype=np.int64),
            **fields}


def load_table2():
    rows = []
    with open(os.path.join(GOLDEN, "table2_rtg_params.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                d, n, m, ct = line.split()
                rows.append((int(d), int(n), int(m), float(ct)))
    return rows
