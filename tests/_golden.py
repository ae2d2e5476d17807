"""Reader for the hand-written fixtures under tests/golden/."""
from __future__ import annotations

import glob
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(path):
    rows, cols, vals = [], [], []
    case = {"path": path}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tag, *rest = line.split()
            if tag == "shape":
                case["shape"] = (int(rest[0]), int(rest[1]))
            elif tag == "mode":
                case["mode"] = rest[0]
            elif tag == "write":
                rows.append(int(rest[0]))
                cols.append(int(rest[1]))
                vals.append(float(rest[2]))
            elif tag == "expect_col_ptr_runs":
                cp = []
                for tok in rest:
                    v, n = tok.split("x")
                    cp += [int(v)] * int(n)
                case["col_ptr"] = np.array(cp, dtype=np.int64)
            elif tag == "expect_row_idx":
                case["row_idx"] = np.array([int(x) for x in rest], dtype=np.int64)
            elif tag == "expect_vals":
                case["vals_expected"] = np.array([float(x) for x in rest], dtype=np.float64)
            else:
                raise ValueError(f"{path}: unknown tag {tag}")
    case["rows"] = np.array(rows, dtype=np.int32)
    case["cols"] = np.array(cols, dtype=np.int32)
    case["vals"] = np.array(vals, dtype=np.float64)
    return case


def all_cases():
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))]
