"""Loads the hand-derived fixtures under tests/golden/."""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _arr(vals, dtype):
    v = [float("nan") if isinstance(t, str) and t == "nan" else t for t in vals]
    return np.array(v, dtype=np.float64 if np.dtype(dtype).kind == "f" else object).astype(dtype)


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        doc = json.load(f)
    cases = []
    for c in doc["cases"]:
        y = _arr(c["y"], c["dtype"])
        x = _arr(c["x"], c["x_dtype"]) if "x" in c else None
        cases.append(dict(algo=c["algo"], x=x, y=y, n_out=c["n_out"], nan=c.get("nan", "propagate"),
                          minmax_ratio=c.get("minmax_ratio", 4), expected=np.array(c["expected"], dtype=np.int64),
                          derivation=c["derivation"]))
    return cases


def all_cases():
    out = []
    for name in sorted(os.listdir(GOLDEN)):
        if name.endswith(".json"):
            for i, c in enumerate(load(name)):
                c["id"] = f"{name[:-5]}-{i}"
                out.append(c)
    return out
