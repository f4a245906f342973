"""Reader for the small text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tag, *vals = line.split()
            rows.setdefault(tag, []).append(vals)
    out = {}
    if "vertex" in rows:
        out["vertices"] = np.array([[float(x) for x in r[1:]] for r in rows["vertex"]], np.float32)
    if "triangle" in rows:
        out["triangles"] = np.array([[int(x) for x in r[1:]] for r in rows["triangle"]], np.int32)
    if "ray" in rows:
        r = np.array([[float(x) for x in r[1:]] for r in rows["ray"]], np.float32)
        out["ray_from"], out["ray_to"] = r[:, 0:3].copy(), r[:, 3:6].copy()
    for tag in ("boolean", "leaf_order", "count"):
        if tag in rows:
            out[tag] = np.array([int(x) for x in rows[tag][0]])
    if "hitpoint" in rows:
        out["hitpoint"] = [(int(r[0]), int(r[1]), np.array([float(x) for x in r[2:]])) for r in rows["hitpoint"]]
    if "leaf_box" in rows:
        out["leaf_box"] = {int(r[0]): np.array([float(x) for x in r[1:]]) for r in rows["leaf_box"]}
    if "internal_box" in rows:
        out["internal_box"] = {(int(r[0]), int(r[1])): np.array([float(x) for x in r[2:]]) for r in rows["internal_box"]}
    return out
