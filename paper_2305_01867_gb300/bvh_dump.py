"""Readable dumps of a built hierarchy (the BVH inspection of Sec. 4.1.1 and
the Graphviz picture of Sec. 4.1.5), from the host arrays LBVH.export()
returns: sorted_keys, perm, left, right, parent, box.

Internal node i has children left[i] / right[i]: an internal index, or leaf j
tagged as (int32)(0x80000000 | j).  Leaf j holds triangle perm[j].  box[] has
6 floats (min xyz, max xyz) per node, internal nodes first, then leaves.

Host code only (numpy); nothing here runs on the GPU.
"""
from __future__ import annotations

import numpy as np

LEAF_TAG = 0x80000000


def _child(ref: int):
    """(is_leaf, index) of a child reference."""
    r = int(ref) & 0xFFFFFFFF
    return (True, r & ~LEAF_TAG) if r & LEAF_TAG else (False, r)


def leaf_ranges(view: dict) -> np.ndarray:
    """[first leaf, last leaf] covered by every internal node (n - 1 rows),
    found by a walk from the root (internal node 0)."""
    n = len(view["perm"])
    rng = np.zeros((max(n - 1, 0), 2), np.int64)
    if n < 2:
        return rng

    def span(ref):
        leaf, i = _child(ref)
        return (i, i) if leaf else tuple(rng[i])

    # children before parents: reverse of a preorder walk
    order, stack = [], [0]
    while stack:
        i = stack.pop()
        order.append(i)
        for ref in (view["left"][i], view["right"][i]):
            leaf, c = _child(ref)
            if not leaf:
                stack.append(c)
    for i in reversed(order):
        a, b = span(view["left"][i]), span(view["right"][i])
        rng[i] = (a[0], b[1])
    return rng


def _box_text(b, digits):
    f = f"{{:.{digits}f}}"
    return (f"x [{f.format(b[0])}, {f.format(b[3])}]  y [{f.format(b[1])}, {f.format(b[4])}]  "
            f"z [{f.format(b[2])}, {f.format(b[5])}]")


def to_text(view: dict, digits: int = 1) -> str:
    """One line per node: internal nodes with their leaf range, box and
    children; leaves with their box and triangle."""
    n = len(view["perm"])
    box = np.asarray(view["box"]).reshape(-1, 6)
    rng = leaf_ranges(view)
    lines = [f"hierarchy over {n} triangles", "internal nodes"]
    for i in range(n - 1):
        kids = []
        for ref in (view["left"][i], view["right"][i]):
            leaf, c = _child(ref)
            kids.append(f"leaf {c}" if leaf else f"node {c}")
        p = int(view["parent"][i])
        lines.append(f"  node {i}{' (root)' if i == 0 else ''}: leaves [{rng[i][0]}, {rng[i][1]}]  "
                     f"{_box_text(box[i], digits)}  children {kids[0]}, {kids[1]}  parent {p}")
    lines.append("leaves")
    for j in range(n):
        p = int(view["parent"][n - 1 + j])
        lines.append(f"  leaf {j}: triangle {int(view['perm'][j])}  {_box_text(box[n - 1 + j], digits)}  parent {p}")
    return "\n".join(lines) + "\n"


def to_dot(view: dict, path: str | None = None) -> str:
    """Graph description in the DOT language: internal nodes as ellipses
    labelled with their leaf range "[a,b]", leaves as boxes labelled
    "[j] t" (leaf j, triangle t).  Written to `path` if given."""
    n = len(view["perm"])
    rng = leaf_ranges(view)
    out = ["digraph bvh {", "  node [fontname=\"Helvetica\"];"]
    for i in range(n - 1):
        out.append(f"  n{i} [shape=ellipse, label=\"[{rng[i][0]},{rng[i][1]}]\"];")
    for j in range(n):
        out.append(f"  l{j} [shape=box, label=\"[{j}] {int(view['perm'][j])}\"];")
    for i in range(n - 1):
        for ref in (view["left"][i], view["right"][i]):
            leaf, c = _child(ref)
            out.append(f"  n{i} -> {'l' if leaf else 'n'}{c};")
    out.append("}")
    text = "\n".join(out) + "\n"
    if path is not None:
        with open(path, "w") as f:
            f.write(text)
    return text
