"""Host-side hierarchy dumps (Sec. 4.1.1 text dump, Sec. 4.1.5 DOT graph),
checked on trees the oracle builds: the Sec. 4.1 worked example must show
the printed structure, and every dump must describe a valid binary tree."""
import re

import numpy as np
import pytest

import oracle
import workloads as W
from golden_io import load

dump = pytest.importorskip("paper_2305_01867_gb300.bvh_dump")


def _edges(dot):
    return re.findall(r"^\s*(n\d+|l\d+) -> (n\d+|l\d+);$", dot, flags=re.M)


def test_case_study1_dot_matches_printed_tree():
    """Sec. 4.1: the root covers leaves [0,3] with children [0,1] and [2,3];
    leaves 0..3 hold triangles 0, 3, 1, 2."""
    g = load("case_study1_sec4_1.txt")
    view = oracle.build_all(g["vertices"], g["triangles"])
    dot = dump.to_dot(view)
    labels = dict(re.findall(r"^\s*(n\d+|l\d+) \[shape=\w+, label=\"([^\"]+)\"\];$", dot, flags=re.M))
    assert labels["n0"] == "[0,3]"
    assert sorted(labels[c] for p, c in _edges(dot) if p == "n0") == ["[0,1]", "[2,3]"]
    assert [labels[f"l{j}"] for j in range(4)] == ["[0] 0", "[1] 3", "[2] 1", "[3] 2"]
    text = dump.to_text(view)
    # the printed boxes of the corrected dump (one decimal)
    assert "node 0 (root): leaves [0, 3]  x [12.0, 13.0]  y [2.0, 3.0]  z [1.0, 1.3]" in text
    assert "leaf 1: triangle 3  x [12.0, 12.5]  y [2.0, 3.0]  z [1.0, 1.2]" in text


@pytest.mark.parametrize("mesh", ["c1", "soup"])
def test_dump_is_a_tree_with_oracle_ranges(mesh):
    if mesh == "c1":
        m = W.config_mesh("c1")
        V, T = m.vertices, m.triangles
    else:
        rng = np.random.default_rng(5)
        V = rng.uniform(0, 1, (3 * 777, 3)).astype(np.float32)
        T = np.arange(3 * 777, dtype=np.int32).reshape(-1, 3)
    view = oracle.build_all(V, T)
    n = len(T)
    r = dump.leaf_ranges(view)
    assert np.array_equal(r[:, 0], view["range_lo"]) and np.array_equal(r[:, 1], view["range_hi"])
    e = _edges(dump.to_dot(view))
    assert len(e) == 2 * (n - 1)
    heads = [c for _, c in e]
    assert len(set(heads)) == len(heads) == 2 * n - 2 and "n0" not in heads
    assert {f"l{j}" for j in range(n)} <= set(heads)
    assert len(dump.to_text(view).splitlines()) == 3 + (n - 1) + n


def test_single_triangle():
    view = oracle.build_all(np.eye(3, dtype=np.float32), np.array([[0, 1, 2]], np.int32))
    dot = dump.to_dot(view)
    assert "l0 [shape=box, label=\"[0] 0\"];" in dot and "->" not in dot
