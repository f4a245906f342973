"""Pins of the oracle's build steps (no GPU): Morton codes (Sec. 3.2),
the sort (Sec. 3.2), the binary radix tree (Sec. 1 / Karras 2012, Sec. 4.2)
and the node boxes (Sec. 4.1, 4.2)."""
import numpy as np
import pytest

import oracle
import workloads as W

LEAF = oracle.LEAF_TAG


def _tri_at(points):
    """Degenerate 'triangles' (three equal vertices) whose centroid is the
    given point exactly: ((p + p) + p) / 3 == p in FP32 for these values."""
    V = np.repeat(np.asarray(points, np.float32), 3, axis=0)
    T = np.arange(len(V), dtype=np.int32).reshape(-1, 3)
    return V, T


@pytest.mark.parametrize("bits", [30, 63])
def test_morton_closed_forms(bits):
    b = bits // 3
    # extent [0,1]^3 fixed by the two corner points; powers of two are exact
    pts = [[0, 0, 0], [1, 1, 1], [0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5], [0.25, 0.5, 0.75]]
    V, T = _tri_at(pts)
    k = oracle.morton(V, T, bits).astype(object)
    assert k[0] == 0
    assert k[1] == (1 << bits) - 1                 # q = 2^b - 1 on every axis
    assert k[2] == 1 << (3 * (b - 1))              # x is bit 0 of each group
    assert k[3] == 1 << (3 * (b - 1) + 1)          # y is bit 1
    assert k[4] == 1 << (3 * (b - 1) + 2)          # z is bit 2 (the high bit)
    # (0.25, 0.5, 0.75): qx = 2^(b-2), qy = 2^(b-1), qz = 2^(b-1) + 2^(b-2)
    expect = (1 << (3 * (b - 2))) | (1 << (3 * (b - 1) + 1)) | (1 << (3 * (b - 1) + 2)) | (1 << (3 * (b - 2) + 2))
    assert k[5] == expect


def test_morton_truncates_and_is_monotone_along_axes():
    xs = (np.arange(0, 1024) + 0.5) / 1024.0
    pts = [[0, 0, 0], [1, 1, 1]] + [[x, 0, 0] for x in xs]
    V, T = _tri_at(pts)
    k = oracle.morton(V, T, 30)[2:]
    # u = (k + 1/2) / 1024 quantises to k: the key is k spread to bits 0,3,6..
    spread = np.array([sum(((q >> i) & 1) << (3 * i) for i in range(10)) for q in range(1024)], np.uint64)
    assert np.array_equal(k, spread)
    for axis in range(3):
        pts = [[0, 0, 0], [1, 1, 1]] + [[x if a == axis else 0.3 for a in range(3)] for x in np.linspace(0, 1, 300)]
        V, T = _tri_at(pts)
        kk = oracle.morton(V, T, 63)[2:]
        assert np.all(np.diff(kk.astype(np.int64)) >= 0)


def test_morton_flat_axis_quantises_to_zero():
    V = np.array([[0, 0, 5], [1, 0, 5], [0, 1, 5], [1, 1, 5]], np.float32)
    T = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    k = oracle.morton(V, T, 30)
    assert np.all((k.astype(np.int64) & 0o4444444444) == 0)    # no z bits


def test_sort_equals_library_stable_sort():
    rng = np.random.default_rng(5)
    for n in (1, 2, 3, 1000, 5000):
        keys = rng.integers(0, 50, n).astype(np.uint64) << np.uint64(rng.integers(0, 30))
        sk, perm = oracle.sort(keys)
        ref = np.argsort(keys, kind="stable")
        assert np.array_equal(perm, ref)
        assert np.array_equal(sk, keys[ref])


def _trie_nodes(keys, n_idx_bits):
    """Independent construction: the branching prefixes of the binary trie of
    the index-augmented keys.  Returns {(a, b): split} over internal nodes."""
    aug = [(int(k) << n_idx_bits) | i for i, k in enumerate(keys)]
    width = max(aug).bit_length() + 1 if len(aug) else 1
    nodes = {}
    # a prefix of length L branches iff keys with that prefix continue with 0
    # and with 1; keys sharing a prefix are contiguous because they are sorted
    for L in range(width):
        groups = {}
        for i, x in enumerate(aug):
            groups.setdefault(x >> (width - L), []).append(i)
        for members in groups.values():
            zeros = [i for i in members if not (aug[i] >> (width - L - 1)) & 1]
            ones = [i for i in members if (aug[i] >> (width - L - 1)) & 1]
            if zeros and ones:
                nodes[(members[0], members[-1])] = zeros[-1]
    return nodes


@pytest.mark.parametrize("seed", range(6))
def test_radix_tree_equals_trie(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 70))
    keys = np.sort(rng.integers(0, 40 if seed % 2 else 1 << 30, n)).astype(np.uint64)
    t = oracle.radix_tree(keys)
    nidx = max(1, (n - 1).bit_length())
    trie = _trie_nodes(keys, nidx)
    got = {}
    for i in range(n - 1):
        a, b = int(t["range_lo"][i]), int(t["range_hi"][i])
        lc = int(t["left"][i]) & 0xFFFFFFFF
        split = (lc & ~LEAF) if lc & LEAF else lc
        got[(a, b)] = split
        # Karras numbering: a node's index is one end of its range, the
        # children are "split" and "split + 1", the root is node 0
        assert i in (a, b)
        rc = int(t["right"][i]) & 0xFFFFFFFF
        assert ((rc & ~LEAF) if rc & LEAF else rc) == split + 1
        assert bool(lc & LEAF) == (split == a) and bool(rc & LEAF) == (split + 1 == b)
    assert got == trie
    assert (int(t["range_lo"][0]), int(t["range_hi"][0])) == (0, n - 1)


def test_tree_invariants_and_refit_brute_force():
    """Sec. 4.2: n - 1 internal nodes are used, every leaf has a parent, the
    root covers [0, n-1]; every box is the bound of the triangles below it."""
    mesh = W.heightfield(12, seed=9)
    b = oracle.build_all(mesh.vertices, mesh.triangles, bits=30)
    n = len(b["perm"])
    par = b["parent"]
    assert par[0] == -1 and np.all(par[1:] >= 0)
    assert sorted(b["perm"].tolist()) == list(range(n))
    kids = np.concatenate([b["left"], b["right"]])
    assert len(set(kids.tolist())) == 2 * (n - 1)          # each node once
    V, T = mesh.vertices, mesh.triangles
    for i in range(n - 1):
        a, c = b["range_lo"][i], b["range_hi"][i]
        pts = V[T[b["perm"][a:c + 1]].ravel()]
        np.testing.assert_array_equal(b["box"][i, :3], pts.min(0))
        np.testing.assert_array_equal(b["box"][i, 3:], pts.max(0))
    # height = deepest leaf, by walking parent links
    depth = []
    for j in range(n):
        d, x = 0, par[n - 1 + j]
        while x != -1:
            d, x = d + 1, par[x]
        depth.append(d)
    assert b["height"] == max(depth)


def test_single_triangle_tree():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    b = oracle.build_all(V, np.array([[0, 1, 2]], np.int32))
    assert b["perm"].tolist() == [0] and b["parent"].tolist() == [-1] and b["height"] == 0
