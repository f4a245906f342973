"""CPU oracle for the ray-segment / triangle-surface intersection method.

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the CPU-baseline leg of
the benchmark call this package; the library under ``paper_2305_01867_gb300``
never does.  It shares no code with the CUDA path.

``rsi_oracle.c`` holds the plain FP64 brute force (every ray against every
triangle, Sec. 1) and plain-definition Morton / sort / radix tree / refit
(Sec. 3.2, 4.1, 4.2); ``mlp.py`` holds the FP64 reference of the proposal
network.  Each function cites the passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsi_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

PAIR_MISS, PAIR_HIT, PAIR_AMBIGUOUS = 0, 1, 2
LEAF_TAG = 0x80000000
TAU = 1e-6


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no fused multiply-add on any host)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_classify_pair.argtypes = [P, P, P, P, P, P]
        lib.oracle_classify_pair.restype = ctypes.c_int
        lib.oracle_query.argtypes = [P, i64, P, i64, P, P, i64, P, P, P, P, P, P, P, P, ctypes.c_int]
        lib.oracle_query.restype = ctypes.c_int
        lib.oracle_extent.argtypes = [P, i64, P, P]
        lib.oracle_extent.restype = ctypes.c_int
        lib.oracle_morton.argtypes = [P, i64, P, i64, ctypes.c_int, P]
        lib.oracle_morton.restype = ctypes.c_int
        lib.oracle_sort.argtypes = [P, i64, P, P]
        lib.oracle_sort.restype = ctypes.c_int
        lib.oracle_radix_tree.argtypes = [P, i64, P, P, P, P, P]
        lib.oracle_radix_tree.restype = ctypes.c_int
        lib.oracle_refit.argtypes = [P, P, P, i64, P, P, P]
        lib.oracle_refit.restype = ctypes.c_int
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_pair_classes.argtypes = [P, i64, P, i64, P, P, i64, P]
        lib.oracle_pair_classes.restype = ctypes.c_int
        _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def classify_pair(s, e, a, b, c):
    """Class of one segment/triangle pair and its Moller quantities.

    Returns (cls, dict(u, v, t, det_rel, dist, incl, w))."""
    lib = _load()
    pts = [_f32(x).reshape(3) for x in (s, e, a, b, c)]
    out = np.zeros(7, dtype=np.float64)
    cls = lib.oracle_classify_pair(*[_ptr(p) for p in pts], _ptr(out))
    keys = ("u", "v", "t", "det_rel", "dist", "incl", "w")
    return int(cls), dict(zip(keys, out.tolist()))


def query(vertices, triangles, ray_from, ray_to, nthreads: int = 0):
    """Brute force over all pairs (Sec. 1).  Returns a dict of per-ray arrays:
    hit, amb_hit (boolean mode), count, amb_count (intercept_count mode, and
    the flag of the barycentric mode), near_tri, near_t, near_point,
    near_dist (barycentric mode: nearest inclusive hit, -1 / NaN if none)."""
    lib = _load()
    V, T = _f32(vertices).reshape(-1, 3), _i32(triangles).reshape(-1, 3)
    F, E = _f32(ray_from).reshape(-1, 3), _f32(ray_to).reshape(-1, 3)
    n = F.shape[0]
    assert E.shape[0] == n
    res = dict(hit=np.zeros(n, np.uint8), amb_hit=np.zeros(n, np.uint8),
               count=np.zeros(n, np.int32), amb_count=np.zeros(n, np.uint8),
               near_tri=np.zeros(n, np.int32), near_t=np.zeros(n, np.float32),
               near_point=np.zeros((n, 3), np.float32), near_dist=np.zeros(n, np.float32))
    rc = lib.oracle_query(_ptr(V), V.shape[0], _ptr(T), T.shape[0], _ptr(F), _ptr(E), n,
                          _ptr(res["hit"]), _ptr(res["amb_hit"]), _ptr(res["count"]),
                          _ptr(res["amb_count"]), _ptr(res["near_tri"]), _ptr(res["near_t"]),
                          _ptr(res["near_point"]), _ptr(res["near_dist"]), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_query: bad arguments (triangle index out of range?)")
    return res


def pair_classes(vertices, triangles, ray_from, ray_to):
    """[n_rays, n_triangles] uint8 class of every pair (PAIR_MISS/HIT/AMBIGUOUS)."""
    lib = _load()
    V, T = _f32(vertices).reshape(-1, 3), _i32(triangles).reshape(-1, 3)
    F, E = _f32(ray_from).reshape(-1, 3), _f32(ray_to).reshape(-1, 3)
    out = np.zeros((F.shape[0], T.shape[0]), np.uint8)
    if lib.oracle_pair_classes(_ptr(V), V.shape[0], _ptr(T), T.shape[0], _ptr(F), _ptr(E), F.shape[0], _ptr(out)) != 0:
        raise ValueError("oracle_pair_classes: triangle index out of range")
    return out


def extent(vertices):
    lib = _load()
    V = _f32(vertices).reshape(-1, 3)
    lo, hi = np.zeros(3, np.float32), np.zeros(3, np.float32)
    if lib.oracle_extent(_ptr(V), V.shape[0], _ptr(lo), _ptr(hi)) != 0:
        raise ValueError("oracle_extent: NaN coordinate")
    return lo, hi


def morton(vertices, triangles, bits: int = 30):
    """Morton codes of triangle centroids (Sec. 3.2), uint64 array."""
    lib = _load()
    V, T = _f32(vertices).reshape(-1, 3), _i32(triangles).reshape(-1, 3)
    keys = np.zeros(T.shape[0], np.uint64)
    if lib.oracle_morton(_ptr(V), V.shape[0], _ptr(T), T.shape[0], int(bits), _ptr(keys)) != 0:
        raise ValueError("oracle_morton: bad arguments")
    return keys


def sort(keys):
    """Stable sort by (key, index) (Sec. 3.2).  Returns (sorted_keys, perm)."""
    lib = _load()
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    sk, perm = np.zeros_like(k), np.zeros(k.shape[0], np.int32)
    lib.oracle_sort(_ptr(k), k.shape[0], _ptr(sk), _ptr(perm))
    return sk, perm


def radix_tree(sorted_keys):
    """Binary radix tree (Karras numbering).  Returns dict(left, right, parent,
    range_lo, range_hi) with leaves tagged by LEAF_TAG."""
    lib = _load()
    k = np.ascontiguousarray(sorted_keys, dtype=np.uint64)
    n = k.shape[0]
    m = max(n - 1, 1)
    left, right = np.zeros(m, np.int32), np.zeros(m, np.int32)
    rlo, rhi = np.zeros(m, np.int32), np.zeros(m, np.int32)
    parent = np.zeros(2 * n - 1, np.int32)
    if lib.oracle_radix_tree(_ptr(k), n, _ptr(left), _ptr(right), _ptr(parent), _ptr(rlo), _ptr(rhi)) != 0:
        raise ValueError("oracle_radix_tree: n < 1")
    if n == 1:
        left, right, rlo, rhi = left[:0], right[:0], rlo[:0], rhi[:0]
    return dict(left=left, right=right, parent=parent, range_lo=rlo, range_hi=rhi)


def refit(vertices, triangles, perm, tree):
    """Node boxes (internal nodes then leaves) and tree height (Sec. 4.1)."""
    lib = _load()
    V, T = _f32(vertices).reshape(-1, 3), _i32(triangles).reshape(-1, 3)
    p = _i32(perm)
    n = p.shape[0]
    left = _i32(tree["left"]) if n > 1 else np.zeros(1, np.int32)
    right = _i32(tree["right"]) if n > 1 else np.zeros(1, np.int32)
    box = np.zeros((2 * n - 1, 6), np.float32)
    h = lib.oracle_refit(_ptr(V), _ptr(T), _ptr(p), n, _ptr(left), _ptr(right), _ptr(box))
    return box, int(h)


def build_all(vertices, triangles, bits: int = 30):
    """The whole plain-definition build: keys, order, tree, boxes."""
    keys = morton(vertices, triangles, bits)
    sk, perm = sort(keys)
    tree = radix_tree(sk)
    box, height = refit(vertices, triangles, perm, tree)
    return dict(keys=keys, sorted_keys=sk, perm=perm, box=box, height=height, **tree)
