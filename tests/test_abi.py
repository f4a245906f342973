"""The C ABI without a GPU: the library builds (nvcc cross-compiles for
sm_103a), loads, exports every function include/rsi.h declares, and rejects
bad arguments on the host before any device work."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    b = __graft_entry__._builder()
    if not b.up_to_date():
        if not shutil.which(b.NVCC) and not os.path.exists(b.NVCC):
            pytest.skip("nvcc not available")
        b.build()
    import paper_2305_01867_gb300 as m
    return m


def test_every_declared_symbol_is_exported(lib):
    names = _declared("rsi.h")
    assert {"lbvh_build", "rsi_query", "rsi_query_host", "lbvh_export", "rsi_last_error"} <= set(names)
    raw = ctypes.CDLL(lib._LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


def test_node_size_is_queried_not_assumed(lib):
    # Sec. 3.2: struct sizes come from the library (bytesInBVHNode)
    assert lib.node_bytes() == 64


def test_host_side_rejections(lib):
    L = lib.lib
    h = ctypes.c_void_p()
    # int64 indices (Sec. 4.1.2) are refused before any device work
    rc = L.lbvh_build(ctypes.c_void_p(16), 3, ctypes.c_void_p(16), 1, 8, 30, None, ctypes.byref(h))
    assert rc == -2 and "int32" in lib.last_error()
    rc = L.lbvh_build(None, 3, None, 1, 4, 30, None, ctypes.byref(h))
    assert rc == -1
    rc = L.lbvh_build(ctypes.c_void_p(16), 3, ctypes.c_void_p(16), 0, 4, 30, None, ctypes.byref(h))
    assert rc == -1
    rc = L.lbvh_build(ctypes.c_void_p(16), 3, ctypes.c_void_p(16), 1, 4, 31, None, ctypes.byref(h))
    assert rc == -1 and "30 or 63" in lib.last_error()
    rc = L.lbvh_build_ex(ctypes.c_void_p(16), 3, ctypes.c_void_p(16), 1, 4, 30, 2, None, ctypes.byref(h))
    assert rc == -1 and "tree_builder" in lib.last_error()
    rc = L.lbvh_build_ex(ctypes.c_void_p(16), 3, ctypes.c_void_p(16), 1, 8, 30, 1, None, ctypes.byref(h))
    assert rc == -2
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    outs = (P * 2)()
    rc = L.lbvh_build_batched(0, None, None, None, None, 4, 30, None, outs)
    assert rc == -1
    vp, tp = (P * 2)(16, 16), (P * 2)(16, None)
    nv, nt = (I64 * 2)(3, 3), (I64 * 2)(1, 1)
    rc = L.lbvh_build_batched(2, vp, nv, tp, nt, 4, 30, None, outs)
    assert rc == -1 and "mesh 1" in lib.last_error() and not outs[0] and not outs[1]
    rc = L.lbvh_build_batched(2, vp, nv, (P * 2)(16, 16), nt, 4, 31, None, outs)
    assert rc == -1
    rc = L.rsi_query(None, None, None, 0, 0, None, None, None, None, None, None)
    assert rc == -1
    assert L.lbvh_free(None) == 0
    # barycentric mode: a handle is required; compaction checks its outputs
    rc = L.rsi_query_nearest(None, None, None, 0, None, None, None, None, None, None, None, None)
    assert rc == -1
    k = ctypes.c_int64(7)
    assert L.rsi_nearest_compact(None, None, None, 0, None, None, None, None, ctypes.byref(k), None) == 0
    assert k.value == 0                        # nothing to compact: no device work
    assert L.rsi_nearest_compact(None, None, None, 10, None, None, None, None, None, None) == -1
    rc = L.rsi_nearest_compact(ctypes.c_void_p(16), None, None, 5, None, None, ctypes.c_void_p(16), None,
                               ctypes.byref(k), None)
    assert rc == -1                            # distances asked for without their input


def test_binding_rejects_before_the_library(lib):
    """Argument checks of the binding that need no GPU."""
    import torch
    V = torch.zeros(4, 3, dtype=torch.float32)
    T = torch.zeros(2, 3, dtype=torch.int32)
    with pytest.raises(ValueError):
        lib.LBVH(V, T, builder="octree")
    with pytest.raises(ValueError):
        lib.build_many([])
    with pytest.raises(TypeError):
        lib.build_many([(V, T)])                      # host tensors
    with pytest.raises(TypeError):
        lib.build_many([(V, T.to(torch.int64))])      # int64 indices (Sec. 4.1.2)
    with pytest.raises(TypeError):
        lib.build_many([(V.to(torch.float64), T)])
