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
    for bad in (4 << 8, (1 << 8) | 2, -1):   # RSI_TREE_TREELETS(4); an unknown builder with passes; negative
        rc = L.lbvh_build_ex(ctypes.c_void_p(16), 3, ctypes.c_void_p(16), 1, 4, 30, bad, None, ctypes.byref(h))
        assert rc == -1 and "tree_builder" in lib.last_error(), bad
    rc = L.lbvh_build_host_ex(ctypes.c_void_p(16), 3, ctypes.c_void_p(16), 1, 4, 30, 4 << 8, None, ctypes.byref(h))
    assert rc == -1 and "tree_builder" in lib.last_error()
    one_p, one_n = (ctypes.c_void_p * 1)(16), (ctypes.c_int64 * 1)(3)
    rc = L.lbvh_build_batched_ex(1, one_p, one_n, one_p, one_n, 4, 30, 4, None, (ctypes.c_void_p * 1)())
    assert rc == -1 and "treelet_passes" in lib.last_error()
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
        lib.LBVH(V, T, treelet_passes=4)
    with pytest.raises(ValueError):
        lib.build_many([])
    with pytest.raises(TypeError):
        lib.build_many([(V, T)])                      # host tensors
    with pytest.raises(TypeError):
        lib.build_many([(V, T.to(torch.int64))])      # int64 indices (Sec. 4.1.2)
    with pytest.raises(TypeError):
        lib.build_many([(V.to(torch.float64), T)])


def test_every_entry_point_rejects_missing_arguments(lib):
    """Each call that takes a handle or buffers answers RSI_ERR_INVALID_ARG
    (-1), with a message naming the call, when one is missing or a size is
    out of range -- before any device work, so no GPU is needed here."""
    L, P = lib.lib, ctypes.c_void_p
    f = ctypes.c_float()
    k = ctypes.c_int64()
    cases = {
        "lbvh_info": lambda: L.lbvh_info(None, None),
        "lbvh_export": lambda: L.lbvh_export(None, None, None),
        "lbvh_build_host": lambda: L.lbvh_build_host(None, 3, None, 1, 4, 30, None, None),
        "rsi_query_host": lambda: L.rsi_query_host(None, None, None, 5, 0, None, None, None, None, None, None),
        "rsi_query_noalloc": lambda: L.rsi_query_noalloc(None, None, None, 5, 0, None, None, None, None, None),
        "rsi_query_nearest": lambda: L.rsi_query_nearest(None, None, None, 5, None, None, None, None, None, None,
                                                         None, None),
        "rsi_nearest_compact": lambda: L.rsi_nearest_compact(None, None, None, -1, None, None, None, None,
                                                             ctypes.byref(k), None),
        "rsi_batch_create": lambda: L.rsi_batch_create(None, 0, 0, None, None, None),
        "rsi_batch_launch": lambda: L.rsi_batch_launch(None, None),
        "rsi_batch_create_rebuild": lambda: L.rsi_batch_create_rebuild(None, 0, None, None, 0, None, None, None),
        "rsi_query_batched": lambda: L.rsi_query_batched(None, 0, None, 0, None, None),
        "rsi_mlp_attach": lambda: L.rsi_mlp_attach(None, None),
        "rsi_batch_post": lambda: L.rsi_batch_post(None, 0, None),
        "rsi_batch_stats": lambda: L.rsi_batch_stats(None, None, None),
        "rsi_autotune": lambda: L.rsi_autotune(None, None, None, 5, 0, None, None, None, None),
        "rsi_batch_autotune": lambda: L.rsi_batch_autotune(None, 0, 0, None, None, None, None),
        "rsi_segment_order": lambda: L.rsi_segment_order(None, None, None, 5, None, None),
        "rsi_mlp_create": lambda: L.rsi_mlp_create(1, None),
        "rsi_mlp_set_params": lambda: L.rsi_mlp_set_params(None, None, None),
        "rsi_mlp_get_params": lambda: L.rsi_mlp_get_params(None, None, None, None),
        "rsi_mlp_forward": lambda: L.rsi_mlp_forward(None, None, None, None, 5, None, None, None),
        "rsi_mlp_status": lambda: L.rsi_mlp_status(None, None),
        "rsi_mlp_activation": lambda: L.rsi_mlp_activation(None, -1, None, None, None, None),
        "rsi_mlp_train_step": lambda: L.rsi_mlp_train_step(None, None, None, None, None, 5, 1e-3, 1, None, None),
        "rsi_mlp_reset_optimizer": lambda: L.rsi_mlp_reset_optimizer(None, None),
        "rsi_cluster_labels": lambda: L.rsi_cluster_labels(None, None, None, 5, None, None),
        "rsi_query_learned": lambda: L.rsi_query_learned(None, None, None, None, 5, None, None, None, None, None),
        "rsi_last_query_ms": lambda: L.rsi_last_query_ms(None, ctypes.byref(f), ctypes.byref(f)),
    }
    for name, call in cases.items():
        assert call() == -1, name
        assert name in lib.last_error(), (name, lib.last_error())
    # releasing nothing is not an error
    assert L.rsi_batch_free(None) == 0 and L.rsi_mlp_free(None) == 0
    # the network's parameter count follows from its shape: 16x128 + 128x128 +
    # 128x256 weights and 128 + 128 + 256 biases
    assert L.rsi_mlp_num_params() == 16 * 128 + 128 * 128 + 128 * 256 + 128 + 128 + 256


def test_struct_layouts_match_the_header(lib):
    """Every structure the binding passes through the ABI has the header's
    layout: the offset of each field and the size of the whole, as a C
    compiler lays out include/rsi.h on this host."""
    import json
    import subprocess
    pairs = {"rsi_options": lib.Options, "rsi_stats": lib.Stats, "rsi_bvh_info": lib.Info,
             "rsi_bvh_host_view": lib.HostView, "rsi_tuning": lib.Tuning, "rsi_ray_batch": lib.RayBatch}
    lines = ['#include <stdio.h>', '#include "rsi.h"', "int main(void) {", 'printf("{");']
    for k, (cname, py) in enumerate(pairs.items()):
        sep = "," if k else ""
        lines.append(f'printf("{sep}\\"{cname}\\": {{\\"size\\": %zu", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf(", \\"{f}\\": %zu", offsetof({cname}, {f}));')
        lines.append('printf("}");')
    lines += ['printf("}\\n");', "return 0; }"]
    scratch = os.path.join(ROOT, "tests", ".abi_layout")
    os.makedirs(scratch, exist_ok=True)
    exe = os.path.join(scratch, f"layout_{os.getpid()}")
    try:
        cc = subprocess.run(["gcc", "-std=c11", "-x", "c", "-", "-I", os.path.join(ROOT, "include"), "-o", exe],
                            input="\n".join(lines), capture_output=True, text=True)
        assert cc.returncode == 0, cc.stderr
        got = json.loads(subprocess.run([exe], capture_output=True, text=True, check=True).stdout)
    finally:
        shutil.rmtree(scratch, ignore_errors=True)
    for cname, py in pairs.items():
        assert got[cname]["size"] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[cname][f] == getattr(py, f).offset, (cname, f)


def test_allocation_failure_injection_on_the_host(lib):
    """With injection at 0, the first allocation of a build from host memory
    fails with RSI_ERR_OOM (-3) before any device work and no handle is
    returned; switched off, the same call goes on to the device."""
    import numpy as np
    L = lib.lib
    V = np.zeros((3, 3), np.float32)
    T = np.array([[0, 1, 2]], np.int32)
    h = ctypes.c_void_p()
    lib.fail_allocations(0)
    try:
        rc = L.lbvh_build_host(V.ctypes.data, 3, T.ctypes.data, 1, 4, 30, None, ctypes.byref(h))
        assert rc == -3 and "injected" in lib.last_error() and not h.value
    finally:
        lib.fail_allocations(None)
    rc = L.lbvh_build_host(V.ctypes.data, 3, T.ctypes.data, 1, 4, 30, None, ctypes.byref(h))
    assert rc == 0 or "injected" not in lib.last_error()
    if rc == 0:
        L.lbvh_free(h)


def test_size_limits_at_the_boundary(lib):
    """The largest sizes the header allows pass the argument checks and the
    next ones are refused, before any device work: n_triangles < 2^30,
    n_vertices <= 2^31, n_rays < 2^31, and RSI_NOALLOC_MAX_RAYS for the
    no-allocation query.  (The accepted build stops at its first allocation,
    refused by the failure-injection hook.)"""
    L, P = lib.lib, ctypes.c_void_p
    h = ctypes.c_void_p()
    fake = P(256)                       # never dereferenced on these paths
    assert L.lbvh_build(fake, 3, fake, 1 << 30, 4, 30, None, ctypes.byref(h)) == -1
    assert "n_triangles" in lib.last_error()
    assert L.lbvh_build(fake, (1 << 31) + 1, fake, 1, 4, 30, None, ctypes.byref(h)) == -1
    lib.fail_allocations(0)
    try:
        assert L.lbvh_build(fake, 1 << 31, fake, (1 << 30) - 1, 4, 30, None, ctypes.byref(h)) == -3
        assert "injected" in lib.last_error() and not h.value
    finally:
        lib.fail_allocations(None)
    big = 1 << 31
    assert L.rsi_query(fake, fake, fake, big, 0, None, fake, None, None, None, None) == -1
    assert "2^31" in lib.last_error()
    assert L.rsi_query_host(fake, fake, fake, big, 1, None, None, fake, None, None, None) == -1
    assert L.rsi_query_nearest(fake, fake, fake, big, None, fake, None, None, None, None, None, None) == -1
    assert L.rsi_query_noalloc(fake, fake, fake, big, 0, None, fake, None, None, None) == -1
    assert L.rsi_query_noalloc(fake, fake, fake, 2_097_152 + 1, 0, None, fake, None, None, None) == -1
    assert "RSI_NOALLOC_MAX_RAYS" in lib.last_error()


def test_binding_refuses_bad_buffers_before_any_call(lib):
    """Buffers the library would read or write through are checked first:
    segments of different shapes or in the wrong memory, outputs of the wrong
    type, too small or not contiguous.  (A handle is never reached: the
    object below has none.)"""
    import torch
    b = lib.LBVH.__new__(lib.LBVH)
    b._h = None
    F = torch.zeros(10, 3, dtype=torch.float32)
    with pytest.raises(TypeError):
        b.query(F, F, "any_hit")                                   # host segments to the device query
    with pytest.raises(TypeError):
        b.nearest(F, F)
    with pytest.raises(ValueError):
        b.query_host(F, F[:5], "any_hit")                           # lengths differ
    with pytest.raises(TypeError):
        b.query_host(F, F, "any_hit", hit=torch.zeros(10, dtype=torch.int32))
    with pytest.raises(ValueError):
        b.query_host(F, F, "count", count=torch.zeros(9, dtype=torch.int32))
    with pytest.raises(TypeError):
        b.query_host(F, F, "any_hit", ambiguous=torch.zeros(20, dtype=torch.uint8)[::2])
    with pytest.raises(TypeError):
        b.query_host(F[:, [0, 2, 1]].t().contiguous().t(), F, "any_hit")   # not contiguous
    with pytest.raises(TypeError):
        lib.query_learned(None, None, F, F)
    with pytest.raises(TypeError):
        lib.activation(torch.zeros(4))


def test_binding_refuses_bad_buffers_of_the_other_calls(lib):
    """As above for the compaction, the batched plans, the network and the
    labels: host tensors, mismatched shapes, wrong element types and sizes are
    refused before the library is called."""
    import numpy as np
    import torch
    F = torch.zeros(6, 3, dtype=torch.float32)
    with pytest.raises(TypeError):
        lib.compact_hits(torch.zeros(6, dtype=torch.int32), None, None)        # host memory
    with pytest.raises(TypeError):
        lib.BatchPlan([(None, F, F)], "any_hit")
    with pytest.raises(TypeError):
        lib.cluster_labels(None, F, F)
    net = lib.MLP.__new__(lib.MLP)
    net._m, net.n_params = None, 16 * 128 + 128 * 128 + 128 * 256 + 128 + 128 + 256
    with pytest.raises(TypeError):
        net.forward(None, F, F)
    with pytest.raises(TypeError):
        net.train_step(None, F, F, torch.zeros(6, 8, dtype=torch.int32))
    with pytest.raises(ValueError):
        net.set_params(np.zeros(10, np.float32))
