"""GB300 (sm_103a) linear-BVH ray-segment / triangle-surface intersection.

A thin binding over the C ABI of ``librsi.so`` (declared in include/rsi.h):
argument checking and marshalling only -- every step of the build and the
query runs in the library's CUDA kernels.  PyTorch supplies device memory
and streams.  If the library is missing this module raises on import; there
is no CPU fallback.

    import paper_2305_01867_gb300 as rsi
    bvh = rsi.LBVH(vertices_cuda_f32, triangles_cuda_i32, morton_bits=30)
    hit = bvh.query(ray_from, ray_to, mode="any_hit")["hit"]       # Sec. 1 boolean
    cnt = bvh.query(ray_from, ray_to, mode="count")["count"]       # intercept_count
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB as _LIB_PATH
from .build import build as build_library

RSI_OK = 0
RSI_ANY_HIT, RSI_COUNT, RSI_NEAREST, RSI_BOTH = 0, 1, 2, 3
NOALLOC_MAX_RAYS = 1 << 21   # RSI_NOALLOC_MAX_RAYS of include/rsi.h
LEAF_TAG = 0x80000000
ERRORS = {-1: "INVALID_ARG", -2: "DTYPE", -3: "OOM", -4: "CUDA", -5: "TIMEOUT", -6: "STACK", -7: "NAN",
          -8: "INDEX", -9: "OVERFLOW"}


class RSIError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("fp32_only", ctypes.c_int), ("block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("collect_stats", ctypes.c_int), ("timeout_ns", ctypes.c_int64), ("time_kernels", ctypes.c_int),
                ("ray_sort_tile", ctypes.c_int), ("node_width", ctypes.c_int), ("fp64_all", ctypes.c_int),
                ("stack", ctypes.c_int), ("order", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("n_rays", ctypes.c_int64), ("node_visits", ctypes.c_int64), ("tri_tests", ctypes.c_int64),
                ("band_rays", ctypes.c_int64), ("ambiguous", ctypes.c_int64), ("tree_height", ctypes.c_int32),
                ("device_error", ctypes.c_int32), ("proposal_confirmed", ctypes.c_int64),
                ("fallback_rays", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [("n_triangles", ctypes.c_int64), ("n_vertices", ctypes.c_int64), ("morton_bits", ctypes.c_int32),
                ("height", ctypes.c_int32), ("device_bytes", ctypes.c_int64), ("extent_lo", ctypes.c_float * 3),
                ("extent_hi", ctypes.c_float * 3), ("max_tri_extent", ctypes.c_float * 3)]


class HostView(ctypes.Structure):
    _fields_ = [("sorted_keys", ctypes.c_void_p), ("perm", ctypes.c_void_p), ("left", ctypes.c_void_p),
                ("right", ctypes.c_void_p), ("parent", ctypes.c_void_p), ("box", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("ray_sort_tile", ctypes.c_int),
                ("stack", ctypes.c_int), ("ms", ctypes.c_float), ("from_cache", ctypes.c_int),
                ("candidates", ctypes.c_int), ("node_width", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RayBatch(ctypes.Structure):
    _fields_ = [("bvh", ctypes.c_void_p), ("d_from", ctypes.c_void_p), ("d_to", ctypes.c_void_p),
                ("n_rays", ctypes.c_int64), ("d_hit", ctypes.c_void_p), ("d_count", ctypes.c_void_p),
                ("d_ambiguous", ctypes.c_void_p)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"librsi.so is not built ({_LIB_PATH}); run paper_2305_01867_gb300.build_library()")
    lib = ctypes.CDLL(_LIB_PATH)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.lbvh_build.argtypes = [P, i64, P, i64, i32, i32, P, ctypes.POINTER(P)]
    lib.lbvh_build_host.argtypes = [P, i64, P, i64, i32, i32, P, ctypes.POINTER(P)]
    lib.lbvh_build_host_ex.argtypes = [P, i64, P, i64, i32, i32, i32, P, ctypes.POINTER(P)]
    lib.lbvh_build_host_ex.restype = ctypes.c_int
    lib.lbvh_build_ex.argtypes = [P, i64, P, i64, i32, i32, i32, P, ctypes.POINTER(P)]
    lib.lbvh_build_ex.restype = ctypes.c_int
    lib.lbvh_build_batched.argtypes = [i32, ctypes.POINTER(P), ctypes.POINTER(i64), ctypes.POINTER(P),
                                       ctypes.POINTER(i64), i32, i32, P, ctypes.POINTER(P)]
    lib.lbvh_build_batched.restype = ctypes.c_int
    lib.lbvh_build_batched_ex.argtypes = [i32, ctypes.POINTER(P), ctypes.POINTER(i64), ctypes.POINTER(P),
                                          ctypes.POINTER(i64), i32, i32, i32, P, ctypes.POINTER(P)]
    lib.lbvh_build_batched_ex.restype = ctypes.c_int
    lib.lbvh_free.argtypes = [P]
    lib.lbvh_info.argtypes = [P, ctypes.POINTER(Info)]
    lib.lbvh_export.argtypes = [P, P, ctypes.POINTER(HostView)]
    lib.lbvh_node_bytes.restype = ctypes.c_size_t
    lib.lbvh_node_bytes.argtypes = []
    for f in (lib.rsi_query, lib.rsi_query_host):
        f.argtypes = [P, P, P, i64, i32, ctypes.POINTER(Options), P, P, P, ctypes.POINTER(Stats), P]
    lib.rsi_query_noalloc.argtypes = [P, P, P, i64, i32, ctypes.POINTER(Options), P, P, P, P]
    lib.rsi_query_nearest.argtypes = [P, P, P, i64, ctypes.POINTER(Options), P, P, P, P, P, ctypes.POINTER(Stats), P]
    lib.rsi_query_nearest.restype = ctypes.c_int
    lib.rsi_nearest_compact.argtypes = [P, P, P, i64, P, P, P, P, ctypes.POINTER(ctypes.c_int64), P]
    lib.rsi_nearest_compact.restype = ctypes.c_int
    lib.rsi_query_noalloc.restype = ctypes.c_int
    lib.rsi_segment_order.argtypes = [P, P, P, i64, P, P]
    lib.rsi_segment_order.restype = ctypes.c_int
    lib.rsi_last_query_ms.argtypes = [P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    lib.rsi_last_query_ms.restype = ctypes.c_int
    lib.rsi_kernel_launches.argtypes = []
    lib.rsi_kernel_launches.restype = ctypes.c_uint64
    lib.rsi_autotune.argtypes = [P, P, P, i64, i32, ctypes.c_char_p, ctypes.POINTER(Options), ctypes.POINTER(Tuning), P]
    lib.rsi_batch_autotune.argtypes = [ctypes.POINTER(RayBatch), i32, i32, ctypes.c_char_p, ctypes.POINTER(Options),
                                       ctypes.POINTER(Tuning), P]
    lib.rsi_batch_autotune.restype = ctypes.c_int
    lib.rsi_autotune.restype = ctypes.c_int
    lib.rsi_batch_create.argtypes = [ctypes.POINTER(RayBatch), i32, i32, ctypes.POINTER(Options), P,
                                     ctypes.POINTER(P)]
    lib.rsi_batch_launch.argtypes = [P, P]
    lib.rsi_batch_create_rebuild.argtypes = [ctypes.POINTER(RayBatch), i32, ctypes.POINTER(P), ctypes.POINTER(P), i32,
                                             ctypes.POINTER(Options), P, ctypes.POINTER(P)]
    lib.rsi_batch_create_rebuild.restype = ctypes.c_int
    lib.rsi_query_batched.argtypes = [ctypes.POINTER(P), i32, ctypes.POINTER(RayBatch), i32, ctypes.POINTER(Options),
                                      P]
    lib.rsi_batch_post.argtypes = [P, i64, P]
    lib.rsi_batch_stats.argtypes = [P, ctypes.POINTER(Stats), P]
    lib.rsi_batch_free.argtypes = [P]
    for name in ("rsi_batch_create", "rsi_batch_launch", "rsi_query_batched", "rsi_batch_post", "rsi_batch_stats",
                 "rsi_batch_free"):
        getattr(lib, name).restype = ctypes.c_int
    lib.rsi_mlp_create.argtypes = [ctypes.c_uint64, ctypes.POINTER(P)]
    lib.rsi_mlp_free.argtypes = [P]
    lib.rsi_mlp_num_params.argtypes = []
    lib.rsi_mlp_set_params.argtypes = [P, P, P]
    lib.rsi_mlp_get_params.argtypes = [P, P, P, P]
    lib.rsi_mlp_forward.argtypes = [P, P, P, P, i64, P, P, P]
    lib.rsi_mlp_status.argtypes = [P, P]
    lib.rsi_mlp_activation.argtypes = [P, i64, P, P, P, P]
    lib.rsi_mlp_activation.restype = ctypes.c_int
    lib.rsi_mlp_train_step.argtypes = [P, P, P, P, P, i64, ctypes.c_float, i32, ctypes.POINTER(ctypes.c_float), P]
    lib.rsi_mlp_reset_optimizer.argtypes = [P, P]
    lib.rsi_mlp_attach.argtypes = [P, P]
    lib.rsi_mlp_attach.restype = ctypes.c_int
    lib.rsi_cluster_labels.argtypes = [P, P, P, i64, P, P]
    lib.rsi_query_learned.argtypes = [P, P, P, P, i64, ctypes.POINTER(Options), P, P, ctypes.POINTER(Stats), P]
    for name in ("rsi_mlp_train_step", "rsi_mlp_reset_optimizer", "rsi_cluster_labels", "rsi_query_learned"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("rsi_mlp_create", "rsi_mlp_free", "rsi_mlp_num_params", "rsi_mlp_set_params", "rsi_mlp_get_params",
                 "rsi_mlp_forward", "rsi_mlp_status"):
        getattr(lib, name).restype = ctypes.c_int
    lib.rsi_last_error.restype = ctypes.c_char_p
    lib.rsi_debug_fail_allocations.argtypes = [i64]
    lib.rsi_debug_fail_allocations.restype = i32
    lib.rsi_last_error.argtypes = []
    for name in ("lbvh_build", "lbvh_build_host", "lbvh_free", "lbvh_info", "lbvh_export", "rsi_query",
                 "rsi_query_host"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()


def last_error() -> str:
    return lib.rsi_last_error().decode()


def check(rc: int):
    if rc != RSI_OK:
        raise RSIError(rc, last_error())


def kernel_launches() -> int:
    """Kernels the library has launched since it was loaded."""
    return int(lib.rsi_kernel_launches())


def fail_allocations(after: int | None):
    """Test hook: the next `after` allocations of the library succeed, the
    later ones fail with RSI_ERR_OOM; None switches injection off."""
    lib.rsi_debug_fail_allocations(-1 if after is None else int(after))


def node_bytes() -> int:
    return int(lib.lbvh_node_bytes())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_out(t, name, dtype, n, device):
    """A caller-supplied buffer the library reads or writes: `dtype`,
    contiguous, at least n elements, on `device` (a torch.device, or "host"
    for host memory).  Only its pointer crosses the ABI, so a wrong buffer is
    refused here.  None passes (an optional buffer left out)."""
    import torch
    if t is None:
        return
    if not isinstance(t, torch.Tensor) or t.dtype != dtype:
        raise TypeError(f"{name} must be a {dtype} tensor")
    if not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous")
    if device == "host":
        if t.is_cuda:
            raise TypeError(f"{name} must be in host memory")
    elif t.device != device:
        raise TypeError(f"{name} must be on {device}")
    if t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} elements, {n} are written")


def _check_segments(ray_from, ray_to):
    """Segment end points for a device call: [n, 3] float32, contiguous,
    equal shapes, both on one GPU."""
    _check_f32x3(ray_from, "ray_from")
    _check_f32x3(ray_to, "ray_to")
    if ray_from.shape != ray_to.shape:
        raise ValueError("ray_from and ray_to differ in shape")
    if not (ray_from.is_cuda and ray_to.is_cuda) or ray_to.device != ray_from.device:
        raise TypeError("segments must be device tensors on one GPU")


def _check_f32x3(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 3:
        raise TypeError(f"{name} must be a float32 tensor of shape [n, 3]")
    if not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous")


def _mode(mode):
    if mode in ("any_hit", "boolean", RSI_ANY_HIT):
        return RSI_ANY_HIT
    if mode in ("count", "intercept_count", RSI_COUNT):
        return RSI_COUNT
    if mode in ("both", RSI_BOTH):
        return RSI_BOTH
    raise ValueError(f"unknown mode {mode!r}")


_TREE_BUILDERS = {"karras": 0, "apetrei": 1}   # RSI_TREE_KARRAS, RSI_TREE_APETREI


class LBVH:
    """A linear BVH over a triangle mesh, built on the GPU (lbvh_build).

    builder: "karras" (radix tree, then refit) or "apetrei" (one bottom-up
    pass, lbvh_build_ex; device inputs only).  Both give the same hierarchy.
    treelet_passes: 0 (the paper's tree) or 1-3 restructuring passes after
    the build (RSI_TREE_TREELETS): same answers, fewer nodes met per segment.
    """

    def __init__(self, vertices, triangles, morton_bits: int = 30, stream=None, builder: str = "karras",
                 treelet_passes: int = 0):
        import torch
        _check_f32x3(vertices, "vertices")
        if not isinstance(triangles, torch.Tensor) or triangles.dim() != 2 or triangles.shape[1] != 3:
            raise TypeError("triangles must be a tensor of shape [n, 3]")
        index_bytes = triangles.element_size()
        if triangles.dtype not in (torch.int32, torch.int64):
            raise TypeError("triangles must hold integer vertex indices")
        self._h = ctypes.c_void_p()
        on_dev = vertices.is_cuda
        if on_dev != triangles.is_cuda:
            raise TypeError("vertices and triangles must both be on the GPU or both on the host")
        if builder not in _TREE_BUILDERS:
            raise ValueError(f"unknown builder {builder!r} (karras or apetrei)")
        if int(treelet_passes) not in (0, 1, 2, 3):
            raise ValueError("treelet_passes must be 0, 1, 2 or 3")
        code = _TREE_BUILDERS[builder] | (int(treelet_passes) << 8)   # | RSI_TREE_TREELETS(passes)
        if builder == "karras" and treelet_passes:
            fn = lib.lbvh_build_ex if on_dev else lib.lbvh_build_host_ex
            check(fn(_ptr(vertices), vertices.shape[0], _ptr(triangles.contiguous()), triangles.shape[0],
                     index_bytes, morton_bits, code, _stream(stream), ctypes.byref(self._h)))
        elif builder == "karras":
            fn = lib.lbvh_build if on_dev else lib.lbvh_build_host
            check(fn(_ptr(vertices), vertices.shape[0], _ptr(triangles.contiguous()), triangles.shape[0],
                     index_bytes, morton_bits, _stream(stream), ctypes.byref(self._h)))
        else:
            if not on_dev:
                raise TypeError("the apetrei builder takes device tensors")
            check(lib.lbvh_build_ex(_ptr(vertices), vertices.shape[0], _ptr(triangles.contiguous()),
                                    triangles.shape[0], index_bytes, morton_bits, code,
                                    _stream(stream), ctypes.byref(self._h)))
        self.n_triangles = triangles.shape[0]

    @classmethod
    def _adopt(cls, handle, n_triangles):
        """Wrap a handle built elsewhere (build_many)."""
        obj = cls.__new__(cls)
        obj._h = handle
        obj.n_triangles = n_triangles
        return obj

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.lbvh_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def attach(self, net):
        """Attach a proposal network (rsi_mlp_attach; None detaches): boolean
        queries on this hierarchy then go through the learned proposal,
        with the same answers."""
        check(lib.rsi_mlp_attach(self._h, net.handle if net is not None else None))
        self._net = net   # keep the network alive while attached

    def info(self) -> dict:
        inf = Info()
        check(lib.lbvh_info(self._h, ctypes.byref(inf)))
        d = {k: getattr(inf, k) for k, _ in Info._fields_}
        for k in ("extent_lo", "extent_hi", "max_tri_extent"):
            d[k] = list(d[k])
        return d

    def export(self, stream=None) -> dict:
        """Host copy of keys, order, children, parents and boxes (Sec. 4.1.1)."""
        import numpy as np
        n = self.n_triangles
        out = dict(sorted_keys=np.zeros(n, np.uint64), perm=np.zeros(n, np.int32),
                   left=np.zeros(max(n - 1, 1), np.int32), right=np.zeros(max(n - 1, 1), np.int32),
                   parent=np.zeros(2 * n - 1, np.int32), box=np.zeros((2 * n - 1, 6), np.float32))
        v = HostView(*[out[k].ctypes.data for k in ("sorted_keys", "perm", "left", "right", "parent", "box")])
        check(lib.lbvh_export(self._h, _stream(stream), ctypes.byref(v)))
        if n == 1:
            out["left"], out["right"] = out["left"][:0], out["right"][:0]
        return out

    def autotune(self, ray_from, ray_to, mode="any_hit", cache_path=None, stream=None) -> dict:
        """Pick block / blocks_per_sm / ray_sort_tile for queries like this one
        (rsi_autotune); the result's keys can be passed straight to query()."""
        _check_f32x3(ray_from, "ray_from")
        _check_f32x3(ray_to, "ray_to")
        opt, res = Options(), Tuning()
        path = cache_path.encode() if cache_path else None
        check(lib.rsi_autotune(self._h, _ptr(ray_from), _ptr(ray_to), ray_from.shape[0], _mode(mode), path,
                               ctypes.byref(opt), ctypes.byref(res), _stream(stream)))
        return res.as_dict()

    def segment_order(self, ray_from, ray_to, out=None, stream=None):
        """A traversal order for these segments (rsi_segment_order): int32
        [n] device tensor, a permutation of 0 .. n - 1 by midpoint cell, to
        pass as query(..., order=...)."""
        import torch
        _check_segments(ray_from, ray_to)
        n = ray_from.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=ray_from.device)
        _check_out(out, "order", torch.int32, n, ray_from.device)
        check(lib.rsi_segment_order(self._h, _ptr(ray_from), _ptr(ray_to), n, _ptr(out), _stream(stream)))
        return out

    def last_query_ms(self):
        """(traversal ms, FP64 re-test ms) of the last query run with time_kernels=True."""
        a, b = ctypes.c_float(), ctypes.c_float()
        check(lib.rsi_last_query_ms(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def query(self, ray_from, ray_to, mode="any_hit", *, fp32_only=False, block=0, blocks_per_sm=0,
              stats=False, hit=None, count=None, ambiguous=None, want_ambiguous=True, time_kernels=False,
              ray_sort_tile=0, node_width=0, fp64_all=False, stack=0, order=None, stream=None):
        """Query segments (device tensors [n, 3] float32).  mode: "any_hit",
        "count" or "both" (one pass answering both; 'ambiguous' then holds
        bit 0 = the boolean mode's flag, bit 1 = the count mode's).  Returns
        a dict with 'hit' (uint8, any-hit answer or count > 0), 'count'
        (int32), 'ambiguous' (uint8) and, with stats=True, 'stats'."""
        import torch
        _check_f32x3(ray_from, "ray_from")
        _check_f32x3(ray_to, "ray_to")
        if ray_from.shape != ray_to.shape:
            raise ValueError("ray_from and ray_to differ in shape")
        if not (ray_from.is_cuda and ray_to.is_cuda):
            raise TypeError("query() takes device tensors; use query_host() for host arrays")
        m = _mode(mode)
        n = ray_from.shape[0]
        dev = ray_from.device
        if hit is None and m in (RSI_ANY_HIT, RSI_BOTH):
            hit = torch.empty(n, dtype=torch.uint8, device=dev)
        if count is None and m in (RSI_COUNT, RSI_BOTH):
            count = torch.empty(n, dtype=torch.int32, device=dev)
        if ambiguous is None and want_ambiguous:
            ambiguous = torch.empty(n, dtype=torch.uint8, device=dev)
        if ray_to.device != dev:
            raise TypeError("ray_from and ray_to must be on the same device")
        _check_out(hit, "hit", torch.uint8, n, dev)
        _check_out(count, "count", torch.int32, n, dev)
        _check_out(ambiguous, "ambiguous", torch.uint8, n, dev)
        _check_out(order, "order", torch.int32, n, dev)
        opt = Options(int(fp32_only), int(block), int(blocks_per_sm), int(stats), 0, int(time_kernels),
                      int(ray_sort_tile), int(node_width), int(fp64_all), int(stack),
                      order.data_ptr() if order is not None else None)
        st = Stats()
        check(lib.rsi_query(self._h, _ptr(ray_from), _ptr(ray_to), n, m, ctypes.byref(opt), _ptr(hit), _ptr(count),
                            _ptr(ambiguous), ctypes.byref(st) if stats else None, _stream(stream)))
        out = {"hit": hit, "count": count, "ambiguous": ambiguous}
        if stats:
            out["stats"] = st.as_dict()
        return out

    def query_host(self, ray_from, ray_to, mode="any_hit", *, fp32_only=False, stats=False, hit=None, count=None,
                   ambiguous=None, want_ambiguous=True, ray_sort_tile=0, stream=None):
        """As query() with host (preferably pinned) tensors; blocks until the
        results are in host memory."""
        import torch
        _check_f32x3(ray_from, "ray_from")
        _check_f32x3(ray_to, "ray_to")
        if ray_from.shape != ray_to.shape:
            raise ValueError("ray_from and ray_to differ in shape")
        if ray_from.is_cuda or ray_to.is_cuda:
            raise TypeError("query_host() takes host tensors; use query() for device tensors")
        m = _mode(mode)
        n = ray_from.shape[0]
        if hit is None and m in (RSI_ANY_HIT, RSI_BOTH):
            hit = torch.empty(n, dtype=torch.uint8)
        if count is None and m in (RSI_COUNT, RSI_BOTH):
            count = torch.empty(n, dtype=torch.int32)
        if ambiguous is None and want_ambiguous:
            ambiguous = torch.empty(n, dtype=torch.uint8)
        _check_out(hit, "hit", torch.uint8, n, "host")
        _check_out(count, "count", torch.int32, n, "host")
        _check_out(ambiguous, "ambiguous", torch.uint8, n, "host")
        opt = Options(int(fp32_only), 0, 0, int(stats), 0, 0, int(ray_sort_tile))
        st = Stats()
        check(lib.rsi_query_host(self._h, _ptr(ray_from), _ptr(ray_to), n, m, ctypes.byref(opt), _ptr(hit),
                                 _ptr(count), _ptr(ambiguous), ctypes.byref(st), _stream(stream)))
        out = {"hit": hit, "count": count, "ambiguous": ambiguous}
        if stats:
            out["stats"] = st.as_dict()
        return out


    def nearest(self, ray_from, ray_to, *, fp32_only=False, block=0, blocks_per_sm=0, stats=False,
                want_t=True, want_point=True, want_dist=True, want_ambiguous=True, time_kernels=False,
                ray_sort_tile=0, node_width=0, fp64_all=False, stream=None):
        """Barycentric mode per segment (rsi_query_nearest): 'tri' (int32, -1
        when no hit), 't', 'point' [n, 3], 'dist' (float32), 'ambiguous'."""
        import torch
        _check_f32x3(ray_from, "ray_from")
        _check_f32x3(ray_to, "ray_to")
        if ray_from.shape != ray_to.shape:
            raise ValueError("ray_from and ray_to differ in shape")
        if not (ray_from.is_cuda and ray_to.is_cuda):
            raise TypeError("nearest() takes device tensors")
        if ray_to.device != ray_from.device:
            raise TypeError("ray_from and ray_to must be on the same device")
        n = ray_from.shape[0]
        dev = ray_from.device
        tri = torch.empty(n, dtype=torch.int32, device=dev)
        t = torch.empty(n, dtype=torch.float32, device=dev) if want_t else None
        point = torch.empty(n, 3, dtype=torch.float32, device=dev) if want_point else None
        dist = torch.empty(n, dtype=torch.float32, device=dev) if want_dist else None
        amb = torch.empty(n, dtype=torch.uint8, device=dev) if want_ambiguous else None
        opt = Options(int(fp32_only), int(block), int(blocks_per_sm), int(stats), 0, int(time_kernels),
                      int(ray_sort_tile), int(node_width), int(fp64_all))
        st = Stats()
        check(lib.rsi_query_nearest(self._h, _ptr(ray_from), _ptr(ray_to), n, ctypes.byref(opt), _ptr(tri), _ptr(t),
                                    _ptr(point), _ptr(dist), _ptr(amb), ctypes.byref(st) if stats else None,
                                    _stream(stream)))
        out = {"tri": tri, "t": t, "point": point, "dist": dist, "ambiguous": amb}
        if stats:
            out["stats"] = st.as_dict()
        return out

    def barycentric(self, ray_from, ray_to, stream=None):
        """The paper's barycentric result (Sec. 2.3): (intersecting_rays,
        distances, hit_triangles, hit_points) for the segments that meet the
        surface, in increasing segment order."""
        r = self.nearest(ray_from, ray_to, want_t=False, want_ambiguous=False, stream=stream)
        return compact_hits(r["tri"], r["dist"], r["point"], stream=stream)


def build_many(meshes, morton_bits: int = 30, stream=None, treelet_passes: int = 0):
    """Hierarchies of many meshes in one build (lbvh_build_batched_ex): meshes
    is a list of (vertices, triangles) device tensors ([n, 3] float32, [m, 3]
    int32); returns one LBVH per mesh, each identical to LBVH(vertices,
    triangles, treelet_passes=treelet_passes)."""
    import torch
    M = len(meshes)
    if M < 1:
        raise ValueError("build_many needs at least one mesh")
    P = ctypes.c_void_p
    vp, tp = (P * M)(), (P * M)()
    nv, nt = (ctypes.c_int64 * M)(), (ctypes.c_int64 * M)()
    keep = []
    for m, (V, T) in enumerate(meshes):
        _check_f32x3(V, "vertices")
        if not isinstance(T, torch.Tensor) or T.dim() != 2 or T.shape[1] != 3 or T.dtype != torch.int32:
            raise TypeError("triangles must be int32 tensors of shape [n, 3]")
        if not (V.is_cuda and T.is_cuda):
            raise TypeError("build_many takes device tensors")
        T = T.contiguous()
        keep.append(T)
        vp[m], tp[m] = V.data_ptr(), T.data_ptr()
        nv[m], nt[m] = V.shape[0], T.shape[0]
    if int(treelet_passes) not in (0, 1, 2, 3):
        raise ValueError("treelet_passes must be 0, 1, 2 or 3")
    out = (P * M)()
    check(lib.lbvh_build_batched_ex(M, vp, nv, tp, nt, 4, morton_bits, int(treelet_passes), _stream(stream), out))
    return [LBVH._adopt(P(out[m]), int(nt[m])) for m in range(M)]


def compact_hits(tri, dist, point, stream=None):
    """rsi_nearest_compact: (segment indices, distances, triangles, points)
    of the entries with tri >= 0, in index order."""
    import torch
    if not isinstance(tri, torch.Tensor) or tri.dim() != 1 or not tri.is_cuda:
        raise TypeError("tri must be a 1-D device tensor")
    n = tri.shape[0]
    dev = tri.device
    _check_out(tri, "tri", torch.int32, n, dev)
    _check_out(dist, "dist", torch.float32, n, dev)
    _check_out(point, "point", torch.float32, 3 * n, dev)
    rays = torch.empty(n, dtype=torch.int32, device=dev)
    tri_o = torch.empty(n, dtype=torch.int32, device=dev)
    dist_o = torch.empty(n, dtype=torch.float32, device=dev) if dist is not None else None
    point_o = torch.empty(n, 3, dtype=torch.float32, device=dev) if point is not None else None
    k = ctypes.c_int64()
    check(lib.rsi_nearest_compact(_ptr(tri), _ptr(dist), _ptr(point), n, _ptr(rays), _ptr(tri_o), _ptr(dist_o),
                                  _ptr(point_o), ctypes.byref(k), _stream(stream)))
    k = k.value
    return (rays[:k], dist_o[:k] if dist_o is not None else None, tri_o[:k],
            point_o[:k] if point_o is not None else None)


class BatchPlan:
    """Many (hierarchy, segments) pairs answered by one graph-launched
    persistent traversal (rsi_batch_create / rsi_batch_launch).

    items: list of (LBVH, ray_from, ray_to) with device tensors.  Outputs
    are allocated here: .hit / .count / .ambiguous are lists of tensors.
    stream_timeout_ns > 0 makes a streaming plan fed by post()."""

    def __init__(self, items, mode="any_hit", *, fp32_only=False, block=0, blocks_per_sm=0, stats=False,
                 stream_timeout_ns=0, node_width=0, ray_sort_tile=0, stack=0, rebuild=None, stream=None):
        import torch
        m = _mode(mode)
        self.mode = m
        self.items = items
        self.hit, self.count, self.ambiguous = [], [], []
        arr = (RayBatch * len(items))()
        for i, (bvh, f, t) in enumerate(items):
            _check_segments(f, t)
            n = f.shape[0]
            h = torch.empty(n, dtype=torch.uint8, device=f.device) if m == RSI_ANY_HIT else None
            c = torch.empty(n, dtype=torch.int32, device=f.device) if m == RSI_COUNT else None
            a = torch.empty(n, dtype=torch.uint8, device=f.device)
            self.hit.append(h)
            self.count.append(c)
            self.ambiguous.append(a)
            arr[i] = RayBatch(bvh.handle.value, f.data_ptr(), t.data_ptr(), n, h.data_ptr() if h is not None else None,
                              c.data_ptr() if c is not None else None, a.data_ptr())
        timeout = -int(stream_timeout_ns) if stream_timeout_ns else 0
        opt = Options(int(fp32_only), int(block), int(blocks_per_sm), int(stats), timeout, 0, int(ray_sort_tile),
                      int(node_width), 0, int(stack))
        self._p = ctypes.c_void_p()
        if rebuild is None:
            check(lib.rsi_batch_create(arr, len(items), m, ctypes.byref(opt), _stream(stream), ctypes.byref(self._p)))
        else:   # (vertices, triangles) device tensors per item: rebuilt in the graph before the query
            if len(rebuild) != len(items):
                raise ValueError("rebuild needs one (vertices, triangles) pair per item")
            vp, tp = (ctypes.c_void_p * len(items))(), (ctypes.c_void_p * len(items))()
            for i, ((bvh, _, _), (V, T)) in enumerate(zip(items, rebuild)):
                _check_f32x3(V, "vertices")
                _check_out(T, "triangles", __import__("torch").int32, 3 * bvh.n_triangles, V.device)
                if V.shape[0] != bvh.info()["n_vertices"] or T.shape != (bvh.n_triangles, 3):
                    raise ValueError(f"rebuild mesh {i} differs in size from its hierarchy")
                vp[i], tp[i] = V.data_ptr(), T.data_ptr()
            self._rebuild = rebuild   # keep the buffers alive
            check(lib.rsi_batch_create_rebuild(arr, len(items), vp, tp, m, ctypes.byref(opt), _stream(stream),
                                               ctypes.byref(self._p)))
        self.total = sum(int(f.shape[0]) for _, f, _ in items)

    def run(self, stream=None):
        check(lib.rsi_batch_launch(self._p, _stream(stream)))

    def post(self, n_ready, stream=None):
        check(lib.rsi_batch_post(self._p, int(n_ready), _stream(stream)))

    def stats(self, stream=None, raise_on_error=True):
        st = Stats()
        rc = lib.rsi_batch_stats(self._p, ctypes.byref(st), _stream(stream))
        if raise_on_error:
            check(rc)
        return st.as_dict()

    def close(self):
        if getattr(self, "_p", None) and self._p.value:
            lib.rsi_batch_free(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def query_batched(items, mode="any_hit", *, hit=None, count=None, ambiguous=None, fp32_only=False, block=0,
                  blocks_per_sm=0, node_width=0, stream=None):
    """The one-call batched query (rsi_query_batched): items is a list of
    (LBVH, ray_from, ray_to) with device tensors; every segment is answered
    against its own hierarchy.  Outputs (lists, one tensor per item) are
    allocated unless given; the library keeps the plan of a call and
    replays it when the same hierarchies, buffers and options come back.
    Returns dict(hit=[...] or None, count=[...] or None, ambiguous=[...])."""
    import torch
    m = _mode(mode)
    k = len(items)
    if k < 1:
        raise ValueError("query_batched needs at least one item")
    hit = list(hit) if hit is not None else [None] * k
    count = list(count) if count is not None else [None] * k
    ambiguous = list(ambiguous) if ambiguous is not None else [None] * k
    hs = (ctypes.c_void_p * k)()
    arr = (RayBatch * k)()
    for i, (bvh, f, t) in enumerate(items):
        _check_segments(f, t)
        n = f.shape[0]
        if m == RSI_ANY_HIT and hit[i] is None:
            hit[i] = torch.empty(n, dtype=torch.uint8, device=f.device)
        if m == RSI_COUNT and count[i] is None:
            count[i] = torch.empty(n, dtype=torch.int32, device=f.device)
        if ambiguous[i] is None:
            ambiguous[i] = torch.empty(n, dtype=torch.uint8, device=f.device)
        _check_out(hit[i], "hit", torch.uint8, n, f.device)
        _check_out(count[i], "count", torch.int32, n, f.device)
        _check_out(ambiguous[i], "ambiguous", torch.uint8, n, f.device)
        hs[i] = bvh.handle.value
        arr[i] = RayBatch(None, f.data_ptr(), t.data_ptr(), n, *(x.data_ptr() if x is not None else None
                                                                 for x in (hit[i], count[i], ambiguous[i])))
    opt = Options(int(fp32_only), int(block), int(blocks_per_sm), 0, 0, 0, 0, int(node_width))
    check(lib.rsi_query_batched(hs, k, arr, m, ctypes.byref(opt), _stream(stream)))
    return {"hit": hit if m == RSI_ANY_HIT else None, "count": count if m == RSI_COUNT else None,
            "ambiguous": ambiguous}


def batch_autotune(items, mode="any_hit", cache_path=None, stream=None) -> dict:
    """Tune batched plans of these (LBVH, ray_from, ray_to) items
    (rsi_batch_autotune): threads per block, blocks per SM, node width,
    in-tile reordering and stack size, timed on a sample of every batch.
    The result's block / blocks_per_sm / node_width / ray_sort_tile / stack
    can be passed straight to BatchPlan."""
    m = _mode(mode)
    arr = (RayBatch * len(items))()
    for i, (bvh, f, t) in enumerate(items):
        _check_segments(f, t)
        arr[i] = RayBatch(bvh.handle.value, f.data_ptr(), t.data_ptr(), f.shape[0], None, None, None)
    opt, res = Options(), Tuning()
    path = cache_path.encode() if cache_path else None
    check(lib.rsi_batch_autotune(arr, len(items), m, path, ctypes.byref(opt), ctypes.byref(res), _stream(stream)))
    return res.as_dict()


MLP_SHAPES = (("W1", (16, 128)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (128, 256)),
              ("b3", (256,)))


class MLP:
    """The cluster-proposal network (rsi_mlp_*): 6 -> 128 -> 128 -> 256,
    BF16 weights, FP32 accumulation, tensor-core inference."""

    def __init__(self, seed: int = 0):
        self._m = ctypes.c_void_p()
        check(lib.rsi_mlp_create(int(seed), ctypes.byref(self._m)))
        self.n_params = int(lib.rsi_mlp_num_params())

    @property
    def handle(self):
        return self._m

    def close(self):
        if getattr(self, "_m", None) and self._m.value:
            lib.rsi_mlp_free(self._m)
            self._m = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def flatten(params: dict):
        import numpy as np
        return np.concatenate([np.asarray(params[k], np.float32).reshape(-1) for k, _ in MLP_SHAPES])

    @staticmethod
    def unflatten(flat):
        import numpy as np
        out, i = {}, 0
        for k, shp in MLP_SHAPES:
            n = int(np.prod(shp))
            out[k] = np.asarray(flat[i:i + n], np.float64).reshape(shp)
            i += n
        return out

    def set_params(self, params, stream=None):
        import numpy as np
        flat = self.flatten(params) if isinstance(params, dict) else np.ascontiguousarray(params, np.float32)
        if flat.size != self.n_params:
            raise ValueError(f"{flat.size} parameters given, the network has {self.n_params}")
        check(lib.rsi_mlp_set_params(self._m, flat.ctypes.data_as(ctypes.c_void_p), _stream(stream)))

    def get_params(self, grads=False, stream=None):
        import numpy as np
        p = np.zeros(self.n_params, np.float32)
        g = np.zeros(self.n_params, np.float32) if grads else None
        check(lib.rsi_mlp_get_params(self._m, p.ctypes.data_as(ctypes.c_void_p),
                                     g.ctypes.data_as(ctypes.c_void_p) if grads else None, _stream(stream)))
        return (self.unflatten(p), self.unflatten(g)) if grads else self.unflatten(p)

    def forward(self, bvh, ray_from, ray_to, logits=True, top4=True, stream=None):
        """Tensor-core inference: dict(logits=[n,256] float32, top4=[n,4] uint8)."""
        import torch
        _check_segments(ray_from, ray_to)
        n = ray_from.shape[0]
        lg = torch.empty(n, 256, dtype=torch.float32, device=ray_from.device) if logits else None
        t4 = torch.empty(n, 4, dtype=torch.uint8, device=ray_from.device) if top4 else None
        check(lib.rsi_mlp_forward(self._m, bvh.handle, _ptr(ray_from), _ptr(ray_to), n, _ptr(lg), _ptr(t4),
                                  _stream(stream)))
        return {"logits": lg, "top4": t4}

    def status(self, stream=None):
        check(lib.rsi_mlp_status(self._m, _stream(stream)))

    def train_step(self, bvh, ray_from, ray_to, labels, lr=1e-3, apply=True, want_loss=False, stream=None):
        """One GPU training step on a batch (labels: [n, 8] int32 bit masks).
        Returns the batch loss when want_loss (synchronizes)."""
        import torch
        _check_segments(ray_from, ray_to)
        n = ray_from.shape[0]
        if not isinstance(labels, torch.Tensor) or labels.dim() != 2 or labels.shape != (n, 8):
            raise TypeError("labels must be an [n, 8] tensor")
        _check_out(labels, "labels", torch.int32, 8 * n, ray_from.device)
        loss = ctypes.c_float()
        check(lib.rsi_mlp_train_step(self._m, bvh.handle, _ptr(ray_from), _ptr(ray_to), _ptr(labels),
                                     ray_from.shape[0], float(lr), int(apply),
                                     ctypes.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value if want_loss else None

    def reset_optimizer(self, stream=None):
        check(lib.rsi_mlp_reset_optimizer(self._m, _stream(stream)))

    def fit(self, bvh, ray_from, ray_to, labels, epochs=1, batch=8192, lr=1e-3, stream=None):
        """Minibatch training over the whole set (in order); returns the
        per-epoch mean loss of the last batches."""
        n = ray_from.shape[0]
        losses = []
        for _ in range(epochs):
            last = []
            for b0 in range(0, n, batch):
                b1 = min(n, b0 + batch)
                want = b0 + batch >= n or (b0 // batch) % 50 == 0
                l = self.train_step(bvh, ray_from[b0:b1], ray_to[b0:b1], labels[b0:b1], lr=lr, want_loss=want,
                                    stream=stream)
                if want:
                    last.append(l)
            losses.append(float(sum(last) / len(last)))
        return losses


def cluster_labels(bvh, ray_from, ray_to, stream=None):
    """[n, 8] int32 bit masks of the clusters each segment meets (rsi_cluster_labels)."""
    import torch
    _check_segments(ray_from, ray_to)
    n = ray_from.shape[0]
    out = torch.empty(n, 8, dtype=torch.int32, device=ray_from.device)
    check(lib.rsi_cluster_labels(bvh.handle, _ptr(ray_from), _ptr(ray_to), n, _ptr(out), _stream(stream)))
    return out


def query_learned(bvh, net, ray_from, ray_to, stats=False, hit=None, ambiguous=None, stream=None, **opts):
    """Boolean query with the learned proposal (rsi_query_learned); answers
    identical to LBVH.query(..., "any_hit")."""
    import torch
    _check_f32x3(ray_from, "ray_from")
    _check_f32x3(ray_to, "ray_to")
    if ray_from.shape != ray_to.shape:
        raise ValueError("ray_from and ray_to differ in shape")
    if not (ray_from.is_cuda and ray_to.is_cuda) or ray_to.device != ray_from.device:
        raise TypeError("query_learned() takes device tensors on one device")
    n = ray_from.shape[0]
    if hit is None:
        hit = torch.empty(n, dtype=torch.uint8, device=ray_from.device)
    if ambiguous is None:
        ambiguous = torch.empty(n, dtype=torch.uint8, device=ray_from.device)
    _check_out(hit, "hit", torch.uint8, n, ray_from.device)
    _check_out(ambiguous, "ambiguous", torch.uint8, n, ray_from.device)
    opt = Options(int(opts.get("fp32_only", 0)), int(opts.get("block", 0)), int(opts.get("blocks_per_sm", 0)),
                  int(stats), 0, 0, 0, int(opts.get("node_width", 0)))
    st = Stats()
    check(lib.rsi_query_learned(bvh.handle, net.handle, _ptr(ray_from), _ptr(ray_to), n, ctypes.byref(opt),
                                _ptr(hit), _ptr(ambiguous), ctypes.byref(st) if stats else None, _stream(stream)))
    out = {"hit": hit, "ambiguous": ambiguous}
    if stats:
        out["stats"] = st.as_dict()
    return out


def activation(z, stream=None):
    """(tanh by the hardware approximation inference uses, CUDA tanhf, GELU
    as inference applies it) of a device float32 vector (rsi_mlp_activation)."""
    import torch
    if not isinstance(z, torch.Tensor) or not z.is_cuda or z.dtype != torch.float32 or not z.is_contiguous():
        raise TypeError("z must be a contiguous float32 device tensor")
    a, b, g = torch.empty_like(z), torch.empty_like(z), torch.empty_like(z)
    check(lib.rsi_mlp_activation(_ptr(z), z.numel(), _ptr(a), _ptr(b), _ptr(g), _stream(stream)))
    return a, b, g
