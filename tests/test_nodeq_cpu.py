"""Compressed child-pair nodes (NodeQ), checked on the CPU (no GPU).

The build kernel k_quantize and the traversal's decode are restated in
numpy: per internal node, the node's own box minimum is the frame origin,
each axis gets the smallest power-of-two step whose 255 multiples cover the
box, and each child plane becomes an 8-bit grid coordinate chosen so that
the traversal's rebuilt value -- fma rounded down for a lower plane, up for
an upper one -- lies outside the exact plane.  Claims: every rebuilt child
box contains the exact one (so culling stays conservative), the right child
is always the left one + 1, and the rebuilt boxes add almost no visits."""
import numpy as np
import pytest

import oracle
import workloads as W

F32, F64 = np.float32, np.float64
LEAF = 0x80000000


def _fma_dir(q, step, o, up):
    """float32 rounding toward +inf (up) or -inf of q * step + o, exactly
    (q * step is exact in float64; the sum's error comes from a two-sum)."""
    p = q.astype(F64) * step.astype(F64)
    o64 = o.astype(F64)
    s = p + o64
    bb = s - p
    err = (p - (s - bb)) + (o64 - bb)            # s + err == p + o exactly
    r = s.astype(F32)
    diff = (r.astype(F64) - s) - err            # sign of r - (p + o)
    if up:
        return np.where(diff < 0, np.nextafter(r, F32(np.inf)), r)
    return np.where(diff > 0, np.nextafter(r, F32(-np.inf)), r)


def _grid_exponent(ext):
    need = ext * (1.0 + 2.0 ** -40)
    k = np.full(ext.shape, -126, np.int64)
    pos = ext > 0
    kk = np.floor(np.log2(np.where(pos, need, 1.0) / 255.0)).astype(np.int64)
    for _ in range(3):                               # fix-ups of the log2 estimate
        kk = np.where(np.ldexp(255.0, kk) < need, kk + 1, kk)
        kk = np.where((kk > -126) & (np.ldexp(255.0, kk - 1) >= need), kk - 1, kk)
    return np.where(pos, np.maximum(kk, -126), k)


def _quant(x, o, step, up):
    q = ((x.astype(F64) - o.astype(F64)) / step.astype(F64))
    q = np.clip(np.ceil(q) if up else np.floor(q), 0, 255)
    for _ in range(300):                             # the kernel's fix-up loops
        if up:
            inc = (q < 255) & (_fma_dir(q.astype(F32), step, o, True) < x)
            dec = (q > 0) & (_fma_dir((q - 1).astype(F32), step, o, True) >= x)
        else:
            dec = (q > 0) & (_fma_dir(q.astype(F32), step, o, False) > x)
            inc = (q < 255) & (_fma_dir((q + 1).astype(F32), step, o, False) <= x)
        if not (inc.any() or dec.any()):
            break
        q = q + inc - dec
    return q.astype(F32)


def quantize(b):
    """Rebuilt child boxes (n-1, 2, 6) and the split / leaf flags of every
    internal node of an oracle hierarchy."""
    n = len(b["perm"])
    box = b["box"]
    refs = []
    cb = np.empty((n - 1, 2, 6), F32)
    for k, arr in enumerate((b["left"], b["right"])):
        ref = arr.astype(np.int64) & 0xFFFFFFFF
        leaf = (ref & LEAF) != 0
        idx = np.where(leaf, n - 1 + (ref & ~LEAF), ref)
        cb[:, k] = box[idx]
        refs.append((ref & ~LEAF, leaf))
    lo = np.minimum(cb[:, 0, 0:3], cb[:, 1, 0:3])
    hi = np.maximum(cb[:, 0, 3:6], cb[:, 1, 3:6])
    k = _grid_exponent(hi.astype(F64) - lo.astype(F64))
    step = np.ldexp(np.ones(k.shape, F32), k.astype(np.int32)).astype(F32)
    out = np.empty_like(cb)
    for c in range(2):
        ql = _quant(cb[:, c, 0:3], lo, step, False)
        qh = _quant(cb[:, c, 3:6], lo, step, True)
        out[:, c, 0:3] = _fma_dir(ql, step, lo, False)
        out[:, c, 3:6] = _fma_dir(qh, step, lo, True)
    return cb, out, refs, k


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_rebuilt_boxes_contain_the_exact_ones(name):
    mesh = W.config_mesh(name)
    b = oracle.build_all(mesh.vertices, mesh.triangles, bits=63 if name == "c3" else 30)
    exact, rebuilt, refs, k = quantize(b)
    assert np.all(rebuilt[:, :, 0:3] <= exact[:, :, 0:3]) and np.all(rebuilt[:, :, 3:6] >= exact[:, :, 3:6])
    (left, _), (right, _) = refs
    assert np.array_equal(right, left + 1)           # one index names both children
    assert k.min() >= -126 and k.max() <= 127
    # the grid is fine: the rebuilt boxes are at most a few steps larger
    grow = (rebuilt[:, :, 3:6] - rebuilt[:, :, 0:3]) - (exact[:, :, 3:6] - exact[:, :, 0:3])
    node_ext = np.maximum(exact[:, :, 3:6].max(1) - exact[:, :, 0:3].min(1), 1e-30)
    assert np.quantile(grow.max(1) / node_ext, 0.99) < 2.5 / 255 * 2


def test_far_from_the_origin_and_flat():
    """Boxes far from the origin (large origin, small extent) and flat axes
    are still contained."""
    rng = np.random.default_rng(3)
    V = (rng.uniform(-1, 1, (300, 3)) * [1e-3, 1e-3, 0.0] + [4096.5, -3e4, 7.25]).astype(F32)
    T = rng.integers(0, 300, (400, 3)).astype(np.int32)
    b = oracle.build_all(V, T, bits=30)
    exact, rebuilt, _, _ = quantize(b)
    assert np.all(rebuilt[:, :, 0:3] <= exact[:, :, 0:3]) and np.all(rebuilt[:, :, 3:6] >= exact[:, :, 3:6])
