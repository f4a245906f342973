"""Barycentric mode on the GPU (nearest crossing: triangle, t, point,
distance; Sec. 1 and Sec. 3.3) against the FP64 brute-force oracle through
the C ABI.

Bar: identical on every segment, ambiguous ones included.  The triangle is
an index decided by floating point, and both sides decide it in FP64 with
the same IEEE operations (the GPU only skips FP64 where FP32 error bounds
already prove the order of the crossings); t, point and distance are FP64
values of the definition rounded once to FP32 on both sides, so they are
compared bit for bit.  At full size the oracle checks a seeded sample plus
every segment the GPU marked ambiguous."""
import numpy as np
import pytest

import oracle
import workloads as W
from golden_io import load

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rsi():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2305_01867_gb300 as m
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _nearest(bvh, F, E, **kw):
    r = bvh.nearest(_dev(F), _dev(E), **kw)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in r.items()}


def _compare(got, ref, idx=None):
    sel = slice(None) if idx is None else idx
    g = {k: v[sel] for k, v in got.items() if isinstance(v, np.ndarray)}
    assert np.array_equal(g["ambiguous"], ref["amb_count"]), "ambiguity marks differ"
    bad = np.flatnonzero(g["tri"] != ref["near_tri"])
    assert bad.size == 0, f"{bad.size} nearest triangles differ, e.g. {bad[:5]}"
    assert np.array_equal(g["t"].view(np.uint32), ref["near_t"].view(np.uint32))
    assert np.array_equal(g["dist"].view(np.uint32), ref["near_dist"].view(np.uint32))
    hit = ref["near_tri"] >= 0
    assert np.array_equal(g["point"][hit].view(np.uint32), ref["near_point"][hit].view(np.uint32))
    assert np.isnan(g["point"][~hit]).all()
    return int(hit.sum())


def test_case_study1_hit_points(rsi):
    """The worked example of Sec. 4.1: the printed intersecting points."""
    g = load("case_study1_sec4_1.txt")
    bvh = rsi.LBVH(_dev(g["vertices"]), _dev(g["triangles"]))
    got = _nearest(bvh, g["ray_from"], g["ray_to"])
    for ray, tri, point in g["hitpoint"]:
        assert got["tri"][ray] == tri
        np.testing.assert_allclose(got["point"][ray], point, atol=2e-6)
    assert (got["tri"] >= 0).tolist() == [bool(b) for b in g["boolean"]]
    _compare(got, oracle.query(g["vertices"], g["triangles"], g["ray_from"], g["ray_to"]))


@pytest.mark.parametrize("bits", [30, 63])
def test_c1_full_parity(rsi, bits):
    """32x32 heightfield, 1e5 segments: every segment checked."""
    mesh = W.config_mesh("c1")
    F, E = W.rays(W.config_rays("c1"), mesh)
    ref = oracle.query(mesh.vertices, mesh.triangles, F, E)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles), morton_bits=bits)
    got = _nearest(bvh, F, E, stats=True)
    assert _compare(got, ref) > 0.3 * len(F)
    assert got["stats"]["device_error"] == 0


def test_grazing_and_multiple_crossings(rsi):
    """Half grazing segments (edges, vertices, near-parallel) on the c1 mesh,
    and long segments that cross the surface several times: the FP64 pass
    settles both the band pairs and crossings too close to order in FP32."""
    mesh = W.config_mesh("c1")
    F, E = W.rays(W.RaySpec("grazing_mix", 30_000, seed=21, grazing_frac=0.5), mesh)
    rng = np.random.default_rng(3)
    m = 5000   # nearly horizontal segments through the relief: several crossings each
    z = rng.uniform(-0.1, 0.1, m)
    F2 = np.c_[rng.uniform(0, 0.2, m), rng.uniform(0, 1, m), z].astype(np.float32)
    E2 = np.c_[rng.uniform(0.8, 1, m), rng.uniform(0, 1, m), z + rng.uniform(-0.02, 0.02, m)].astype(np.float32)
    F, E = np.concatenate([F, F2]), np.concatenate([E, E2])
    ref = oracle.query(mesh.vertices, mesh.triangles, F, E)
    assert (ref["count"][-m:] > 1).sum() > 1000
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    got = _nearest(bvh, F, E, stats=True)
    _compare(got, ref)
    assert got["stats"]["band_rays"] > 0 and got["ambiguous"].sum() > 0


def test_c2_sample_and_compaction(rsi):
    """100x100 heightfield, 2e5 segments of the 1e7-segment batch; the
    compacted (rays, distances, triangles, points) form of Sec. 2.3."""
    mesh = W.config_mesh("c2")
    F, E = W.rays(W.config_rays("c2", 200_000), mesh)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    got = _nearest(bvh, F, E)
    rng = np.random.default_rng(12)
    marked = np.flatnonzero(got["ambiguous"])
    idx = np.unique(np.concatenate([rng.choice(len(F), 8000, replace=False), marked[:2000]]))
    sub = oracle.query(mesh.vertices, mesh.triangles, F[idx], E[idx])
    _compare(got, sub, idx)
    rays, dist, tri, point = bvh.barycentric(_dev(F), _dev(E))
    want = np.flatnonzero(got["tri"] >= 0)
    assert np.array_equal(rays.cpu().numpy(), want)
    assert np.array_equal(tri.cpu().numpy(), got["tri"][want])
    assert np.array_equal(dist.cpu().numpy(), got["dist"][want])
    assert np.array_equal(point.cpu().numpy(), got["point"][want])


def test_c3_grazing_sample(rsi):
    """300x300 jittered heightfield, 63-bit codes, 1% grazing segments."""
    mesh = W.config_mesh("c3")
    F, E = W.rays(W.config_rays("c3"), mesh, start=0, count=100_000)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles), morton_bits=63)
    got = _nearest(bvh, F, E)
    rng = np.random.default_rng(13)
    marked = np.flatnonzero(got["ambiguous"])
    assert len(marked) > 50
    idx = np.unique(np.concatenate([rng.choice(len(F), 1200, replace=False), marked[:1200]]))
    _compare(got, oracle.query(mesh.vertices, mesh.triangles, F[idx], E[idx]), idx)


def test_degenerate_inputs(rsi):
    """One triangle (the tree is a single leaf), coincident plates (equal t:
    lower index), zero-length and NaN segments, an empty batch."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]] * 3, np.float32)
    V[3:6, 2] = 0.5
    T = np.arange(9, dtype=np.int32).reshape(3, 3)[[1, 0, 2]]   # plates at z = 0.5, 0, 0
    F = np.array([[0.2, 0.2, -1], [0.2, 0.2, 1], [0.2, 0.2, 0.3], [0.6, 0.6, -1], [np.nan, 0, 0]], np.float32)
    E = np.array([[0.2, 0.2, 1], [0.2, 0.2, -1], [0.2, 0.2, 0.3], [0.6, 0.6, 1], [1, 1, 1]], np.float32)
    for tris in (T, T[:1]):
        ref = oracle.query(V, tris, F, E)
        bvh = rsi.LBVH(_dev(V), _dev(tris))
        got = _nearest(bvh, F, E)
        _compare(got, ref)
    assert got["ambiguous"][4] == 1 and got["tri"][4] == -1
    empty = bvh.nearest(torch.empty(0, 3, device="cuda"), torch.empty(0, 3, device="cuda"))
    assert empty["tri"].numel() == 0
    rays, dist, tri, point = rsi.compact_hits(empty["tri"], empty["dist"], empty["point"])
    assert rays.numel() == 0


def test_options_change_nothing(rsi):
    """Launch shapes and in-tile segment reordering leave every answer as is;
    the uncorrected FP32 decisions still name a triangle the segment meets."""
    mesh = W.config_mesh("c2")
    F, E = W.rays(W.config_rays("c2", 100_003), mesh)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    base = _nearest(bvh, F, E)
    for kw in (dict(ray_sort_tile=4096), dict(block=64, blocks_per_sm=2)):
        other = _nearest(bvh, F, E, **kw)
        for k in ("tri", "t", "dist", "ambiguous"):
            assert np.array_equal(base[k].view(np.uint8), other[k].view(np.uint8)), (kw, k)
    plain = _nearest(bvh, F, E, fp32_only=True)
    same = (plain["tri"] == base["tri"]).mean()
    assert same > 0.999
    # the nearest mode has its own entry point: rsi_query refuses it
    dF, dE, out = _dev(F), _dev(E), torch.empty(len(F), dtype=torch.int32, device="cuda")
    rc = rsi.lib.rsi_query(bvh.handle, rsi._ptr(dF), rsi._ptr(dE), len(F), rsi.RSI_NEAREST, None, None,
                           rsi._ptr(out), None, None, rsi._stream(None))
    assert rc == -1
