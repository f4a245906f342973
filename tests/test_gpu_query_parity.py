"""GPU queries (FP32 traversal + FP64 re-test) against the FP64 brute-force
oracle through the C ABI.

Bar: hit flags and crossing counts identical on every segment the oracle
does not mark ambiguous; the ambiguous marks themselves identical (the FP64
re-test evaluates the definition with the same IEEE operations).  At full
size the oracle checks a seeded sample plus every segment the GPU marked."""
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


def _gpu_both(rsi, bvh, F, E, **kw):
    dF, dE = _dev(F), _dev(E)
    a = bvh.query(dF, dE, "any_hit", **kw)
    c = bvh.query(dF, dE, "count", hit=torch.empty(len(F), dtype=torch.uint8, device="cuda"), **kw)
    torch.cuda.synchronize()
    return dict(hit=a["hit"].cpu().numpy(), amb_hit=a["ambiguous"].cpu().numpy(),
                count=c["count"].cpu().numpy(), amb_count=c["ambiguous"].cpu().numpy(),
                hit_from_count=c["hit"].cpu().numpy() if c["hit"] is not None else None)


def _compare(got, ref, idx=None, allow_amb_mismatch=0):
    sel = slice(None) if idx is None else idx
    g = {k: (v[sel] if v is not None else None) for k, v in got.items()}
    # the ambiguity marks follow the definition; identical by construction
    assert int(np.sum(g["amb_hit"] != ref["amb_hit"])) <= allow_amb_mismatch
    assert int(np.sum(g["amb_count"] != ref["amb_count"])) <= allow_amb_mismatch
    ok_h = (ref["amb_hit"] == 0) & (g["amb_hit"] == 0)
    ok_c = (ref["amb_count"] == 0) & (g["amb_count"] == 0)
    bad_h = np.flatnonzero(g["hit"][ok_h] != ref["hit"][ok_h])
    bad_c = np.flatnonzero(g["count"][ok_c] != ref["count"][ok_c])
    assert bad_h.size == 0, f"{bad_h.size} hit flags differ"
    assert bad_c.size == 0, f"{bad_c.size} counts differ"
    return int(ok_h.sum()), int(ok_c.sum())


def test_case_study1_and_canopy(rsi):
    for name, expect_key in (("case_study1_sec4_1.txt", "boolean"), ("canopy_sec4_1_5.txt", "count")):
        g = load(name)
        bvh = rsi.LBVH(_dev(g["vertices"]), _dev(g["triangles"]))
        got = _gpu_both(rsi, bvh, g["ray_from"], g["ray_to"])
        if expect_key == "boolean":
            assert got["hit"].tolist() == g["boolean"].tolist()
        else:
            assert got["count"].tolist() == g["count"].tolist()
        assert got["amb_hit"].sum() == 0 and got["amb_count"].sum() == 0


@pytest.mark.parametrize("node_width", [2, 3, 4])
@pytest.mark.parametrize("bits", [30, 63])
def test_c1_full_parity(rsi, bits, node_width):
    """32x32 heightfield, 1e5 segments: every segment checked, with the
    child-pair and the four-wide traversal."""
    mesh = W.config_mesh("c1")
    F, E = W.rays(W.config_rays("c1"), mesh)
    ref = oracle.query(mesh.vertices, mesh.triangles, F, E)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles), morton_bits=bits)
    got = _gpu_both(rsi, bvh, F, E, node_width=node_width)
    nh, nc = _compare(got, ref)
    assert nh > 0.99 * len(F)
    assert np.array_equal(got["hit_from_count"], (got["count"] > 0).astype(np.uint8))
    # ambiguous segments: both sides report the closed-interval reading
    amb = ref["amb_count"] == 1
    assert np.array_equal(got["count"][amb], ref["count"][amb])


def test_small_meshes_and_ragged_sizes(rsi):
    """Single triangle, two triangles, tiny heightfields; odd ray counts."""
    rng = np.random.default_rng(1)
    cases = [(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), np.array([[0, 1, 2]], np.int32))]
    m = W.heightfield(2, seed=5)
    cases.append((m.vertices, m.triangles))
    for n in (3, 7, 40):
        m = W.heightfield(n, seed=n)
        cases.append((m.vertices, m.triangles))
    for V, T in cases:
        for nr in (1, 31, 257, 5003):
            F = rng.uniform(-0.2, 1.2, (nr, 3)).astype(np.float32)
            E = rng.uniform(-0.2, 1.2, (nr, 3)).astype(np.float32)
            F[:, 2] -= 0.6
            E[:, 2] += 0.6
            ref = oracle.query(V, T, F, E)
            bvh = rsi.LBVH(_dev(V), _dev(T))
            for w in (2, 4):
                _compare(_gpu_both(rsi, bvh, F, E, node_width=w), ref)


def test_edge_vertex_and_degenerate_segments(rsi):
    """Segments through vertices and edges of a heightfield, zero-length
    segments, segments lying in a face, NaN segments."""
    m = W.heightfield(9, seed=4)
    V, T = m.vertices, m.triangles
    rng = np.random.default_rng(2)
    P = []
    for j in range(len(T)):
        a, b, c = V[T[j]].astype(np.float64)
        P += [a, 0.5 * (a + b), (a + b + c) / 3]
    P = np.array(P)
    F = (P + [0, 0, -1]).astype(np.float32)
    E = (P + [0, 0, 1]).astype(np.float32)
    Z = P[:50].astype(np.float32)                                    # zero length on the surface
    a, b, c = V[T[0]]
    inface = np.stack([a + 0.1 * (b - a), a + 0.8 * (c - a)]).astype(np.float32)
    F = np.concatenate([F, Z, inface[:1], [[np.nan, 0, 0]]]).astype(np.float32)
    E = np.concatenate([E, Z, inface[1:], [[0, 0, 1]]]).astype(np.float32)
    ref = oracle.query(V, T, F, E)
    bvh = rsi.LBVH(_dev(V), _dev(T))
    got = _gpu_both(rsi, bvh, F, E)
    _compare(got, ref)
    assert ref["amb_count"].sum() > len(T)          # vertex and edge crossings
    assert got["hit"][-1] == 0 and got["amb_hit"][-1] == 1   # NaN: undefined


def test_c2_full_size_sampled(rsi):
    """100x100 heightfield with bumps, 1e7 segments (50% crossing, 50% above)
    in the launch configuration the benchmark times: a seeded sample plus
    every segment the GPU marked ambiguous, checked against the oracle."""
    mesh = W.config_mesh("c2")
    spec = W.config_rays("c2")
    F, E = W.rays(spec, mesh)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    got = _gpu_both(rsi, bvh, F, E)
    rng = np.random.default_rng(12)
    marked = np.flatnonzero(got["amb_hit"] | got["amb_count"])
    idx = np.unique(np.concatenate([rng.choice(len(F), 12000, replace=False), marked[:2000]]))
    ref = oracle.query(mesh.vertices, mesh.triangles, F[idx], E[idx])
    _compare(got, ref, idx)
    # the other half of the workload: segments above the surface never hit
    above = np.minimum(F[:, 2], E[:, 2]) > mesh.z_max
    assert got["hit"][above].sum() == 0 and got["count"][above].sum() == 0


def test_c3_grazing_sample(rsi):
    """300x300 jittered heightfield (178,802 triangles): a 2e5-segment slice
    of the 1e8-segment batch with 1% grazing segments, every grazing-prone
    segment the GPU marked plus a sample checked by the oracle."""
    mesh = W.config_mesh("c3")
    spec = W.config_rays("c3")
    F, E = W.rays(spec, mesh, start=0, count=200_000)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles), morton_bits=63)
    got = _gpu_both(rsi, bvh, F, E)
    rng = np.random.default_rng(13)
    marked = np.flatnonzero(got["amb_hit"] | got["amb_count"])
    assert len(marked) > 100
    idx = np.unique(np.concatenate([rng.choice(len(F), 1500, replace=False), marked[:1500]]))
    ref = oracle.query(mesh.vertices, mesh.triangles, F[idx], E[idx])
    _compare(got, ref, idx)


def test_fp32_only_flips_are_rare(rsi):
    """Without the FP64 re-test, FP32 decisions flip on a small fraction of
    grazing segments (the Epilogue reports ~1e-6 overall); with it, none."""
    mesh = W.config_mesh("c1")
    spec = W.RaySpec("grazing_mix", 50_000, seed=21, grazing_frac=0.5)
    F, E = W.rays(spec, mesh)
    ref = oracle.query(mesh.vertices, mesh.triangles, F, E)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    plain = bvh.query(_dev(F), _dev(E), "any_hit", fp32_only=True)["hit"].cpu().numpy()
    ok = ref["amb_hit"] == 0
    flips = int(np.sum(plain[ok] != ref["hit"][ok]))
    assert flips < 0.01 * ok.sum()
    _compare(_gpu_both(rsi, bvh, F, E), ref)


def test_stats_and_host_path(rsi):
    mesh = W.config_mesh("c1")
    F, E = W.rays(W.config_rays("c1", 20000), mesh)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    r = bvh.query(_dev(F), _dev(E), "count", stats=True)
    st = r["stats"]
    assert st["n_rays"] == len(F) and st["node_visits"] >= len(F) and st["tri_tests"] > 0
    assert st["device_error"] == 0 and st["tree_height"] == bvh.info()["height"]
    h = bvh.query_host(torch.from_numpy(F).pin_memory(), torch.from_numpy(E).pin_memory(), "count")
    assert np.array_equal(h["count"].numpy(), r["count"].cpu().numpy())
    assert np.array_equal(h["ambiguous"].numpy(), r["ambiguous"].cpu().numpy())
    # empty batch is a no-op
    e = bvh.query(torch.empty(0, 3, device="cuda"), torch.empty(0, 3, device="cuda"), "any_hit")
    assert e["hit"].numel() == 0


@pytest.mark.parametrize("block,bps", [(64, 2), (128, 16), (256, 1), (32, 64)])
def test_launch_shapes_agree(rsi, block, bps):
    mesh = W.config_mesh("c1")
    F, E = W.rays(W.config_rays("c1", 30011), mesh)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    base = bvh.query(_dev(F), _dev(E), "count")["count"].cpu().numpy()
    other = bvh.query(_dev(F), _dev(E), "count", block=block, blocks_per_sm=bps)["count"].cpu().numpy()
    assert np.array_equal(base, other)


def test_bad_launch_shape_rejected(rsi):
    mesh = W.config_mesh("c1")
    F, E = W.rays(W.config_rays("c1", 100), mesh)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    for block in (512, 48, 1024):
        with pytest.raises(rsi.RSIError) as e:
            bvh.query(_dev(F), _dev(E), "any_hit", block=block)
        assert e.value.code == -1


@pytest.mark.parametrize("tile", [256, 1000, 4096, 8192])
def test_ray_sort_tile_changes_nothing(rsi, tile):
    """Reordering segments inside tiles before traversal leaves every answer
    unchanged (ragged last tile included)."""
    mesh = W.config_mesh("c2")
    F, E = W.rays(W.config_rays("c2", 200_003), mesh)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    dF, dE = _dev(F), _dev(E)
    for mode, key in (("any_hit", "hit"), ("count", "count")):
        a = bvh.query(dF, dE, mode)
        b = bvh.query(dF, dE, mode, ray_sort_tile=tile)
        assert torch.equal(a[key], b[key]) and torch.equal(a["ambiguous"], b["ambiguous"])
    with pytest.raises(rsi.RSIError):
        bvh.query(dF, dE, "any_hit", ray_sort_tile=100)


def test_host_path_streams_chunks(rsi):
    """Host buffers, several 2M-segment chunks and a ragged tail, staged
    whole or through recycled slots: the same answers and counters as the
    device-buffer query."""
    mesh = W.config_mesh("c2")
    F, E = W.rays(W.config_rays("c2", 5_000_007), mesh)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    pF, pE = torch.from_numpy(F).pin_memory(), torch.from_numpy(E).pin_memory()
    for mode, key in (("any_hit", "hit"), ("count", "count")):
        d = bvh.query(_dev(F), _dev(E), mode, stats=True)
        # the whole batch staged on the device, then (with in-tile reordering)
        # 2M-segment chunks recycled through two staging slots
        for tile in (0, 2048):
            h = bvh.query_host(pF, pE, mode, stats=True, ray_sort_tile=tile)
            assert np.array_equal(h[key].numpy(), d[key].cpu().numpy()), (mode, tile)
            assert np.array_equal(h["ambiguous"].numpy(), d["ambiguous"].cpu().numpy()), (mode, tile)
            assert h["stats"]["band_rays"] == d["stats"]["band_rays"], (mode, tile)
            assert h["stats"]["ambiguous"] == d["stats"]["ambiguous"], (mode, tile)
    # pageable (not page-locked) host memory works too, only slower
    h = bvh.query_host(torch.from_numpy(F), torch.from_numpy(E), "any_hit")
    assert np.array_equal(h["hit"].numpy(), bvh.query(_dev(F), _dev(E), "any_hit")["hit"].cpu().numpy())


def test_node_widths_agree_on_c2(rsi):
    """Child-pair and four-wide traversal give identical outputs, all modes,
    on 2^21 segments of the c2 workload; a bad width is rejected."""
    mesh = W.config_mesh("c2")
    F, E = W.rays(W.config_rays("c2"), mesh, count=1 << 21)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    dF, dE = _dev(F), _dev(E)
    for mode in ("any_hit", "count"):
        a = bvh.query(dF, dE, mode, node_width=2, stats=True)
        b = bvh.query(dF, dE, mode, node_width=4, stats=True)
        for k in ("hit", "count", "ambiguous"):
            if a[k] is not None:
                assert torch.equal(a[k], b[k]), (mode, k)
        # the four-wide walk fetches fewer nodes for the same answers
        assert b["stats"]["node_visits"] < a["stats"]["node_visits"]
        assert b["stats"]["band_rays"] == a["stats"]["band_rays"]
        # compressed nodes: the same answers from boxes that are only ever larger
        q = bvh.query(dF, dE, mode, node_width=3, stats=True)
        for k in ("hit", "count", "ambiguous"):
            if a[k] is not None:
                assert torch.equal(a[k], q[k]), (mode, k)
        if mode == "count":   # every overlap is visited: larger boxes, at least the same visits
            assert a["stats"]["node_visits"] <= q["stats"]["node_visits"]
        assert q["stats"]["node_visits"] <= 1.05 * a["stats"]["node_visits"]
    na, nb = bvh.nearest(dF, dE, node_width=2), bvh.nearest(dF, dE, node_width=4)
    nq = bvh.nearest(dF, dE, node_width=3)
    for k in ("tri", "t", "dist", "ambiguous"):
        assert torch.equal(na[k], nb[k]), k
        assert torch.equal(na[k], nq[k]), k
    assert torch.equal(torch.nan_to_num(na["point"], nan=-7.0), torch.nan_to_num(nb["point"], nan=-7.0))
    with pytest.raises(rsi.RSIError):
        bvh.query(dF, dE, "any_hit", node_width=5)


@pytest.mark.parametrize("m", [6_000, 40_000])
def test_fp64_pass_overflow_paths_match_oracle(rsi, m):
    """Segments lying in an exactly flat surface: every triangle they cross
    is an ambiguous pair, so every segment goes to the FP64 pass. 6,000 (a
    queue the warp-per-segment collect takes) or 40,000 (the thread-per-
    segment collect) of them exceed the pass's per-segment list (4,096
    entries at these sizes) and its pair list, and the long ones cross more
    than 32 triangles: those segments are settled by the warp-per-segment
    kernel instead. All modes must still equal the oracle, ambiguous marks
    included."""
    n = 21
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    V = np.stack([i.ravel() / (n - 1), j.ravel() / (n - 1), np.zeros(n * n)], 1).astype(np.float32)
    T = W.grid_triangles(n)
    rng = np.random.default_rng(11)
    F = np.zeros((m, 3), np.float32)
    E = np.zeros((m, 3), np.float32)
    F[:, :2] = rng.uniform(0.02, 0.98, (m, 2))
    L = np.where(rng.uniform(size=m) < 0.1, 0.9, rng.uniform(0.05, 0.3, m))
    ang = rng.uniform(0, 2 * np.pi, m)
    E[:, 0] = F[:, 0] + L * np.cos(ang)
    E[:, 1] = F[:, 1] + L * np.sin(ang)
    # and 2,000 steep segments through grid vertices and edge midpoints:
    # several inclusive crossings at one t (merged to one; the nearest is
    # the lowest triangle id)
    k = 2000
    g = rng.integers(1, 2 * (n - 1), (k, 2)) / (2.0 * (n - 1))
    tilt = rng.uniform(-0.2, 0.2, (k, 2))
    F2 = np.concatenate([g - 0.3 * tilt, -0.3 * np.ones((k, 1))], 1).astype(np.float32)
    E2 = np.concatenate([g + 0.2 * tilt, 0.2 * np.ones((k, 1))], 1).astype(np.float32)
    F, E = np.concatenate([F, F2]), np.concatenate([E, E2])
    ref = oracle.query(V, T, F, E)
    assert ref["count"][m:].sum() > 500 and (ref["near_tri"][m:] >= 0).sum() > 500
    assert ref["amb_count"].sum() > 4096
    bvh = rsi.LBVH(_dev(V), _dev(T))
    got = _gpu_both(rsi, bvh, F, E)
    _compare(got, ref)
    st = bvh.query(_dev(F), _dev(E), "count", stats=True)["stats"]
    assert st["band_rays"] > 4096 and st["device_error"] == 0
    # ambiguous segments: both sides give the closed-interval reading
    amb = ref["amb_count"] == 1
    assert np.array_equal(got["count"][amb], ref["count"][amb])
    nr = bvh.nearest(_dev(F), _dev(E))
    assert np.array_equal(nr["tri"].cpu().numpy(), ref["near_tri"])
    assert np.array_equal(nr["t"].cpu().numpy(), ref["near_t"])


def test_fp64_pass_long_pair_list_matches_oracle(rsi):
    """6e5 segments over an exactly flat surface, 1e5 of them lying in it:
    the FP64 pass lists more than 2^17 (segment, triangle) pairs, so the
    undecided ones are settled in a separate pass of their own; the rest
    lie above the surface. Every mode equals the oracle on every segment."""
    n = 21
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    V = np.stack([i.ravel() / (n - 1), j.ravel() / (n - 1), np.zeros(n * n)], 1).astype(np.float32)
    T = W.grid_triangles(n)
    rng = np.random.default_rng(12)
    m, k = 600_000, 100_000
    F = rng.uniform(0.0, 1.0, (m, 3)).astype(np.float32)
    E = (F + rng.uniform(-0.05, 0.05, (m, 3))).astype(np.float32)
    F[:, 2] += 0.5
    E[:, 2] = F[:, 2] + 0.1
    L = rng.uniform(0.05, 0.3, k)
    ang = rng.uniform(0, 2 * np.pi, k)
    F[:k, 2] = 0.0
    E[:k, 0] = F[:k, 0] + L * np.cos(ang)
    E[:k, 1] = F[:k, 1] + L * np.sin(ang)
    E[:k, 2] = 0.0
    ref = oracle.query(V, T, F, E)
    bvh = rsi.LBVH(_dev(V), _dev(T))
    _compare(_gpu_both(rsi, bvh, F, E), ref)
    st = bvh.query(_dev(F), _dev(E), "count", stats=True)["stats"]
    assert st["band_rays"] >= 0.9 * k and st["device_error"] == 0
    nr = bvh.nearest(_dev(F), _dev(E))
    assert np.array_equal(nr["tri"].cpu().numpy(), ref["near_tri"])


@pytest.mark.parametrize("n", [1, 31, 1 << 18, (1 << 18) + 1, (1 << 18) + (1 << 21) + 7])
def test_host_path_chunk_boundaries(rsi, n):
    """The whole-batch host path at its chunk boundaries (a first chunk of
    2^18 segments, then 2^21): the same results as the device path, with and
    without the FP64 re-test."""
    mesh = W.config_mesh("c2")
    F, E = W.rays(W.config_rays("c2", n), mesh)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    pF, pE = torch.from_numpy(F).pin_memory(), torch.from_numpy(E).pin_memory()
    for fp32_only in (False, True):
        for mode, key in (("any_hit", "hit"), ("count", "count")):
            d = bvh.query(_dev(F), _dev(E), mode, fp32_only=fp32_only)
            h = bvh.query_host(pF, pE, mode, fp32_only=fp32_only, stats=True)
            assert np.array_equal(h[key].numpy(), d[key].cpu().numpy()), (n, mode, fp32_only)
            assert np.array_equal(h["ambiguous"].numpy(), d["ambiguous"].cpu().numpy()), (n, mode, fp32_only)
            assert h["stats"]["n_rays"] == n and h["stats"]["device_error"] == 0


@pytest.mark.parametrize("mode", ["any_hit", "count", "both"])
def test_host_path_pinned_outputs(rsi, mode):
    """Page-locked host outputs: the FP32 answers are copied out chunk by
    chunk (2^21 segments) as the traversal finishes them and the queued
    segments' answers are written into the host arrays after the FP64 pass --
    every entry equals the device path's, on the grazing c3 mix (many queued
    segments), on a short c2 batch and on a c3 batch of three output chunks."""
    for cfg, n, bits in (("c3", 600_000, 63), ("c2", 70_001, 30), ("c3", 4_500_001, 63)):
        mesh = W.config_mesh(cfg)
        F, E = W.rays(W.config_rays(cfg), mesh, count=n)
        bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles), morton_bits=bits)
        d = bvh.query(_dev(F), _dev(E), mode)
        outs = {}
        if mode in ("any_hit", "both"):
            outs["hit"] = torch.empty(n, dtype=torch.uint8).pin_memory()
        if mode in ("count", "both"):
            outs["count"] = torch.empty(n, dtype=torch.int32).pin_memory()
        outs["ambiguous"] = torch.empty(n, dtype=torch.uint8).pin_memory()
        for t in outs.values():
            t.fill_(0xAB if t.dtype == torch.uint8 else -7)   # stale values must not survive
        h = bvh.query_host(torch.from_numpy(F).pin_memory(), torch.from_numpy(E).pin_memory(), mode,
                           stats=True, **outs)
        assert h["stats"]["band_rays"] > 0
        for k, t in outs.items():
            assert torch.equal(t, d[k].cpu()), (cfg, mode, k)


def test_host_path_whole_batch_above_2_26(rsi):
    """A host batch of 2^26 + 12,345 segments (1.6 GB of segments in, 64
    chunks): staged whole, its answers in both modes at once equal the
    device path's on every segment.  Segments drawn on the device from a
    seeded generator over the c1 mesh's box (the bulk is what is tested)."""
    n = (1 << 26) + 12_345
    mesh = W.config_mesh("c1")
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles))
    lo = torch.tensor(mesh.vertices.min(0), device="cuda")
    hi = torch.tensor(mesh.vertices.max(0), device="cuda")
    g = torch.Generator(device="cuda").manual_seed(2626)
    span = (hi - lo) * 1.2
    dF = (lo - 0.1 * (hi - lo) + torch.rand(n, 3, device="cuda", generator=g) * span).contiguous()
    dE = (lo - 0.1 * (hi - lo) + torch.rand(n, 3, device="cuda", generator=g) * span).contiguous()
    d = bvh.query(dF, dE, "both")
    pF, pE = dF.cpu().pin_memory(), dE.cpu().pin_memory()
    del dF, dE
    h = bvh.query_host(pF, pE, "both", stats=True)
    assert h["stats"]["n_rays"] == n and h["stats"]["device_error"] == 0
    for k in ("hit", "count", "ambiguous"):
        assert torch.equal(h[k], d[k].cpu()), k
    assert int(d["hit"].sum()) > n // 10


@pytest.mark.parametrize("cfg,n", [("c2", 10_000_000), ("c3", 2_000_000), ("c3", 4_000_000)])
def test_fp32_decisions_equal_fp64_everywhere(rsi, cfg, n):
    """Every segment of a full-size batch (c2: all 1e7; c3: 2e6 and 4e6
    slices with 1 % grazing segments -- the larger one queues over 32,768
    segments in the count mode, so the default path takes the long-queue
    collect) answered twice: by the default path (FP32 with certified
    decisions, FP64 for the band) and with every segment settled by the FP64
    re-test. All outputs of all three modes must be identical -- the claim
    that a certain FP32 decision is the FP64 decision, checked on every
    segment rather than on an oracle sample."""
    mesh = W.config_mesh(cfg)
    F, E = W.rays(W.config_rays(cfg), mesh, count=n)
    bvh = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles), morton_bits=63 if cfg == "c3" else 30)
    dF, dE = _dev(F), _dev(E)
    for mode, key in (("any_hit", "hit"), ("count", "count")):
        a = bvh.query(dF, dE, mode, stats=True)
        if cfg == "c3" and n > 3_000_000 and mode == "count":
            assert a["stats"]["band_rays"] >= 32768   # the long-queue collect ran
        b = bvh.query(dF, dE, mode, fp64_all=True, stats=True)
        assert b["stats"]["band_rays"] == n
        assert torch.equal(a[key], b[key]), mode
        assert torch.equal(a["ambiguous"], b["ambiguous"]), mode
    a, b = bvh.nearest(dF, dE), bvh.nearest(dF, dE, fp64_all=True)
    for k in ("tri", "t", "dist", "ambiguous"):
        assert torch.equal(a[k], b[k]), k
    assert torch.equal(torch.nan_to_num(a["point"], nan=-7.0), torch.nan_to_num(b["point"], nan=-7.0))
    with pytest.raises(rsi.RSIError):
        bvh.query(dF[:10], dE[:10], "any_hit", fp64_all=True, fp32_only=True)


@pytest.mark.parametrize("stack", [64, 128])
def test_stack_size_leaves_answers_unchanged(rsi, stack):
    """A larger traversal stack than the tree needs (a tuning choice) gives
    the same answers in both modes; sizes other than 0/32/64/128 are refused."""
    m = W.config_mesh("c1")
    F, E = W.rays(W.config_rays("c1", 50_000), m)
    bvh = rsi.LBVH(torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.triangles).cuda())
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    for mode, key in (("any_hit", "hit"), ("count", "count")):
        a, b = bvh.query(dF, dE, mode), bvh.query(dF, dE, mode, stack=stack)
        assert torch.equal(a[key], b[key]) and torch.equal(a["ambiguous"], b["ambiguous"])
    with pytest.raises(rsi.RSIError):
        bvh.query(dF, dE, "any_hit", stack=48)
    bvh.close()


def test_segment_order_is_a_permutation_and_keeps_answers(rsi):
    """rsi_segment_order writes a permutation of the batch sorted by midpoint
    cell; queries walking the segments in that order give the answers of
    the input order at the segments' own indices, in all three modes."""
    m = W.config_mesh("c2")
    n = 300_007
    F, E = W.rays(W.config_rays("c2", n), m)
    bvh = rsi.LBVH(torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.triangles).cuda())
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    order = bvh.segment_order(dF, dE)
    o = order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(n))
    # cells are non-decreasing along the order (32^3 grid over the extent, z-order)
    info = bvh.info()
    lo, hi = np.array(info["extent_lo"], np.float32), np.array(info["extent_hi"], np.float32)
    mid = (F[o] + E[o]) * np.float32(0.5)
    q = np.clip(((mid - lo) * (np.float32(32.0) / (hi - lo))).astype(np.float32), 0, 31).astype(np.int64)
    key = np.zeros(n, np.int64)
    for b in range(5):
        for a in range(3):
            key |= ((q[:, a] >> b) & 1) << (3 * b + a)
    assert np.all(np.diff(key) >= 0)
    for mode, k in (("any_hit", "hit"), ("count", "count")):
        a, b = bvh.query(dF, dE, mode), bvh.query(dF, dE, mode, order=order)
        assert torch.equal(a[k], b[k]) and torch.equal(a["ambiguous"], b["ambiguous"]), mode
    with pytest.raises(rsi.RSIError):
        bvh.query(dF, dE, "any_hit", order=order, ray_sort_tile=2048)
    bvh.close()


def _both_matches(rsi, bvh, dF, dE):
    """RSI_BOTH against the two separate queries on every segment: the hit
    flag is the boolean answer, the count the count answer, and the
    ambiguity byte carries both modes' flags (bit 0 boolean, bit 1 count)."""
    a = bvh.query(dF, dE, "any_hit")
    c = bvh.query(dF, dE, "count")
    b = bvh.query(dF, dE, "both")
    assert torch.equal(b["hit"], a["hit"])
    assert torch.equal(b["count"], c["count"])
    assert torch.equal(b["ambiguous"] & 1, a["ambiguous"])
    assert torch.equal(b["ambiguous"] >> 1, c["ambiguous"])
    return b


def test_both_modes_in_one_pass_c1_against_oracle(rsi):
    """The combined pass on the c1 workload, every segment against the
    oracle's boolean and intercept_count answers (Sec. 1)."""
    m = W.config_mesh("c1")
    F, E = W.rays(W.config_rays("c1"), m)
    F[11] = np.nan    # undefined segment: ambiguous in both modes, hit 0, count 0
    bvh = rsi.LBVH(torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.triangles).cuda())
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    b = _both_matches(rsi, bvh, dF, dE)
    ref = oracle.query(m.vertices, m.triangles, F, E)
    amb = b["ambiguous"].cpu().numpy()
    hit, cnt = b["hit"].cpu().numpy(), b["count"].cpu().numpy()
    assert np.array_equal(amb & 1, ref["amb_hit"]) and np.array_equal(amb >> 1, ref["amb_count"])
    ok_h, ok_c = ref["amb_hit"] == 0, ref["amb_count"] == 0
    assert np.array_equal(hit[ok_h], ref["hit"][ok_h]) and np.array_equal(cnt[ok_c], ref["count"][ok_c])
    assert amb[11] == 3 and hit[11] == 0 and cnt[11] == 0
    bvh.close()


def test_both_modes_in_one_pass_grazing_and_host(rsi):
    """On a grazing-heavy slice of the c3 recipe (1 % of the segments end
    within 1e-6 of an edge or vertex or run nearly parallel to a face) the
    two modes' ambiguity flags differ on many segments; the combined pass
    still equals both separate queries, on device and host buffers."""
    m = W.config_mesh("c3")
    F, E = W.rays(W.config_rays("c3"), m, 0, 1 << 20)
    bvh = rsi.LBVH(torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.triangles).cuda(), morton_bits=63)
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    b = _both_matches(rsi, bvh, dF, dE)
    amb = b["ambiguous"].cpu().numpy()
    assert ((amb >> 1) != (amb & 1)).sum() > 100   # count-ambiguous segments settled by a decisive hit
    h = bvh.query_host(torch.from_numpy(F).pin_memory(), torch.from_numpy(E).pin_memory(), "both")
    for k in ("hit", "count", "ambiguous"):
        assert torch.equal(h[k], b[k].cpu()), k
    bvh.close()
