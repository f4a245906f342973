"""Restructured hierarchies (lbvh_build_ex with RSI_TREE_TREELETS): the tree
stays a valid hierarchy over the same leaves, its summed node surface goes
down, and every query answers exactly as on the paper's tree and as the
oracle does."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
LEAF = 0x80000000


@pytest.fixture(scope="module")
def rsi():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2305_01867_gb300 as m
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _slot(ref, n):
    ref = np.asarray(ref, np.int64) & 0xFFFFFFFF
    return np.where(ref & LEAF, n - 1 + (ref & ~LEAF), ref)


def _check_tree(ex, plain, n):
    """A binary tree over the same leaves: every node but the root is the
    child of exactly one node, parents agree, boxes are the unions of their
    children's, everything is reachable from the root; leaves unchanged."""
    if n == 1:
        return
    L, R = _slot(ex["left"], n), _slot(ex["right"], n)
    kids = np.concatenate([L, R])
    assert np.array_equal(np.sort(kids), np.arange(1, 2 * n - 1))      # each non-root node once
    par = ex["parent"].astype(np.int64)
    assert par[0] == -1
    assert np.array_equal(par[L], np.arange(n - 1)) and np.array_equal(par[R], np.arange(n - 1))
    box = ex["box"]
    assert np.array_equal(box[: n - 1, :3], np.minimum(box[L, :3], box[R, :3]))
    assert np.array_equal(box[: n - 1, 3:], np.maximum(box[L, 3:], box[R, 3:]))
    assert np.array_equal(box[n - 1:], plain["box"][n - 1:])              # leaves and their order
    assert np.array_equal(ex["perm"], plain["perm"])
    assert np.array_equal(box[0], plain["box"][0])
    seen, st = np.zeros(2 * n - 1, bool), [0]                              # reachable, no cycle
    while st:
        i = st.pop()
        assert not seen[i]
        seen[i] = True
        if i < n - 1:
            st += [L[i], R[i]]
    assert seen.all()


def _sah(ex, n):
    b = ex["box"][: n - 1].astype(np.float64)
    e = b[:, 3:] - b[:, :3]
    return float((e[:, 0] * e[:, 1] + e[:, 1] * e[:, 2] + e[:, 2] * e[:, 0]).sum())


def _answers(bvh, dF, dE):
    out = {}
    for mode in ("any_hit", "count", "both"):
        r = bvh.query(dF, dE, mode)
        out[mode] = {k: v.cpu().numpy() for k, v in r.items() if v is not None}
    nr = bvh.nearest(dF, dE)
    out["nearest"] = {k: nr[k].cpu().numpy() for k in ("tri", "t", "dist")}
    return out


def _same(a, b):
    for mode in a:
        for k in a[mode]:
            assert np.array_equal(a[mode][k], b[mode][k]), (mode, k)


@pytest.mark.parametrize("cfg", ["c1", "c2", "c3"])
@pytest.mark.parametrize("passes", [1, 2, 3])
def test_restructured_tree_is_valid_and_tighter(rsi, cfg, passes):
    mesh = W.config_mesh(cfg)
    bits = 63 if cfg == "c3" else 30
    dV, dT = _dev(mesh.vertices), _dev(mesh.triangles)
    n = len(mesh.triangles)
    plain = rsi.LBVH(dV, dT, morton_bits=bits).export()
    t = rsi.LBVH(dV, dT, morton_bits=bits, treelet_passes=passes)
    ex = t.export()
    _check_tree(ex, plain, n)
    assert _sah(ex, n) < 0.9 * _sah(plain, n)
    assert t.info()["height"] >= int(np.ceil(np.log2(n)))
    # the same restructured tree from the single-pass builder and on a second build
    again = rsi.LBVH(dV, dT, morton_bits=bits, treelet_passes=passes, builder="apetrei").export()
    for k in ("left", "right", "parent", "box"):
        assert np.array_equal(again[k], ex[k]), k


def test_answers_equal_plain_tree_and_oracle_c1(rsi):
    """c1 (all 1e5 segments): boolean, count, both and nearest answers on the
    restructured tree equal the plain tree's and the oracle's."""
    mesh = W.config_mesh("c1")
    F, E = W.rays(W.config_rays("c1"), mesh)
    dV, dT, dF, dE = _dev(mesh.vertices), _dev(mesh.triangles), _dev(F), _dev(E)
    plain = _answers(rsi.LBVH(dV, dT), dF, dE)
    for passes in (1, 3):
        _same(_answers(rsi.LBVH(dV, dT, treelet_passes=passes), dF, dE), plain)
    ref = oracle.query(mesh.vertices, mesh.triangles, F, E)
    a = plain["both"]
    keep = ref["amb_hit"] == 0
    assert np.array_equal(a["hit"][keep], ref["hit"][keep])
    keep = ref["amb_count"] == 0
    assert np.array_equal(plain["count"]["count"][keep], ref["count"][keep])


def test_answers_equal_plain_tree_c2_c3(rsi):
    """1e6 segments of c2 and of the grazing c3 mix, all modes and node widths."""
    for cfg, bits in (("c2", 30), ("c3", 63)):
        mesh = W.config_mesh(cfg)
        F, E = W.rays(W.config_rays(cfg), mesh, count=1_000_000)
        dV, dT, dF, dE = _dev(mesh.vertices), _dev(mesh.triangles), _dev(F), _dev(E)
        plain = _answers(rsi.LBVH(dV, dT, morton_bits=bits), dF, dE)
        t = rsi.LBVH(dV, dT, morton_bits=bits, treelet_passes=2)
        _same(_answers(t, dF, dE), plain)
        for w in (3, 4):
            r = t.query(dF, dE, "both", node_width=w)
            for k in ("hit", "count", "ambiguous"):
                assert np.array_equal(r[k].cpu().numpy(), plain["both"][k]), (cfg, w, k)


def test_restructuring_cuts_node_visits(rsi):
    mesh = W.config_mesh("c2")
    F, E = W.rays(W.config_rays("c2"), mesh, count=1_000_000)
    dV, dT, dF, dE = _dev(mesh.vertices), _dev(mesh.triangles), _dev(F), _dev(E)
    v0 = rsi.LBVH(dV, dT).query(dF, dE, "count", stats=True)["stats"]["node_visits"]
    v1 = rsi.LBVH(dV, dT, treelet_passes=1).query(dF, dE, "count", stats=True)["stats"]["node_visits"]
    assert v1 < 0.85 * v0, (v0, v1)


@pytest.mark.parametrize("n_tri", [1, 2, 3, 6, 7, 8, 13, 64, 1000])
def test_small_meshes(rsi, n_tri):
    """Meshes around the treelet size: valid trees, answers as the oracle's."""
    rng = np.random.default_rng(n_tri)
    V = rng.uniform(-1, 1, (3 * n_tri, 3)).astype(np.float32)
    T = np.arange(3 * n_tri, dtype=np.int32).reshape(n_tri, 3)
    F = rng.uniform(-1.5, 1.5, (4000, 3)).astype(np.float32)
    E = rng.uniform(-1.5, 1.5, (4000, 3)).astype(np.float32)
    dV, dT, dF, dE = _dev(V), _dev(T), _dev(F), _dev(E)
    plain = rsi.LBVH(dV, dT)
    t = rsi.LBVH(dV, dT, treelet_passes=3)
    _check_tree(t.export(), plain.export(), n_tri)
    _same(_answers(t, dF, dE), _answers(plain, dF, dE))
    ref = oracle.query(V, T, F, E)
    r = t.query(dF, dE, "count")
    keep = ref["amb_count"] == 0
    assert np.array_equal(r["count"].cpu().numpy()[keep], ref["count"][keep])


def test_host_mesh_build(rsi):
    """lbvh_build_host_ex: the same restructured tree from a host mesh."""
    mesh = W.config_mesh("c1")
    a = rsi.LBVH(_dev(mesh.vertices), _dev(mesh.triangles), treelet_passes=2).export()
    b = rsi.LBVH(torch.from_numpy(mesh.vertices), torch.from_numpy(mesh.triangles), treelet_passes=2).export()
    for k in ("left", "right", "parent", "box"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("passes", [1, 2])
def test_batched_build_equals_single_builds(rsi, passes):
    """One batched build with restructuring (lbvh_build_batched_ex) gives
    every mesh -- meshes of 1, 2, 3, 8 and thousands of triangles, 30- and
    63-bit codes -- the restructured hierarchy its own build gives it, bit for
    bit, and the same answers."""
    rng = np.random.default_rng(5)
    meshes = []
    for n_tri in (1, 2, 3, 8, 500):
        V = rng.uniform(-1, 1, (3 * n_tri, 3)).astype(np.float32)
        meshes.append((V, np.arange(3 * n_tri, dtype=np.int32).reshape(n_tri, 3)))
    for name in ("c1", "c2"):
        m = W.config_mesh(name)
        meshes.append((m.vertices, m.triangles))
    dev = [(_dev(V), _dev(T)) for V, T in meshes]
    for bits in (30, 63):
        many = rsi.build_many(dev, morton_bits=bits, treelet_passes=passes)
        for k, ((V, T), b) in enumerate(zip(dev, many)):
            one = rsi.LBVH(V, T, morton_bits=bits, treelet_passes=passes)
            e1, e2 = one.export(), b.export()
            for key in e1:
                assert np.array_equal(e1[key], e2[key]), (bits, k, key)
            assert one.info()["height"] == b.info()["height"], (bits, k)
            one.close()
        m = W.config_mesh("c2")
        F, E = W.rays(W.config_rays("c2"), m, count=200_000)
        dF, dE = _dev(F), _dev(E)
        plain = _answers(rsi.LBVH(dev[-1][0], dev[-1][1], morton_bits=bits), dF, dE)
        _same(_answers(many[-1], dF, dE), plain)
        out = rsi.query_batched([(b, dF, dE) for b in many[-2:]], "count")
        assert np.array_equal(out["count"][-1].cpu().numpy(), plain["count"]["count"])
        for b in many:
            b.close()


def test_rebuild_plan_repeats_the_restructuring(rsi):
    """A rebuilding plan over restructured hierarchies rebuilds them with the
    same passes: after the meshes move, a launch answers as fresh
    restructured builds do and the hierarchies equal them bit for bit."""
    jobs = W.batched_meshes(n_meshes=4, seed=6, max_rays=30_000)
    meshes = [(torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.triangles).cuda()) for m, _ in jobs]
    rays = [W.rays(spec, m) for m, spec in jobs]
    bvhs = rsi.build_many(meshes, treelet_passes=1)
    items = [(b, torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()) for b, (F, E) in zip(bvhs, rays)]
    plan = rsi.BatchPlan(items, "count", rebuild=meshes)
    for V, _ in meshes:                   # move the meshes before the first launch
        V[:, 2] *= 1.3
        V[:, :2] += 0.007
    plan.run()
    assert plan.stats()["device_error"] == 0
    for i, ((b, f, t), (V, T)) in enumerate(zip(items, meshes)):
        fresh = rsi.LBVH(V, T, treelet_passes=1)
        ref = fresh.query(f, t, "count")
        assert torch.equal(plan.count[i], ref["count"]) and torch.equal(plan.ambiguous[i], ref["ambiguous"]), i
        e1, e2 = fresh.export(), b.export()
        for k in e1:
            assert np.array_equal(e1[k], e2[k]), (i, k)
        assert fresh.info()["height"] == b.info()["height"], i
        fresh.close()
    plan.close()
    for b in bvhs:
        b.close()
