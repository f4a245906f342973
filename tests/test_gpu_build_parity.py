"""GPU build (extent, Morton, sort, radix tree, refit) against the oracle,
bit for bit, through the C ABI.  Sizes span several sort tiles, ragged tails,
a single triangle and forced duplicate Morton codes, and both sort plans: up
to 524,288 keys one launch per pass over at most 128 tiles of 256 * R keys
(sizes on either side of the R steps and of that limit), above it three
launches per pass over tiles of 4096 keys.  Both tree
constructions are checked: Karras + refit, and the single bottom-up pass
(Apetrei; Sec. 4.2), which must give the same hierarchy."""
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


def _soup(n, seed, dup_frac=0.0):
    """n random small triangles in [0,1]^3; a fraction share one centroid
    cell so their Morton codes collide."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, 1, (n, 3))
    off = rng.uniform(-0.01, 0.01, (n, 3, 3))
    k = int(n * dup_frac)
    if k:   # identical triangles: identical codes
        c[:k] = c[0]
        off[:k] = off[0]
    V = (c[:, None, :] + off).reshape(-1, 3).astype(np.float32)
    T = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    return V, T


def _meshes():
    g = load("case_study1_sec4_1.txt")
    yield "case_study1", g["vertices"], g["triangles"]
    for n in (1, 2, 3, 255, 256, 257, 1023, 1024, 1025, 4097, 9000, 32768, 32769, 65537, 524288, 524289):
        V, T = _soup(n, seed=n)
        yield f"soup{n}", V, T
    V, T = _soup(5000, seed=3, dup_frac=0.3)
    yield "dups", V, T
    m = W.config_mesh("c1")
    yield "c1", m.vertices, m.triangles
    m = W.config_mesh("c2")
    yield "c2", m.vertices, m.triangles
    m = W.config_mesh("c3")                 # 178,802 triangles, jittered grid
    yield "c3", m.vertices, m.triangles


@pytest.mark.parametrize("builder", ["karras", "apetrei"])
@pytest.mark.parametrize("bits", [30, 63])
def test_build_bit_exact(rsi, bits, builder):
    for name, V, T in _meshes():
        ref = oracle.build_all(V, T, bits=bits)
        bvh = rsi.LBVH(torch.from_numpy(V).cuda(), torch.from_numpy(T).cuda(), morton_bits=bits, builder=builder)
        got = bvh.export()
        n = len(T)
        assert np.array_equal(got["sorted_keys"], ref["sorted_keys"]), name
        assert np.array_equal(got["perm"], ref["perm"]), name
        if n > 1:
            assert np.array_equal(got["left"], ref["left"]), name
            assert np.array_equal(got["right"], ref["right"]), name
        assert np.array_equal(got["parent"], ref["parent"]), name
        assert np.array_equal(got["box"].view(np.uint32), ref["box"].view(np.uint32)), name
        info = bvh.info()
        assert info["height"] == ref["height"], name
        lo, hi = oracle.extent(V)
        assert np.array_equal(np.array(info["extent_lo"], np.float32), lo), name
        assert np.array_equal(np.array(info["extent_hi"], np.float32), hi), name
        bvh.close()


def test_case_study1_leaf_order_on_gpu(rsi):
    """Sec. 4.1: leaves hold T0, T3, T1, T2 and every leaf has a parent."""
    g = load("case_study1_sec4_1.txt")
    bvh = rsi.LBVH(torch.from_numpy(g["vertices"]).cuda(), torch.from_numpy(g["triangles"]).cuda())
    got = bvh.export()
    assert got["perm"].tolist() == g["leaf_order"].tolist()
    assert got["parent"][0] == -1 and np.all(got["parent"][1:] >= 0)


def test_build_errors(rsi):
    V = torch.zeros(3, 3, dtype=torch.float32, device="cuda")
    V[1, 0] = 1
    V[2, 1] = 1
    T64 = torch.tensor([[0, 1, 2]], dtype=torch.int64, device="cuda")
    with pytest.raises(rsi.RSIError) as e:       # the int64 mix-up of Sec. 4.1.2
        rsi.LBVH(V, T64)
    assert e.value.code == -2
    with pytest.raises(rsi.RSIError) as e:
        rsi.LBVH(V, torch.tensor([[0, 1, 5]], dtype=torch.int32, device="cuda"))
    assert e.value.code == -8
    Vn = V.clone()
    Vn[0, 2] = float("nan")
    with pytest.raises(rsi.RSIError) as e:
        rsi.LBVH(Vn, torch.tensor([[0, 1, 2]], dtype=torch.int32, device="cuda"))
    assert e.value.code == -7
    with pytest.raises(rsi.RSIError) as e:
        rsi.LBVH(V, torch.tensor([[0, 1, 2]], dtype=torch.int32, device="cuda"), morton_bits=32)
    assert e.value.code == -1
    # the library keeps working after rejected calls
    b = rsi.LBVH(V, torch.tensor([[0, 1, 2]], dtype=torch.int32, device="cuda"))
    assert b.info()["n_triangles"] == 1


def test_build_from_host_equals_device(rsi):
    m = W.config_mesh("c1")
    a = rsi.LBVH(torch.from_numpy(m.vertices), torch.from_numpy(m.triangles)).export()
    b = rsi.LBVH(torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.triangles).cuda()).export()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("bits", [30, 63])
def test_apetrei_queries_equal_karras(rsi, bits):
    """The packed traversal nodes and leaf triangles (not exported) are the
    same too: every answer of both modes agrees on the c1 workload, and the
    hierarchy stays identical over repeated builds (the range-end slots are
    reset each time)."""
    m = W.config_mesh("c1")
    F, E = W.rays(W.config_rays("c1"), m)
    dV, dT = torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.triangles).cuda()
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    a = rsi.LBVH(dV, dT, morton_bits=bits)
    ea = a.export()
    qa = [a.query(dF, dE, mode) for mode in ("any_hit", "count")]
    for _ in range(3):
        b = rsi.LBVH(dV, dT, morton_bits=bits, builder="apetrei")
        eb = b.export()
        for k in ea:
            assert np.array_equal(ea[k], eb[k]), k
        assert a.info()["height"] == b.info()["height"]
        for mode, ra in zip(("any_hit", "count"), qa):
            rb = b.query(dF, dE, mode)
            for k in ra:
                if isinstance(ra[k], torch.Tensor):
                    assert torch.equal(ra[k], rb[k]), (mode, k)
        nb = b.nearest(dF, dE)
        na = a.nearest(dF, dE)
        assert torch.equal(na["tri"], nb["tri"]) and torch.equal(na["t"], nb["t"])
        b.close()
    a.close()


def test_apetrei_rejects_host_inputs(rsi):
    m = W.config_mesh("c1")
    with pytest.raises(TypeError):
        rsi.LBVH(torch.from_numpy(m.vertices), torch.from_numpy(m.triangles), builder="apetrei")
    with pytest.raises(ValueError):
        rsi.LBVH(torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.triangles).cuda(), builder="x")


def test_dumps_of_gpu_hierarchy_equal_oracle(rsi):
    """The text and DOT dumps (Sec. 4.1.1, 4.1.5) of the exported GPU
    hierarchy are those of the oracle's tree, for both builders."""
    from paper_2305_01867_gb300 import bvh_dump
    for name in ("case_study1", "c1"):
        if name == "c1":
            m = W.config_mesh("c1")
            V, T = m.vertices, m.triangles
        else:
            g = load("case_study1_sec4_1.txt")
            V, T = g["vertices"], g["triangles"]
        ref = oracle.build_all(V, T)
        for builder in ("karras", "apetrei"):
            got = rsi.LBVH(torch.from_numpy(V).cuda(), torch.from_numpy(T).cuda(), builder=builder).export()
            assert bvh_dump.to_text(got, digits=6) == bvh_dump.to_text(ref, digits=6), (name, builder)
            assert bvh_dump.to_dot(got) == bvh_dump.to_dot(ref), (name, builder)


@pytest.mark.parametrize("bits", [30, 63])
def test_build_many_equals_single_builds(rsi, bits):
    """One batched build of meshes of very different sizes (1, 2 and 3
    triangles, duplicate codes, heightfields) gives every mesh the hierarchy
    a build of its own gives it, bit for bit, and the same answers."""
    meshes = [(V, T) for name, V, T in _meshes()]
    m2 = W.heightfield(7, seed=9, n_bumps=1)
    meshes.append((m2.vertices, m2.triangles))
    dev = [(torch.from_numpy(V).cuda(), torch.from_numpy(np.ascontiguousarray(T)).cuda()) for V, T in meshes]
    many = rsi.build_many(dev, morton_bits=bits)
    assert len(many) == len(dev)
    for k, ((V, T), b) in enumerate(zip(dev, many)):
        one = rsi.LBVH(V, T, morton_bits=bits)
        e1, e2 = one.export(), b.export()
        for key in e1:
            assert np.array_equal(e1[key], e2[key]), (k, key)
        i1, i2 = one.info(), b.info()
        for key in ("height", "extent_lo", "extent_hi", "max_tri_extent", "n_triangles"):
            assert i1[key] == i2[key], (k, key)
        one.close()
    # the packed nodes and triangles answer the same (c1 and c2 meshes)
    m = W.config_mesh("c1")
    F, E = W.rays(W.config_rays("c1"), m)
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    k1 = [i for i, (V, T) in enumerate(meshes) if len(T) == len(m.triangles)][0]
    ref = rsi.LBVH(dev[k1][0], dev[k1][1], morton_bits=bits)
    for mode in ("any_hit", "count"):
        a, b = ref.query(dF, dE, mode), many[k1].query(dF, dE, mode)
        key = "hit" if mode == "any_hit" else "count"
        assert torch.equal(a[key], b[key]) and torch.equal(a["ambiguous"], b["ambiguous"])
    for b in many:
        b.close()


def test_build_many_reports_the_bad_mesh(rsi):
    good = W.heightfield(5, seed=1)
    V = torch.from_numpy(good.vertices).cuda()
    T = torch.from_numpy(good.triangles).cuda()
    bad_T = T.clone()
    bad_T[3, 1] = 10_000
    with pytest.raises(rsi.RSIError) as e:
        rsi.build_many([(V, T), (V, bad_T), (V, T)])
    assert e.value.code == -8 and "mesh 1" in str(e.value)
    # the library keeps working
    assert len(rsi.build_many([(V, T)])) == 1


@pytest.mark.parametrize("bits", [30, 63])
def test_build_many_c4_meshes_equal_oracle(rsi, bits):
    """The 64 heightfields of the batching workload (1e3 to 1e5 triangles
    each, 1.16e6 in all), built by one batched build: every mesh's keys,
    order, children, parents, boxes, height and extent equal the oracle's
    plain-definition build bit for bit (Sec. 3.2 codes and sort, Sec. 4.2
    tree and boxes)."""
    jobs = W.batched_meshes(64, seed=4, max_rays=1)
    dev = [(torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.triangles).cuda()) for m, _ in jobs]
    many = rsi.build_many(dev, morton_bits=bits)
    for k, ((m, _), b) in enumerate(zip(jobs, many)):
        ref = oracle.build_all(m.vertices, m.triangles, bits=bits)
        got = b.export()
        for key in ("sorted_keys", "perm", "left", "right", "parent"):
            assert np.array_equal(got[key], ref[key]), (k, key)
        assert np.array_equal(got["box"].view(np.uint32), ref["box"].view(np.uint32)), k
        info = b.info()
        assert info["height"] == ref["height"], k
        lo, hi = oracle.extent(m.vertices)
        assert np.array_equal(np.array(info["extent_lo"], np.float32), lo), k
        assert np.array_equal(np.array(info["extent_hi"], np.float32), hi), k
        b.close()
