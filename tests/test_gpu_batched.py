"""Batched queries (many meshes, one persistent launch under a CUDA graph,
device work queue) through the C ABI: every answer equals the single-mesh
query's, which the oracle pins; streaming through posts gives the same
answers; a queue nobody feeds ends with RSI_ERR_TIMEOUT instead of hanging."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rsi():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2305_01867_gb300 as m
    return m


@pytest.fixture(scope="module")
def scene(rsi):
    """Eight meshes of uneven size (log-uniform triangle and segment counts,
    segments capped at 40,000 per mesh) plus an empty batch."""
    items, host = [], []
    for mesh, spec in W.batched_meshes(n_meshes=8, seed=4, max_rays=40_000):
        F, E = W.rays(spec, mesh)
        bvh = rsi.LBVH(torch.from_numpy(mesh.vertices).cuda(), torch.from_numpy(mesh.triangles).cuda())
        items.append((bvh, torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()))
        host.append((mesh, F, E))
    bvh0 = items[0][0]
    items.insert(3, (bvh0, torch.empty(0, 3, device="cuda"), torch.empty(0, 3, device="cuda")))
    host.insert(3, (host[0][0], np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32)))
    return items, host


@pytest.mark.parametrize("node_width,tile,stack", [(2, 0, 0), (4, 0, 0), (2, 2048, 0), (4, 8192, 128),
                                                   (2, 0, 64)])
@pytest.mark.parametrize("mode", ["any_hit", "count"])
def test_batched_equals_single_queries(rsi, scene, mode, node_width, tile, stack):
    """The batched plan (child-pair or four-wide nodes, with or without the
    in-tile reordering of each batch, any stack size) answers as the single
    queries (child-pair by default) do."""
    items, host = scene
    plan = rsi.BatchPlan(items, mode, node_width=node_width, ray_sort_tile=tile, stack=stack)
    for rep in range(2):   # the graph replays
        plan.run()
        torch.cuda.synchronize()
        for i, (bvh, f, t) in enumerate(items):
            ref = bvh.query(f, t, mode)
            key = "hit" if mode == "any_hit" else "count"
            got = plan.hit[i] if mode == "any_hit" else plan.count[i]
            assert torch.equal(got, ref[key]), (rep, i)
            assert torch.equal(plan.ambiguous[i], ref["ambiguous"]), (rep, i)
    st = plan.stats()
    assert st["n_rays"] == sum(int(f.shape[0]) for _, f, _ in items) and st["device_error"] == 0
    plan.close()


def test_batched_against_oracle_sample(rsi, scene):
    items, host = scene
    plan = rsi.BatchPlan(items, "count")
    plan.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for i in (0, 5):
        mesh, F, E = host[i]
        idx = rng.choice(len(F), 400, replace=False)
        ref = oracle.query(mesh.vertices, mesh.triangles, F[idx], E[idx])
        cnt = plan.count[i].cpu().numpy()[idx]
        amb = plan.ambiguous[i].cpu().numpy()[idx]
        assert np.array_equal(amb, ref["amb_count"])
        ok = ref["amb_count"] == 0
        assert np.array_equal(cnt[ok], ref["count"][ok])


def test_streamed_plan_matches(rsi, scene):
    """Segments copied in chunks on a second stream and posted one chunk at a
    time while the persistent kernel is already running."""
    items, host = scene
    ref_plan = rsi.BatchPlan(items, "any_hit")
    ref_plan.run()
    # destination buffers filled only by the streamed copies
    dst = [(bvh, torch.full_like(f, float("nan")), torch.full_like(t, float("nan"))) for bvh, f, t in items]
    plan = rsi.BatchPlan(dst, "any_hit", stream_timeout_ns=5_000_000_000)
    src = [(torch.from_numpy(F).pin_memory(), torch.from_numpy(E).pin_memory()) for _, F, E in host]
    copy = torch.cuda.Stream()
    torch.cuda.synchronize()   # the NaN fills are done before any copy lands
    plan.run()
    posted = 0
    with torch.cuda.stream(copy):
        for (bvh, df, dt), (hf, ht) in zip(dst, src):
            df.copy_(hf, non_blocking=True)
            dt.copy_(ht, non_blocking=True)
            posted += df.shape[0]
            plan.post(posted, stream=copy)
    torch.cuda.synchronize()
    assert plan.stats()["device_error"] == 0
    for i in range(len(items)):
        assert torch.equal(plan.hit[i], ref_plan.hit[i]) and torch.equal(plan.ambiguous[i], ref_plan.ambiguous[i])


def test_unfed_queue_times_out_without_hanging(rsi, scene):
    """Failure detection without a GPU fault: a streaming plan that nobody
    feeds ends after its 2 ms budget with RSI_ERR_TIMEOUT; outputs stay
    untouched and the device keeps working."""
    items, host = scene
    plan = rsi.BatchPlan(items[:2], "any_hit", stream_timeout_ns=2_000_000)
    for h in plan.hit:
        h.fill_(77)
    plan.run()
    torch.cuda.synchronize()
    st = plan.stats(raise_on_error=False)
    assert st["device_error"] == -5
    assert all(int((h == 77).sum()) == h.numel() for h in plan.hit)
    with pytest.raises(rsi.RSIError) as e:
        plan.stats()
    assert e.value.code == -5
    bvh, f, t = items[0]
    assert bvh.query(f, t, "any_hit")["hit"].numel() == f.shape[0]


def test_bad_plans_rejected(rsi, scene):
    items, _ = scene
    with pytest.raises(rsi.RSIError):
        rsi.BatchPlan(items, "any_hit", block=512)
    plan = rsi.BatchPlan(items[:2], "any_hit")
    with pytest.raises(rsi.RSIError):
        plan.post(10)   # not a streaming plan


@pytest.mark.parametrize("mode", ["any_hit", "count"])
def test_one_call_batched_query(rsi, scene, mode):
    """rsi_query_batched(hs, n_meshes, batches, mode, opt, stream): the call
    shape of the boundary.  The first call plans (and keeps the plan), the
    second replays it; both answer as the single queries do.  A freed
    hierarchy drops the kept plans that name it, and a new hierarchy --
    possibly at the same address -- gets a plan of its own."""
    items, host = scene
    key = "hit" if mode == "any_hit" else "count"
    refs = [bvh.query(f, t, mode) for bvh, f, t in items]
    out = None
    for rep in range(2):
        out = rsi.query_batched(items, mode, hit=out["hit"] if out else None, count=out["count"] if out else None,
                                ambiguous=out["ambiguous"] if out else None)
        torch.cuda.synchronize()
        for i, ref in enumerate(refs):
            assert torch.equal(out[key][i], ref[key]), (rep, i)
            assert torch.equal(out["ambiguous"][i], ref["ambiguous"]), (rep, i)
    # a fresh hierarchy of mesh 0 in place of the first one: answers still right
    mesh0, F0, E0 = host[0]
    fresh = rsi.LBVH(torch.from_numpy(mesh0.vertices).cuda(), torch.from_numpy(mesh0.triangles).cuda())
    items2 = [(fresh, items[0][1], items[0][2])] + items[1:]
    out2 = rsi.query_batched(items2, mode)
    torch.cuda.synchronize()
    assert torch.equal(out2[key][0], refs[0][key])
    fresh.close()   # drops the plan that names it; the next call plans again
    fresh = rsi.LBVH(torch.from_numpy(mesh0.vertices).cuda(), torch.from_numpy(mesh0.triangles).cuda())
    items3 = [(fresh, items[0][1], items[0][2])] + items[1:]
    out3 = rsi.query_batched(items3, mode, hit=out2["hit"], count=out2["count"], ambiguous=out2["ambiguous"])
    torch.cuda.synchronize()
    for i, ref in enumerate(refs):
        assert torch.equal(out3[key][i], ref[key]) and torch.equal(out3["ambiguous"][i], ref["ambiguous"]), i
    fresh.close()


def test_one_call_batched_query_rejections(rsi, scene):
    import ctypes
    items, _ = scene
    bvh, f, t = items[0]
    hs = (ctypes.c_void_p * 1)(bvh.handle.value)
    other = items[1][0]
    arr = (rsi.RayBatch * 1)()
    arr[0] = rsi.RayBatch(other.handle.value, f.data_ptr(), t.data_ptr(), f.shape[0], None, None, None)
    assert rsi.lib.rsi_query_batched(hs, 1, arr, rsi.RSI_ANY_HIT, None, None) == -1   # bvh neither NULL nor hs[0]
    assert "bvh" in rsi.last_error()
    opt = rsi.Options(0, 0, 0, 0, -1000)
    arr[0] = rsi.RayBatch(None, f.data_ptr(), t.data_ptr(), 0, None, None, None)
    assert rsi.lib.rsi_query_batched(hs, 1, arr, rsi.RSI_ANY_HIT, ctypes.byref(opt), None) == -1
    assert "streaming" in rsi.last_error()


@pytest.mark.parametrize("mode", ["any_hit", "count"])
def test_rebuild_and_query_in_one_graph(rsi, mode):
    """rsi_batch_create_rebuild: each launch rebuilds every hierarchy in place
    from its mesh buffers, then queries, in one graph.  After the vertices
    move, a launch gives what a fresh build and query of the moved meshes
    give, and the rebuilt hierarchies equal fresh builds bit for bit; a NaN
    vertex is reported by the plan's stats with its mesh."""
    jobs = W.batched_meshes(n_meshes=5, seed=5, max_rays=30_000)
    meshes = [(torch.from_numpy(m.vertices).cuda(), torch.from_numpy(m.triangles).cuda()) for m, _ in jobs]
    rays = [W.rays(spec, m) for m, spec in jobs]
    bvhs = rsi.build_many(meshes)
    items = [(b, torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()) for b, (F, E) in zip(bvhs, rays)]
    key = "hit" if mode == "any_hit" else "count"
    plan = rsi.BatchPlan(items, mode, rebuild=meshes)

    def check_against_fresh():
        plan.run()
        st = plan.stats()                 # synchronizes, refreshes the hierarchies' summaries
        assert st["device_error"] == 0
        for i, ((b, f, t), (V, T)) in enumerate(zip(items, meshes)):
            fresh = rsi.LBVH(V, T)
            ref = fresh.query(f, t, mode)
            got = plan.hit[i] if mode == "any_hit" else plan.count[i]
            assert torch.equal(got, ref[key]) and torch.equal(plan.ambiguous[i], ref["ambiguous"]), i
            e1, e2 = fresh.export(), b.export()
            for k in e1:
                assert np.array_equal(e1[k], e2[k]), (i, k)
            i1, i2 = fresh.info(), b.info()
            for k in ("height", "extent_lo", "extent_hi", "max_tri_extent"):
                assert i1[k] == i2[k], (i, k)
            fresh.close()

    check_against_fresh()
    for V, _ in meshes:                   # move the meshes: stretch the relief, shift the grid
        V[:, 2] *= 1.7
        V[:, :2] += 0.013
    check_against_fresh()
    keep = meshes[2][0][4, 1].item()
    meshes[2][0][4, 1] = float("nan")
    plan.run()
    with pytest.raises(rsi.RSIError) as e:
        plan.stats()
    assert e.value.code == -7 and "mesh 2" in str(e.value)
    meshes[2][0][4, 1] = keep
    check_against_fresh()
    plan.close()
    for b in bvhs:
        b.close()
