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


@pytest.mark.parametrize("node_width", [2, 4])
@pytest.mark.parametrize("mode", ["any_hit", "count"])
def test_batched_equals_single_queries(rsi, scene, mode, node_width):
    """The batched plan (child-pair or four-wide nodes) answers as the
    single queries (child-pair by default) do."""
    items, host = scene
    plan = rsi.BatchPlan(items, mode, node_width=node_width)
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
