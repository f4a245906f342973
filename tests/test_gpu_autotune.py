"""The autotuner: times candidate launch shapes and in-tile reorderings on a
sample, caches the winner in a JSON file, and its choice changes no answer."""
import json

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rsi():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2305_01867_gb300 as m
    return m


def test_autotune_caches_and_keeps_results(rsi, tmp_path):
    mesh = W.config_mesh("c2")
    F, E = W.rays(W.config_rays("c2", 500_000), mesh)
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    bvh = rsi.LBVH(torch.from_numpy(mesh.vertices).cuda(), torch.from_numpy(mesh.triangles).cuda())
    cache = str(tmp_path / "tune.json")
    t1 = bvh.autotune(dF, dE, "count", cache_path=cache)
    assert t1["from_cache"] == 0 and t1["candidates"] >= 6 and t1["ms"] > 0
    h = bvh.info()["height"]
    assert t1["node_width"] in (2, 3, 4)
    assert t1["stack"] >= (3 * ((h + 2) // 2) if t1["node_width"] == 4 else h + 1)
    t2 = bvh.autotune(dF, dE, "count", cache_path=cache)
    assert t2["from_cache"] == 1 and t2["candidates"] == 0
    for k in ("block", "blocks_per_sm", "ray_sort_tile", "node_width", "stack"):
        assert t1[k] == t2[k]
    d = json.load(open(cache))
    assert len(d) == 1 and list(d.values())[0]["block"] == t1["block"]
    base = bvh.query(dF, dE, "count")
    tuned = bvh.query(dF, dE, "count", block=t1["block"], blocks_per_sm=t1["blocks_per_sm"],
                      ray_sort_tile=t1["ray_sort_tile"], node_width=t1["node_width"])
    assert torch.equal(base["count"], tuned["count"]) and torch.equal(base["ambiguous"], tuned["ambiguous"])


def test_batch_autotune_picks_a_plan_and_keeps_results(rsi, tmp_path):
    """The batched plan's tuner (launch shape, node width, in-tile
    reordering, stack size) on meshes of uneven size: its choice is cached,
    holds the deepest tree's walk, and a plan with it answers as the
    default plan does."""
    items = []
    for mesh, spec in W.batched_meshes(n_meshes=6, seed=4, max_rays=60_000):
        F, E = W.rays(spec, mesh)
        bvh = rsi.LBVH(torch.from_numpy(mesh.vertices).cuda(), torch.from_numpy(mesh.triangles).cuda())
        items.append((bvh, torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()))
    cache = str(tmp_path / "tune_batched.json")
    t1 = rsi.batch_autotune(items, "count", cache_path=cache)
    assert t1["from_cache"] == 0 and t1["candidates"] >= 8 and t1["ms"] > 0
    h = max(b.info()["height"] for b, _, _ in items)
    need = 3 * ((h + 2) // 2) if t1["node_width"] == 4 else h + 1
    assert t1["stack"] in (32, 64, 128) and t1["stack"] >= need
    assert t1["ray_sort_tile"] in (0, 8192) and t1["node_width"] in (2, 4)
    t2 = rsi.batch_autotune(items, "count", cache_path=cache)
    assert t2["from_cache"] == 1 and all(t1[k] == t2[k] for k in ("block", "blocks_per_sm", "node_width",
                                                                    "ray_sort_tile", "stack"))
    base = rsi.BatchPlan(items, "count")
    tuned = rsi.BatchPlan(items, "count", block=t1["block"], blocks_per_sm=t1["blocks_per_sm"],
                          node_width=t1["node_width"], ray_sort_tile=t1["ray_sort_tile"], stack=t1["stack"])
    base.run()
    tuned.run()
    torch.cuda.synchronize()
    for i in range(len(items)):
        assert torch.equal(base.count[i], tuned.count[i]) and torch.equal(base.ambiguous[i], tuned.ambiguous[i])
    base.close()
    tuned.close()
