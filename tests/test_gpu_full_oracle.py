"""Every segment of the 1e7-segment c2 batch against the oracle, in all three
modes: the exhaustive search of Sec. 1 on 2e11 segment/triangle pairs, about
three minutes of FP64 brute force on 16 host cores.

Part of the default GPU run; RSI_SKIP_FULL_ORACLE=1 skips it for quick local
iterations.  The bar: ambiguity marks identical; hit flags and counts
identical on every unmarked segment; the nearest crossing (triangle, t,
point, distance) identical on every segment."""
import os

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rsi():
    if os.environ.get("RSI_SKIP_FULL_ORACLE") == "1":
        pytest.skip("RSI_SKIP_FULL_ORACLE=1")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2305_01867_gb300 as m
    return m


def test_c2_every_segment(rsi):
    mesh = W.config_mesh("c2")
    F, E = W.rays(W.config_rays("c2"), mesh)
    n = len(F)
    bvh = rsi.LBVH(torch.from_numpy(mesh.vertices).cuda(), torch.from_numpy(mesh.triangles).cuda())
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    a = bvh.query(dF, dE, "any_hit")
    c = bvh.query(dF, dE, "count")
    b = bvh.query(dF, dE, "both")
    nr = bvh.nearest(dF, dE)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in (("hit", a["hit"]), ("amb_hit", a["ambiguous"]),
                                            ("count", c["count"]), ("amb_count", c["ambiguous"]),
                                            ("both_hit", b["hit"]), ("both_count", b["count"]),
                                            ("both_amb", b["ambiguous"]),
                                            ("near_tri", nr["tri"]), ("near_t", nr["t"]),
                                            ("near_point", nr["point"]), ("near_dist", nr["dist"]))}
    bvh.close()
    ref = oracle.query(mesh.vertices, mesh.triangles, F, E)
    assert np.array_equal(got["amb_hit"], ref["amb_hit"])
    assert np.array_equal(got["amb_count"], ref["amb_count"])
    ok_h, ok_c = ref["amb_hit"] == 0, ref["amb_count"] == 0
    assert np.array_equal(got["hit"][ok_h], ref["hit"][ok_h])
    assert np.array_equal(got["count"][ok_c], ref["count"][ok_c])
    # the combined pass (RSI_BOTH): both answers and both flags from one traversal
    assert np.array_equal(got["both_amb"] & 1, ref["amb_hit"]) and np.array_equal(got["both_amb"] >> 1, ref["amb_count"])
    assert np.array_equal(got["both_hit"][ok_h], ref["hit"][ok_h])
    assert np.array_equal(got["both_count"][ok_c], ref["count"][ok_c])
    assert np.array_equal(got["near_tri"], ref["near_tri"])
    hit = ref["near_tri"] >= 0
    for k in ("near_t", "near_dist"):
        assert np.array_equal(got[k].view(np.uint32), ref[k].view(np.uint32)), k
    assert np.array_equal(got["near_point"][hit].view(np.uint32), ref["near_point"][hit].view(np.uint32))
    assert np.isnan(got["near_point"][~hit]).all()
    assert ok_c.sum() > n - 1000 and got["hit"].sum() > n // 3
