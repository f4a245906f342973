"""rsi_query_noalloc: the query entry point for callers that cannot allocate
device memory while they query (e.g. a plugin inside an application that
owns all device memory, or a real-time loop).  It must give the same
results as rsi_query, call after call, from its fixed scratch array."""
import ctypes

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


def _noalloc(rsi, bvh, dF, dE, mode, hit=None, count=None, amb=None):
    rc = rsi.lib.rsi_query_noalloc(bvh.handle, ctypes.c_void_p(dF.data_ptr()), ctypes.c_void_p(dE.data_ptr()),
                                   dF.shape[0], mode, None,
                                   ctypes.c_void_p(hit.data_ptr()) if hit is not None else None,
                                   ctypes.c_void_p(count.data_ptr()) if count is not None else None,
                                   ctypes.c_void_p(amb.data_ptr()) if amb is not None else None,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def test_noalloc_matches_rsi_query_twice(rsi):
    mesh = W.config_mesh("c2")
    F, E = W.rays(W.config_rays("c2", 300_007), mesh)
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    bvh = rsi.LBVH(torch.from_numpy(mesh.vertices).cuda(), torch.from_numpy(mesh.triangles).cuda())
    ref_a = bvh.query(dF, dE, "any_hit")
    ref_c = bvh.query(dF, dE, "count")
    n = len(F)
    for call in range(2):
        hit = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        amb = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        cnt = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        amb_c = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        free0 = torch.cuda.mem_get_info()[0]
        if call == 1:
            # set-up done on the first call: from now on any allocation the
            # library attempts fails (RSI_ERR_OOM), even one its memory pool
            # could serve from cached blocks without touching free memory
            rsi.fail_allocations(0)
        try:
            assert _noalloc(rsi, bvh, dF, dE, rsi.RSI_ANY_HIT, hit=hit, amb=amb) == 0, rsi.last_error()
            assert _noalloc(rsi, bvh, dF, dE, rsi.RSI_COUNT, count=cnt, amb=amb_c) == 0, rsi.last_error()
            torch.cuda.synchronize()
        finally:
            rsi.fail_allocations(None)
        if call == 1:   # and nothing outside the library's pool was taken either
            assert torch.cuda.mem_get_info()[0] == free0
        # flags and counts are integers: the bar is exact equality
        assert torch.equal(hit, ref_a["hit"]) and torch.equal(amb, ref_a["ambiguous"])
        assert torch.equal(cnt, ref_c["count"]) and torch.equal(amb_c, ref_c["ambiguous"])
    assert int(ref_c["ambiguous"].sum()) >= 0 and int(ref_a["hit"].sum()) > 0


def test_noalloc_rejects_oversize_batches(rsi):
    mesh = W.config_mesh("c1")
    bvh = rsi.LBVH(torch.from_numpy(mesh.vertices).cuda(), torch.from_numpy(mesh.triangles).cuda())
    n = rsi.NOALLOC_MAX_RAYS + 1
    dF = torch.zeros(n, 3, device="cuda")
    hit = torch.zeros(n, dtype=torch.uint8, device="cuda")
    rc = _noalloc(rsi, bvh, dF, dF, rsi.RSI_ANY_HIT, hit=hit)
    assert rc == -1 and "RSI_NOALLOC_MAX_RAYS" in rsi.last_error()


def test_noalloc_grazing_batch_at_the_cap(rsi):
    """A full-size call (RSI_NOALLOC_MAX_RAYS segments) from the jittered
    300 x 300 mesh with 1 % grazing segments: many segments go to the FP64
    re-test, which here runs from the fixed array.  Both modes equal
    rsi_query on every segment, with every library allocation failing, and
    a sample (all marked ambiguous segments up to 400, plus 600 others)
    equals the oracle."""
    import oracle
    mesh = W.config_mesh("c3")
    n = rsi.NOALLOC_MAX_RAYS
    F, E = W.rays(W.config_rays("c3"), mesh, 0, n)
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    bvh = rsi.LBVH(torch.from_numpy(mesh.vertices).cuda(), torch.from_numpy(mesh.triangles).cuda(), morton_bits=63)
    ref_a = bvh.query(dF, dE, "any_hit", stats=True)
    ref_c = bvh.query(dF, dE, "count", stats=True)
    assert ref_c["stats"]["band_rays"] > 10_000   # the FP64 pass has real work
    hit = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    amb = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    cnt = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    amb_c = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    assert _noalloc(rsi, bvh, dF, dE, rsi.RSI_COUNT, count=cnt, amb=amb_c) == 0, rsi.last_error()   # set-up
    rsi.fail_allocations(0)
    try:
        for _ in range(2):
            assert _noalloc(rsi, bvh, dF, dE, rsi.RSI_ANY_HIT, hit=hit, amb=amb) == 0, rsi.last_error()
            assert _noalloc(rsi, bvh, dF, dE, rsi.RSI_COUNT, count=cnt, amb=amb_c) == 0, rsi.last_error()
            torch.cuda.synchronize()
            assert torch.equal(hit, ref_a["hit"]) and torch.equal(amb, ref_a["ambiguous"])
            assert torch.equal(cnt, ref_c["count"]) and torch.equal(amb_c, ref_c["ambiguous"])
    finally:
        rsi.fail_allocations(None)
    got_amb = amb_c.cpu().numpy()
    rng = np.random.default_rng(5)
    marked = np.flatnonzero(got_amb)[:400]
    idx = np.unique(np.concatenate([marked, rng.choice(n, 600, replace=False)]))
    ref = oracle.query(mesh.vertices, mesh.triangles, F[idx], E[idx])
    h, a = hit.cpu().numpy()[idx], amb.cpu().numpy()[idx]
    c, ac = cnt.cpu().numpy()[idx], got_amb[idx]
    assert np.array_equal(a, ref["amb_hit"]) and np.array_equal(ac, ref["amb_count"])
    assert np.array_equal(h[a == 0], ref["hit"][a == 0])
    assert np.array_equal(c[ac == 0], ref["count"][ac == 0])
    bvh.close()
