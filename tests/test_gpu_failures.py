"""Failure paths on the GPU without a GPU fault: allocation failures injected
on the host (rsi_debug_fail_allocations) surface as RSI_ERR_OOM at the call
that needed the memory, release what that call had taken, launch nothing,
and leave the library usable -- the same answers afterwards.  (The device
side of failure detection, a work-queue wait that runs out, is tested in
test_gpu_batched.py.)"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsi():
    import paper_2305_01867_gb300 as m
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return m


def test_injected_allocation_failures(rsi):
    mesh = W.heightfield(20, seed=5, n_bumps=1)
    F, E = W.rays(W.RaySpec("cross_above", 5000, seed=5), mesh)
    V, T = torch.from_numpy(mesh.vertices).cuda(), torch.from_numpy(mesh.triangles).cuda()
    dF, dE = torch.from_numpy(F).cuda(), torch.from_numpy(E).cuda()
    pF, pE = torch.from_numpy(F).pin_memory(), torch.from_numpy(E).pin_memory()

    def pipeline():
        bvh = rsi.LBVH(V, T)
        try:
            a = bvh.query(dF, dE, "any_hit")
            c = bvh.query(dF, dE, "count")
            nr = bvh.nearest(dF, dE)
            hc = torch.empty(len(F), dtype=torch.int32).pin_memory()
            ha = torch.empty(len(F), dtype=torch.uint8).pin_memory()
            bvh.query_host(pF, pE, "count", count=hc, ambiguous=ha)
            torch.cuda.synchronize()
            return [a["hit"].cpu(), a["ambiguous"].cpu(), c["count"].cpu(), c["ambiguous"].cpu(),
                    nr["tri"].cpu(), nr["t"].cpu(), hc.clone(), ha.clone()]
        finally:
            bvh.close()

    ref = pipeline()
    failed = []
    for k in range(8):
        rsi.fail_allocations(k)
        try:
            pipeline()
        except rsi.RSIError as e:
            assert e.code == -3, (k, e)
            failed.append(k)
        finally:
            rsi.fail_allocations(None)
    assert 0 in failed and len(failed) >= 2, failed
    got = pipeline()
    for x, y in zip(got, ref):
        assert torch.equal(x, y)
    assert torch.equal(got[2], got[6])          # host-buffer and device-buffer counts agree
