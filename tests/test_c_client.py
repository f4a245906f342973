"""The C ABI used from plain C (tests/c_abi_client.c): the header compiles as
C11 and the client links against librsi.so (no GPU); on a GPU the client's
answers, built and queried from host memory, equal the oracle's."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2305_01867_gb300")
SCRATCH = os.path.join(ROOT, "tests", ".c_client")


@pytest.fixture(scope="module")
def client():
    import __graft_entry__
    b = __graft_entry__._builder()
    if not b.up_to_date():
        if not shutil.which(b.NVCC) and not os.path.exists(b.NVCC):
            pytest.skip("nvcc not available")
        b.build()
    os.makedirs(SCRATCH, exist_ok=True)
    exe = os.path.join(SCRATCH, f"c_abi_client_{os.getpid()}")
    cc = subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-O2", os.path.join(ROOT, "tests", "c_abi_client.c"),
                         "-I", os.path.join(ROOT, "include"), "-L", PKG, "-lrsi", f"-Wl,-rpath,{PKG}", "-o", exe],
                        capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    yield exe
    shutil.rmtree(SCRATCH, ignore_errors=True)


def test_client_compiles_and_links(client):
    assert os.access(client, os.X_OK)


@pytest.mark.gpu
def test_client_answers_equal_the_oracle(client):
    import oracle
    import workloads as W
    mesh = W.heightfield(40, seed=17, n_bumps=3)
    F, E = W.rays(W.RaySpec("cross_above", 30_000, seed=17), mesh)
    F[5] = F[6]                                          # a zero-length segment
    E[5] = F[5]
    inp, out = os.path.join(SCRATCH, "in.bin"), os.path.join(SCRATCH, "out.bin")
    n = len(F)
    with open(inp, "wb") as f:
        np.array([len(mesh.vertices), len(mesh.triangles), n], np.int64).tofile(f)
        for a in (mesh.vertices, mesh.triangles, F, E):
            np.ascontiguousarray(a).tofile(f)
    r = subprocess.run([client, inp, out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    raw = np.fromfile(out, np.uint8)
    assert raw.size == 7 * n
    hit, amb_h = raw[:n], raw[n:2 * n]
    cnt, amb_c = raw[2 * n:6 * n].view(np.int32), raw[6 * n:]
    ref = oracle.query(mesh.vertices, mesh.triangles, F, E)
    assert np.array_equal(amb_h, ref["amb_hit"]) and np.array_equal(amb_c, ref["amb_count"])
    ok_h, ok_c = ref["amb_hit"] == 0, ref["amb_count"] == 0
    assert np.array_equal(hit[ok_h], ref["hit"][ok_h])
    assert np.array_equal(cnt[ok_c], ref["count"][ok_c])
    assert hit[5] == 0 and cnt[5] == 0 and hit.sum() > 1000
