"""The seeded synthetic inputs follow the recipe they are documented with
(no GPU): mesh sizes and triangulation, the crossing / above split and the
lengths of the segments, the grazing mix, regeneration of any sub-range,
and the realised totals of the many-mesh configuration."""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("name,nv,nt", [("c1", 1024, 1922), ("c2", 10_000, 19_602), ("c3", 90_000, 178_802),
                                        ("paper", 14_874, 29_260)])
def test_mesh_sizes(name, nv, nt):
    m = W.config_mesh(name)
    assert m.vertices.shape == (nv, 3) and m.triangles.shape == (nt, 3)
    assert m.vertices.dtype == np.float32 and m.triangles.dtype == np.int32


def test_grid_layout_and_triangulation():
    """Vertex j n + i sits at (i / (n-1), j / (n-1)); cell (i, j) is split into
    (v_ij, v_i+1,j, v_i+1,j+1) and (v_ij, v_i+1,j+1, v_i,j+1); the triangles
    tile the unit square once, all facing up."""
    n = 7
    m = W.heightfield(n, seed=3)
    V = m.vertices.astype(np.float64)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    np.testing.assert_allclose(V[:, 0], (i / (n - 1)).ravel(), atol=1e-7)
    np.testing.assert_allclose(V[:, 1], (j / (n - 1)).ravel(), atol=1e-7)
    T = m.triangles
    assert T[0].tolist() == [0, 1, n + 1] and T[1].tolist() == [0, n + 1, n]
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    cross_z = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert np.all(cross_z > 0)
    assert abs(0.5 * cross_z.sum() - 1.0) < 1e-9


def test_relief_amplitude():
    """Four sinusoids of amplitude 0.1 (|z| <= 0.4), plus up to 8 bumps of
    height <= 0.2 on the larger meshes."""
    assert np.abs(W.config_mesh("c1").vertices[:, 2]).max() <= 0.4 + 1e-6
    for name in ("c2", "c3", "paper"):
        z = W.config_mesh(name).vertices[:, 2]
        assert z.min() >= -0.4 - 1e-6 and z.max() <= 0.4 + 8 * 0.2 + 1e-6


def test_crossing_and_above_segments():
    """c2 segments: lengths in [0.05, 1]; about half lie wholly above the
    surface's highest vertex, the others pass through a point of the mesh, so
    their lower end is no higher than the mesh top."""
    mesh = W.config_mesh("c2")
    F, E = W.rays(W.config_rays("c2", 200_000), mesh)
    L = np.linalg.norm(E.astype(np.float64) - F, axis=1)
    assert L.min() >= 0.05 - 1e-6 and L.max() <= 1.0 + 1e-6
    above = np.minimum(F[:, 2], E[:, 2]) > mesh.z_max
    assert abs(above.mean() - 0.5) < 0.01
    assert np.all(np.minimum(F[~above, 2], E[~above, 2]) <= mesh.z_max + 1e-6)


def test_crossing_segments_meet_the_surface():
    """Per the oracle, every crossing segment of a small sample meets the
    surface (or grazes it), and no segment above it does."""
    mesh = W.config_mesh("c1")
    F, E = W.rays(W.RaySpec("cross_above", 3000, seed=21), mesh)
    above = np.minimum(F[:, 2], E[:, 2]) > mesh.z_max
    r = oracle.query(mesh.vertices, mesh.triangles, F, E)
    assert np.all(r["hit"][~above] == 1)
    assert np.all(r["hit"][above] == 0) and np.all(r["amb_count"][above] == 0)


def test_grazing_segments_sit_in_the_band():
    """The grazing mix (end point within 1e-6 of an edge or a vertex, or a
    segment within 1e-6 of a face and tilted by <= 1e-6) puts most of its
    segments in the oracle's ambiguity band; the c3 batch has about 1 % of
    them."""
    mesh = W.config_mesh("c1")
    F, E = W.rays(W.RaySpec("grazing_mix", 3000, seed=22, grazing_frac=1.0), mesh)
    r = oracle.query(mesh.vertices, mesh.triangles, F, E)
    assert r["amb_count"].mean() > 0.5
    m3 = W.config_mesh("c3")
    F3, _ = W.ray_chunk(W.config_rays("c3"), m3, 0)
    plain, _ = W.ray_chunk(W.RaySpec("cross_above", W.CHUNK, seed=3), m3, 0)
    # rows replaced by grazing segments differ from the plain draw of the same chunk
    assert 0.008 < np.mean(np.any(F3 != plain, axis=1)) < 0.012


def test_any_sub_range_regenerates_exactly():
    """Rows are drawn in chunks of 2^20 seeded by (seed, chunk): a sub-range
    or a scattered index set across a chunk boundary equals the same rows of
    the whole batch."""
    mesh = W.config_mesh("c1")
    spec = W.RaySpec("cross_above", W.CHUNK + 5000, seed=9)
    F, E = W.rays(spec, mesh)
    f, e = W.rays(spec, mesh, start=W.CHUNK - 100, count=300)
    assert np.array_equal(f, F[W.CHUNK - 100:W.CHUNK + 200]) and np.array_equal(e, E[W.CHUNK - 100:W.CHUNK + 200])
    idx = np.array([W.CHUNK + 4999, 7, W.CHUNK, 123_456, W.CHUNK - 1])
    f, e = W.rays_at(spec, mesh, idx)
    assert np.array_equal(f, F[idx]) and np.array_equal(e, E[idx])
    F2, _ = W.rays(W.RaySpec("cross_above", 1000, seed=10), mesh)
    assert not np.array_equal(F2, F[:1000])


def test_many_mesh_configuration_totals():
    """64 meshes with log-uniform triangle and segment counts; the realised
    totals are the ones the measurements quote (1.16e6 triangles, 7.7e7
    segments)."""
    jobs = W.batched_meshes(64, seed=4)
    nt = sum(len(m.triangles) for m, _ in jobs)
    nr = sum(s.n for _, s in jobs)
    assert len(jobs) == 64 and nt == 1_161_888 and nr == 76_748_244
    sizes = np.array([len(m.triangles) for m, _ in jobs])
    assert sizes.min() >= 800 and sizes.max() <= 2 * 10 ** 5
