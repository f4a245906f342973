"""Seeded synthetic workloads: heightfield meshes and segment batches.

Shared by the tests, the smoke check and the benchmark; holds none of the
intersection method's arithmetic (only how inputs are drawn).  They stand in
for the paper's surface generator and 10 M-ray data set (Sec. 3.3, Sec. 4.2),
which are not available: a ~2e4-triangle heightfield and 1e7 segments keep
the paper's order of scale.

Meshes: an n x n vertex grid over [0, 1]^2, vertex index j * n + i at
(i / (n-1), j / (n-1)), cell (i, j) split into (v_ij, v_i+1j, v_i+1j+1) and
(v_ij, v_i+1j+1, v_ij+1); height = sum of 4 seeded sinusoids of amplitude
0.1 (+ optional Gaussian bumps; optional xy jitter of the vertices).

Segments are produced in chunks of 2**20 whose generator is seeded by
(seed, chunk index), so any sub-range can be regenerated on its own (the
oracle checks samples of batches too large for it).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CHUNK = 1 << 20


@dataclass
class Mesh:
    vertices: np.ndarray   # float32 [N_v, 3]
    triangles: np.ndarray  # int32 [N_t, 3]
    n: int
    seed: int
    params: dict = field(default_factory=dict)

    @property
    def z_max(self) -> float:
        return float(self.vertices[:, 2].max())

    @property
    def z_min(self) -> float:
        return float(self.vertices[:, 2].min())


def grid_triangles(n: int, ny: int | None = None) -> np.ndarray:
    ny = n if ny is None else ny
    i, j = np.meshgrid(np.arange(n - 1), np.arange(ny - 1), indexing="xy")
    i, j = i.ravel(), j.ravel()
    v00 = j * n + i
    v10 = j * n + i + 1
    v11 = (j + 1) * n + i + 1
    v01 = (j + 1) * n + i
    t = np.empty((2 * (n - 1) * (ny - 1), 3), np.int32)
    t[0::2] = np.stack([v00, v10, v11], 1)
    t[1::2] = np.stack([v00, v11, v01], 1)
    return t


def heightfield(n: int, seed: int, n_bumps: int = 0, jitter: float = 0.0, ny: int | None = None) -> Mesh:
    """n x n (or n x ny) heightfield over [0, 1]^2: 4 sinusoids
    0.1 sin(2 pi (fx x + fy y) + phi) with fx, fy ~ U(-3, 3),
    phi ~ U(0, 2 pi); n_bumps Gaussian bumps of height U(0.05, 0.2) and width
    U(0.03, 0.1); xy jitter ~ U(+-jitter cell)."""
    ny = n if ny is None else ny
    rng = np.random.default_rng([seed, 0x4D455348])
    fx, fy = rng.uniform(-3, 3, 4), rng.uniform(-3, 3, 4)
    phi = rng.uniform(0, 2 * math.pi, 4)
    bumps = [(rng.uniform(0, 1), rng.uniform(0, 1), rng.uniform(0.05, 0.2), rng.uniform(0.03, 0.1))
             for _ in range(n_bumps)]
    i, j = np.meshgrid(np.arange(n), np.arange(ny), indexing="xy")
    x = (i.ravel() / (n - 1)).astype(np.float64)
    y = (j.ravel() / (ny - 1)).astype(np.float64)
    if jitter > 0:
        x = x + rng.uniform(-jitter, jitter, x.shape) / (n - 1)
        y = y + rng.uniform(-jitter, jitter, y.shape) / (ny - 1)
    z = np.zeros_like(x)
    for k in range(4):
        z += 0.1 * np.sin(2 * math.pi * (fx[k] * x + fy[k] * y) + phi[k])
    for (cx, cy, h, s) in bumps:
        z += h * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s * s))
    V = np.stack([x, y, z], 1).astype(np.float32)
    params = dict(fx=fx.tolist(), fy=fy.tolist(), phi=phi.tolist(), bumps=bumps, jitter=jitter)
    return Mesh(V, grid_triangles(n, ny), n, seed, params)


def _unit_vectors(rng, m):
    v = rng.normal(size=(m, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _points_on_mesh(rng, mesh: Mesh, m):
    """Uniform points over the mesh's xy footprint, lifted onto the mesh."""
    V = mesh.vertices.astype(np.float64)
    T = mesh.triangles
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    area = 0.5 * np.abs((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))
    cdf = np.cumsum(area)
    tri = np.minimum(np.searchsorted(cdf, rng.uniform(0, cdf[-1], m)), len(T) - 1)
    r1, r2 = rng.uniform(size=m), rng.uniform(size=m)
    flip = r1 + r2 > 1
    r1[flip], r2[flip] = 1 - r1[flip], 1 - r2[flip]
    p = a[tri] + r1[:, None] * (b[tri] - a[tri]) + r2[:, None] * (c[tri] - a[tri])
    return p, tri


def _chunk_uniform_box(rng, m):
    """Segments of the small configuration: start and end xy ~ U[0,1]^2
    independently, start z ~ U(-0.5, 0), end z ~ U(0.2, 0.7)."""
    f = np.empty((m, 3)); t = np.empty((m, 3))
    f[:, 0:2] = rng.uniform(0, 1, (m, 2)); t[:, 0:2] = rng.uniform(0, 1, (m, 2))
    f[:, 2] = rng.uniform(-0.5, 0.0, m); t[:, 2] = rng.uniform(0.2, 0.7, m)
    return f, t


def _chunk_cross_above(rng, mesh: Mesh, m, frac_cross=0.5):
    """Half the segments cross the surface, half lie wholly above it:
    crossing: a point p on the mesh, a random unit direction, length
    L ~ U(0.05, 1), p at fraction s ~ U(0, 1) along the segment;
    above: midpoint xy ~ U[0,1]^2 at z >= z_max + L/2 + 0.01."""
    L = rng.uniform(0.05, 1.0, m)
    d = _unit_vectors(rng, m)
    cross = rng.uniform(size=m) < frac_cross
    p, _ = _points_on_mesh(rng, mesh, m)
    s = rng.uniform(size=m)
    f = p - (s * L)[:, None] * d
    t = p + ((1 - s) * L)[:, None] * d
    mid = np.empty((m, 3))
    mid[:, 0:2] = rng.uniform(0, 1, (m, 2))
    mid[:, 2] = mesh.z_max + L / 2 + 0.01 + rng.uniform(0, 0.2, m)
    fa = mid - (L / 2)[:, None] * d
    ta = mid + (L / 2)[:, None] * d
    f = np.where(cross[:, None], f, fa)
    t = np.where(cross[:, None], t, ta)
    return f, t


def _chunk_grazing(rng, mesh: Mesh, m):
    """Grazing segments, a third each: an end point within 1e-6 of an edge,
    within 1e-6 of a vertex, or a segment nearly parallel to a face (direction
    in the face plane tilted by <= 1e-6, passing within 1e-6 of the face)."""
    V = mesh.vertices.astype(np.float64)
    T = mesh.triangles
    tri = rng.integers(0, len(T), m)
    a, b, c = V[T[tri, 0]], V[T[tri, 1]], V[T[tri, 2]]
    kind = rng.integers(0, 3, m)
    L = rng.uniform(0.05, 1.0, m)
    d = _unit_vectors(rng, m)
    off = _unit_vectors(rng, m) * rng.uniform(0, 1e-6, m)[:, None]
    # kind 0: near an edge
    edge = rng.integers(0, 3, m)
    P = np.stack([a, b, c], 1)
    e0 = P[np.arange(m), edge]
    e1 = P[np.arange(m), (edge + 1) % 3]
    lam = rng.uniform(size=m)[:, None]
    p_edge = e0 + lam * (e1 - e0) + off
    # kind 1: near a vertex
    p_vert = e0 + off
    # kind 2: nearly parallel to the face
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    inplane = d - (d * n).sum(1, keepdims=True) * n
    inplane /= np.linalg.norm(inplane, axis=1, keepdims=True)
    tilt = rng.uniform(-1e-6, 1e-6, m)[:, None]
    dpar = inplane + tilt * n
    dpar /= np.linalg.norm(dpar, axis=1, keepdims=True)
    r1, r2 = rng.uniform(size=m), rng.uniform(size=m)
    flip = r1 + r2 > 1
    r1[flip], r2[flip] = 1 - r1[flip], 1 - r2[flip]
    p_face = a + r1[:, None] * (b - a) + r2[:, None] * (c - a) + n * rng.uniform(-1e-6, 1e-6, m)[:, None]
    s = rng.uniform(size=m)
    f = np.empty((m, 3)); t = np.empty((m, 3))
    # end point near an edge / a vertex: the segment ends (or starts) there
    at_end = rng.uniform(size=m) < 0.5
    for k, p in ((0, p_edge), (1, p_vert)):
        sel = kind == k
        other = p - L[:, None] * d
        f[sel] = np.where(at_end[sel, None], other[sel], p[sel])
        t[sel] = np.where(at_end[sel, None], p[sel], (p + L[:, None] * d)[sel])
    sel = kind == 2
    f[sel] = (p_face - (s * L)[:, None] * dpar)[sel]
    t[sel] = (p_face + ((1 - s) * L)[:, None] * dpar)[sel]
    return f, t


@dataclass
class RaySpec:
    kind: str            # "uniform_box" | "cross_above" | "grazing_mix"
    n: int
    seed: int
    grazing_frac: float = 0.0


def ray_chunk(spec: RaySpec, mesh: Mesh, c: int):
    """Chunk c (rows c*CHUNK .. ) of a segment batch: float32 (from, to)."""
    m = min(CHUNK, spec.n - c * CHUNK)
    rng = np.random.default_rng([spec.seed, 0x52415953, c])
    if spec.kind == "uniform_box":
        f, t = _chunk_uniform_box(rng, m)
    elif spec.kind == "cross_above":
        f, t = _chunk_cross_above(rng, mesh, m)
    elif spec.kind == "grazing_mix":
        f, t = _chunk_cross_above(rng, mesh, m)
        g = rng.uniform(size=m) < spec.grazing_frac
        ng = int(g.sum())
        if ng:
            gf, gt = _chunk_grazing(rng, mesh, ng)
            f[g], t[g] = gf, gt
    else:
        raise ValueError(spec.kind)
    return f.astype(np.float32), t.astype(np.float32)


def rays(spec: RaySpec, mesh: Mesh, start: int = 0, count: int | None = None, out=None):
    """Rows [start, start + count) of the batch as float32 [count, 3] pairs.
    `out` may be a pair of preallocated (e.g. pinned) float32 arrays."""
    if count is None:
        count = spec.n - start
    if out is None:
        F = np.empty((count, 3), np.float32)
        E = np.empty((count, 3), np.float32)
    else:
        F, E = out
    c0, c1 = start // CHUNK, (start + count + CHUNK - 1) // CHUNK
    for c in range(c0, c1):
        f, t = ray_chunk(spec, mesh, c)
        lo = max(start, c * CHUNK)
        hi = min(start + count, c * CHUNK + len(f))
        F[lo - start:hi - start] = f[lo - c * CHUNK:hi - c * CHUNK]
        E[lo - start:hi - start] = t[lo - c * CHUNK:hi - c * CHUNK]
    return F, E


def _chunk_task(args):
    spec, mesh, c = args
    return ray_chunk(spec, mesh, c)


def rays_many(jobs, workers: int | None = None):
    """Several whole batches [(mesh, spec), ...] generated chunk by chunk in
    a pool of spawned processes (start it before the process touches a GPU).
    Returns [(from, to), ...] in job order, identical to rays()."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    tasks = [(spec, mesh, c) for mesh, spec in jobs for c in range((spec.n + CHUNK - 1) // CHUNK)]
    workers = workers or min(32, os.cpu_count() or 1)
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_chunk_task, tasks, chunksize=1))
    out, k = [], 0
    for mesh, spec in jobs:
        nc = (spec.n + CHUNK - 1) // CHUNK
        fs = [parts[k + i][0] for i in range(nc)]
        ts = [parts[k + i][1] for i in range(nc)]
        k += nc
        F = np.concatenate(fs) if fs else np.zeros((0, 3), np.float32)
        E = np.concatenate(ts) if ts else np.zeros((0, 3), np.float32)
        out.append((F, E))
    return out


def rays_at(spec: RaySpec, mesh: Mesh, idx: np.ndarray):
    """Rows idx (any order) of the batch, regenerating only their chunks."""
    idx = np.asarray(idx, np.int64)
    F = np.empty((len(idx), 3), np.float32)
    E = np.empty((len(idx), 3), np.float32)
    chunks = idx // CHUNK
    for c in np.unique(chunks):
        f, t = ray_chunk(spec, mesh, int(c))
        sel = chunks == c
        F[sel] = f[idx[sel] - c * CHUNK]
        E[sel] = t[idx[sel] - c * CHUNK]
    return F, E


# ---------------------------------------------------------------- configs
def config_mesh(name: str) -> Mesh:
    if name == "c1":
        return heightfield(32, seed=1)
    if name == "c2":
        return heightfield(100, seed=2, n_bumps=8)
    if name == "c3":
        return heightfield(300, seed=3, n_bumps=8, jitter=0.3)
    if name == "paper":
        # the paper's test surface has 14,874 vertices and 29,260 triangles
        # (Sec. 3.3); a 111 x 134 vertex grid has exactly those counts
        return heightfield(111, seed=6, n_bumps=8, ny=134)
    raise ValueError(name)


def config_rays(name: str, n: int | None = None) -> RaySpec:
    if name == "c1":
        return RaySpec("uniform_box", n or 100_000, seed=1)
    if name == "c2":
        return RaySpec("cross_above", n or 10_000_000, seed=2)
    if name == "c3":
        return RaySpec("grazing_mix", n or 100_000_000, seed=3, grazing_frac=0.01)
    if name == "paper":
        return RaySpec("cross_above", n or 10_000_000, seed=6)
    raise ValueError(name)


CONFIG_DOC = {
    "c1": "32x32-vertex heightfield (1,922 triangles), 1e5 segments z from U(-0.5,0) to U(0.2,0.7)",
    "c2": "100x100-vertex heightfield with 8 bumps (19,602 triangles), 1e7 segments: 50% crossing, 50% above",
    "c3": "300x300-vertex jittered heightfield (178,802 triangles), 1e8 segments, 1% grazing",
    "paper": "111x134-vertex heightfield with 8 bumps (14,874 vertices, 29,260 triangles, the counts of the "
             "paper's surface), 1e7 segments: 50% crossing, 50% above",
}


def batched_meshes(n_meshes: int = 64, seed: int = 4, max_rays: int | None = None):
    """Many independent meshes with uneven sizes: triangle counts and ray
    counts log-uniform in [1e3, 1e5] and [1e4, 1e7]; grid n =
    round(sqrt(T / 2)) + 1; crossing/above segments per mesh."""
    rng = np.random.default_rng([seed, 0x42415443])
    tri = np.exp(rng.uniform(math.log(1e3), math.log(1e5), n_meshes))
    nr = np.exp(rng.uniform(math.log(1e4), math.log(1e7), n_meshes)).astype(np.int64)
    if max_rays is not None:
        nr = np.minimum(nr, max_rays)
    out = []
    for m in range(n_meshes):
        g = int(round(math.sqrt(tri[m] / 2))) + 1
        mesh = heightfield(g, seed=seed * 1000 + m, n_bumps=4)
        out.append((mesh, RaySpec("cross_above", int(nr[m]), seed=seed * 1000 + m)))
    return out
