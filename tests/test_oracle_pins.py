"""Pins of the CPU oracle to things other than itself (no GPU).

* the paper's worked example (Sec. 4.1): printed hit points, boolean result,
  leaf order, leaf and internal boxes;
* the canopy surface of Sec. 4.1.5 (counts follow from our patch geometry);
* closed forms of axis-aligned cases (t, u, v known by hand);
* a closed box: convexity fixes every crossing count;
* exact rational orientation predicates (a different formula: signed
  volumes instead of Moller's cross/dot products) on near-boundary pairs;
* the degenerate cases the method has (edge, vertex, end point, parallel,
  zero-area triangle, zero-length segment).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from golden_io import load

MISS, HIT, AMB = oracle.PAIR_MISS, oracle.PAIR_HIT, oracle.PAIR_AMBIGUOUS


# ------------------------------------------------------------ worked example
def test_case_study1_boolean_and_hit_points():
    g = load("case_study1_sec4_1.txt")
    r = oracle.query(g["vertices"], g["triangles"], g["ray_from"], g["ray_to"])
    assert r["hit"].tolist() == g["boolean"].tolist()
    assert r["amb_hit"].sum() == 0 and r["amb_count"].sum() == 0
    for ray, tri, point in g["hitpoint"]:
        assert r["near_tri"][ray] == tri
        s, e = g["ray_from"][ray].astype(np.float64), g["ray_to"][ray].astype(np.float64)
        p = s + float(r["near_t"][ray]) * (e - s)
        # the printed points carry 2 decimals; FP32 vertices round at ~1e-7
        np.testing.assert_allclose(p, point, atol=2e-6)
        np.testing.assert_allclose(r["near_point"][ray], point, atol=2e-6)
        assert abs(r["near_dist"][ray] - np.linalg.norm(np.asarray(point) - s)) < 2e-6
        assert r["count"][ray] == 1


def test_case_study1_leaf_order_and_boxes():
    g = load("case_study1_sec4_1.txt")
    b = oracle.build_all(g["vertices"], g["triangles"], bits=30)
    assert b["perm"].tolist() == g["leaf_order"].tolist()
    b63 = oracle.build_all(g["vertices"], g["triangles"], bits=63)
    assert b63["perm"].tolist() == g["leaf_order"].tolist()
    n = len(b["perm"])
    for leaf, box in g["leaf_box"].items():
        got = b["box"][n - 1 + leaf]
        np.testing.assert_allclose(got[[0, 3, 1, 4, 2, 5]], box, atol=1e-6)
    ranges = {(int(a), int(c)): i for i, (a, c) in enumerate(zip(b["range_lo"], b["range_hi"]))}
    assert set(ranges) == set(g["internal_box"])
    for rng, box in g["internal_box"].items():
        got = b["box"][ranges[rng]]
        np.testing.assert_allclose(got[[0, 3, 1, 4, 2, 5]], box, atol=1e-6)
    # root covers all leaves (Sec. 4.2: bounds reach the top of the tree)
    assert ranges[(0, 3)] == 0


def test_canopy_counts():
    g = load("canopy_sec4_1_5.txt")
    r = oracle.query(g["vertices"], g["triangles"], g["ray_from"], g["ray_to"])
    assert r["count"].tolist() == g["count"].tolist()
    assert r["amb_count"].sum() == 0
    assert r["hit"].tolist() == (g["count"] > 0).astype(int).tolist()


# ------------------------------------------------------------ closed forms
TRI = ([0, 0, 0], [1, 0, 0], [0, 1, 0])


@pytest.mark.parametrize("x,y,z0,z1", [(0.25, 0.25, -1, 3), (0.1, 0.6, -2, 0.5), (0.7, 0.2, 1, -1)])
def test_axis_aligned_closed_form(x, y, z0, z1):
    cls, q = oracle.classify_pair([x, y, z0], [x, y, z1], *TRI)
    assert cls == HIT
    t = -z0 / (z1 - z0)
    assert q["t"] == pytest.approx(t, abs=1e-12)
    x64, y64 = float(np.float32(x)), float(np.float32(y))
    assert q["u"] == pytest.approx(x64, abs=1e-12)   # weight of b = x
    assert q["v"] == pytest.approx(y64, abs=1e-12)   # weight of c = y
    assert q["w"] == pytest.approx(1 - x64 - y64, abs=1e-12)


@pytest.mark.parametrize("name,s,e,expect", [
    ("edge u=0 side", [0.0, 0.5, -1], [0.0, 0.5, 1], AMB),
    ("edge v=0 side", [0.5, 0.0, -1], [0.5, 0.0, 1], AMB),
    ("hypotenuse", [0.5, 0.5, -1], [0.5, 0.5, 1], AMB),
    ("vertex", [0.0, 0.0, -1], [0.0, 0.0, 1], AMB),
    ("vertex b", [1.0, 0.0, -1], [1.0, 0.0, 1], AMB),
    ("start on face t=0", [0.25, 0.25, 0], [0.25, 0.25, 1], AMB),
    ("end on face t=1", [0.25, 0.25, -1], [0.25, 0.25, 0], AMB),
    ("in-plane through face", [0.1, 0.1, 0], [0.3, 0.3, 0], AMB),
    ("in-plane far away", [2.0, 2.0, 0], [3.0, 3.0, 0], MISS),
    ("parallel above", [0.2, 0.2, 0.5], [0.4, 0.2, 0.5], MISS),
    ("outside footprint", [2.0, 2.0, -1], [2.0, 2.0, 1], MISS),
    ("stops short", [0.25, 0.25, 0.5], [0.25, 0.25, 1], MISS),
    ("just inside edge", [0.5, 1e-3, -1], [0.5, 1e-3, 1], HIT),
    ("just outside edge", [0.5, -1e-3, -1], [0.5, -1e-3, 1], MISS),
    ("zero-length on face", [0.25, 0.25, 0], [0.25, 0.25, 0], MISS),
])
def test_degenerate_and_boundary_cases(name, s, e, expect):
    cls, _ = oracle.classify_pair(s, e, *TRI)
    assert cls == expect, name


def test_zero_area_triangle_never_hits():
    a, b = [0, 0, 0], [1, 0, 0]
    c = [2, 0, 0]                       # collinear: the normal is exactly zero
    cls, _ = oracle.classify_pair([0.5, 0, -1], [0.5, 0, 1], a, b, c)
    assert cls == MISS


def test_nearly_parallel_uses_distance():
    # direction tilted by 1e-8 rad out of the plane z = 0, 0.1 above it: the
    # distance 0.1 >> tau |d| so it is a decisive miss, though det_rel < tau
    cls, q = oracle.classify_pair([-1, 0.2, 0.1], [1, 0.2, 0.1 + 2e-8], *TRI)
    assert abs(q["det_rel"]) <= oracle.TAU and q["dist"] > 0.09 and cls == MISS
    # the same segment 1e-9 above the face is within the band: ambiguous
    cls, q = oracle.classify_pair([-1, 0.2, 0.0], [1, 0.2, 2e-8], *TRI)
    assert cls == AMB


# ------------------------------------------------------------ closed box
def _cube():
    V = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], np.float32)
    q = [(0, 1, 3, 2), (4, 5, 7, 6), (0, 1, 5, 4), (2, 3, 7, 6), (0, 2, 6, 4), (1, 3, 7, 5)]
    T = []
    for a, b, c, d in q:
        T += [(a, b, c), (a, c, d)]
    return V, np.array(T, np.int32)


def test_closed_box_crossing_parity():
    V, T = _cube()
    rng = np.random.default_rng(7)
    n = 4000
    F = rng.uniform(-1, 2, (n, 3)).astype(np.float32)
    E = rng.uniform(-1, 2, (n, 3)).astype(np.float32)
    inside = lambda P: np.all((P > 0) & (P < 1), axis=1)
    # force a quarter of the segments to start inside
    F[: n // 4] = rng.uniform(0.05, 0.95, (n // 4, 3)).astype(np.float32)
    r = oracle.query(V, T, F, E)
    ok = r["amb_count"] == 0
    assert ok.mean() > 0.95
    fi, ei = inside(F), inside(E)
    cnt = r["count"]
    # a convex closed surface: through-segments cross 0 or 2 times, a segment
    # with exactly one end inside crosses once, both inside: never
    both_out = ok & ~fi & ~ei
    one_in = ok & (fi ^ ei)
    both_in = ok & fi & ei
    assert set(np.unique(cnt[both_out])) <= {0, 2}
    assert np.all(cnt[one_in] == 1)
    assert np.all(cnt[both_in] == 0)
    assert np.all(r["hit"][ok] == (cnt[ok] > 0))
    assert both_out.sum() > 500 and one_in.sum() > 500


def test_crossings_through_shared_edges_and_vertices_count_once():
    """The reading of "unique intersections" (Sec. 1) pinned by convexity: a
    segment from inside the closed box to outside crosses its surface at
    exactly one point, also where that point is a vertex (3 to 6 triangles
    meet there), an edge, or the diagonal splitting a face, so the distinct
    crossing points number 1 although several triangles report a hit; a
    segment along the main diagonal, both ends outside, crosses at 2
    vertices.  The rays are ambiguous (they meet edges), and the count is the
    closed-interval one."""
    V, T = _cube()
    c = np.full(3, 0.5)
    corners = [np.array(v, float) for v in V]
    edges = [(corners[i] + corners[j]) / 2 for i in range(8) for j in range(i + 1, 8)
             if np.sum(corners[i] != corners[j]) == 1]
    diag = []
    for a, b, cc in T.reshape(-1, 2, 3)[:, 0]:      # first triangle of each face: (a, b, c), diagonal a-c
        diag += [(corners[a] + corners[cc]) / 2, 0.75 * corners[a] + 0.25 * corners[cc]]
    targets = corners + edges + diag
    assert len(edges) == 12 and len(diag) == 12
    F = np.array([c] * len(targets), np.float32)
    E = np.array([c + 2 * (p - c) for p in targets], np.float32)
    r = oracle.query(V, T, F, E)
    assert r["count"].tolist() == [1] * len(targets)
    assert r["amb_count"].all() and r["hit"].all()
    incl = [sum(oracle.classify_pair(F[i], E[i], *V[t])[1]["incl"] for t in T) for i in range(len(targets))]
    assert min(incl) >= 2 and max(incl) >= 3           # several triangles report each point
    r = oracle.query(V, T, [[-0.5, -0.5, -0.5]], [[1.5, 1.5, 1.5]])
    assert r["count"][0] == 2 and r["amb_count"][0] == 1


# ------------------------------------------------------------ exact predicates
def _F(x):
    return [Fraction(float(v)) for v in x]


def _orient(a, b, c, d):
    ab = [b[i] - a[i] for i in range(3)]
    ac = [c[i] - a[i] for i in range(3)]
    ad = [d[i] - a[i] for i in range(3)]
    return (ab[0] * (ac[1] * ad[2] - ac[2] * ad[1]) - ab[1] * (ac[0] * ad[2] - ac[2] * ad[0])
            + ab[2] * (ac[0] * ad[1] - ac[1] * ad[0]))


def _exact_class(s, e, a, b, c, tau=Fraction(1, 10 ** 6)):
    """Exact classification from signed volumes.  Returns (cls, guard) where
    guard is False when a margin sits so near a threshold that FP64 rounding
    could flip it, or when the pair is on the nearly-parallel branch (there
    the threshold is an irrational distance and is not checked here)."""
    s, e, a, b, c = map(_F, (s, e, a, b, c))
    d = [e[i] - s[i] for i in range(3)]
    e1 = [b[i] - a[i] for i in range(3)]
    e2 = [c[i] - a[i] for i in range(3)]
    n = [e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]]
    dot = lambda x, y: sum(x[i] * y[i] for i in range(3))
    det = -dot(d, n)                                      # e1 . (d x e2)
    den2 = dot(d, d) * dot(e1, e1) * dot(e2, e2)
    # nearly parallel (|det_rel| <= tau, with a relative guard of 1e-6 so that
    # FP64 rounding of det_rel cannot cross the threshold): not checked here
    if det == 0 or det * det <= tau * tau * den2 * (1 + Fraction(1, 10 ** 6)):
        return None, False
    # plane side of the end points: t = S_s / (S_s - S_e)
    Ss, Se = _orient(a, b, c, s), _orient(a, b, c, e)
    t = Ss / (Ss - Se)
    # barycentric weights of the line's plane point, from the volumes spanned
    # by the segment and each edge: weight of a ~ (s,e,b,c), b ~ (s,e,c,a),
    # c ~ (s,e,a,b)
    Oa, Ob, Oc = _orient(s, e, b, c), _orient(s, e, c, a), _orient(s, e, a, b)
    tot = Oa + Ob + Oc
    w, u, v = Oa / tot, Ob / tot, Oc / tot
    marg = min(abs(x - y) for x in (u, v, w, t) for y in (tau, -tau))
    marg = min(marg, abs(t - (1 - tau)), abs(t - (1 + tau)))
    guard = marg > Fraction(1, 10 ** 12)
    if u > tau and v > tau and w > tau and tau < t < 1 - tau:
        return HIT, guard
    if u < -tau or v < -tau or w < -tau or t < -tau or t > 1 + tau:
        return MISS, guard
    return AMB, guard


def _near_boundary_pairs(rng, n):
    """Triangles of random shape and size; segments aimed at a point of the
    triangle's edge, vertex or interior, displaced by 1e-9..1e-3 of the size,
    with random length and a random split of the segment at that point."""
    out = []
    for _ in range(n):
        a = rng.uniform(-1, 1, 3); b = a + rng.uniform(-0.3, 0.3, 3); c = a + rng.uniform(-0.3, 0.3, 3)
        kind = rng.integers(0, 4)
        lam = rng.uniform()
        if kind == 0:
            p = a + lam * (b - a)
        elif kind == 1:
            p = (a, b, c)[rng.integers(0, 3)].copy()
        elif kind == 2:
            r1, r2 = rng.uniform(size=2)
            if r1 + r2 > 1:
                r1, r2 = 1 - r1, 1 - r2
            p = a + r1 * (b - a) + r2 * (c - a)
        else:
            p = b + lam * (c - b)
        p = p + rng.normal(size=3) * 10.0 ** rng.uniform(-9, -3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        L = rng.uniform(0.01, 2.0)
        f = rng.choice([rng.uniform(), 0.0, 1.0, rng.uniform(-1e-6, 1e-6), 1 + rng.uniform(-1e-6, 1e-6)])
        s = p - f * L * d
        e = p + (1 - f) * L * d
        out.append([x.astype(np.float32) for x in (s, e, a, b, c)])
    return out


def test_oracle_matches_exact_predicates():
    rng = np.random.default_rng(11)
    checked = {HIT: 0, MISS: 0, AMB: 0}
    for s, e, a, b, c in _near_boundary_pairs(rng, 3000):
        exact, guard = _exact_class(s, e, a, b, c)
        cls, _ = oracle.classify_pair(s, e, a, b, c)
        if exact is None:
            # nearly parallel: a decisive hit would contradict the definition
            assert cls != HIT
            continue
        if guard:
            assert cls == exact
            checked[exact] += 1
    assert min(checked.values()) > 100, checked


def test_query_aggregates_pairs():
    """The per-ray answer is the aggregate of the per-pair classes."""
    g = load("canopy_sec4_1_5.txt")
    rng = np.random.default_rng(3)
    F = rng.uniform([11.8, 1.8, 0.5], [13.2, 3.2, 2.0], (300, 3)).astype(np.float32)
    E = rng.uniform([11.8, 1.8, 0.5], [13.2, 3.2, 2.0], (300, 3)).astype(np.float32)
    r = oracle.query(g["vertices"], g["triangles"], F, E)
    V, T = g["vertices"], g["triangles"]
    for i in range(len(F)):
        cls = [oracle.classify_pair(F[i], E[i], *V[T[j]])[0] for j in range(len(T))]
        nh, na = cls.count(HIT), cls.count(AMB)
        assert r["amb_count"][i] == (na > 0)
        assert r["amb_hit"][i] == (nh == 0 and na > 0)
        if na == 0:
            assert r["count"][i] == nh and r["hit"][i] == (nh > 0)


def test_shared_edge_counted_once_on_ambiguous_ray():
    """Reading of "unique intersections" (Sec. 1): a segment through the
    shared edge of two triangles is one crossing point (parity unpinned)."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], np.float32)
    T = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    r = oracle.query(V, T, [[0.5, 0.5, -1]], [[0.5, 0.5, 1]])
    assert r["amb_count"][0] == 1 and r["count"][0] == 1 and r["hit"][0] == 1


def test_answers_do_not_depend_on_the_thread_count():
    """The brute force splits the segments into contiguous ranges, one per
    thread: every split gives the same arrays as one thread."""
    g = load("canopy_sec4_1_5.txt")
    rng = np.random.default_rng(4)
    F = rng.uniform([11.8, 1.8, 0.5], [13.2, 3.2, 2.0], (257, 3)).astype(np.float32)
    E = rng.uniform([11.8, 1.8, 0.5], [13.2, 3.2, 2.0], (257, 3)).astype(np.float32)
    one = oracle.query(g["vertices"], g["triangles"], F, E, nthreads=1)
    for k in (2, 3, 7, 300):
        many = oracle.query(g["vertices"], g["triangles"], F, E, nthreads=k)
        for key in one:
            assert np.array_equal(one[key], many[key], equal_nan=True), (k, key)


def test_bad_index_rejected():
    V = np.zeros((3, 3), np.float32)
    with pytest.raises(ValueError):
        oracle.query(V, [[0, 1, 3]], [[0, 0, 0]], [[0, 0, 1]])


# ------------------------------------------------------------ nearest hit (barycentric mode)
def _plates(zs):
    """One right triangle [0,1]^2 (lower half) per height z, listed in the given order."""
    V, T = [], []
    for z in zs:
        k = len(V)
        V += [[0, 0, z], [1, 0, z], [0, 1, z]]
        T.append([k, k + 1, k + 2])
    return np.array(V, np.float32), np.array(T, np.int32)


def test_nearest_of_stacked_plates():
    """Three parallel plates listed out of order: the nearest crossing of a
    vertical segment is the first plate met from the start point, in both
    directions (Sec. 1, barycentric mode: triangle, distance, point)."""
    V, T = _plates([0.5, 0.0, 0.25])
    F = np.array([[0.25, 0.25, -1.0], [0.25, 0.25, 1.0], [0.25, 0.25, 0.75]], np.float32)
    E = np.array([[0.25, 0.25, 1.0], [0.25, 0.25, -1.0], [0.25, 0.25, 2.0]], np.float32)
    r = oracle.query(V, T, F, E)
    assert r["near_tri"].tolist() == [1, 0, -1]
    assert r["near_t"][:2].tolist() == [0.5, 0.25] and r["near_t"][2] == -1
    np.testing.assert_array_equal(r["near_point"][:2], [[0.25, 0.25, 0.0], [0.25, 0.25, 0.5]])
    assert np.isnan(r["near_point"][2]).all()
    assert r["near_dist"].tolist() == [1.0, 0.5, -1.0]
    assert r["count"].tolist() == [3, 3, 0] and r["amb_count"].sum() == 0


def test_nearest_equal_t_takes_lower_index():
    V, T = _plates([0.0, 0.3, 0.0, 0.0])     # plates 0, 2 and 3 coincide
    r = oracle.query(V, T, [[0.2, 0.2, -1.0]], [[0.2, 0.2, 1.0]])
    assert r["near_tri"][0] == 0 and r["near_t"][0] == 0.5


def test_nearest_on_heightfield_closed_form():
    """Vertical segments through a piecewise-linear surface cross it once:
    the crossing is the plane of the triangle whose footprint holds (x, y),
    found here by solving 2x2 systems (a different formula from Moller's)."""
    rng = np.random.default_rng(5)
    n = 6
    xs = np.linspace(0.0, 1.0, n)
    gx, gy = np.meshgrid(xs, xs, indexing="xy")
    gz = rng.uniform(-0.2, 0.2, gx.shape)
    V = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1).astype(np.float32)
    T = []
    for j in range(n - 1):
        for i in range(n - 1):
            a, b, c, d = j * n + i, j * n + i + 1, (j + 1) * n + i + 1, (j + 1) * n + i
            T += [(a, b, c), (a, c, d)]
    T = np.array(T, np.int32)
    P = rng.uniform(0.01, 0.99, (300, 2))
    F = np.c_[P, np.full(300, -1.0)].astype(np.float32)
    E = np.c_[P, np.full(300, 1.0)].astype(np.float32)
    r = oracle.query(V, T, F, E)
    V64 = V.astype(np.float64)
    for k in range(300):
        x, y = float(F[k, 0]), float(F[k, 1])
        want = None
        for j, tri in enumerate(T):
            a, b, c = V64[tri]
            lam = np.linalg.solve(np.array([[b[0] - a[0], c[0] - a[0]], [b[1] - a[1], c[1] - a[1]]]),
                                  np.array([x - a[0], y - a[1]]))
            if lam.min() > 1e-6 and lam.sum() < 1 - 1e-6:   # strictly inside the footprint
                z = a[2] + lam[0] * (b[2] - a[2]) + lam[1] * (c[2] - a[2])
                want = (j, z)
        if want is None:
            continue    # on a footprint edge: ambiguous by construction
        j, z = want
        assert r["near_tri"][k] == j and r["amb_count"][k] == 0
        assert abs(r["near_t"][k] - (z + 1.0) / 2.0) < 1e-6
        np.testing.assert_allclose(r["near_point"][k], [x, y, z], atol=1e-6)
        assert abs(r["near_dist"][k] - (z + 1.0)) < 1e-6


# ------------------------------------------------------------ the nearly-parallel branch
def test_nearest_none_when_every_crossing_lies_past_the_end():
    """A segment that stops before the plates it points at meets none of
    them: the inclusive test needs t <= 1 as well as t >= 0 (Sec. 1: a ray is
    the segment between its two end points)."""
    V, T = _plates([0.5, 0.0, 0.25])
    r = oracle.query(V, T, [[0.25, 0.25, -1.0]], [[0.25, 0.25, -0.5]])
    assert r["near_tri"][0] == -1 and r["count"][0] == 0 and r["hit"][0] == 0
    cls, q = oracle.classify_pair([0.25, 0.25, -1.0], [0.25, 0.25, -0.5], *TRI)
    assert cls == MISS and q["incl"] == 0 and q["t"] == 2.0


def test_det_rel_is_scale_free_closed_form():
    """det_rel = det / (|d||e1||e2|) is the sine of the segment's elevation
    over the plane times sin(e1, e2): for the unit right triangle and a
    segment rising 2h over a run of L it is -2h / |d|.  A 1000-long segment
    tilted by 1e-7 through the middle of the face is in the parallel branch
    (|det_rel| <= tau) and, as it meets the face, ambiguous; the same tilt
    over a unit run gives the same class."""
    for half, h in [(500.0, 5e-5), (0.5, 5e-8)]:
        s = np.array([0.25 - half, 0.25, -h], np.float32)
        e = np.array([0.25 + half, 0.25, h], np.float32)
        cls, q = oracle.classify_pair(s, e, *TRI)
        d = e.astype(np.float64) - s.astype(np.float64)
        assert q["det_rel"] == pytest.approx(-d[2] / np.linalg.norm(d), rel=1e-12)
        assert abs(q["det_rel"]) < oracle.TAU and cls == AMB and q["dist"] == 0.0


@pytest.mark.parametrize("z,expect", [(1e-4, AMB), (9e-4, AMB), (1.1e-3, MISS), (2e-3, MISS)])
def test_parallel_band_is_relative_to_segment_length(z, expect):
    """An exactly parallel segment of length 1000 passing over the face at
    height z is z away from it; the band is tau |d| = 1e-3 wide."""
    s, e = [-500.0, 0.25, z], [500.0, 0.25, z]
    cls, q = oracle.classify_pair(s, e, *TRI)
    assert q["dist"] == pytest.approx(float(np.float32(z)), rel=1e-12)
    assert cls == expect


def test_skew_pass_beside_an_edge_closed_form():
    """A segment rising with slope 0.9e-6 along y = 0.5, from x = -0.1 to
    x = 0.45, passes over the edge x = 0 of the unit right triangle at height
    3e-7 and ends over the face at 7.05e-7.  Its nearest approach is to the
    inside of that edge: the distance between the two lines, z(0) /
    sqrt(1 + slope^2).  That is within tau |d| = 5.5e-7 (ambiguous), while
    the end point alone (7.05e-7) is not."""
    s = np.array([-0.1, 0.5, 3e-7 - 0.1 * 0.9e-6], np.float32)
    e = np.array([0.45, 0.5, 3e-7 + 0.45 * 0.9e-6], np.float32)
    cls, q = oracle.classify_pair(s, e, *TRI)
    s64, e64 = s.astype(np.float64), e.astype(np.float64)
    slope = (e64[2] - s64[2]) / (e64[0] - s64[0])
    z0 = s64[2] + (0.0 - s64[0]) * slope
    assert abs(q["det_rel"]) < oracle.TAU and q["incl"] == 0
    assert q["dist"] == pytest.approx(z0 / np.sqrt(1 + slope * slope), rel=1e-9)
    assert cls == AMB


def _nearly_parallel_pairs(rng, n):
    """Random triangles and segments tilted by up to 2e-6 rad out of the
    triangle's plane, offset from it by up to 3e-6 |d|, passing over, beside
    or across the face: both sides of the det_rel and distance bands."""
    out = []
    while len(out) < n:
        a, b, c = rng.uniform(-1, 1, (3, 3))
        nrm = np.cross(b - a, c - a)
        if np.linalg.norm(nrm) < 0.2:
            continue
        nrm /= np.linalg.norm(nrm)
        u = (b - a) / np.linalg.norm(b - a)
        w = np.cross(nrm, u)
        phi = rng.uniform(0, 2 * np.pi)
        d = np.cos(phi) * u + np.sin(phi) * w
        d = d + rng.uniform(-2e-6, 2e-6) * nrm
        d /= np.linalg.norm(d)
        L = rng.uniform(0.05, 3.0)
        cen = (a + b + c) / 3
        p = cen + rng.uniform(-1, 1) * u + rng.uniform(-1, 1) * w + rng.uniform(-3e-6, 3e-6) * L * nrm
        f = rng.uniform(0, 1)
        out.append([x.astype(np.float32) for x in (p - f * L * d, p + (1 - f) * L * d, a, b, c)])
    return out


def test_classification_is_scale_free():
    """The margins are relative (det_rel, tau |d|), so scaling the whole
    configuration by a power of two -- exact in FP32 and FP64 -- changes no
    class, leaves u, v, t, det_rel unchanged bit for bit and scales the
    distance exactly."""
    rng = np.random.default_rng(21)
    n_par = 0
    for s, e, a, b, c in _nearly_parallel_pairs(rng, 1500) + _near_boundary_pairs(rng, 500):
        cls, q = oracle.classify_pair(s, e, a, b, c)
        n_par += q["dist"] >= 0
        for k in (-5, 7):
            f = np.float32(2.0 ** k)
            cls_k, q_k = oracle.classify_pair(s * f, e * f, a * f, b * f, c * f)
            assert cls_k == cls
            assert (q_k["u"], q_k["v"], q_k["t"], q_k["det_rel"]) == (q["u"], q["v"], q["t"], q["det_rel"])
            assert q_k["dist"] == (q["dist"] * 2.0 ** k if q["dist"] >= 0 else q["dist"])
    assert n_par > 500


def _point_triangle_distance_qp(p, a, b, c):
    """|p - closest point of the triangle|, by minimising |a + u e1 + v e2 - p|
    over u, v >= 0, u + v <= 1: the unconstrained minimiser (2x2 normal
    equations) if feasible, else the best of the three clamped edges."""
    e1, e2, r = b - a, c - a, p - a
    G = np.array([[e1 @ e1, e1 @ e2], [e1 @ e2, e2 @ e2]])
    u, v = np.linalg.solve(G, [e1 @ r, e2 @ r])
    if u >= 0 and v >= 0 and u + v <= 1:
        return np.linalg.norm(a + u * e1 + v * e2 - p)
    best = np.inf
    for x, y in ((a, b), (b, c), (c, a)):
        g = y - x
        tt = min(max((p - x) @ g / (g @ g), 0.0), 1.0)
        best = min(best, np.linalg.norm(x + tt * g - p))
    return best


def _segment_triangle_distance_search(s, e, a, b, c):
    """Minimum over the segment of the point-triangle distance, a convex
    function of the segment parameter: golden-section search."""
    f = lambda x: _point_triangle_distance_qp(s + x * (e - s), a, b, c)
    lo, hi = 0.0, 1.0
    g = (np.sqrt(5) - 1) / 2
    x1, x2 = hi - g * (hi - lo), lo + g * (hi - lo)
    f1, f2 = f(x1), f(x2)
    for _ in range(90):
        if f1 < f2:
            hi, x2, f2 = x2, x1, f1
            x1 = hi - g * (hi - lo)
            f1 = f(x1)
        else:
            lo, x1, f1 = x1, x2, f2
            x2 = lo + g * (hi - lo)
            f2 = f(x2)
    return min(f1, f2, f(0.0), f(1.0))


def test_parallel_branch_distance_brute_force():
    """On the nearly-parallel branch the oracle's distance (end points
    against the face, the segment against the three edges) equals a direct
    minimisation of the point-triangle distance along the segment."""
    rng = np.random.default_rng(23)
    checked = 0
    for s, e, a, b, c in _nearly_parallel_pairs(rng, 600):
        cls, q = oracle.classify_pair(s, e, a, b, c)
        if q["dist"] < 0 or q["incl"]:
            continue
        P = [x.astype(np.float64) for x in (s, e, a, b, c)]
        ref = _segment_triangle_distance_search(*P)
        L = np.linalg.norm(P[1] - P[0])
        assert abs(q["dist"] - ref) <= 1e-10 * L + 1e-9 * ref
        checked += 1
    assert checked > 200


def test_decisive_hit_settles_boolean_mode():
    """Boolean mode needs one hit: a decisive crossing of one plate settles
    the answer although the segment also runs through an edge of another
    (not ambiguous), while intercept_count is ambiguous on that ray and
    counts both crossing points.  Without the decisive plate the boolean
    answer rests on the edge alone and is ambiguous."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0],
                  [0.25, 0, 0.5], [1, 0, 0.5], [0.25, 1, 0.5]], np.float32)
    T = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    F, E = [[0.25, 0.25, -1.0]], [[0.25, 0.25, 1.0]]
    r = oracle.query(V, T, F, E)
    assert (r["hit"][0], r["amb_hit"][0], r["amb_count"][0], r["count"][0]) == (1, 0, 1, 2)
    assert r["near_tri"][0] == 0 and r["near_t"][0] == 0.5
    r = oracle.query(V, T[1:], F, E)
    assert (r["hit"][0], r["amb_hit"][0], r["amb_count"][0], r["count"][0]) == (1, 1, 1, 1)


# ------------------------------------------------------------ surface extent
def test_extent_equals_library_minmax():
    """Per-axis minimum and maximum over all vertices (Sec. 3.3), against
    numpy's reductions, including one vertex, all-negative coordinates and
    the extreme vertex first or last."""
    rng = np.random.default_rng(9)
    cases = [rng.uniform(-5, 5, (100, 3)), rng.uniform(-9, -1, (50, 3)), rng.uniform(1, 9, (50, 3)),
             np.array([[3.0, -2.0, 7.0]])]
    sorted_desc = np.sort(rng.uniform(-1, 1, (20, 3)), axis=0)[::-1]
    cases += [sorted_desc, sorted_desc[::-1].copy()]
    for V in cases:
        V = V.astype(np.float32)
        lo, hi = oracle.extent(V)
        assert lo.tolist() == V.min(0).tolist() and hi.tolist() == V.max(0).tolist()
    with pytest.raises(ValueError):
        oracle.extent(np.array([[0, 0, 0], [np.nan, 1, 1]], np.float32))
