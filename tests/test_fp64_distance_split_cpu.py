"""The definition's segment-to-triangle distance, as the warp-wide FP64 kernel
splits it over lanes, equals the serial evaluation term for term.

The FP64 classification of an undecided pair (Epilogue: the definition in
double precision) needs, for a nearly parallel pair, the distance from the
segment to the triangle: the smallest of the two end points' distances to
the triangle and the three edge-to-segment distances.  The warp form
evaluates the distinct terms side by side -- the nine point-to-segment
distances (end points to edges, vertices to the segment), the three
interior closest approaches of the segment and an edge, and the two end
points' plane distances where their projections fall inside -- and takes
their minimum.  This restates both forms in plain double-precision Python
(the same operations in the same order, no fused multiply-adds) and checks
that they agree bit for bit on random, nearly parallel and touching pairs:
a dropped or duplicated term, or a wrong end point or edge, fails it."""
import math
import random


def sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def add(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def scale(a, t):
    return (a[0] * t, a[1] * t, a[2] * t)


def dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def norm(a):
    return math.sqrt(dot(a, a))


def clamp01(x):
    return 0.0 if x < 0.0 else (1.0 if x > 1.0 else x)


def pt_seg(p, a, b):
    ab = sub(b, a)
    len2 = dot(ab, ab)
    t = clamp01(dot(sub(p, a), ab) / len2) if len2 > 0.0 else 0.0
    return norm(sub(p, add(a, scale(ab, t))))


def interior(p0, p1, q0, q1):
    """The closest approach of two segments strictly by their interiors, or None."""
    u, v, w0 = sub(p1, p0), sub(q1, q0), sub(p0, q0)
    a, b, c = dot(u, u), dot(u, v), dot(v, v)
    d, e = dot(u, w0), dot(v, w0)
    den = a * c - b * b
    if den > 0.0:
        s = (b * e - c * d) / den
        t = (a * e - b * d) / den
        if 0.0 <= s <= 1.0 and 0.0 <= t <= 1.0:
            return norm(sub(add(w0, scale(u, s)), scale(v, t)))
    return None


def seg_seg(p0, p1, q0, q1):
    best = pt_seg(p0, q0, q1)
    for d in (pt_seg(p1, q0, q1), pt_seg(q0, p0, p1), pt_seg(q1, p0, p1)):
        if d < best:
            best = d
    d = interior(p0, p1, q0, q1)
    if d is not None and d < best:
        best = d
    return best


def plane_part(p, a, b, c):
    """The distance to the triangle's plane when the projection of p falls inside, else None."""
    n = cross(sub(b, a), sub(c, a))
    nn = dot(n, n)
    h = dot(sub(p, a), n) / nn
    proj = sub(p, scale(n, h))
    s0 = dot(cross(sub(b, a), sub(proj, a)), n)
    s1 = dot(cross(sub(c, b), sub(proj, b)), n)
    s2 = dot(cross(sub(a, c), sub(proj, c)), n)
    if s0 >= 0.0 and s1 >= 0.0 and s2 >= 0.0:
        return abs(h) * math.sqrt(nn)
    return None


def pt_tri(p, a, b, c):
    d = plane_part(p, a, b, c)
    if d is not None:
        return d
    best = pt_seg(p, a, b)
    for e in (pt_seg(p, b, c), pt_seg(p, c, a)):
        if e < best:
            best = e
    return best


def serial_distance(s, e, a, b, c):
    best = pt_tri(s, a, b, c)
    for d in (pt_tri(e, a, b, c), seg_seg(s, e, a, b), seg_seg(s, e, b, c), seg_seg(s, e, c, a)):
        if d < best:
            best = d
    return best


def split_distance(s, e, a, b, c):
    edges = ((a, b), (b, c), (c, a))
    terms = [pt_seg(p, q0, q1) for p in (s, e) for q0, q1 in edges]
    terms += [pt_seg(v, s, e) for v in (a, b, c)]
    terms += [interior(s, e, q0, q1) for q0, q1 in edges]
    terms += [plane_part(p, a, b, c) for p in (s, e)]
    return min(t for t in terms if t is not None)


def _pairs(seed, count):
    rng = random.Random(seed)
    out = []
    for i in range(count):
        a = tuple(rng.uniform(-1, 1) for _ in range(3))
        b = tuple(rng.uniform(-1, 1) for _ in range(3))
        c = tuple(rng.uniform(-1, 1) for _ in range(3))
        kind = i % 4
        if kind == 0:     # anywhere
            s = tuple(rng.uniform(-2, 2) for _ in range(3))
            e = tuple(rng.uniform(-2, 2) for _ in range(3))
        else:             # in or near the triangle's plane (nearly parallel)
            n = cross(sub(b, a), sub(c, a))
            nl = norm(n)
            off = 0.0 if kind == 1 else rng.uniform(-1e-7, 1e-7) * (10.0 ** rng.randint(0, 6))
            def in_plane():
                u, v = rng.uniform(-0.5, 1.5), rng.uniform(-0.5, 1.5)
                q = add(a, add(scale(sub(b, a), u), scale(sub(c, a), v)))
                return add(q, scale(n, off / nl))
            s, e = in_plane(), in_plane()
            if kind == 3:   # one end on an edge or a vertex
                s = rng.choice((a, b, c, scale(add(a, b), 0.5)))
        out.append((s, e, a, b, c))
    return out


def test_split_distance_equals_serial_bit_for_bit():
    for s, e, a, b, c in _pairs(2305, 4000):
        if norm(cross(sub(b, a), sub(c, a))) == 0.0 or s == e:
            continue
        d1, d2 = serial_distance(s, e, a, b, c), split_distance(s, e, a, b, c)
        assert d1 == d2, (s, e, a, b, c, d1, d2)


def test_split_distance_catches_a_missing_term():
    """Dropping the vertex-to-segment terms changes the minimum on some pair:
    the split test above is sensitive to the set of terms."""
    def without_vertices(s, e, a, b, c):
        edges = ((a, b), (b, c), (c, a))
        terms = [pt_seg(p, q0, q1) for p in (s, e) for q0, q1 in edges]
        terms += [interior(s, e, q0, q1) for q0, q1 in edges]
        terms += [plane_part(p, a, b, c) for p in (s, e)]
        return min(t for t in terms if t is not None)
    differ = sum(serial_distance(*p) != without_vertices(*p) for p in _pairs(7, 4000)
                 if norm(cross(sub(p[3], p[2]), sub(p[4], p[2]))) > 0.0 and p[0] != p[1])
    assert differ > 0
