"""The certified double-float finishing pass of the barycentric mode, checked
on the CPU against the oracle (no GPU).

For a hitting segment the pass computes t = T / det, the point s + t d and
the distance t |d| (Sec. 1, barycentric mode) as pairs of FP32 numbers
(Knuth's two-sum, Dekker's fast two-sum, FMA products), together with a
bound on their distance from the FP64 evaluation of the definition.  When no
FP32 rounding boundary lies within that bound it writes the FP32 roundings
directly; otherwise the segment goes to the FP64 kernel.  The claim: every
result it certifies equals the FP32 rounding of the FP64 value -- the
oracle's.  The pass's operations are restated here in numpy float32 (a fused
multiply-add emulated exactly from float64 with a two-sum error term) and
run over hitting segments of many scales, positions and angles.
"""
import numpy as np
import pytest

import oracle

F32, F64 = np.float32, np.float64


# ------------------------------------------------------------ float32 primitives
def _fma(a, b, c):
    """a * b + c rounded once to float32 (ties to even)."""
    p = a.astype(F64) * b.astype(F64)            # exact: 24 + 24 bits
    c64 = c.astype(F64)
    s = p + c64
    bb = s - p
    err = (p - (s - bb)) + (c64 - bb)            # s + err == p + c exactly
    r = s.astype(F32)
    r64 = r.astype(F64)
    lo = np.where(r64 > s, np.nextafter(r, F32(-np.inf)), r)
    hi = np.where(r64 < s, np.nextafter(r, F32(np.inf)), r)
    mid = (r64 != s) & ((lo.astype(F64) + hi.astype(F64)) / 2 == s)
    # s is a midpoint of two float32 numbers: the sign of err decides
    return np.where(mid & (err > 0), hi, np.where(mid & (err < 0), lo, r))


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _fast(a, b):
    s = a + b
    return s, b - (s - a)


def _add(x, y):
    sh, sl = _two_sum(x[0], y[0])
    return _fast(sh, sl + (x[1] + y[1]))


def _neg(x):
    return -x[0], -x[1]


def _mul(x, y):
    p = x[0] * y[0]
    e = _fma(x[0], y[0], -p)
    e = _fma(x[0], y[1], e)
    e = _fma(x[1], y[0], e)
    return _fast(p, e)


def _div(x, y):
    q1 = x[0] / y[0]
    r = _add(x, _neg(_mul((q1, np.zeros_like(q1)), y)))
    return _fast(q1, r[0] / y[0])


def _sqrt(x):
    s = np.sqrt(x[0])
    z = np.zeros_like(s)
    r = _add(x, _neg(_mul((s, z), (s, z))))
    return _fast(s, r[0] / (F32(2) * s))


def _diff(a, b):
    return _two_sum(a, -b)


def _round_certain(v, r):
    """(certified, value): v[0] when every real within r of v rounds to it."""
    h = np.abs(v[0])
    ok = (h >= F32(1.17549435e-38)) & (h < F32(1e30))
    gap = np.minimum(np.nextafter(h, F32(np.inf)) - h, h - np.nextafter(h, F32(0)))
    bound = np.abs(v[1]).astype(F64) + r.astype(F64)
    bound32 = bound.astype(F32)
    bound32 = np.where(bound32.astype(F64) < bound, np.nextafter(bound32, F32(np.inf)), bound32)   # rounded up
    return ok & (bound32 < F32(0.5) * gap), v[0]


def nearest_ff(s, e, a, b, c):
    """Certified flag and (t, px, py, pz, dist) per segment, as the pass computes them."""
    d = [_diff(e[:, k], s[:, k]) for k in range(3)]
    e1 = [_diff(b[:, k], a[:, k]) for k in range(3)]
    e2 = [_diff(c[:, k], a[:, k]) for k in range(3)]
    sv = [_diff(s[:, k], a[:, k]) for k in range(3)]
    cr = lambda x, y, i, j: _add(_mul(x[i], y[j]), _neg(_mul(x[j], y[i])))
    p = [cr(d, e2, 1, 2), cr(d, e2, 2, 0), cr(d, e2, 0, 1)]
    det = _add(_add(_mul(e1[0], p[0]), _mul(e1[1], p[1])), _mul(e1[2], p[2]))
    q = [cr(sv, e1, 1, 2), cr(sv, e1, 2, 0), cr(sv, e1, 0, 1)]
    T = _add(_add(_mul(e2[0], q[0]), _mul(e2[1], q[1])), _mul(e2[2], q[2]))
    ad, a1, a2, asv = ([np.abs(v[k][0]) for k in range(3)] for v in (d, e1, e2, sv))
    Md = F32(1.001) * (a1[0] * (ad[1] * a2[2] + ad[2] * a2[1]) + a1[1] * (ad[2] * a2[0] + ad[0] * a2[2])
                       + a1[2] * (ad[0] * a2[1] + ad[1] * a2[0]))
    MT = F32(1.001) * (a2[0] * (asv[1] * a1[2] + asv[2] * a1[1]) + a2[1] * (asv[2] * a1[0] + asv[0] * a1[2])
                       + a2[2] * (asv[0] * a1[1] + asv[1] * a1[0]))
    cu = F32(8.0) * F32(1.1102230e-16) + F32(9.0949470e-13)
    D = np.abs(det[0])
    ok = cu * Md < F32(0.01) * D
    t = _div(T, det)
    at = np.abs(t[0])
    rt = F32(1.02) * (cu * (MT + at * Md) / D + (F32(1.1102230e-16) + F32(9.0949470e-13)) * at)
    pts = [_add((s[:, k], np.zeros_like(at)), _mul(d[k], t)) for k in range(3)]
    nrm = _sqrt(_add(_add(_mul(d[0], d[0]), _mul(d[1], d[1])), _mul(d[2], d[2])))
    dist = _mul(t, nrm)
    cp = F32(1.8189894e-12)
    rp = [F32(1.02) * (ad[k] * rt + cp * (np.abs(s[:, k]) + ad[k] * at)) for k in range(3)]
    rd = F32(1.02) * (np.abs(nrm[0]) * rt + cp * np.abs(dist[0]))
    outs = [_round_certain(t, rt)] + [_round_certain(pts[k], rp[k]) for k in range(3)] + [_round_certain(dist, rd)]
    cert = ok.copy()
    for c_, _ in outs:
        cert &= c_
    return cert, np.stack([v for _, v in outs], 1)


# ------------------------------------------------------------ hitting segments
def _hitting_pairs(rng, n):
    """Triangles of size 10^-2..10^3 placed up to 10^3 from the origin;
    segments through an interior point at t in (0.02, 0.98), at any angle,
    a sixth of them within 10^-5..10^-2 rad of the plane."""
    S, E, A, B, C = [], [], [], [], []
    while len(S) < n:
        scale = 10.0 ** rng.uniform(-2, 3)
        off = rng.normal(size=3) * 10.0 ** rng.uniform(0, 3)
        a = off + scale * rng.uniform(-1, 1, 3)
        b = a + scale * rng.uniform(-1, 1, 3)
        c = a + scale * rng.uniform(-1, 1, 3)
        nrm = np.cross(b - a, c - a)
        if np.linalg.norm(nrm) < 1e-2 * scale * scale:
            continue
        nrm /= np.linalg.norm(nrm)
        w = rng.dirichlet([2, 2, 2])
        p = w[0] * a + w[1] * b + w[2] * c
        if rng.uniform() < 1 / 6:
            u = np.cross(nrm, rng.normal(size=3))
            u /= np.linalg.norm(u)
            dvec = u + 10.0 ** rng.uniform(-5, -2) * nrm
        else:
            dvec = rng.normal(size=3)
        dvec /= np.linalg.norm(dvec)
        L = scale * 10.0 ** rng.uniform(-1, 1)
        t = rng.uniform(0.02, 0.98)
        for lst, v in zip((S, E, A, B, C), (p - t * L * dvec, p + (1 - t) * L * dvec, a, b, c)):
            lst.append(v.astype(F32))
    return [np.stack(x) for x in (S, E, A, B, C)]


@pytest.fixture(scope="module")
def finished():
    rng = np.random.default_rng(41)
    S, E, A, B, C = _hitting_pairs(rng, 12000)
    ref = np.full((len(S), 5), np.nan, F32)
    hit = np.zeros(len(S), bool)
    for i in range(len(S)):
        r = oracle.query(np.stack([A[i], B[i], C[i]]), [[0, 1, 2]], S[i:i + 1], E[i:i + 1], nthreads=1)
        if r["near_tri"][0] == 0:
            hit[i] = True
            ref[i] = [r["near_t"][0], *r["near_point"][0], r["near_dist"][0]]
    with np.errstate(all="ignore"):
        cert, val = nearest_ff(S, E, A, B, C)
    return hit, ref, cert, val


def test_certified_results_equal_the_fp64_roundings(finished):
    """(Without the certificate's radius, about 1 in 1,500 of these results
    would be certified wrongly.)"""
    hit, ref, cert, val = finished
    sel = hit & cert
    assert np.array_equal(val[sel].view(np.uint32), ref[sel].view(np.uint32))


def test_most_hits_are_certified(finished):
    """Only hits near a rounding boundary or at a grazing angle are left to
    the FP64 kernel."""
    hit, _, cert, _ = finished
    assert hit.sum() > 11000
    assert cert[hit].mean() > 0.85
