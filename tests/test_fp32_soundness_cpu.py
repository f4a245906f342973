"""The two arguments that make the FP32 traversal exact, checked on the CPU
against the oracle (no GPU).

1. Culling: a (segment, triangle) pair that is a hit or ambiguous in the FP64
   definition is never pruned.  Its segment, extended to t in [-tau, 1 + tau],
   meets the triangle's box widened per axis by tau |d|_1 + 2 tau D_axis
   (D_axis the box side): at a non-parallel pair the plane point has
   barycentric weights >= -tau; at a parallel one some point of the segment
   lies within tau |d| of the triangle.  The traversal pads node boxes by
   4 tau (|d|_1 + D_max,axis) and rounds outward, so it keeps every such box.
2. Certainty: the FP32 Moller-Trumbore test (Sec. 1) decides on numerators
   with forward error bounds (16 u times the same expression in magnitudes);
   a pair it calls a certain hit or a certain miss has that class in FP64.

3. The FP64 re-test first tries the same numerator test in double precision
   (bound 32 u, tau widened by 1e-9 relative); its certain answers must be
   the class the definition's own FP64 evaluation gives.

The formulas are restated here in numpy float32 / float64 -- each dot and
cross product in two evaluation orders, plain and with fused multiply-adds,
since the compiler may contract either way -- and run over near-boundary,
nearly-parallel and near-threshold pairs whose class the oracle gives.
"""
import numpy as np
import pytest

import oracle
from test_oracle_pins import _near_boundary_pairs, _nearly_parallel_pairs

MISS, HIT, AMB = oracle.PAIR_MISS, oracle.PAIR_HIT, oracle.PAIR_AMBIGUOUS
BAND = 2
TAU = 1e-6

F32, F64 = np.float32, np.float64
kU = F32(2.0 ** -24)
kErrK = F32(16.0) * kU
kTauHi = F32(1.000001e-6)
kSlabGrow = F32(1.000002)


# ------------------------------------------------------------ float32 restatement
def _fma(a, b, c):
    """Single-rounded a * b + c (the product is exact in float64)."""
    return (a.astype(F64) * b.astype(F64) + c.astype(F64)).astype(F32)


def _dot(a, b, fused):
    if fused:
        return _fma(a[:, 2], b[:, 2], _fma(a[:, 1], b[:, 1], a[:, 0] * b[:, 0]))
    return (a[:, 0] * b[:, 0] + a[:, 1] * b[:, 1]) + a[:, 2] * b[:, 2]


def _cross(a, b, fused, sign=-1):
    """a x b (sign -1), or the same products added (sign +1: the magnitude bound)."""
    out = np.empty_like(a)
    for k, (i, j) in enumerate(((1, 2), (2, 0), (0, 1))):
        if fused:
            out[:, k] = _fma(a[:, i], b[:, j], F32(sign) * (a[:, j] * b[:, i]))
        else:
            out[:, k] = a[:, i] * b[:, j] + F32(sign) * (a[:, j] * b[:, i])
    return out


def tri_fp32(s, e, a, b, c, fused):
    """Certain hit / certain miss / band of each pair, as the traversal decides."""
    d, e1, e2, sv = e - s, b - a, c - a, s - a
    p = _cross(d, e2, fused)
    det = _dot(e1, p, fused)
    q = _cross(sv, e1, fused)
    T = _dot(e2, q, fused)
    ad, ae1, ae2, asv = np.abs(d), np.abs(e1), np.abs(e2), np.abs(sv)
    pa, qa = _cross(ad, ae2, fused, +1), _cross(asv, ae1, fused, +1)
    errdet = kErrK * _dot(ae1, pa, fused) + F32(1e-35)
    errT = kErrK * _dot(ae2, qa, fused) + F32(1e-35)
    dl1 = (ad[:, 0] + ad[:, 1]) + ad[:, 2]
    n1 = lambda x: (x[:, 0] + x[:, 1]) + x[:, 2]
    thr = ((kTauHi * (dl1 * n1(ae1))) * n1(ae2)) * F32(1.000001)
    Tm = T - det
    errTm = (errT + errdet) + F32(2.0) * kU * (np.abs(T) + np.abs(det))
    U, V = _dot(sv, p, fused), _dot(d, q, fused)
    miss0 = ((T > 0) == (Tm > 0)) & (np.minimum(np.abs(T) - errT, np.abs(Tm) - errTm) > thr)
    D = np.abs(det)
    sure = D - errdet > thr
    sg = np.where(det > 0, F32(1), F32(-1))
    errU = kErrK * _dot(asv, pa, fused) + F32(1e-35)
    errV = kErrK * _dot(ad, qa, fused) + F32(1e-35)
    Us, Vs, Ts = sg * U, sg * V, sg * T
    Ws = (D - Us) - Vs
    errW = ((errdet + errU) + errV) + F32(2.0) * kU * ((D + np.abs(U)) + np.abs(V))
    Tms = D - Ts
    lim = kTauHi * (D + errdet) * F32(1.000001)
    hit = sure & (Us - errU > lim) & (Vs - errV > lim) & (Ws - errW > lim) & (Ts - errT > lim) & (Tms - errTm > lim)
    miss1 = sure & ((Us + errU < -lim) | (Vs + errV < -lim) | (Ws + errW < -lim) | (Ts + errT < -lim)
                    | (Tms + errTm < -lim))
    return np.where(miss0, MISS, np.where(hit, HIT, np.where(miss1, MISS, BAND)))


def tri_certain_hit(s, e, a, b, c, fused):
    """The verification's certain-hit test: the numerators' signs first,
    then the same bounds as tri_fp32's hit branch."""
    d, e1, e2, sv = e - s, b - a, c - a, s - a
    p = _cross(d, e2, fused)
    det = _dot(e1, p, fused)
    q = _cross(sv, e1, fused)
    T = _dot(e2, q, fused)
    U, V = _dot(sv, p, fused), _dot(d, q, fused)
    D = np.abs(det)
    sg = np.where(det > 0, F32(1), F32(-1))
    Us, Vs, Ts = sg * U, sg * V, sg * T
    Ws = (D - Us) - Vs
    Tms = D - Ts
    signs = (Us > 0) & (Vs > 0) & (Ws > 0) & (Ts > 0) & (Tms > 0)
    ad, ae1, ae2, asv = np.abs(d), np.abs(e1), np.abs(e2), np.abs(sv)
    pa, qa = _cross(ad, ae2, fused, +1), _cross(asv, ae1, fused, +1)
    errdet = kErrK * _dot(ae1, pa, fused) + F32(1e-35)
    n1 = lambda x: (x[:, 0] + x[:, 1]) + x[:, 2]
    dl1 = (ad[:, 0] + ad[:, 1]) + ad[:, 2]
    thr = ((kTauHi * (dl1 * n1(ae1))) * n1(ae2)) * F32(1.000001)
    sure = D - errdet > thr
    errT = kErrK * _dot(ae2, qa, fused) + F32(1e-35)
    errTm = (errT + errdet) + F32(2.0) * kU * (np.abs(T) + np.abs(det))
    errU = kErrK * _dot(asv, pa, fused) + F32(1e-35)
    errV = kErrK * _dot(ad, qa, fused) + F32(1e-35)
    errW = ((errdet + errU) + errV) + F32(2.0) * kU * ((D + np.abs(U)) + np.abs(V))
    lim = kTauHi * (D + errdet) * F32(1.000001)
    return signs & sure & (Us - errU > lim) & (Vs - errV > lim) & (Ws - errW > lim) & (Ts - errT > lim) & (
        Tms - errTm > lim)


def _round_dir(exact, up):
    """float32 rounding of a float64 value toward +inf (up) or -inf."""
    r = exact.astype(F32)
    if up:
        return np.where(r.astype(F64) < exact, np.nextafter(r, F32(np.inf)), r)
    return np.where(r.astype(F64) > exact, np.nextafter(r, F32(-np.inf)), r)


def slab_pass(s, e, lo, hi, dmax):
    """The traversal's padded slab test of one box per segment (no sum is
    left for the compiler to contract: the planes are single FMAs and the
    interval test one product)."""
    d = e - s
    inv = np.where(np.abs(d) < F32(1e-20), np.copysign(F32(1e20), d), F32(1) / np.where(d == 0, F32(1), d))
    dl1 = (np.abs(d[:, 0]) + np.abs(d[:, 1])) + np.abs(d[:, 2])
    k = F32(4.0) * kTauHi
    pad = _round_dir(k.astype(F64) * _round_dir(dl1[:, None].astype(F64) + dmax.astype(F64), True).astype(F64), True)
    slo = _round_dir(s.astype(F64) + pad.astype(F64), True)
    shi = _round_dir(s.astype(F64) - pad.astype(F64), False)
    # one FMA per plane with offsets rounded toward the conservative side:
    # down for the entry plane (lower plane when inv >= 0), up for the exit one
    pos = inv >= 0
    plo = -slo.astype(F64) * inv.astype(F64)          # exact products in float64
    phi = -shi.astype(F64) * inv.astype(F64)
    olo = np.where(pos, _round_dir(plo, False), _round_dir(plo, True))
    ohi = np.where(pos, _round_dir(phi, True), _round_dir(phi, False))
    t0, t1 = _fma(lo, inv, olo), _fma(hi, inv, ohi)
    # the segment's part [0, 1] meets the box when max(tn, 0) <= min(tf, 1) x grow
    tn = np.maximum(np.minimum(t0, t1).max(axis=1), F32(0))
    tf = np.minimum(np.maximum(t0, t1).min(axis=1), F32(1))
    return tn <= tf * kSlabGrow


# ------------------------------------------------------------ float64 restatement
def _two_prod(a, b):
    """a * b = p + e exactly (Dekker's splitting)."""
    p = a * b
    sp = 134217729.0                          # 2^27 + 1
    ah = a * sp - (a * sp - a)
    al = a - ah
    bh = b * sp - (b * sp - b)
    bl = b - bh
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _fma64(a, b, c):
    """a * b + c with one final rounding (up to rare double roundings)."""
    p, pe = _two_prod(a, b)
    s = p + c
    bb = s - p
    se = (p - (s - bb)) + (c - bb)
    return s + (se + pe)


def tri_certain64(s, e, a, b, c, fused):
    """The FP64 pass's certain test: the FP32 one in double precision with
    the bound 32 u (u = 2^-53) and tau widened by 1e-9 relative."""
    u, tau = 2.0 ** -53, TAU * (1 + 1e-9)
    K = 32 * u
    s, e, a, b, c = (x.astype(F64) for x in (s, e, a, b, c))
    d, e1, e2, sv = e - s, b - a, c - a, s - a

    def dot(x, y):
        if fused:
            return _fma64(x[:, 2], y[:, 2], _fma64(x[:, 1], y[:, 1], x[:, 0] * y[:, 0]))
        return x[:, 0] * y[:, 0] + x[:, 1] * y[:, 1] + x[:, 2] * y[:, 2]

    def cross(x, y, sign=-1.0):
        out = np.empty_like(x)
        for k, (i, j) in enumerate(((1, 2), (2, 0), (0, 1))):
            out[:, k] = _fma64(x[:, i], y[:, j], sign * (x[:, j] * y[:, i])) if fused else \
                x[:, i] * y[:, j] + sign * (x[:, j] * y[:, i])
        return out

    p, q = cross(d, e2), cross(sv, e1)
    det, T, U, V = dot(e1, p), dot(e2, q), dot(sv, p), dot(d, q)
    ad, a1, a2, asv = np.abs(d), np.abs(e1), np.abs(e2), np.abs(sv)
    pa, qa = cross(ad, a2, 1.0), cross(asv, a1, 1.0)
    errdet = K * dot(a1, pa) + 1e-300
    errT = K * dot(a2, qa) + 1e-300
    thr = tau * (ad.sum(1) * a1.sum(1)) * a2.sum(1)
    Tm = T - det
    errTm = errT + errdet + 4 * u * (np.abs(T) + np.abs(det))
    miss0 = ((T > 0) == (Tm > 0)) & (np.minimum(np.abs(T) - errT, np.abs(Tm) - errTm) > thr)
    D = np.abs(det)
    sure = D - errdet > thr
    sg = np.where(det > 0, 1.0, -1.0)
    errU, errV = K * dot(asv, pa) + 1e-300, K * dot(ad, qa) + 1e-300
    Us, Vs, Ts = sg * U, sg * V, sg * T
    Ws = D - Us - Vs
    errW = errdet + errU + errV + 4 * u * (D + np.abs(U) + np.abs(V))
    Tms = D - Ts
    lim = tau * (D + errdet)
    hit = sure & (Us - errU > lim) & (Vs - errV > lim) & (Ws - errW > lim) & (Ts - errT > lim) & (Tms - errTm > lim)
    miss1 = sure & ((Us + errU < -lim) | (Vs + errV < -lim) | (Ws + errW < -lim) | (Ts + errT < -lim)
                    | (Tms + errTm < -lim))
    return np.where(miss0, MISS, np.where(hit, HIT, np.where(miss1, MISS, BAND)))


# ------------------------------------------------------------ pairs
def _margin_pairs(rng, n):
    """Segments through a plane point with one barycentric weight, or t, within
    a few tau of a decision threshold (-tau, tau, 1 - tau, 1 + tau)."""
    out = []
    while len(out) < n:
        a = rng.uniform(-1, 1, 3)
        b, c = a + rng.uniform(-0.5, 0.5, 3), a + rng.uniform(-0.5, 0.5, 3)
        nrm = np.cross(b - a, c - a)
        if np.linalg.norm(nrm) < 1e-3:
            continue
        w3 = rng.dirichlet([1, 1, 1])
        k = rng.integers(0, 3)
        w3[k] = rng.choice([-1, 1]) * TAU * rng.uniform(0.25, 3.0)
        w3[(k + 1) % 3] = 1 - w3[k] - w3[(k + 2) % 3]
        p = w3[0] * a + w3[1] * b + w3[2] * c
        dvec = rng.normal(size=3)
        dvec /= np.linalg.norm(dvec)
        L = 10.0 ** rng.uniform(-2, 0.5)
        t = rng.choice([rng.uniform(0.1, 0.9), TAU * rng.uniform(-3, 3), 1 + TAU * rng.uniform(-3, 3)])
        out.append([x.astype(F32) for x in (p - t * L * dvec, p + (1 - t) * L * dvec, a, b, c)])
    return out


@pytest.fixture(scope="module")
def pairs():
    rng = np.random.default_rng(31)
    P = _near_boundary_pairs(rng, 8000) + _nearly_parallel_pairs(rng, 6000) + _margin_pairs(rng, 12000)
    res = [oracle.classify_pair(*x) for x in P]
    cls = np.array([r[0] for r in res])
    S, E, A, B, C = (np.stack([x[i] for x in P]) for i in range(5))
    det_rel = np.array([abs(r[1]["det_rel"]) for r in res])
    return S, E, A, B, C, cls, det_rel


@pytest.mark.parametrize("fused", [False, True])
def test_certain_fp32_decisions_are_fp64_decisions(pairs, fused):
    S, E, A, B, C, cls, det_rel = pairs
    with np.errstate(all="ignore"):
        got = tri_fp32(S, E, A, B, C, fused)
    assert np.all(cls[got == HIT] == HIT)
    assert np.all(cls[got == MISS] == MISS)
    # every ambiguous pair lands in the band; the pairs are built to sit near
    # the thresholds, yet thousands are still decided in FP32
    assert np.all(got[cls == AMB] == BAND)
    assert (got == HIT).sum() > 1000 and (got == MISS).sum() > 1000


@pytest.mark.parametrize("fused", [False, True])
def test_verification_hits_are_the_traversals_certain_hits(pairs, fused):
    """The learned query's verification test (sign test first) confirms
    exactly the pairs the traversal's test calls certain hits, so every
    hit it confirms is a decisive hit of the definition."""
    S, E, A, B, C, cls, det_rel = pairs
    with np.errstate(all="ignore"):
        full = tri_fp32(S, E, A, B, C, fused)
        quick = tri_certain_hit(S, E, A, B, C, fused)
    assert np.array_equal(quick, full == HIT)
    assert np.all(cls[quick] == HIT) and quick.sum() > 1000


def test_hit_or_ambiguous_pairs_meet_the_widened_box(pairs):
    """Argument 1 in FP64: the extended segment meets the triangle's box
    widened by tau |d|_1 + 2 tau D per axis."""
    S, E, A, B, C, cls, det_rel = pairs
    keep = cls != MISS
    s, e = S[keep].astype(F64), E[keep].astype(F64)
    V = np.stack([A[keep], B[keep], C[keep]], 1).astype(F64)
    lo, hi = V.min(1), V.max(1)
    d = e - s
    pad = TAU * np.abs(d).sum(1, keepdims=True) + 2 * TAU * (hi - lo)
    lo, hi = lo - pad, hi + pad
    with np.errstate(all="ignore"):
        t0 = np.where(d != 0, (lo - s) / d, np.where((s >= lo) & (s <= hi), -np.inf, np.inf))
        t1 = np.where(d != 0, (hi - s) / d, np.where((s >= lo) & (s <= hi), np.inf, -np.inf))
    tn = np.maximum(np.minimum(t0, t1).max(1), -TAU)
    tf = np.minimum(np.maximum(t0, t1).min(1), 1 + TAU)
    assert np.all(tn <= tf + 1e-12 * (1 + np.abs(tf)))
    assert keep.sum() > 2000


def test_traversal_slab_keeps_every_hit_or_ambiguous_pair(pairs):
    """Argument 1 as the traversal computes it in FP32, with the box of the
    triangle alone and its own box sides as D_max (the tightest padding any
    node of a hierarchy can get)."""
    S, E, A, B, C, cls, det_rel = pairs
    keep = cls != MISS
    V = np.stack([A[keep], B[keep], C[keep]], 1)
    lo, hi = V.min(1), V.max(1)
    with np.errstate(all="ignore"):
        ok = slab_pass(S[keep], E[keep], lo, hi, hi - lo)
    assert ok.all(), np.flatnonzero(~ok)[:10]
    # and the test does prune: most decisive misses' boxes are rejected
    miss = cls == MISS
    Vm = np.stack([A[miss], B[miss], C[miss]], 1)
    with np.errstate(all="ignore"):
        pruned = ~slab_pass(S[miss], E[miss], Vm.min(1), Vm.max(1), Vm.max(1) - Vm.min(1))
    assert pruned.sum() > 0


@pytest.mark.parametrize("fused", [False, True])
def test_certain_fp64_decisions_are_the_definitions(pairs, fused):
    """The FP64 pass decides most queued pairs without square roots or
    divisions; each certain decision must be the class the definition's own
    FP64 evaluation gives (the oracle's).  Of the decisive pairs clear of
    the parallel branch (|det_rel| > 2 tau), it leaves almost none to the
    definition, where the FP32 test leaves half of these adversarial pairs."""
    S, E, A, B, C, cls, det_rel = pairs
    with np.errstate(all="ignore"):
        got = tri_certain64(S, E, A, B, C, fused)
    assert np.all(cls[got == HIT] == HIT)
    assert np.all(cls[got == MISS] == MISS)
    assert np.all(got[cls == AMB] == BAND)
    clear = (cls != AMB) & (det_rel > 2 * TAU)
    assert clear.sum() > 10000 and (got[clear] == BAND).sum() < 0.001 * clear.sum()


def _padded_slab_exact(s, e, lo, hi, pad):
    """Does the segment meet the padded box [lo - pad, hi + pad]?  Float64
    slab arithmetic on the float32 inputs (a reference far finer than the
    float32 test's own rounding)."""
    s, e = s.astype(F64), e.astype(F64)
    d = e - s
    blo, bhi = lo.astype(F64) - pad.astype(F64), hi.astype(F64) + pad.astype(F64)
    with np.errstate(all="ignore"):
        inside = (s >= blo) & (s <= bhi)
        t0 = np.where(d != 0, (blo - s) / d, np.where(inside, -np.inf, np.inf))
        t1 = np.where(d != 0, (bhi - s) / d, np.where(inside, np.inf, -np.inf))
    tn = np.minimum(t0, t1).max(1)
    tf = np.maximum(t0, t1).min(1)
    return (tn <= tf) & (tn <= 1.0) & (tf >= 0.0)


def test_slab_accepts_every_box_the_segment_touches():
    """The traversal's FP32 slab test (one FMA per plane, offsets rounded
    toward the conservative side, interval grown by 2e-6) never rejects a padded
    box the segment meets: boxes shrunk to a point on the segment and then
    pushed out by exactly the padding, so the segment grazes the padded box's
    faces, edges or corners; segments near and far from the origin, some
    nearly parallel to an axis."""
    rng = np.random.default_rng(17)
    n = 300_000
    scale = np.where(rng.uniform(size=(n, 1)) < 0.5, 1.0, 1e3)
    shift = np.where(rng.uniform(size=(n, 1)) < 0.3, rng.uniform(-5e3, 5e3, (n, 3)), 0.0)
    s = (rng.uniform(-1, 1, (n, 3)) * scale + shift).astype(F32)
    d = rng.normal(size=(n, 3)) * rng.uniform(0.05, 1.0, (n, 1)) * scale
    flat = rng.uniform(size=(n, 3)) < 0.1
    d = np.where(flat, d * rng.choice([0.0, 1e-9, 1e-5], size=(n, 3)), d)
    e = (s.astype(F64) + d).astype(F32)
    dmax = (rng.uniform(0, 0.05, (n, 3)) * scale).astype(F32)
    # the kernel's padding, rounded as it rounds it
    dd = e - s
    dl1 = (np.abs(dd[:, 0]) + np.abs(dd[:, 1])) + np.abs(dd[:, 2])
    k = F32(4.0) * kTauHi
    pad = _round_dir(k.astype(F64) * _round_dir(dl1[:, None].astype(F64) + dmax.astype(F64), True).astype(F64), True)
    t = rng.uniform(-2e-6, 1 + 2e-6, (n, 1))
    c = s.astype(F64) + t * (e.astype(F64) - s.astype(F64))
    sign = rng.choice([-1.0, 1.0], size=(n, 3))
    q = (c + sign * pad.astype(F64)).astype(F32)           # a point box whose padded cube touches c
    exact = _padded_slab_exact(s, e, q, q, pad)
    with np.errstate(all="ignore"):
        got = slab_pass(s, e, q, q, dmax)
    assert exact.sum() > n // 4
    assert np.all(got[exact]), int((exact & ~got).sum())
