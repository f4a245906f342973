// query.cu -- per-segment BVH search with Moller-Trumbore tests (Sec. 1:
// the tree yields candidate triangles, each tested with Moller-Trumbore;
// boolean and intercept_count modes), in two passes:
//
//  k_query_fp32  one lane per segment in a warp-coherent persistent loop:
//                stack traversal of the child-pair nodes with a padded,
//                outward-rounded slab test, and an FP32 Moller test that
//                carries a forward error bound.  Each pair comes out as a
//                certain decisive hit, a certain decisive miss, or "band"
//                (the FP32 value is too close to a decision boundary or to
//                the 1e-6 margin to be trusted, the Epilogue's concern).
//                Segments with a band pair and no certain answer are queued.
//  k_query_fp64  one warp per queued segment: re-traverses it, and classifies
//                the candidate pairs 32 at a time in FP64 with the outcome
//                the definition gives (decisive hit / decisive miss /
//                ambiguous, margin 1e-6).
//
// Culling never drops a pair that could be a hit or ambiguous: node boxes
// are padded by 4e-6 (|d|_1 + the largest triangle extent), which covers
// the margin band, and the slab interval is widened by 1e-6 relative, which
// covers FP32 rounding of the slab arithmetic.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "rsi_internal.cuh"

namespace rsi {

struct QueryArgs {
    const Node* nodes;
    const Tri* tris;
    int64_t n_tri;
    const float* from;
    const float* to;
    int64_t n_rays;
    uint8_t* hit;
    int32_t* count;
    uint8_t* amb;
    int32_t* band_ids;
    const int32_t* perm;   // traversal order of the segments, or NULL
    DevCounters* ctr;
    float dmax0, dmax1, dmax2;
    int fp32_only;
};

namespace {

constexpr float kU = 5.9604645e-8f;        // unit roundoff of FP32, 2^-24
constexpr float kErrK = 16.0f * kU;        // bound factor of a dot(cross) in FP32
constexpr float kTauHi = 1.000001e-6f;     // tau, rounded up
constexpr float kWiden = 1e-6f;            // relative widening of slab intervals

enum { kMiss = 0, kHit = 1, kBand = 2 };

struct SegF {
    float3 s, d, inv, slo, shi;   // slo = s + pad (up), shi = s - pad (down)
    float dl1;                    // |d|_1
};

__device__ __forceinline__ float safe_inv(float x) {
    return fabsf(x) < 1e-20f ? copysignf(1e20f, x) : 1.0f / x;
}

__device__ __forceinline__ SegF make_seg(float3 s, float3 e, float dmx, float dmy, float dmz) {
    SegF g;
    g.s = s;
    g.d = make_float3(e.x - s.x, e.y - s.y, e.z - s.z);
    g.inv = make_float3(safe_inv(g.d.x), safe_inv(g.d.y), safe_inv(g.d.z));
    g.dl1 = fabsf(g.d.x) + fabsf(g.d.y) + fabsf(g.d.z);
    const float k = 4.0f * kTauHi;
    float px = __fmul_ru(k, __fadd_ru(g.dl1, dmx));
    float py = __fmul_ru(k, __fadd_ru(g.dl1, dmy));
    float pz = __fmul_ru(k, __fadd_ru(g.dl1, dmz));
    g.slo = make_float3(__fadd_ru(s.x, px), __fadd_ru(s.y, py), __fadd_ru(s.z, pz));
    g.shi = make_float3(__fsub_rd(s.x, px), __fsub_rd(s.y, py), __fsub_rd(s.z, pz));
    return g;
}

// Does the segment pass through the padded box?  The padded slab [lo - pad,
// hi + pad] becomes parameters (lo - (s + pad)) / d and (hi - (s - pad)) / d
// with the shifted origins rounded outward; the interval is then widened.
__device__ __forceinline__ bool slab(const float4& bmin, const float4& bmax, const SegF& g) {
    float t0x = (bmin.x - g.slo.x) * g.inv.x, t1x = (bmax.x - g.shi.x) * g.inv.x;
    float t0y = (bmin.y - g.slo.y) * g.inv.y, t1y = (bmax.y - g.shi.y) * g.inv.y;
    float t0z = (bmin.z - g.slo.z) * g.inv.z, t1z = (bmax.z - g.shi.z) * g.inv.z;
    float tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fminf(t0z, t1z));
    float tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fmaxf(t0z, t1z));
    tn = tn - fabsf(tn) * kWiden;
    tf = tf + fabsf(tf) * kWiden;
    return tn <= tf && tn <= 1.0f && tf >= 0.0f;
}

__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 f3(const float4& v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 abs3(float3 a) { return make_float3(fabsf(a.x), fabsf(a.y), fabsf(a.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
// |a| x |b| with every product added: bounds the magnitude of each term.
__device__ __forceinline__ float3 cross_abs(float3 a, float3 b) {
    return make_float3(a.y * b.z + a.z * b.y, a.z * b.x + a.x * b.z, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// FP32 Moller-Trumbore with forward error bounds.  With d, e1, e2, sv each
// rounded once and every quantity a dot of a cross, |fl(x) - x| <= 8 u M_x
// where M_x is the same expression in absolute values; kErrK doubles that.
// Decisions are taken on the numerators against the denominator so the
// bounds stay linear:  u > tau  <=>  sign(det) U > tau |det|,  etc.
__device__ __forceinline__ int tri_fp32(const SegF& g, const Tri& tr, bool want_plain, bool& plain_hit) {
    float3 a = f3(tr.v0);
    float3 e1 = sub3(f3(tr.v1), a), e2 = sub3(f3(tr.v2), a);
    float3 sv = sub3(g.s, a);
    float3 p = cross3(g.d, e2);
    float det = dot3(e1, p);
    float3 q = cross3(sv, e1);
    float T = dot3(e2, q);
    float3 ad = abs3(g.d), ae1 = abs3(e1), ae2 = abs3(e2), asv = abs3(sv);
    float3 pa = cross_abs(ad, ae2), qa = cross_abs(asv, ae1);
    float errdet = kErrK * dot3(ae1, pa) + 1e-35f;
    float errT = kErrK * dot3(ae2, qa) + 1e-35f;
    // tau * |d| |e1| |e2| bounded above with 1-norms (no square roots)
    float thr = kTauHi * (g.dl1 * (ae1.x + ae1.y + ae1.z)) * (ae2.x + ae2.y + ae2.z) * 1.000001f;
    float Tm = T - det;
    float errTm = errT + errdet + 2.0f * kU * (fabsf(T) + fabsf(det));
    float U = dot3(sv, p), V = dot3(g.d, q);
    plain_hit = false;
    if (want_plain && det != 0.0f) {   // the uncorrected FP32 decision (fp32_only)
        float u = U / det, v = V / det, t = T / det;
        plain_hit = u >= 0.0f && v >= 0.0f && u + v <= 1.0f && t >= 0.0f && t <= 1.0f;
    }
    // both end points strictly on one side of the plane, farther than
    // tau |d| |n| (|n| <= |e1||e2|): a decisive miss on either branch
    if ((T > 0.0f) == (Tm > 0.0f) && fminf(fabsf(T) - errT, fabsf(Tm) - errTm) > thr) return kMiss;
    float D = fabsf(det);
    if (D - errdet > thr) {   // |det_rel| > tau for certain
        float sg = det > 0.0f ? 1.0f : -1.0f;
        float errU = kErrK * dot3(asv, pa) + 1e-35f;
        float errV = kErrK * dot3(ad, qa) + 1e-35f;
        float Us = sg * U, Vs = sg * V, Ts = sg * T;
        float Ws = D - Us - Vs;
        float errW = errdet + errU + errV + 2.0f * kU * (D + fabsf(U) + fabsf(V));
        float Tms = D - Ts;
        float lim = kTauHi * (D + errdet) * 1.000001f;
        if (Us - errU > lim && Vs - errV > lim && Ws - errW > lim && Ts - errT > lim && Tms - errTm > lim)
            return kHit;
        if (Us + errU < -lim || Vs + errV < -lim || Ws + errW < -lim || Ts + errT < -lim || Tms + errTm < -lim)
            return kMiss;
    }
    return kBand;
}

__device__ __forceinline__ void load_node(const Node* __restrict__ nodes, int i, float4& a, float4& b, float4& c,
                                          float4& d) {
    const float4* p = reinterpret_cast<const float4*>(nodes + i);
    a = __ldg(p);
    b = __ldg(p + 1);
    c = __ldg(p + 2);
    d = __ldg(p + 3);
}

__device__ __forceinline__ Tri load_tri(const Tri* __restrict__ tris, int j) {
    const float4* p = reinterpret_cast<const float4*>(tris + j);
    Tri t;
    t.v0 = __ldg(p);
    t.v1 = __ldg(p + 1);
    t.v2 = __ldg(p + 2);
    return t;
}

__device__ __forceinline__ void raise_error(DevCounters* c, int code) { atomicCAS(&c->error, 0, code); }

__device__ __forceinline__ bool bad3(float3 a) {
    return !(isfinite(a.x) && isfinite(a.y) && isfinite(a.z));
}

// ---------------------------------------------------------------- FP64
// The definition in FP64 with explicit round-to-nearest operations in the
// order the definition is written, so that no multiply-add is fused.
struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 dsub(D3 a, D3 b) { return {__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z)}; }
__device__ __forceinline__ D3 dadd(D3 a, D3 b) { return {__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y), __dadd_rn(a.z, b.z)}; }
__device__ __forceinline__ D3 dscale(D3 a, double s) { return {__dmul_rn(a.x, s), __dmul_rn(a.y, s), __dmul_rn(a.z, s)}; }
__device__ __forceinline__ double ddot(D3 a, D3 b) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)), __dmul_rn(a.z, b.z));
}
__device__ __forceinline__ D3 dcross(D3 a, D3 b) {
    return {__dsub_rn(__dmul_rn(a.y, b.z), __dmul_rn(a.z, b.y)), __dsub_rn(__dmul_rn(a.z, b.x), __dmul_rn(a.x, b.z)),
            __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x))};
}
__device__ __forceinline__ double dnorm(D3 a) { return __dsqrt_rn(ddot(a, a)); }
__device__ __forceinline__ double clamp01d(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }
__device__ __forceinline__ D3 d3of(float4 v) { return {(double)v.x, (double)v.y, (double)v.z}; }

__device__ double pt_seg(D3 p, D3 a, D3 b) {
    D3 ab = dsub(b, a);
    double len2 = ddot(ab, ab);
    double t = len2 > 0.0 ? clamp01d(__ddiv_rn(ddot(dsub(p, a), ab), len2)) : 0.0;
    return dnorm(dsub(p, dadd(a, dscale(ab, t))));
}

__device__ double seg_seg(D3 p0, D3 p1, D3 q0, D3 q1) {
    double best = pt_seg(p0, q0, q1);
    double d = pt_seg(p1, q0, q1);
    if (d < best) best = d;
    d = pt_seg(q0, p0, p1);
    if (d < best) best = d;
    d = pt_seg(q1, p0, p1);
    if (d < best) best = d;
    D3 u = dsub(p1, p0), v = dsub(q1, q0), w0 = dsub(p0, q0);
    double a = ddot(u, u), b = ddot(u, v), c = ddot(v, v);
    double dd = ddot(u, w0), e = ddot(v, w0);
    double den = __dsub_rn(__dmul_rn(a, c), __dmul_rn(b, b));
    if (den > 0.0) {
        double s = __ddiv_rn(__dsub_rn(__dmul_rn(b, e), __dmul_rn(c, dd)), den);
        double t = __ddiv_rn(__dsub_rn(__dmul_rn(a, e), __dmul_rn(b, dd)), den);
        if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
            d = dnorm(dsub(dadd(w0, dscale(u, s)), dscale(v, t)));
            if (d < best) best = d;
        }
    }
    return best;
}

__device__ double pt_tri(D3 p, D3 a, D3 b, D3 c) {
    D3 n = dcross(dsub(b, a), dsub(c, a));
    double nn = ddot(n, n);
    double h = __ddiv_rn(ddot(dsub(p, a), n), nn);
    D3 proj = dsub(p, dscale(n, h));
    double s0 = ddot(dcross(dsub(b, a), dsub(proj, a)), n);
    double s1 = ddot(dcross(dsub(c, b), dsub(proj, b)), n);
    double s2 = ddot(dcross(dsub(a, c), dsub(proj, c)), n);
    if (s0 >= 0.0 && s1 >= 0.0 && s2 >= 0.0) return __dmul_rn(fabs(h), __dsqrt_rn(nn));
    double best = pt_seg(p, a, b);
    double d = pt_seg(p, b, c);
    if (d < best) best = d;
    d = pt_seg(p, c, a);
    if (d < best) best = d;
    return best;
}

// Class of a pair in FP64 (decisive hit / decisive miss / ambiguous), the
// inclusive (closed-interval) hit and its t.
__device__ int classify_fp64(D3 s, D3 e, D3 a, D3 b, D3 c, double& t_out, bool& incl) {
    const double tau = kTauD;
    D3 d = dsub(e, s);
    D3 e1 = dsub(b, a), e2 = dsub(c, a);
    D3 n = dcross(e1, e2);
    incl = false;
    t_out = 0.0;
    if ((d.x == 0.0 && d.y == 0.0 && d.z == 0.0) || (n.x == 0.0 && n.y == 0.0 && n.z == 0.0)) return kMiss;
    D3 p = dcross(d, e2);
    double det = ddot(e1, p);
    D3 sv = dsub(s, a);
    D3 q = dcross(sv, e1);
    double det_rel = __ddiv_rn(det, __dmul_rn(__dmul_rn(dnorm(d), dnorm(e1)), dnorm(e2)));
    double u = 0.0, v = 0.0, t = 0.0, w = 0.0;
    if (det != 0.0) {
        u = __ddiv_rn(ddot(sv, p), det);
        v = __ddiv_rn(ddot(d, q), det);
        t = __ddiv_rn(ddot(e2, q), det);
        w = __dsub_rn(__dsub_rn(1.0, u), v);
        incl = (u >= 0.0 && v >= 0.0 && w >= 0.0 && t >= 0.0 && t <= 1.0);
    }
    t_out = t;
    if (fabs(det_rel) > tau) {
        if (u > tau && v > tau && w > tau && t > tau && t < 1.0 - tau) return kHit;
        if (u < -tau || v < -tau || w < -tau || t < -tau || t > 1.0 + tau) return kMiss;
        return kBand;   // ambiguous
    }
    double dist;
    if (incl) {
        dist = 0.0;
    } else {
        dist = pt_tri(s, a, b, c);
        double dd = pt_tri(e, a, b, c);
        if (dd < dist) dist = dd;
        dd = seg_seg(s, e, a, b);
        if (dd < dist) dist = dd;
        dd = seg_seg(s, e, b, c);
        if (dd < dist) dist = dd;
        dd = seg_seg(s, e, c, a);
        if (dd < dist) dist = dd;
    }
    return dist > __dmul_rn(tau, dnorm(d)) ? kMiss : kBand;
}

constexpr int kWarpChunk = 64;   // segments a warp takes per atomic
constexpr int kRefillMin = 4;    // refill once this many lanes of a warp are idle

constexpr int kLeafMin = 12;     // run the triangle tests once this many lanes hold one
constexpr int kDone = 0x7FFFFFFF;  // "no next node" (node indices stay below 2^30)

// Warp-coherent persistent traversal with deferred leaf tests.  Each lane
// holds its next reference (internal node >= 0, leaf ~j < 0, or kDone) and a
// one-entry leaf slot.  Every iteration a lane whose next reference is an
// internal node fetches it and tests both child boxes (the nearer-listed hit
// child becomes next, the other is pushed; leaves travel as references too);
// a lane whose next reference is a leaf parks it in its slot if the slot is
// free.  The warp runs the triangle tests of all parked leaves together once
// kLeafMin lanes hold one or no lane can move on without it, so node work and
// triangle work both run with most lanes active.  Lanes whose segment is done
// are refilled together from a per-warp chunk of segment indices (one atomic
// per chunk).  A segment with a band pair and no certain answer is queued for
// k_query_fp64 (count mode stops at the first band pair).
template <int MODE, bool STATS, int STACK>
__global__ void __launch_bounds__(256, 4) k_query_fp32(QueryArgs A) {
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int n_rays = (int)A.n_rays;
    unsigned long long visits = 0, tests = 0;
    int wbase = 0, wend = 0;     // warp-uniform chunk [wbase, wend)
    bool exhausted = false;      // warp-uniform
    int ray = -1;
    SegF g;
    int next = kDone, slot = -1, sp = 0;
    int stack[STACK];
    int cnt = 0, plain_cnt = 0;
    bool found = false, band = false, stop = false;
    while (true) {
        unsigned idle = __ballot_sync(kFull, ray < 0);
        if (!exhausted && (__popc(idle) >= kRefillMin || idle == kFull)) {
            while (idle) {
                if (wbase >= wend) {
                    unsigned long long b = 0;
                    if (lane == 0) b = atomicAdd(&A.ctr->next_ray, (unsigned long long)kWarpChunk);
                    b = __shfl_sync(kFull, b, 0);
                    if (b >= (unsigned long long)n_rays) {
                        exhausted = true;
                        break;
                    }
                    wbase = (int)b;
                    wend = min(wbase + kWarpChunk, n_rays);
                }
                const int take = min(__popc(idle), wend - wbase);
                bool mine = false;
                if ((idle >> lane) & 1u) {
                    const int rank = __popc(idle & lt);
                    if (rank < take) {
                        ray = A.perm ? __ldg(A.perm + wbase + rank) : wbase + rank;
                        mine = true;
                    }
                }
                wbase += take;
                if (mine) {
                    const int64_t r = ray;
                    float3 s = make_float3(__ldg(A.from + 3 * r), __ldg(A.from + 3 * r + 1), __ldg(A.from + 3 * r + 2));
                    float3 e = make_float3(__ldg(A.to + 3 * r), __ldg(A.to + 3 * r + 1), __ldg(A.to + 3 * r + 2));
                    if (bad3(s) || bad3(e)) {   // undefined answer: reported as ambiguous
                        if (A.hit) A.hit[r] = 0;
                        if (MODE == RSI_COUNT) A.count[r] = 0;
                        if (A.amb) A.amb[r] = 1;
                        ray = -1;
                    } else {
                        g = make_seg(s, e, A.dmax0, A.dmax1, A.dmax2);
                        next = A.n_tri == 1 ? ~0 : 0;
                        slot = -1;
                        sp = 0;
                        cnt = plain_cnt = 0;
                        found = band = stop = false;
                    }
                }
                idle = __ballot_sync(kFull, ray < 0);
            }
        }
        const bool active = ray >= 0;
        const unsigned act = __ballot_sync(kFull, active);
        if (act == 0) {
            if (exhausted) break;
            continue;
        }
        // node step
        if (active && next != kDone && next >= 0) {
            float4 lmin, lmax, rmin, rmax;
            load_node(A.nodes, next, lmin, lmax, rmin, rmax);
            if (STATS) ++visits;
            const int lref = __float_as_int(lmin.w), rref = __float_as_int(lmax.w);
            const bool hl = slab(lmin, lmax, g), hr = slab(rmin, rmax, g);
            if (hl && hr) {
                if (sp < STACK) {
                    stack[sp++] = rref;
                    next = lref;
                } else {   // cannot happen with STACK > tree height; queued
                    raise_error(A.ctr, RSI_ERR_STACK);
                    band = true;
                    stop = true;
                }
            } else if (hl) {
                next = lref;
            } else if (hr) {
                next = rref;
            } else {
                next = sp > 0 ? stack[--sp] : kDone;
            }
        }
        // park a leaf reference
        if (active && !stop && next < 0 && slot < 0) {
            slot = ~next;
            next = sp > 0 ? stack[--sp] : kDone;
        }
        // leaf phase: all parked leaves of the warp at once
        const unsigned pend = __ballot_sync(kFull, active && slot >= 0);
        const unsigned moving = __ballot_sync(kFull, active && !stop && next != kDone && (next >= 0 || slot < 0));
        if (pend && (__popc(pend) >= kLeafMin || moving == 0)) {
            if (slot >= 0) {
                if (STATS) ++tests;
                const Tri tr = load_tri(A.tris, slot);
                bool plain;
                int c = tri_fp32(g, tr, A.fp32_only != 0, plain);
                plain_cnt += plain;
                if (c == kBand && !A.fp32_only) {   // settled by the FP64 pass
                    band = true;
                    if (MODE == RSI_COUNT) stop = true;
                } else if (c == kHit) {
                    ++cnt;
                    if (MODE == RSI_ANY_HIT) {
                        found = true;
                        stop = true;
                    }
                }
                slot = -1;
            }
        }
        if (active && (stop || (next == kDone && slot < 0))) {
            const int64_t r = ray;
            if (A.fp32_only) {   // plain FP32 closed-interval decisions, no re-test
                if (MODE == RSI_ANY_HIT) A.hit[r] = (uint8_t)(found || plain_cnt > 0);
                else {
                    A.count[r] = plain_cnt;
                    if (A.hit) A.hit[r] = (uint8_t)(plain_cnt > 0);
                }
                if (A.amb) A.amb[r] = 0;
            } else if (MODE == RSI_ANY_HIT && found) {
                A.hit[r] = 1;
                if (A.amb) A.amb[r] = 0;
            } else if (band) {
                int pos = atomicAdd(&A.ctr->band_count, 1);
                A.band_ids[pos] = ray;
            } else {
                if (MODE == RSI_ANY_HIT) A.hit[r] = 0;
                else {
                    A.count[r] = cnt;
                    if (A.hit) A.hit[r] = (uint8_t)(cnt > 0);
                }
                if (A.amb) A.amb[r] = 0;
            }
            ray = -1;
        }
    }
    if (STATS) {
        for (int off = 16; off; off >>= 1) {
            visits += __shfl_xor_sync(kFull, visits, off);
            tests += __shfl_xor_sync(kFull, tests, off);
        }
        if (lane == 0) {
            atomicAdd(&A.ctr->node_visits, visits);
            atomicAdd(&A.ctr->tri_tests, tests);
        }
    }
}

// Certain decisions in FP64 without square roots or divisions: the FP32 test
// above in double precision, with the bound factor 32 u (u = 2^-53) and a
// 1e-9 relative slack on tau, so that a certain answer is also the answer
// the definition's own FP64 rounding gives.  kBand = undecided.
__device__ __forceinline__ int tri_certain64(D3 s, D3 e, D3 a, D3 b, D3 c) {
    const double u = 1.1102230246251565e-16, K = 32.0 * u, tau = kTauD * (1.0 + 1e-9);
    const double dx = e.x - s.x, dy = e.y - s.y, dz = e.z - s.z;
    const double e1x = b.x - a.x, e1y = b.y - a.y, e1z = b.z - a.z;
    const double e2x = c.x - a.x, e2y = c.y - a.y, e2z = c.z - a.z;
    const double sx = s.x - a.x, sy = s.y - a.y, sz = s.z - a.z;
    const double px = dy * e2z - dz * e2y, py = dz * e2x - dx * e2z, pz = dx * e2y - dy * e2x;
    const double qx = sy * e1z - sz * e1y, qy = sz * e1x - sx * e1z, qz = sx * e1y - sy * e1x;
    const double det = e1x * px + e1y * py + e1z * pz;
    const double T = e2x * qx + e2y * qy + e2z * qz;
    const double U = sx * px + sy * py + sz * pz, V = dx * qx + dy * qy + dz * qz;
    const double adx = fabs(dx), ady = fabs(dy), adz = fabs(dz);
    const double a1x = fabs(e1x), a1y = fabs(e1y), a1z = fabs(e1z);
    const double a2x = fabs(e2x), a2y = fabs(e2y), a2z = fabs(e2z);
    const double asx = fabs(sx), asy = fabs(sy), asz = fabs(sz);
    const double pax = ady * a2z + adz * a2y, pay = adz * a2x + adx * a2z, paz = adx * a2y + ady * a2x;
    const double qax = asy * a1z + asz * a1y, qay = asz * a1x + asx * a1z, qaz = asx * a1y + asy * a1x;
    const double errdet = K * (a1x * pax + a1y * pay + a1z * paz) + 1e-300;
    const double errT = K * (a2x * qax + a2y * qay + a2z * qaz) + 1e-300;
    const double thr = tau * ((adx + ady + adz) * (a1x + a1y + a1z)) * (a2x + a2y + a2z);
    const double Tm = T - det;
    const double errTm = errT + errdet + 4.0 * u * (fabs(T) + fabs(det));
    if ((T > 0.0) == (Tm > 0.0) && fmin(fabs(T) - errT, fabs(Tm) - errTm) > thr) return kMiss;
    const double D = fabs(det);
    if (D - errdet > thr) {
        const double sg = det > 0.0 ? 1.0 : -1.0;
        const double errU = K * (asx * pax + asy * pay + asz * paz) + 1e-300;
        const double errV = K * (adx * qax + ady * qay + adz * qaz) + 1e-300;
        const double Us = sg * U, Vs = sg * V, Ts = sg * T;
        const double Ws = D - Us - Vs;
        const double errW = errdet + errU + errV + 4.0 * u * (D + fabs(U) + fabs(V));
        const double Tms = D - Ts;
        const double lim = tau * (D + errdet);
        if (Us - errU > lim && Vs - errV > lim && Ws - errW > lim && Ts - errT > lim && Tms - errTm > lim)
            return kHit;
        if (Us + errU < -lim || Vs + errV < -lim || Ws + errW < -lim || Ts + errT < -lim || Tms + errTm < -lim)
            return kMiss;
    }
    return kBand;
}

// t of the definition with its own operations (so that crossings merge
// exactly as the definition merges them).
__device__ __forceinline__ double t_of_definition(D3 s, D3 e, D3 a, D3 b, D3 c) {
    D3 d = dsub(e, s);
    D3 e1 = dsub(b, a), e2 = dsub(c, a);
    D3 p = dcross(d, e2);
    double det = ddot(e1, p);
    D3 q = dcross(dsub(s, a), e1);
    return __ddiv_rn(ddot(e2, q), det);
}

// The queued segments, one warp each: lane 0 walks the tree and keeps the
// leaves the FP32 test does not reject for certain (up to 32 at a time);
// the lanes then classify those pairs side by side in FP64 -- a certain
// decision from the numerators where possible, the definition itself
// otherwise -- and the warp combines the classes.  A decisive hit ends a
// boolean query; otherwise the closed-interval answer of an ambiguous
// segment counts distinct crossings (t merged within 1e-9).
template <int MODE, int STACK>
__global__ void __launch_bounds__(128) k_query_fp64(QueryArgs A) {
    constexpr int kWarps = 4;
    __shared__ double s_t[kWarps][kMaxInclusive];
    __shared__ int s_cand[kWarps][32];
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nb = *(volatile int*)&A.ctr->band_count;
    for (int k = blockIdx.x * kWarps + w; k < nb; k += gridDim.x * kWarps) {
        const int64_t r = A.band_ids[k];
        const float3 s = make_float3(A.from[3 * r], A.from[3 * r + 1], A.from[3 * r + 2]);
        const float3 e = make_float3(A.to[3 * r], A.to[3 * r + 1], A.to[3 * r + 2]);
        const SegF g = make_seg(s, e, A.dmax0, A.dmax1, A.dmax2);
        const D3 sd = {(double)s.x, (double)s.y, (double)s.z}, ed = {(double)e.x, (double)e.y, (double)e.z};
        int n_hit = 0, n_amb = 0, n_incl = 0;
        bool overflow = false;
        int node = 0, sp = 0;
        int stack[STACK];
        bool trav_done = false;
        while (true) {
            int nc = 0;
            if (lane == 0) {
                if (A.n_tri == 1) {
                    s_cand[w][nc++] = 0;
                    trav_done = true;
                }
                while (!trav_done && nc <= 30) {
                    float4 lmin, lmax, rmin, rmax;
                    load_node(A.nodes, node, lmin, lmax, rmin, rmax);
                    const int lref = __float_as_int(lmin.w), rref = __float_as_int(lmax.w);
                    bool hl = slab(lmin, lmax, g), hr = slab(rmin, rmax, g);
                    bool plain;
                    if (hl && lref < 0) {
                        hl = false;
                        if (tri_fp32(g, load_tri(A.tris, ~lref), false, plain) != kMiss) s_cand[w][nc++] = ~lref;
                    }
                    if (hr && rref < 0) {
                        hr = false;
                        if (tri_fp32(g, load_tri(A.tris, ~rref), false, plain) != kMiss) s_cand[w][nc++] = ~rref;
                    }
                    if (hl && hr) {
                        if (sp < STACK) {
                            stack[sp++] = rref;
                            node = lref;
                        } else {
                            raise_error(A.ctr, RSI_ERR_STACK);
                            trav_done = true;
                        }
                    } else if (hl) {
                        node = lref;
                    } else if (hr) {
                        node = rref;
                    } else if (sp > 0) {
                        node = stack[--sp];
                    } else {
                        trav_done = true;
                    }
                }
            }
            nc = __shfl_sync(kFull, nc, 0);
            trav_done = __shfl_sync(kFull, trav_done ? 1 : 0, 0) != 0;
            __syncwarp();
            int cls = -1;
            bool incl = false;
            double t = 0.0;
            if (lane < nc) {
                const Tri tr = load_tri(A.tris, s_cand[w][lane]);
                const D3 a = d3of(tr.v0), b = d3of(tr.v1), c = d3of(tr.v2);
                cls = tri_certain64(sd, ed, a, b, c);
                if (cls == kHit) {
                    incl = true;
                    t = t_of_definition(sd, ed, a, b, c);
                } else if (cls == kBand) {
                    cls = classify_fp64(sd, ed, a, b, c, t, incl);
                }
            }
            const unsigned mh = __ballot_sync(kFull, cls == kHit);
            const unsigned ma = __ballot_sync(kFull, cls == kBand);
            const unsigned mi = __ballot_sync(kFull, incl);
            if (incl) {
                const int pos = n_incl + __popc(mi & lt);
                if (pos < kMaxInclusive) s_t[w][pos] = t;
                else overflow = true;
            }
            n_hit += __popc(mh);
            n_amb += __popc(ma);
            n_incl += __popc(mi);
            overflow = __any_sync(kFull, overflow);
            __syncwarp();
            if ((MODE == RSI_ANY_HIT && mh) || trav_done) break;
        }
        if (lane == 0) {
            if (overflow) raise_error(A.ctr, RSI_ERR_OVERFLOW);
            const int m = min(n_incl, kMaxInclusive);
            if (MODE == RSI_ANY_HIT) {
                const bool amb = n_hit == 0 && n_amb > 0;
                A.hit[r] = (uint8_t)(n_hit > 0 || (amb && n_incl > 0));
                if (A.amb) A.amb[r] = (uint8_t)amb;
                if (amb) atomicAdd(&A.ctr->ambiguous, 1ull);
            } else {
                const bool amb = n_amb > 0;
                int count = n_hit;
                if (amb) {
                    double* ts = s_t[w];
                    for (int i = 1; i < m; ++i) {   // insertion sort of the crossing parameters
                        const double x = ts[i];
                        int k2 = i - 1;
                        while (k2 >= 0 && ts[k2] > x) {
                            ts[k2 + 1] = ts[k2];
                            --k2;
                        }
                        ts[k2 + 1] = x;
                    }
                    count = 0;
                    for (int i = 0; i < m; ++i)
                        if (i == 0 || __dsub_rn(ts[i], ts[i - 1]) > kTMerge) ++count;
                    atomicAdd(&A.ctr->ambiguous, 1ull);
                }
                A.count[r] = count;
                if (A.hit) A.hit[r] = (uint8_t)(count > 0);
                if (A.amb) A.amb[r] = (uint8_t)amb;
            }
        }
        __syncwarp();
    }
}

// In-tile reordering of segments for warp coherence: a counting sort of each
// tile by the top 10 bits of the 30-bit Morton code of the segment midpoint
// (normalised by the mesh extent).  perm[base .. base + m) becomes a
// permutation of the tile's indices; order inside a cell is arbitrary, which
// is harmless because every segment's answer is independent of the order.
constexpr int kSortBins = 1024;
constexpr int kMaxSortTile = 8192;

__device__ __forceinline__ uint32_t spread10q(uint32_t x) {
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void __launch_bounds__(256) k_ray_tile_sort(const float* __restrict__ from, const float* __restrict__ to,
                                                       int n, int tile, float lox, float loy, float loz, float sx,
                                                       float sy, float sz, int32_t* __restrict__ perm) {
    __shared__ int cnt[kSortBins];
    __shared__ unsigned short key[kMaxSortTile];
    __shared__ int wsum[8];
    const int tid = threadIdx.x;
    for (int i = tid; i < kSortBins; i += 256) cnt[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * tile;
    const int m = (int)min((int64_t)tile, (int64_t)n - base);
    for (int i = tid; i < m; i += 256) {
        const int64_t r = base + i;
        float mx = 0.5f * (from[3 * r] + to[3 * r]);
        float my = 0.5f * (from[3 * r + 1] + to[3 * r + 1]);
        float mz = 0.5f * (from[3 * r + 2] + to[3 * r + 2]);
        uint32_t qx = (uint32_t)fminf(fmaxf((mx - lox) * sx, 0.0f), 1023.0f);
        uint32_t qy = (uint32_t)fminf(fmaxf((my - loy) * sy, 0.0f), 1023.0f);
        uint32_t qz = (uint32_t)fminf(fmaxf((mz - loz) * sz, 0.0f), 1023.0f);   // NaN -> 0
        uint32_t k = (spread10q(qx) | (spread10q(qy) << 1) | (spread10q(qz) << 2)) >> 20;
        key[i] = (unsigned short)k;
        atomicAdd(&cnt[k], 1);
    }
    __syncthreads();
    // exclusive scan of the 1024 bins: 4 per thread, then across warps
    int v0 = cnt[4 * tid], v1 = cnt[4 * tid + 1], v2 = cnt[4 * tid + 2], v3 = cnt[4 * tid + 3];
    int tot = v0 + v1 + v2 + v3, inc = tot;
    const int lane = tid & 31, w = tid >> 5;
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int wpre = 0;
    for (int j = 0; j < w; ++j) wpre += wsum[j];
    int ex = wpre + inc - tot;
    cnt[4 * tid] = ex;
    cnt[4 * tid + 1] = ex + v0;
    cnt[4 * tid + 2] = ex + v0 + v1;
    cnt[4 * tid + 3] = ex + v0 + v1 + v2;
    __syncthreads();
    for (int i = tid; i < m; i += 256) {
        int pos = atomicAdd(&cnt[key[i]], 1);
        perm[base + pos] = (int32_t)(base + i);
    }
}

__global__ void k_reset_query(DevCounters* c) {
    c->band_count = 0;
    c->next_ray = 0;
    c->error = 0;
    c->node_visits = c->tri_tests = c->ambiguous = 0;
}

template <int MODE, bool STATS, int STACK>
void launch_fp32(const QueryArgs& A, int grid, int block, cudaStream_t s) {
    k_query_fp32<MODE, STATS, STACK><<<grid, block, 0, s>>>(A);
}

template <int MODE, bool STATS>
void launch_fp32_stack(const QueryArgs& A, int height, int grid, int block, cudaStream_t s) {
    if (height < 32) launch_fp32<MODE, STATS, 32>(A, grid, block, s);
    else if (height < 64) launch_fp32<MODE, STATS, 64>(A, grid, block, s);
    else launch_fp32<MODE, STATS, 128>(A, grid, block, s);
}

template <int MODE>
void launch_fp64(const QueryArgs& A, int height, int grid, cudaStream_t s) {
    if (height < 32) k_query_fp64<MODE, 32><<<grid, 128, 0, s>>>(A);
    else if (height < 64) k_query_fp64<MODE, 64><<<grid, 128, 0, s>>>(A);
    else k_query_fp64<MODE, 128><<<grid, 128, 0, s>>>(A);
}

}  // namespace

// Launch the two passes for one batch of segments already on the device.
int query_device(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n, int mode, const rsi_options* opt,
                 uint8_t* d_hit, int32_t* d_count, uint8_t* d_amb, int32_t* band_ids, int32_t* perm_scratch,
                 DevCounters* ctr, cudaStream_t s) {
    rsi_options o = {};
    if (opt) o = *opt;
    if (h->height >= 127) return fail(RSI_ERR_STACK, "rsi_query: tree height exceeds the 128-entry traversal stack");
    QueryArgs A;
    A.nodes = h->nodes;
    A.tris = h->tris;
    A.n_tri = h->n_tri;
    A.from = d_from;
    A.to = d_to;
    A.n_rays = n;
    A.hit = d_hit;
    A.count = d_count;
    A.amb = d_amb;
    A.band_ids = band_ids;
    A.perm = nullptr;
    A.ctr = ctr;
    A.dmax0 = h->dmax[0];
    A.dmax1 = h->dmax[1];
    A.dmax2 = h->dmax[2];
    A.fp32_only = o.fp32_only;
    if (o.block != 0 && (o.block < 32 || o.block > 256 || o.block % 32 != 0))
        return fail(RSI_ERR_INVALID_ARG, "rsi_query: block must be a multiple of 32 in [32, 256]");
    if (o.blocks_per_sm < 0) return fail(RSI_ERR_INVALID_ARG, "rsi_query: blocks_per_sm < 0");
    const int block = o.block > 0 ? o.block : 256;
    const int bps = o.blocks_per_sm > 0 ? o.blocks_per_sm : 8;
    int64_t want = (n + block - 1) / block;
    int64_t cap = (int64_t)device_sm_count() * bps;
    int grid = (int)std::max<int64_t>(1, std::min(want, cap));
    if (o.time_kernels && !h->ev[0]) {
        for (auto& e : h->ev) RSI_CUDA_TRY(cudaEventCreate(&e));
    }
    h->timed = o.time_kernels != 0;
    if (o.ray_sort_tile != 0) {
        if (o.ray_sort_tile < 256 || o.ray_sort_tile > kMaxSortTile)
            return fail(RSI_ERR_INVALID_ARG, "rsi_query: ray_sort_tile must be 0 or in [256, 8192]");
        if (!perm_scratch) return fail(RSI_ERR_INVALID_ARG, "rsi_query: ray_sort_tile needs scratch");
        float sc[3];
        for (int a = 0; a < 3; ++a) sc[a] = h->hi[a] > h->lo[a] ? 1024.0f / (h->hi[a] - h->lo[a]) : 0.0f;
        k_ray_tile_sort<<<grid_for(n, o.ray_sort_tile), 256, 0, s>>>(d_from, d_to, (int)n, o.ray_sort_tile, h->lo[0],
                                                                     h->lo[1], h->lo[2], sc[0], sc[1], sc[2],
                                                                     perm_scratch);
        note_launches(1);
        A.perm = perm_scratch;
    }
    k_reset_query<<<1, 1, 0, s>>>(ctr);
    if (h->timed) RSI_CUDA_TRY(cudaEventRecord(h->ev[0], s));
    if (mode == RSI_ANY_HIT) {
        if (o.collect_stats) launch_fp32_stack<RSI_ANY_HIT, true>(A, h->height, grid, block, s);
        else launch_fp32_stack<RSI_ANY_HIT, false>(A, h->height, grid, block, s);
    } else {
        if (o.collect_stats) launch_fp32_stack<RSI_COUNT, true>(A, h->height, grid, block, s);
        else launch_fp32_stack<RSI_COUNT, false>(A, h->height, grid, block, s);
    }
    if (h->timed) RSI_CUDA_TRY(cudaEventRecord(h->ev[1], s));
    if (!o.fp32_only) {
        if (mode == RSI_ANY_HIT) launch_fp64<RSI_ANY_HIT>(A, h->height, device_sm_count() * 4, s);
        else launch_fp64<RSI_COUNT>(A, h->height, device_sm_count() * 4, s);
    }
    if (h->timed) RSI_CUDA_TRY(cudaEventRecord(h->ev[2], s));
    note_launches(o.fp32_only ? 2 : 3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rsi_query launch");
    return RSI_OK;
}

int ensure_band_capacity(rsi_bvh_t h, int64_t n, cudaStream_t s) {
    if (h->band_cap >= n) return RSI_OK;
    int64_t cap = std::max<int64_t>(n, 1 << 16);
    if (h->band_ids) {
        RSI_CUDA_TRY(cudaStreamSynchronize(s));
        cudaFree(h->band_ids);
        h->band_ids = nullptr;
        h->band_cap = 0;
    }
    if (cudaMalloc(&h->band_ids, 8 * (size_t)cap) != cudaSuccess) {   // band list, then permutation
        cudaGetLastError();
        return fail(RSI_ERR_OOM, "rsi_query: band list allocation failed");
    }
    h->band_cap = cap;
    return RSI_OK;
}

int read_stats(rsi_bvh_t h, DevCounters* ctr, int64_t n, rsi_stats* st, cudaStream_t s) {
    RSI_CUDA_TRY(cudaMemcpyAsync(h->h_ctr, ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    RSI_CUDA_TRY(cudaStreamSynchronize(s));
    const DevCounters& c = *h->h_ctr;
    if (st) {
        st->n_rays = n;
        st->node_visits = (int64_t)c.node_visits;
        st->tri_tests = (int64_t)c.tri_tests;
        st->band_rays = c.band_count;
        st->ambiguous = (int64_t)c.ambiguous;
        st->tree_height = h->height;
        st->device_error = c.error;
    }
    if (c.error) return fail(c.error, "rsi_query: device error " + std::to_string(c.error));
    return RSI_OK;
}

}  // namespace rsi

extern "C" int rsi_last_query_ms(rsi_bvh_t h, float* traverse_ms, float* retest_ms) {
    if (!h) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_last_query_ms: NULL handle");
    float a = -1.0f, b = -1.0f;
    if (h->timed && h->ev[0]) {
        RSI_CUDA_TRY(cudaEventSynchronize(h->ev[2]));
        RSI_CUDA_TRY(cudaEventElapsedTime(&a, h->ev[0], h->ev[1]));
        RSI_CUDA_TRY(cudaEventElapsedTime(&b, h->ev[1], h->ev[2]));
    }
    if (traverse_ms) *traverse_ms = a;
    if (retest_ms) *retest_ms = b;
    return RSI_OK;
}

static int check_query_args(rsi_bvh_t h, const void* from, const void* to, int64_t n, int mode, const void* hit,
                            const void* count) {
    if (!h) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query: NULL handle");
    if (n < 0 || n > 0x7FFFFFFFll) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query: need 0 <= n_rays < 2^31");
    if (mode != RSI_ANY_HIT && mode != RSI_COUNT) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query: bad mode");
    if (n > 0 && (!from || !to)) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query: NULL segment pointer");
    if (n > 0 && mode == RSI_ANY_HIT && !hit) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query: any-hit needs hit");
    if (n > 0 && mode == RSI_COUNT && !count) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query: count needs count");
    return RSI_OK;
}

extern "C" int rsi_query(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays, int mode,
                         const rsi_options* opt, uint8_t* d_hit, int32_t* d_count, uint8_t* d_ambiguous,
                         rsi_stats* stats, void* stream) {
    int rc = check_query_args(h, d_from, d_to, n_rays, mode, d_hit, d_count);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_rays == 0) {
        if (stats) *stats = rsi_stats{};
        return RSI_OK;
    }
    rc = rsi::ensure_band_capacity(h, n_rays, s);
    if (rc) return rc;
    rc = rsi::query_device(h, d_from, d_to, n_rays, mode, opt, d_hit, d_count, d_ambiguous, h->band_ids,
                           h->band_ids + h->band_cap, h->ctr, s);
    if (rc) return rc;
    if (stats) return rsi::read_stats(h, h->ctr, n_rays, stats, s);
    return RSI_OK;
}

extern "C" int rsi_query_host(rsi_bvh_t h, const float* h_from, const float* h_to, int64_t n_rays, int mode,
                              const rsi_options* opt, uint8_t* h_hit, int32_t* h_count, uint8_t* h_ambiguous,
                              rsi_stats* stats, void* stream) {
    int rc = check_query_args(h, h_from, h_to, n_rays, mode, h_hit, h_count);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_rays == 0) {
        if (stats) *stats = rsi_stats{};
        return RSI_OK;
    }
    rc = rsi::ensure_band_capacity(h, n_rays, s);
    if (rc) return rc;
    const size_t bf = 12 * (size_t)n_rays;
    float *df = nullptr, *dt = nullptr;
    uint8_t *dh = nullptr, *da = nullptr;
    int32_t* dc = nullptr;
    bool ok = cudaMallocAsync(&df, bf, s) == cudaSuccess && cudaMallocAsync(&dt, bf, s) == cudaSuccess;
    if (ok && h_hit) ok = cudaMallocAsync(&dh, n_rays, s) == cudaSuccess;
    if (ok && h_ambiguous) ok = cudaMallocAsync(&da, n_rays, s) == cudaSuccess;
    if (ok && mode == RSI_COUNT) ok = cudaMallocAsync(&dc, 4 * (size_t)n_rays, s) == cudaSuccess;
    if (ok) {
        ok = cudaMemcpyAsync(df, h_from, bf, cudaMemcpyHostToDevice, s) == cudaSuccess &&
             cudaMemcpyAsync(dt, h_to, bf, cudaMemcpyHostToDevice, s) == cudaSuccess;
        if (!ok) rc = rsi::cuda_fail(cudaGetLastError(), "rsi_query_host copy in");
    } else {
        cudaGetLastError();
        rc = rsi::fail(RSI_ERR_OOM, "rsi_query_host: staging allocation failed");
    }
    if (rc == RSI_OK)
        rc = rsi::query_device(h, df, dt, n_rays, mode, opt, dh, dc, da, h->band_ids, h->band_ids + h->band_cap,
                               h->ctr, s);
    if (rc == RSI_OK) {
        bool c_ok = true;
        if (h_hit) c_ok &= cudaMemcpyAsync(h_hit, dh, n_rays, cudaMemcpyDeviceToHost, s) == cudaSuccess;
        if (h_ambiguous) c_ok &= cudaMemcpyAsync(h_ambiguous, da, n_rays, cudaMemcpyDeviceToHost, s) == cudaSuccess;
        if (mode == RSI_COUNT) c_ok &= cudaMemcpyAsync(h_count, dc, 4 * (size_t)n_rays, cudaMemcpyDeviceToHost, s) == cudaSuccess;
        if (!c_ok) rc = rsi::cuda_fail(cudaGetLastError(), "rsi_query_host copy out");
    }
    for (void* p : {(void*)df, (void*)dt, (void*)dh, (void*)da, (void*)dc})
        if (p) cudaFreeAsync(p, s);
    if (rc) return rc;
    rsi_stats tmp;
    return rsi::read_stats(h, h->ctr, n_rays, stats ? stats : &tmp, s);
}

// ---------------------------------------------------------------- no-alloc
// rsi_query_noalloc: the same two passes with their scratch (counters, then
// the FP64 queue) in this file-scope array instead of handle memory.
namespace {

constexpr size_t kNoallocHeader = 256;
constexpr size_t kNoallocBytes = kNoallocHeader + 4 * (size_t)RSI_NOALLOC_MAX_RAYS;
static_assert(sizeof(rsi::DevCounters) <= kNoallocHeader, "counters fit the header");
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (host code only sees a host-side stand-in for the symbol).
int noalloc_scratch(void** out) {
    int dev = 0;
    RSI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_noalloc: device id >= 64");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return rsi::cuda_fail(e, "rsi_query_noalloc: cudaGetSymbolAddress");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return RSI_OK;
}

}  // namespace

extern "C" int rsi_query_noalloc(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays, int mode,
                                 const rsi_options* opt, uint8_t* d_hit, int32_t* d_count, uint8_t* d_ambiguous,
                                 void* stream) {
    int rc = check_query_args(h, d_from, d_to, n_rays, mode, d_hit, d_count);
    if (rc) return rc;
    if (n_rays > (int64_t)RSI_NOALLOC_MAX_RAYS)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_noalloc: n_rays " + std::to_string(n_rays) +
                                                  " exceeds RSI_NOALLOC_MAX_RAYS (" +
                                                  std::to_string(RSI_NOALLOC_MAX_RAYS) + "); split the batch");
    if (n_rays == 0) return RSI_OK;
    void* base = nullptr;
    rc = noalloc_scratch(&base);
    if (rc) return rc;
    rsi_options o = {};
    if (opt) o = *opt;
    o.time_kernels = 0;
    o.collect_stats = 0;
    o.ray_sort_tile = 0;
    auto* ctr = reinterpret_cast<rsi::DevCounters*>(base);
    auto* band = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(base) + kNoallocHeader);
    return rsi::query_device(h, d_from, d_to, n_rays, mode, &o, d_hit, d_count, d_ambiguous, band, nullptr, ctr,
                             (cudaStream_t)stream);
}
