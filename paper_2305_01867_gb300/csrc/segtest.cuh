// segtest.cuh -- the FP32 segment / box / triangle tests shared by the
// traversal (query.cu) and the learned proposal's verification (mlp.cu):
// Moller-Trumbore (Sec. 1) with a forward error bound, so that every FP32
// decision it calls certain equals the FP64 decision of the definition, and
// the padded, outward-rounded slab test that culls boxes conservatively.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rsi_internal.cuh"

namespace rsi {
namespace segtest {

constexpr float kU = 5.9604645e-8f;        // unit roundoff of FP32, 2^-24
constexpr float kErrK = 16.0f * kU;        // bound factor of a dot(cross) in FP32
constexpr float kTauHi = 1.000001e-6f;     // tau, rounded up
constexpr float kSlabGrow = 1.000002f;     // growth of the slab interval's upper end

enum { kMiss = 0, kHit = 1, kBand = 2 };

struct SegF {
    float3 s, d, inv;
    float3 olo, ohi;   // slab offsets of the lower / upper planes (see make_seg)
    float dl1;         // |d|_1
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
    // the padded slab [lo - pad, hi + pad] gives the parameters (lo - slo) inv
    // and (hi - shi) inv, slo = s + pad and shi = s - pad rounded outward.  Each
    // is evaluated as one FMA, b inv + o, with the offset o = -slo inv (or
    // -shi inv) rounded toward the conservative side: down for the plane the
    // segment enters through (the lower plane when inv >= 0, the upper one
    // otherwise), up for the plane it leaves through.  The FMA's exact sum is
    // then never inside (lo - slo) inv, so only its single rounding remains,
    // which the growth of the interval covers (see slab6).
    const float3 slo = make_float3(__fadd_ru(s.x, px), __fadd_ru(s.y, py), __fadd_ru(s.z, pz));
    const float3 shi = make_float3(__fsub_rd(s.x, px), __fsub_rd(s.y, py), __fsub_rd(s.z, pz));
    g.olo = make_float3(g.inv.x >= 0.0f ? __fmul_rd(-slo.x, g.inv.x) : __fmul_ru(-slo.x, g.inv.x),
                        g.inv.y >= 0.0f ? __fmul_rd(-slo.y, g.inv.y) : __fmul_ru(-slo.y, g.inv.y),
                        g.inv.z >= 0.0f ? __fmul_rd(-slo.z, g.inv.z) : __fmul_ru(-slo.z, g.inv.z));
    g.ohi = make_float3(g.inv.x >= 0.0f ? __fmul_ru(-shi.x, g.inv.x) : __fmul_rd(-shi.x, g.inv.x),
                        g.inv.y >= 0.0f ? __fmul_ru(-shi.y, g.inv.y) : __fmul_rd(-shi.y, g.inv.y),
                        g.inv.z >= 0.0f ? __fmul_ru(-shi.z, g.inv.z) : __fmul_rd(-shi.z, g.inv.z));
    return g;
}

// Three-input minimum / maximum (one instruction on sm_100 and later).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Does the segment pass through the padded box?  One FMA per plane (the
// offsets of make_seg) gives the entry and exit parameters per axis; the
// segment's part [0, 1] of the line meets the box when
//     max(tn, 0) <= min(tf, 1) x kSlabGrow.
// Each computed parameter is within one rounding (relative 2^-24) of the
// exact one, on the conservative side of the padded plane, so whenever the
// exact interval [max(tn, 0), min(tf, 1)] is non-empty the computed left
// side is at most (1 + 2^-24) / (1 - 2^-24) times the right one before the
// growth, well inside kSlabGrow (2e-6): no box the segment meets is culled.
__device__ __forceinline__ bool slab6(float xlo, float ylo, float zlo, float xhi, float yhi, float zhi,
                                      const SegF& g) {
    const float t0x = fmaf(xlo, g.inv.x, g.olo.x), t1x = fmaf(xhi, g.inv.x, g.ohi.x);
    const float t0y = fmaf(ylo, g.inv.y, g.olo.y), t1y = fmaf(yhi, g.inv.y, g.ohi.y);
    const float t0z = fmaf(zlo, g.inv.z, g.olo.z), t1z = fmaf(zhi, g.inv.z, g.ohi.z);
    const float tn = fmaxf(max3f(fminf(t0x, t1x), fminf(t0y, t1y), fminf(t0z, t1z)), 0.0f);
    const float tf = fminf(min3f(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fmaxf(t0z, t1z)), 1.0f);
    return tn <= tf * kSlabGrow;
}
__device__ __forceinline__ bool slab(const float4& bmin, const float4& bmax, const SegF& g) {
    return slab6(bmin.x, bmin.y, bmin.z, bmax.x, bmax.y, bmax.z, g);
}
// The same test, also giving the length of the parameter interval inside the box.
__device__ __forceinline__ bool slab_len(const float4& bmin, const float4& bmax, const SegF& g, float& len) {
    const float t0x = fmaf(bmin.x, g.inv.x, g.olo.x), t1x = fmaf(bmax.x, g.inv.x, g.ohi.x);
    const float t0y = fmaf(bmin.y, g.inv.y, g.olo.y), t1y = fmaf(bmax.y, g.inv.y, g.ohi.y);
    const float t0z = fmaf(bmin.z, g.inv.z, g.olo.z), t1z = fmaf(bmax.z, g.inv.z, g.ohi.z);
    const float tn = fmaxf(max3f(fminf(t0x, t1x), fminf(t0y, t1y), fminf(t0z, t1z)), 0.0f);
    const float tf = fminf(min3f(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fmaxf(t0z, t1z)), 1.0f);
    len = tf - tn;
    return tn <= tf * kSlabGrow;
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
//
// For a certain hit, `tlo`/`thi` (when given) receive bounds of the exact t
// (numerator and denominator bounds divided with directed rounding), and
// `tplain` the plain FP32 t of a plain hit.
__device__ __forceinline__ int tri_fp32(const SegF& g, const Tri& tr, bool want_plain, bool& plain_hit,
                                        float* tlo = nullptr, float* thi = nullptr, float* tplain = nullptr) {
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
        if (tplain) *tplain = t;
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
        if (Us - errU > lim && Vs - errV > lim && Ws - errW > lim && Ts - errT > lim && Tms - errTm > lim) {
            if (tlo) {   // 0 < Ts - errT <= Ts_exact, 0 < D - errdet <= D_exact
                *tlo = __fdiv_rd(__fsub_rd(Ts, errT), __fadd_ru(D, errdet));
                *thi = __fdiv_ru(__fadd_ru(Ts, errT), __fsub_rd(D, errdet));
            }
            return kHit;
        }
        if (Us + errU < -lim || Vs + errV < -lim || Ws + errW < -lim || Ts + errT < -lim || Tms + errTm < -lim)
            return kMiss;
    }
    return kBand;
}

// tri_fp32's certain-hit decision alone (true exactly when tri_fp32 returns
// kHit), for the proposal's verification: the numerators come first and a
// pair whose signs already rule out a hit (a certain hit needs Us, Vs, Ws,
// Ts and D - Ts all above their bounds, so all positive) is rejected before
// any error bound is formed.
__device__ __forceinline__ bool tri_certain_hit(const SegF& g, const Tri& tr) {
    const float3 a = f3(tr.v0);
    const float3 e1 = sub3(f3(tr.v1), a), e2 = sub3(f3(tr.v2), a);
    const float3 sv = sub3(g.s, a);
    const float3 p = cross3(g.d, e2);
    const float det = dot3(e1, p);
    const float3 q = cross3(sv, e1);
    const float T = dot3(e2, q);
    const float U = dot3(sv, p), V = dot3(g.d, q);
    const float D = fabsf(det);
    const float sg = det > 0.0f ? 1.0f : -1.0f;
    const float Us = sg * U, Vs = sg * V, Ts = sg * T;
    const float Ws = D - Us - Vs;
    const float Tms = D - Ts;
    if (!(Us > 0.0f && Vs > 0.0f && Ws > 0.0f && Ts > 0.0f && Tms > 0.0f)) return false;
    const float3 ad = abs3(g.d), ae1 = abs3(e1), ae2 = abs3(e2), asv = abs3(sv);
    const float3 pa = cross_abs(ad, ae2), qa = cross_abs(asv, ae1);
    const float errdet = kErrK * dot3(ae1, pa) + 1e-35f;
    const float thr = kTauHi * (g.dl1 * (ae1.x + ae1.y + ae1.z)) * (ae2.x + ae2.y + ae2.z) * 1.000001f;
    if (!(D - errdet > thr)) return false;   // |det_rel| > tau not certain
    const float errT = kErrK * dot3(ae2, qa) + 1e-35f;
    const float errTm = errT + errdet + 2.0f * kU * (fabsf(T) + fabsf(det));
    const float errU = kErrK * dot3(asv, pa) + 1e-35f;
    const float errV = kErrK * dot3(ad, qa) + 1e-35f;
    const float errW = errdet + errU + errV + 2.0f * kU * (D + fabsf(U) + fabsf(V));
    const float lim = kTauHi * (D + errdet) * 1.000001f;
    return Us - errU > lim && Vs - errV > lim && Ws - errW > lim && Ts - errT > lim && Tms - errTm > lim;
}

// 32-byte read-only load (sm_100 and later): one lane reads one whole L1
// sector in a single request instead of two 16-byte halves.  p must be
// 32-byte aligned (nodes and triangles are 64-byte aligned).
__device__ __forceinline__ void ld32B(const void* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

__device__ __forceinline__ void load_node(const Node* __restrict__ nodes, int i, float4& a, float4& b, float4& c,
                                          float4& d) {
    const float4* p = reinterpret_cast<const float4*>(nodes + i);
    ld32B(p, a, b);
    ld32B(p + 2, c, d);
}

__device__ __forceinline__ Tri load_tri(const Tri* __restrict__ tris, int j) {
    const float4* p = reinterpret_cast<const float4*>(tris + j);
    Tri t;
    ld32B(p, t.v0, t.v1);
    ld32B(p + 2, t.v2, t.pad);
    return t;
}

__device__ __forceinline__ void raise_error(DevCounters* c, int code) { atomicCAS(&c->error, 0, code); }

__device__ __forceinline__ bool bad3(float3 a) {
    return !(isfinite(a.x) && isfinite(a.y) && isfinite(a.z));
}

// First leaf of proposal cluster c: the clusters are 256 equal ranges of
// the Morton-ordered leaves, cluster(leaf j) = floor(256 j / n_tri).
__device__ __forceinline__ int cluster_begin(int c, int64_t n_tri) { return (int)(((int64_t)c * n_tri + 255) / 256); }

}  // namespace segtest
}  // namespace rsi
