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
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "rsi_internal.cuh"
#include "segtest.cuh"

namespace rsi {

// [traversal kernel: begin] (data layout, device helpers and the FP32 traversal kernel)
struct QueryArgs {
    const Node* nodes;
    const Node4* nodes4;   // four-wide nodes of the same hierarchy
    const NodeQ* nodesq;   // compressed child-pair nodes (single queries)
    const Tri* tris;
    int64_t n_tri;
    const float* from;
    const float* to;
    int64_t n_rays;
    uint8_t* hit;
    int32_t* count;
    uint8_t* amb;
    int32_t* near;         // nearest mode: leaf of the nearest hit, -1 none (ids after k_nearest_finish)
    int32_t* band_ids;
    const int32_t* perm;   // traversal order of the segments, or NULL
    const int* n_dev;      // number of segments read from device memory, or NULL
    DevCounters* ctr;
    float dmax0, dmax1, dmax2;
    int fp32_only;
    int amb_bits;          // RSI_BOTH (count pass): amb = boolean-mode flag | count-mode flag << 1
    unsigned int* done;    // host-buffer queries (the DONE traversal): finished segments per output
                           // chunk of 2^done_shift, in device memory the host polls with copies
    int done_shift;
};

// One (hierarchy, segment batch, outputs) triple of a batched query.
struct BatchDesc {
    const Node* nodes;
    const Node4* nodes4;
    const Tri* tris;
    const float* from;
    const float* to;
    uint8_t* hit;
    int32_t* count;
    uint8_t* amb;
    int n_tri;
    int n_rays;
    int ray_begin;   // first global segment index of this batch
    float dmax0, dmax1, dmax2;
};

struct BatchArgs {
    const BatchDesc* desc;
    const int* begins;   // [n_batches + 1] prefix of the batch sizes
    int n_batches;
    int total;
    long long timeout_ns;
    int streamed;        // 1: segments become available as the host posts them
    const int32_t* perm; // [total] batch-local segment of each global index (in-tile reordering), or NULL
};

namespace {

using namespace segtest;   // FP32 segment, box and triangle tests (segtest.cuh)


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

// Host-buffer queries: finished segments are counted per output chunk into
// device counters that the host polls (by copying them out) to copy out the
// chunks already answered.  A lane notes its finished segments in two
// (chunk, count) slots; the warp adds them up per chunk and posts them
// together, once a slot of some lane holds 64 or the second slot is in use,
// and at the end: a warp barrier, then one fence by the posting lane (which
// makes the warp's result writes visible at GPU scope, where the copy engine
// reads them, before the count) and one atomic per chunk.
struct DoneSlots {
    int c0 = -1, c1 = -1;
    unsigned n0 = 0, n1 = 0;
};
__device__ __forceinline__ void done_note(const QueryArgs& A, int64_t r, DoneSlots& d) {
    const int k = (int)(r >> A.done_shift);
    if (d.n0 == 0 || k == d.c0) {
        d.c0 = k;
        ++d.n0;
    } else if (d.n1 == 0 || k == d.c1) {
        d.c1 = k;
        ++d.n1;
    } else {   // a third chunk before the warp's next post (rare): posted alone
        __threadfence();
        atomicAdd(A.done + k, 1u);
    }
}
__device__ __forceinline__ void done_post_slot(const QueryArgs& A, int c, unsigned n, int lane) {
    const unsigned m = __match_any_sync(0xffffffffu, n ? c : -1);
    const unsigned sum = __reduce_add_sync(m, n);
    if (n && lane == __ffs(m) - 1) {
        __threadfence();
        atomicAdd(A.done + c, sum);
    }
}
// All lanes of the warp call it (converged); `force` posts whatever is held.
__device__ __forceinline__ void done_post(const QueryArgs& A, DoneSlots& d, int lane, bool force) {
    const bool want = force ? (d.n0 | d.n1) != 0 : (d.n1 != 0 || d.n0 >= 64);
    if (!__ballot_sync(0xffffffffu, want)) return;
    __syncwarp();   // the warp's result writes happen before the posting lanes' fences
    done_post_slot(A, d.c0, d.n0, lane);
    done_post_slot(A, d.c1, d.n1, lane);
    d = DoneSlots();
}

constexpr int kWarpChunk = 64;   // segments a warp takes per atomic
constexpr int kRefillMin = 4;    // refill once this many lanes of a warp are idle

// Batch holding global segment index gi: the last b with begins[b] <= gi.
__device__ __forceinline__ int find_batch(const BatchArgs& B, int gi) {
    int lo = 0, hi = B.n_batches - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(B.begins + mid) <= gi) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait (lane 0) until the host has posted segments up to `need`;
// false when the budget ran out (RSI_ERR_TIMEOUT is raised) or another warp
// already timed out.
__device__ __noinline__ bool wait_ready(DevCounters* c, unsigned long long need, long long budget_ns) {
    const unsigned long long t0 = global_ns();
    while (ld_acquire_u64(&c->ready) < need) {
        if (*(volatile int*)&c->error == RSI_ERR_TIMEOUT) return false;
        if ((long long)(global_ns() - t0) > budget_ns) {
            atomicCAS(&c->error, 0, RSI_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(1000);
    }
    return true;
}

constexpr int kLeafMin = 10;     // run the triangle tests once this many lanes hold one
constexpr int kNodeSteps = 4;    // node steps per round of the traversal loop
constexpr int kSharedStack = 32; // a stack of this depth lives in shared memory
constexpr int kDone = 0x7FFFFFFF;  // "no next node" (node indices stay below 2^30)

// Dynamic shared memory of a traversal launch: the 32-entry stacks of the
// block's threads, else none.
inline size_t trav_smem_bytes(int stack, int block) {
    return stack == kSharedStack ? sizeof(int) * (size_t)kSharedStack * (size_t)block : 0;
}

// Warp-coherent persistent traversal with deferred leaf tests.  In the
// boolean mode, when both children pass, the walk goes first into the one
// whose box holds the longer stretch of the segment (a hit there is more
// likely, and the first certain hit ends the segment).  Each lane
// holds its next reference (internal node >= 0, leaf ~j < 0, or kDone) and a
// one-entry leaf slot.  Every iteration a lane whose next reference is an
// internal node fetches it and tests both child boxes (the nearer-listed hit
// child becomes next, the other is pushed; leaves travel as references too);
// a lane whose next reference is a leaf parks it in its slot if the slot is
// free.  The warp runs the triangle tests of all parked leaves together once
// kLeafMin lanes hold one or no lane can move on without it, so node work and
// triangle work both run with most lanes active.  Lanes whose segment is done
// are refilled together from a per-warp chunk of segment indices (one atomic
// per chunk).  Each round of the loop runs kNodeSteps node steps (a lane
// parks the leaf it reaches between them), so the refill and leaf-phase
// ballots are paid once per round; the child-pair step updates the walk
// with selects rather than branches.  A 32-entry stack lives in shared
// memory, one column per thread ([entry][thread]: a warp's accesses are
// free of bank conflicts whatever the lanes' depths), deeper ones in local
// memory.  A segment with a band pair and no certain answer is queued for
// k_query_fp64 (count and nearest modes stop at the first band pair).  The
// nearest mode visits every pair like the count mode and keeps the certain
// hit with the smallest upper bound on t; the answer is certain when every
// other certain hit's lower bound lies above it, else the segment is queued.
//
// NW 1: the node step fetches four-wide nodes (Node4): up to four child boxes
// per fetch; the first child that passes becomes next and the others are
// pushed, so children are still visited in leaf order.  NW 2: compressed
// child-pair nodes (NodeQ, one 32-byte load); the child boxes are rebuilt
// with outward rounding, so they contain the exact ones, and the walk is the
// child-pair walk.  NW 0: child-pair nodes (Node).
#ifndef RSI_TRAV_MIN_BLOCKS
#define RSI_TRAV_MIN_BLOCKS 4   // resident 256-thread blocks per SM the register budget is sized for
#endif
template <int MODE, bool STATS, int STACK, bool BATCHED, int NW, bool DONE = false>
__global__ void __launch_bounds__(256, BATCHED ? 3 : RSI_TRAV_MIN_BLOCKS) k_query_fp32(QueryArgs A, BatchArgs B) {
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int n_rays = BATCHED ? B.total : (A.n_dev ? *A.n_dev : (int)A.n_rays);
    // BATCHED: the lane's batch and its hierarchy (uniform kernel arguments otherwise)
    int l_batch = 0, l_ntri = 0;
    const Node* l_nodes = nullptr;
    const Node4* l_nodes4 = nullptr;
    const Tri* l_tris = nullptr;
    unsigned long long visits = 0, tests = 0;
    int wbase = 0, wend = 0;     // warp-uniform chunk [wbase, wend)
    bool exhausted = false;      // warp-uniform
    int ray = -1;
    SegF g;
    // traversal stack: the top entry is cached in a register (`top`, kDone =
    // empty) so that a pop hands over the next node at once; the entries
    // below it live in shared memory (STACK == kSharedStack: entry i of this
    // thread at s_stack[i * blockDim.x + threadIdx.x]) or local memory
    int next = kDone, slot = -1, sp = 0, top = kDone;
    extern __shared__ int s_stack[];
    constexpr bool kShared = STACK == kSharedStack;
    int l_stack[kShared ? 1 : STACK];
    int* const s_col = s_stack + threadIdx.x;
    const int s_stride = blockDim.x;
#define RSI_STK(i) (*(kShared ? s_col + (i) * s_stride : &l_stack[(i)]))
    int cnt = 0, plain_cnt = 0;
    bool found = false, band = false, stop = false;
    // nearest mode: best certain hit (leaf n1, t in [lo1, hi1]), smallest lower
    // bound m2 of the other certain hits, and the plain FP32 nearest (fp32_only)
    int n1 = -1, pbest = -1;
    float lo1 = 0.0f, hi1 = 0.0f, m2 = 0.0f, pbt = 0.0f;
    DoneSlots dn;   // DONE (host-buffer queries): the lane's finished segments not yet posted
    while (true) {
        if (DONE) done_post(A, dn, lane, false);
        unsigned idle = __ballot_sync(kFull, ray < 0);
        bool refilled = false;
        if (!exhausted && (__popc(idle) >= kRefillMin || idle == kFull)) {
            refilled = true;
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
                    // in 64 bits: the last chunk of a batch near 2^31 segments must not wrap
                    wend = (int)min((long long)wbase + kWarpChunk, (long long)n_rays);
                    if (B.streamed) {   // device work queue fed by the host (batched plans, host-buffer queries)
                        bool ok = true;
                        if (lane == 0) ok = wait_ready(A.ctr, (unsigned long long)wend, B.timeout_ns);
                        if (!__shfl_sync(kFull, ok ? 1 : 0, 0)) {
                            exhausted = true;
                            break;
                        }
                    }
                }
                const int take = min(__popc(idle), wend - wbase);
                bool mine = false;
                if ((idle >> lane) & 1u) {
                    const int rank = __popc(idle & lt);
                    if (rank < take) {
                        if (BATCHED) {
                            const int gi = wbase + rank;
                            l_batch = find_batch(B, gi);
                            ray = B.perm ? __ldg(B.perm + gi) : gi - __ldg(B.begins + l_batch);
                        } else {
                            ray = A.perm ? __ldg(A.perm + wbase + rank) : wbase + rank;
                        }
                        mine = true;
                    }
                }
                wbase += take;
                if (mine) {
                    const int64_t r = ray;
                    const float* from = A.from;
                    const float* to = A.to;
                    float dm0 = A.dmax0, dm1 = A.dmax1, dm2 = A.dmax2;
                    if (BATCHED) {
                        const BatchDesc& bd = B.desc[l_batch];
                        from = bd.from;
                        to = bd.to;
                        dm0 = bd.dmax0;
                        dm1 = bd.dmax1;
                        dm2 = bd.dmax2;
                        l_nodes = bd.nodes;
                        l_nodes4 = bd.nodes4;
                        l_tris = bd.tris;
                        l_ntri = bd.n_tri;
                    }
                    float3 s = make_float3(__ldg(from + 3 * r), __ldg(from + 3 * r + 1), __ldg(from + 3 * r + 2));
                    float3 e = make_float3(__ldg(to + 3 * r), __ldg(to + 3 * r + 1), __ldg(to + 3 * r + 2));
                    if (bad3(s) || bad3(e)) {   // undefined answer: reported as ambiguous
                        uint8_t* hit = BATCHED ? B.desc[l_batch].hit : A.hit;
                        int32_t* count = BATCHED ? B.desc[l_batch].count : A.count;
                        uint8_t* amb = BATCHED ? B.desc[l_batch].amb : A.amb;
                        if (hit) hit[r] = 0;
                        if (MODE == RSI_COUNT) count[r] = 0;
                        if (MODE == RSI_NEAREST) A.near[r] = -1;
                        if (amb) amb[r] = A.amb_bits ? 3 : 1;
                        if (DONE) done_note(A, r, dn);
                        ray = -1;
                    } else {
                        g = make_seg(s, e, dm0, dm1, dm2);
                        next = (BATCHED ? l_ntri : A.n_tri) == 1 ? ~0 : 0;
                        slot = -1;
                        sp = 0;
                        top = kDone;
                        cnt = plain_cnt = 0;
                        found = band = stop = false;
                        if (MODE == RSI_NEAREST) {
                            n1 = pbest = -1;
                            lo1 = hi1 = m2 = pbt = __int_as_float(0x7f800000);
                        }
                    }
                }
                idle = __ballot_sync(kFull, ray < 0);
            }
        }
        const bool active = ray >= 0;
        const unsigned act = refilled ? __ballot_sync(kFull, active) : ~idle;
        if (act == 0) {
            if (exhausted) break;
            continue;
        }
#pragma unroll
        for (int step = 0; step < kNodeSteps; ++step) {
            // node step
            if (NW == 1 && active && next != kDone && next >= 0) {
                const float4* p = reinterpret_cast<const float4*>((BATCHED ? l_nodes4 : A.nodes4) + next);
                float4 xl, xh, yl, yh, zl, zh, rff, pad;
                ld32B(p, xl, xh);
                ld32B(p + 2, yl, yh);
                ld32B(p + 4, zl, zh);
                ld32B(p + 6, rff, pad);
                const int4 rf = make_int4(__float_as_int(rff.x), __float_as_int(rff.y), __float_as_int(rff.z),
                                          __float_as_int(rff.w));
                if (STATS) ++visits;
                const bool h0 = slab6(xl.x, yl.x, zl.x, xh.x, yh.x, zh.x, g);
                const bool h1 = slab6(xl.y, yl.y, zl.y, xh.y, yh.y, zh.y, g) && rf.y != kEmpty4;
                const bool h2 = slab6(xl.z, yl.z, zl.z, xh.z, yh.z, zh.z, g) && rf.z != kEmpty4;
                const bool h3 = slab6(xl.w, yl.w, zl.w, xh.w, yh.w, zh.w, g) && rf.w != kEmpty4;
                int nx = h3 ? rf.w : kDone;
                bool over = false;
#define RSI_PUSH_HIT(HC, RC)           \
    if (HC) {                          \
        if (nx != kDone) {             \
            if (top != kDone) {        \
                if (sp < STACK) {      \
                    RSI_STK(sp) = top; \
                    ++sp;              \
                } else {               \
                    over = true;       \
                }                      \
            }                          \
            top = nx;                  \
        }                              \
        nx = (RC);                     \
    }
                RSI_PUSH_HIT(h2, rf.z)
                RSI_PUSH_HIT(h1, rf.y)
                RSI_PUSH_HIT(h0, rf.x)
#undef RSI_PUSH_HIT
                if (over) {   // cannot happen with STACK >= 3 x the four-wide levels; queued
                    raise_error(A.ctr, RSI_ERR_STACK);
                    band = true;
                    stop = true;
                }
                if (nx != kDone) {
                    next = nx;
                } else {
                    next = top;
                    top = sp > 0 ? RSI_STK(sp - 1) : kDone;
                    sp = sp > 0 ? sp - 1 : 0;
                }
            }
            if (NW != 1 && active && next != kDone && next >= 0) {
                float4 lmin, lmax, rmin, rmax;
                int lref, rref;
                if (NW == 2) {
                    float4 fa, fb;
                    ld32B(reinterpret_cast<const float4*>(A.nodesq + next), fa, fb);
                    const unsigned meta = __float_as_uint(fa.w);
                    const float sx = __uint_as_float((meta & 0xFFu) << 23);
                    const float sy = __uint_as_float(((meta >> 8) & 0xFFu) << 23);
                    const float sz = __uint_as_float(((meta >> 16) & 0xFFu) << 23);
                    const unsigned w0 = __float_as_uint(fb.x), w1 = __float_as_uint(fb.y), w2 = __float_as_uint(fb.z);
                    const int split = __float_as_int(fb.w);
#define RSI_QB(W, K) __uint2float_rn(((W) >> (8 * (K))) & 0xFFu)
                    lmin = make_float4(__fmaf_rd(RSI_QB(w0, 0), sx, fa.x), __fmaf_rd(RSI_QB(w0, 1), sy, fa.y),
                                       __fmaf_rd(RSI_QB(w0, 2), sz, fa.z), 0.0f);
                    lmax = make_float4(__fmaf_ru(RSI_QB(w0, 3), sx, fa.x), __fmaf_ru(RSI_QB(w1, 0), sy, fa.y),
                                       __fmaf_ru(RSI_QB(w1, 1), sz, fa.z), 0.0f);
                    rmin = make_float4(__fmaf_rd(RSI_QB(w1, 2), sx, fa.x), __fmaf_rd(RSI_QB(w1, 3), sy, fa.y),
                                       __fmaf_rd(RSI_QB(w2, 0), sz, fa.z), 0.0f);
                    rmax = make_float4(__fmaf_ru(RSI_QB(w2, 1), sx, fa.x), __fmaf_ru(RSI_QB(w2, 2), sy, fa.y),
                                       __fmaf_ru(RSI_QB(w2, 3), sz, fa.z), 0.0f);
#undef RSI_QB
                    lref = (meta >> 24) & 1u ? ~split : split;
                    rref = (meta >> 25) & 1u ? ~(split + 1) : split + 1;
                } else {
                    load_node(BATCHED ? l_nodes : A.nodes, next, lmin, lmax, rmin, rmax);
                    lref = __float_as_int(lmin.w);
                    rref = __float_as_int(lmax.w);
                }
                if (STATS) ++visits;
                bool hl, hr;
                if (MODE == RSI_ANY_HIT) {   // boolean: the child the segment spends longer in first
                    float ll, lr;
                    hl = slab_len(lmin, lmax, g, ll);
                    hr = slab_len(rmin, rmax, g, lr);
                    if (hl && hr && lr > ll) {
                        const int tmp = lref;
                        lref = rref;
                        rref = tmp;
                    }
                } else {
                    hl = slab(lmin, lmax, g);
                    hr = slab(rmin, rmax, g);
                }
                // both children: go left, the right one becomes the cached top
                // and the old top is pushed; one child: go there; none: pop
                const bool both = hl && hr, any = hl || hr;
                const int t0 = top;
                if (both && t0 != kDone) {
                    if (sp < STACK) {
                        RSI_STK(sp) = t0;
                        ++sp;
                    } else {   // cannot happen with STACK > tree height; queued
                        raise_error(A.ctr, RSI_ERR_STACK);
                        band = true;
                        stop = true;
                    }
                }
                int popped = kDone;
                if (!any && sp > 0) {
                    --sp;
                    popped = RSI_STK(sp);
                }
                next = any ? (hl ? lref : rref) : t0;
                top = both ? rref : (any ? t0 : popped);
            }
            // park a leaf reference
            if (active && !stop && next < 0 && slot < 0) {
                slot = ~next;
                next = top;
                top = sp > 0 ? RSI_STK(sp - 1) : kDone;
                sp = sp > 0 ? sp - 1 : 0;
            }
        }   // node steps
        // leaf phase: all parked leaves of the warp at once, once kLeafMin
        // lanes hold one or no lane can move on without it
        const unsigned pend = __ballot_sync(kFull, active && slot >= 0);
        if (pend && (__popc(pend) >= kLeafMin ||
                     __ballot_sync(kFull, active && !stop && next != kDone && (next >= 0 || slot < 0)) == 0)) {
            if (slot >= 0) {
                if (STATS) ++tests;
                const Tri tr = load_tri(BATCHED ? l_tris : A.tris, slot);
                bool plain;
                float tlo, thi, tpl;
                const bool near = MODE == RSI_NEAREST;
                int c = tri_fp32(g, tr, A.fp32_only != 0, plain, near ? &tlo : nullptr, near ? &thi : nullptr,
                                 near ? &tpl : nullptr);
                plain_cnt += plain;
                if (near && plain && tpl < pbt) {
                    pbt = tpl;
                    pbest = slot;
                }
                if (c == kBand && !A.fp32_only) {   // settled by the FP64 pass
                    band = true;
                    if (MODE != RSI_ANY_HIT) stop = true;
                } else if (c == kHit) {
                    ++cnt;
                    if (MODE == RSI_ANY_HIT) {
                        found = true;
                        stop = true;
                    }
                    if (near) {
                        if (thi < hi1) {
                            m2 = fminf(m2, lo1);
                            n1 = slot;
                            lo1 = tlo;
                            hi1 = thi;
                        } else {
                            m2 = fminf(m2, tlo);
                        }
                    }
                }
                slot = -1;
            }
        }
        if (active && (stop || (next == kDone && slot < 0))) {
            const int64_t r = ray;
            uint8_t* hit = BATCHED ? B.desc[l_batch].hit : A.hit;
            int32_t* count = BATCHED ? B.desc[l_batch].count : A.count;
            uint8_t* amb = BATCHED ? B.desc[l_batch].amb : A.amb;
            if (A.fp32_only) {   // plain FP32 closed-interval decisions, no re-test
                if (MODE == RSI_ANY_HIT) hit[r] = (uint8_t)(found || plain_cnt > 0);
                else if (MODE == RSI_COUNT) {
                    count[r] = plain_cnt;
                    if (hit) hit[r] = (uint8_t)(plain_cnt > 0);
                } else {
                    A.near[r] = pbest;
                }
                if (amb) amb[r] = 0;
            } else if (MODE == RSI_ANY_HIT && found) {
                hit[r] = 1;
                if (amb) amb[r] = 0;
            } else if (band || (MODE == RSI_NEAREST && n1 >= 0 && !(m2 > hi1))) {
                int pos = atomicAdd(&A.ctr->band_count, 1);
                A.band_ids[pos] = BATCHED ? ray + __ldg(B.begins + l_batch) : ray;
            } else {
                if (MODE == RSI_ANY_HIT) hit[r] = 0;
                else if (MODE == RSI_COUNT) {
                    count[r] = cnt;
                    if (hit) hit[r] = (uint8_t)(cnt > 0);
                } else {
                    A.near[r] = n1;
                }
                if (amb) amb[r] = 0;
            }
            if (DONE) done_note(A, r, dn);
            ray = -1;
        }
    }
    if (DONE) done_post(A, dn, lane, true);
#undef RSI_STK
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

// [traversal kernel: end]

}  // namespace

// Scratch of the pair-parallel FP64 pass: the (segment, triangle) pairs that
// the FP32 test could not reject for certain, listed per queued segment
// ("band entry" k = position in the FP64 queue).
struct PairScratch {
    int32_t* seg_off;     // [seg_cap] first pair of band entry k
    int32_t* seg_cnt;     // [seg_cap] its number of pairs; -1: left to k_query_fp64
    int32_t* pair_seg;    // [pair_cap] band entry of pair i (-1: slot unused)
    int32_t* pair_leaf;   // [pair_cap] leaf (triangle in leaf order) of pair i
    double* pair_t;       // [pair_cap] t of pair i when it is an inclusive crossing
    uint8_t* pair_cls;    // [pair_cap] class of pair i, | 4 when inclusive, | 8 when its t is not computed
    int32_t* todo;        // [pair_cap] pairs for the FP64 classification
    int32_t* hard;        // [pair_cap] pairs the certain FP64 test left undecided
    int32_t* fb_ids;      // [queue capacity] segments left to k_query_fp64
    int seg_cap, pair_cap;
    int fp32_hits;        // 1: a certain FP32 hit is entered as a hit without the FP64 step
};

namespace {

// classify_fp64 evaluated by a whole warp on one pair (every lane passes the
// same pair and gets the same answer): the same FP64 operations, spread over
// the lanes.  On GB300 a warp's FP64 instruction occupies the FP64 pipe the
// same for 1 or 32 active lanes, so one pair's definition costs the warp
// about as much as 32 pairs' would; here the three norms, the three
// quotients and the distance terms run side by side.  The distance from the
// segment to the triangle is the smallest of: the distance of an end point
// to the triangle's plane where its projection falls inside the triangle,
// the nine point-to-segment distances between the end points and the edges
// and between the vertices and the segment, and the interior closest
// approaches of the segment and each edge -- the same set of terms whose
// minimum classify_fp64 takes (its point-to-triangle terms use the same
// point-to-edge distances), and a minimum does not depend on order.
__device__ int classify_fp64_warp(D3 s, D3 e, D3 a, D3 b, D3 c, double& t_out, bool& incl) {
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const double tau = kTauD;
    const D3 d = dsub(e, s);
    const D3 e1 = dsub(b, a), e2 = dsub(c, a);
    const D3 n = dcross(e1, e2);
    incl = false;
    t_out = 0.0;
    if ((d.x == 0.0 && d.y == 0.0 && d.z == 0.0) || (n.x == 0.0 && n.y == 0.0 && n.z == 0.0)) return kMiss;
    const D3 p = dcross(d, e2);
    const double det = ddot(e1, p);
    const D3 sv = dsub(s, a);
    const D3 q = dcross(sv, e1);
    // lanes 0-2: |d|, |e1|, |e2|; lanes 3-5: u, v, t
    const D3 nv = lane == 0 ? d : (lane == 1 ? e1 : e2);
    const double nrm = lane < 3 ? dnorm(nv) : 0.0;
    const D3 qa = lane == 3 ? sv : (lane == 4 ? d : e2);
    const D3 qb = lane == 3 ? p : q;
    const double quo = (lane >= 3 && lane < 6 && det != 0.0) ? __ddiv_rn(ddot(qa, qb), det) : 0.0;
    const double nd = __shfl_sync(kFull, nrm, 0), n1 = __shfl_sync(kFull, nrm, 1), n2 = __shfl_sync(kFull, nrm, 2);
    const double det_rel = __ddiv_rn(det, __dmul_rn(__dmul_rn(nd, n1), n2));
    double u = 0.0, v = 0.0, t = 0.0, w = 0.0;
    if (det != 0.0) {
        u = __shfl_sync(kFull, quo, 3);
        v = __shfl_sync(kFull, quo, 4);
        t = __shfl_sync(kFull, quo, 5);
        w = __dsub_rn(__dsub_rn(1.0, u), v);
        incl = (u >= 0.0 && v >= 0.0 && w >= 0.0 && t >= 0.0 && t <= 1.0);
    }
    t_out = t;
    if (fabs(det_rel) > tau) {
        if (u > tau && v > tau && w > tau && t > tau && t < 1.0 - tau) return kHit;
        if (u < -tau || v < -tau || w < -tau || t < -tau || t > 1.0 + tau) return kMiss;
        return kBand;   // ambiguous
    }
    if (incl) return kBand;   // distance 0, never above tau |d|
    // the distance terms: lanes 0-8 point to segment, 9-11 interior approaches, 12-13 planes
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    double dist = inf;
    if (lane < 9) {   // lanes 0-5: end point lane / 3 to edge lane % 3; 6-8: vertex lane - 6 to the segment
        const int ei = lane < 6 ? lane % 3 : lane - 6;
        const D3 v0 = ei == 0 ? a : (ei == 1 ? b : c), v1 = ei == 0 ? b : (ei == 1 ? c : a);
        const D3 pt = lane < 6 ? (lane < 3 ? s : e) : v0;
        dist = pt_seg(pt, lane < 6 ? v0 : s, lane < 6 ? v1 : e);
    } else if (lane < 12) {
        const int ei = lane - 9;
        const D3 q0 = ei == 0 ? a : (ei == 1 ? b : c), q1 = ei == 0 ? b : (ei == 1 ? c : a);
        const D3 uu = dsub(e, s), vv = dsub(q1, q0), w0 = dsub(s, q0);
        const double aa = ddot(uu, uu), bb = ddot(uu, vv), cc = ddot(vv, vv);
        const double dd = ddot(uu, w0), ee = ddot(vv, w0);
        const double den = __dsub_rn(__dmul_rn(aa, cc), __dmul_rn(bb, bb));
        if (den > 0.0) {
            const double ss = __ddiv_rn(__dsub_rn(__dmul_rn(bb, ee), __dmul_rn(cc, dd)), den);
            const double tt = __ddiv_rn(__dsub_rn(__dmul_rn(aa, ee), __dmul_rn(bb, dd)), den);
            if (ss >= 0.0 && ss <= 1.0 && tt >= 0.0 && tt <= 1.0) dist = dnorm(dsub(dadd(w0, dscale(uu, ss)), dscale(vv, tt)));
        }
    } else if (lane < 14) {
        const D3 pp = lane == 12 ? s : e;
        const D3 nn3 = dcross(dsub(b, a), dsub(c, a));
        const double nn = ddot(nn3, nn3);
        const double h = __ddiv_rn(ddot(dsub(pp, a), nn3), nn);
        const D3 proj = dsub(pp, dscale(nn3, h));
        const double s0 = ddot(dcross(dsub(b, a), dsub(proj, a)), nn3);
        const double s1 = ddot(dcross(dsub(c, b), dsub(proj, b)), nn3);
        const double s2 = ddot(dcross(dsub(a, c), dsub(proj, c)), nn3);
        if (s0 >= 0.0 && s1 >= 0.0 && s2 >= 0.0) dist = __dmul_rn(fabs(h), __dsqrt_rn(nn));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const double x = __shfl_xor_sync(kFull, dist, o);
        dist = x < dist ? x : dist;
    }
    return dist > __dmul_rn(tau, nd) ? kMiss : kBand;
}

// Ambiguity byte of a count-mode result.  In RSI_BOTH the count pass also
// answers the boolean mode: its hit flag (count > 0) is the boolean answer,
// and a segment is ambiguous for the boolean mode when it is for the count
// mode and no pair is a decisive hit (a decisive hit settles the boolean
// answer alone); bit 0 carries that flag, bit 1 the count mode's.
__device__ __forceinline__ uint8_t both_modes_amb(int amb_bits, bool amb, int n_decisive_hits) {
    if (!amb_bits) return (uint8_t)amb;
    return (uint8_t)((amb ? 2 : 0) | (amb && n_decisive_hits == 0 ? 1 : 0));
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
// segment counts distinct crossings (t merged within 1e-9).  The nearest
// mode keeps the inclusive hit of smallest (t, triangle id).
template <int MODE, int STACK, bool BATCHED>
__global__ void __launch_bounds__(128) k_query_fp64(QueryArgs A, BatchArgs B, const int* __restrict__ n_list) {
    constexpr int kWarps = 4;
    __shared__ double s_t[kWarps][kMaxInclusive];
    __shared__ int s_cand[kWarps][32];
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nb = *(volatile const int*)n_list;   // entries of A.band_ids to settle
    for (int k = blockIdx.x * kWarps + w; k < nb; k += gridDim.x * kWarps) {
        QueryArgs Q = A;   // this segment's hierarchy and outputs
        int64_t r = A.band_ids[k];
        if (BATCHED) {
            const int b = find_batch(B, (int)r);
            const BatchDesc& bd = B.desc[b];
            r -= __ldg(B.begins + b);
            Q.nodes = bd.nodes;
            Q.tris = bd.tris;
            Q.n_tri = bd.n_tri;
            Q.from = bd.from;
            Q.to = bd.to;
            Q.hit = bd.hit;
            Q.count = bd.count;
            Q.amb = bd.amb;
            Q.dmax0 = bd.dmax0;
            Q.dmax1 = bd.dmax1;
            Q.dmax2 = bd.dmax2;
        }
        const float3 s = make_float3(Q.from[3 * r], Q.from[3 * r + 1], Q.from[3 * r + 2]);
        const float3 e = make_float3(Q.to[3 * r], Q.to[3 * r + 1], Q.to[3 * r + 2]);
        const SegF g = make_seg(s, e, Q.dmax0, Q.dmax1, Q.dmax2);
        const D3 sd = {(double)s.x, (double)s.y, (double)s.z}, ed = {(double)e.x, (double)e.y, (double)e.z};
        int n_hit = 0, n_amb = 0, n_incl = 0;
        bool overflow = false;
        double best_t = __longlong_as_double(0x7ff0000000000000ll);   // nearest mode (lane 0)
        int best_id = 0x7FFFFFFF, best_leaf = -1;
        int node = 0, sp = 0;
        int stack[STACK];
        bool trav_done = false;
        while (true) {
            int nc = 0;
            if (lane == 0) {
                if (Q.n_tri == 1) {
                    s_cand[w][nc++] = 0;
                    trav_done = true;
                }
                while (!trav_done && nc <= 30) {
                    float4 lmin, lmax, rmin, rmax;
                    load_node(Q.nodes, node, lmin, lmax, rmin, rmax);
                    const int lref = __float_as_int(lmin.w), rref = __float_as_int(lmax.w);
                    bool hl = slab(lmin, lmax, g), hr = slab(rmin, rmax, g);
                    bool plain;
                    if (hl && lref < 0) {
                        hl = false;
                        if (tri_fp32(g, load_tri(Q.tris, ~lref), false, plain) != kMiss) s_cand[w][nc++] = ~lref;
                    }
                    if (hr && rref < 0) {
                        hr = false;
                        if (tri_fp32(g, load_tri(Q.tris, ~rref), false, plain) != kMiss) s_cand[w][nc++] = ~rref;
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
            int cls = -1, my_id = 0x7FFFFFFF;
            bool incl = false;
            double t = 0.0;
            if (lane < nc) {
                const Tri tr = load_tri(Q.tris, s_cand[w][lane]);
                my_id = __float_as_int(tr.v0.w);
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
            if (MODE == RSI_COUNT && incl) {
                const int pos = n_incl + __popc(mi & lt);
                if (pos < kMaxInclusive) s_t[w][pos] = t;
                else overflow = true;
            }
            if (MODE == RSI_NEAREST && mi) {   // warp minimum of (t, id) over the inclusive hits
                double bt = incl ? t : __longlong_as_double(0x7ff0000000000000ll);
                int bid = incl ? my_id : 0x7FFFFFFF;
                int bl = incl ? s_cand[w][lane] : -1;
                for (int off = 16; off; off >>= 1) {
                    const double ot = __shfl_xor_sync(kFull, bt, off);
                    const int oid = __shfl_xor_sync(kFull, bid, off);
                    const int ol = __shfl_xor_sync(kFull, bl, off);
                    if (ot < bt || (ot == bt && oid < bid)) {
                        bt = ot;
                        bid = oid;
                        bl = ol;
                    }
                }
                if (bt < best_t || (bt == best_t && bid < best_id)) {
                    best_t = bt;
                    best_id = bid;
                    best_leaf = bl;
                }
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
                Q.hit[r] = (uint8_t)(n_hit > 0 || (amb && n_incl > 0));
                if (Q.amb) Q.amb[r] = (uint8_t)amb;
                if (amb) atomicAdd(&A.ctr->ambiguous, 1ull);
            } else if (MODE == RSI_NEAREST) {
                Q.near[r] = best_leaf;
                if (Q.amb) Q.amb[r] = (uint8_t)(n_amb > 0);
                if (n_amb > 0) atomicAdd(&A.ctr->ambiguous, 1ull);
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
                Q.count[r] = count;
                if (Q.hit) Q.hit[r] = (uint8_t)(count > 0);
                if (Q.amb) Q.amb[r] = both_modes_amb(A.amb_bits, amb, n_hit);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- pair-parallel FP64 pass
// The same settlement of the queued segments as k_query_fp64 in three steps
// that keep the lanes busy: (1) the pairs of each queued segment are listed
// -- for queues of up to 32,767 segments by one warp per segment whose lanes
// walk the boxes together (every round each lane takes one node of the
// warp's node list), for longer queues (whose walks are long and many) by
// one thread per segment -- with the
// FP32 test on each reached leaf: a certain miss is dropped; with
// P.fp32_hits (boolean and count modes) a certain FP32 hit is entered as a
// hit at once, the FP32 test being sound, and only the undecided pairs are
// listed for step 2; (2) one thread per listed pair classifies it in FP64 --
// the certain numerator test, else the definition -- so FP64 instructions
// run with full warps (a warp's FP64 instruction costs the same however many
// lanes take part); (3) one thread per segment combines its pairs exactly as
// k_query_fp64 does; the count mode's ambiguous segments (whose distinct
// crossings need every crossing's t) are listed with the certain hits whose
// t is still to compute, one thread per such pair computes it, and one
// thread per listed segment counts the crossings.  Segments with more
// than kCandMax candidates, or that do not fit the scratch, go to
// k_query_fp64 through the fallback list.
constexpr int kCandMax = 32;
constexpr int kThreadQueue = 32768;   // from this queue length on, one thread per segment collects
constexpr uint8_t kTPending = 8;      // pair_cls flag: inclusive hit whose t is not computed yet

// Band entry gidx (a segment index, global over the batches when batched):
// its index r within its batch and that batch's hierarchy and outputs.
template <bool BATCHED>
__device__ __forceinline__ QueryArgs band_segment(const QueryArgs& A, const BatchArgs& B, int64_t gidx, int64_t& r) {
    QueryArgs Q = A;
    r = gidx;
    if (BATCHED) {
        const int b = find_batch(B, (int)gidx);
        const BatchDesc& bd = B.desc[b];
        r -= __ldg(B.begins + b);
        Q.nodes = bd.nodes;
        Q.nodes4 = bd.nodes4;
        Q.tris = bd.tris;
        Q.n_tri = bd.n_tri;
        Q.from = bd.from;
        Q.to = bd.to;
        Q.hit = bd.hit;
        Q.count = bd.count;
        Q.amb = bd.amb;
        Q.dmax0 = bd.dmax0;
        Q.dmax1 = bd.dmax1;
        Q.dmax2 = bd.dmax2;
    }
    return Q;
}

// Class byte of a listed candidate and whether it waits for the FP64 step.
__device__ __forceinline__ bool pair_preset(const PairScratch& P, bool fp32_hit, uint8_t& cls) {
    const bool pre = P.fp32_hits && fp32_hit;
    cls = pre ? (uint8_t)(kHit | 4 | kTPending) : (uint8_t)0;
    return !pre;
}

// Lanes in `want` append `item` to list[] (count in *counter), one atomic per warp.
__device__ __forceinline__ void warp_append(bool want, int32_t item, int32_t* list, int* counter) {
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(kFull, want);
    if (!m) return;
    int base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(kFull, base, __ffs(m) - 1);
    if (want) list[base + __popc(m & ((1u << lane) - 1u))] = item;
}

constexpr int kFront = 256;   // a warp's node list; a walk that needs more goes to k_query_fp64
template <bool BATCHED>
__global__ void __launch_bounds__(128, 12) k_band_collect(QueryArgs A, BatchArgs B, PairScratch P) {
    constexpr int kWarps = 4, kLeafBuf = 96;
    __shared__ int s_front[kWarps][kFront];     // nodes still to open
    __shared__ int s_leaf[kWarps][kLeafBuf];    // leaves whose box the segment passes, not yet tested
    __shared__ int s_cand[kWarps][kCandMax];    // leaves the FP32 test does not reject
    __shared__ uint8_t s_hit[kWarps][kCandMax]; // ... and whether it is a certain FP32 hit
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int nb = *(volatile int*)&A.ctr->band_count;
    if (nb >= kThreadQueue) return;   // k_band_collect_threads takes long queues
    for (int k = blockIdx.x * kWarps + w; k < nb; k += gridDim.x * kWarps) {
        int64_t r;
        const QueryArgs Q = band_segment<BATCHED>(A, B, A.band_ids[k], r);
        const float3 s = make_float3(Q.from[3 * r], Q.from[3 * r + 1], Q.from[3 * r + 2]);
        const float3 e = make_float3(Q.to[3 * r], Q.to[3 * r + 1], Q.to[3 * r + 2]);
        const SegF g = make_seg(s, e, Q.dmax0, Q.dmax1, Q.dmax2);
        bool over = k >= P.seg_cap;   // warp-uniform
        int nc = 0, nf = 0, nl = 0;                        // warp-uniform list lengths
        if (!over) {
            if (Q.n_tri == 1) {
                if (lane == 0) s_leaf[w][0] = 0;
                nl = 1;
            } else {
                if (lane == 0) s_front[w][0] = 0;
                nf = 1;
            }
        }
        __syncwarp();
        while (!over && (nf > 0 || nl > 0)) {
            if (nf > 0) {   // open up to 32 nodes, one per lane
                const int m = min(32, nf);
                const int node = lane < m ? s_front[w][nf - 1 - lane] : 0;
                nf -= m;
                __syncwarp();   // the entries are read before the pushes below overwrite them
                bool hl = false, hr = false;
                int lref = 0, rref = 0;
                if (lane < m) {
                    float4 lmin, lmax, rmin, rmax;
                    load_node(Q.nodes, node, lmin, lmax, rmin, rmax);
                    lref = __float_as_int(lmin.w);
                    rref = __float_as_int(lmax.w);
                    hl = slab(lmin, lmax, g);
                    hr = slab(rmin, rmax, g);
                }
                const unsigned il = __ballot_sync(kFull, hl && lref >= 0), ir = __ballot_sync(kFull, hr && rref >= 0);
                const unsigned ll = __ballot_sync(kFull, hl && lref < 0), lr = __ballot_sync(kFull, hr && rref < 0);
                const int npush = __popc(il) + __popc(ir), nleaf = __popc(ll) + __popc(lr);
                if (nf + npush > kFront) {
                    over = true;   // k_query_fp64 walks it with its own stack
                } else {
                    if ((il >> lane) & 1u) s_front[w][nf + __popc(il & lt)] = lref;
                    if ((ir >> lane) & 1u) s_front[w][nf + __popc(il) + __popc(ir & lt)] = rref;
                    if ((ll >> lane) & 1u) s_leaf[w][nl + __popc(ll & lt)] = ~lref;
                    if ((lr >> lane) & 1u) s_leaf[w][nl + __popc(ll) + __popc(lr & lt)] = ~rref;
                    nf += npush;
                    nl += nleaf;   // below 32 + 64 (tested below once 32 wait)
                }
                __syncwarp();
            }
            // the FP32 test on the reached leaves, 32 at a time, once 32 wait or the walk is over
            while (!over && (nl >= 32 || (nf == 0 && nl > 0))) {
                const int t = min(32, nl);
                int leaf = 0, cls = kMiss;
                if (lane < t) {
                    bool plain;
                    leaf = s_leaf[w][nl - 1 - lane];
                    cls = tri_fp32(g, load_tri(Q.tris, leaf), false, plain);
                }
                nl -= t;
                const unsigned mk = __ballot_sync(kFull, cls != kMiss);
                if (nc + __popc(mk) > kCandMax) {
                    over = true;
                } else {
                    if (cls != kMiss) {
                        s_cand[w][nc + __popc(mk & lt)] = leaf;
                        s_hit[w][nc + __popc(mk & lt)] = (uint8_t)(cls == kHit);
                    }
                    nc += __popc(mk);
                }
                __syncwarp();
            }
        }
        int base = -1;
        // reserve nc pairs; the counter is read first so that it cannot run far past the capacity
        if (lane == 0 && !over && *(volatile int*)&A.ctr->pair_count <= P.pair_cap - nc) {
            base = atomicAdd(&A.ctr->pair_count, nc);
            if (base > P.pair_cap - nc) {
                for (int i = base; i < P.pair_cap && i < base + nc; ++i) P.pair_seg[i] = -1;
                base = -1;
            }
        }
        base = __shfl_sync(kFull, base, 0);
        if (base >= 0) {
            bool undecided = false;
            if (lane < nc) {
                uint8_t cls;
                undecided = pair_preset(P, s_hit[w][lane] != 0, cls);
                P.pair_seg[base + lane] = k;
                P.pair_leaf[base + lane] = s_cand[w][lane];
                P.pair_cls[base + lane] = cls;
            }
            warp_append(undecided, base + lane, P.todo, &A.ctr->todo_count);
            if (lane == 0) {
                P.seg_off[k] = base;
                P.seg_cnt[k] = nc;
            }
        } else if (lane == 0) {
            if (k < P.seg_cap) P.seg_cnt[k] = -1;
            P.fb_ids[atomicAdd(&A.ctr->fb_count, 1)] = A.band_ids[k];
        }
        __syncwarp();
    }
}

// Step 1 for long queues: one thread per queued segment walks the tree and
// tests the reached leaves itself; the warp reserves its pairs and lists its
// undecided ones with one atomic each.
template <int STACK, bool BATCHED>
__global__ void __launch_bounds__(128) k_band_collect_threads(QueryArgs A, BatchArgs B, PairScratch P) {
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nb = *(volatile int*)&A.ctr->band_count;
    if (nb < kThreadQueue) return;   // k_band_collect takes short queues
    const int stride = gridDim.x * blockDim.x;
    for (int k0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); k0 < nb; k0 += stride) {   // warp-uniform
        const int k = k0 + lane;
        int cand[kCandMax];
        unsigned hits = 0;   // bit i: cand[i] is a certain FP32 hit
        int nc = 0;
        bool over = k >= P.seg_cap;
        if (k < nb && !over) {
            int64_t r;
            const QueryArgs Q = band_segment<BATCHED>(A, B, A.band_ids[k], r);
            const float3 s = make_float3(Q.from[3 * r], Q.from[3 * r + 1], Q.from[3 * r + 2]);
            const float3 e = make_float3(Q.to[3 * r], Q.to[3 * r + 1], Q.to[3 * r + 2]);
            const SegF g = make_seg(s, e, Q.dmax0, Q.dmax1, Q.dmax2);
            bool plain;
            if (Q.n_tri == 1) {
                const int c = tri_fp32(g, load_tri(Q.tris, 0), false, plain);
                if (c != kMiss) {
                    hits = c == kHit ? 1u : 0u;
                    cand[nc++] = 0;
                }
            } else {
                int node = 0, sp = 0;
                int stack[STACK];
                while (true) {
                    float4 lmin, lmax, rmin, rmax;
                    load_node(Q.nodes, node, lmin, lmax, rmin, rmax);
                    const int lref = __float_as_int(lmin.w), rref = __float_as_int(lmax.w);
                    bool hl = slab(lmin, lmax, g), hr = slab(rmin, rmax, g);
                    if (hl && lref < 0) {
                        hl = false;
                        const int c = tri_fp32(g, load_tri(Q.tris, ~lref), false, plain);
                        if (c != kMiss) {
                            if (nc == kCandMax) {
                                over = true;
                                break;
                            }
                            hits |= (c == kHit ? 1u : 0u) << nc;
                            cand[nc++] = ~lref;
                        }
                    }
                    if (hr && rref < 0) {
                        hr = false;
                        const int c = tri_fp32(g, load_tri(Q.tris, ~rref), false, plain);
                        if (c != kMiss) {
                            if (nc == kCandMax) {
                                over = true;
                                break;
                            }
                            hits |= (c == kHit ? 1u : 0u) << nc;
                            cand[nc++] = ~rref;
                        }
                    }
                    if (hl && hr) {
                        if (sp == STACK) {   // k_query_fp64 raises RSI_ERR_STACK for it
                            over = true;
                            break;
                        }
                        stack[sp++] = rref;
                        node = lref;
                    } else if (hl) {
                        node = lref;
                    } else if (hr) {
                        node = rref;
                    } else if (sp > 0) {
                        node = stack[--sp];
                    } else {
                        break;
                    }
                }
            }
        }
        // the warp's pairs: one reservation; if the scratch cannot take them all, every segment of
        // the warp goes to the fallback list (the counter is read first so that it cannot run far
        // past the capacity)
        const bool want = k < nb && !over;
        int incl = want ? nc : 0;   // inclusive scan of the pair counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        int base = -1;
        if (lane == 0 && total > 0 && *(volatile int*)&A.ctr->pair_count <= P.pair_cap - total) {
            base = atomicAdd(&A.ctr->pair_count, total);
            if (base > P.pair_cap - total) {
                for (int i = base; i < P.pair_cap && i < base + total; ++i) P.pair_seg[i] = -1;
                base = -1;
            }
        }
        base = total > 0 ? __shfl_sync(kFull, base, 0) : 0;
        const bool placed = want && base >= 0;
        int n_undec = 0;
        if (placed) {
            const int off = base + incl - nc;
            for (int i = 0; i < nc; ++i) {
                uint8_t cls;
                n_undec += pair_preset(P, (hits >> i) & 1u, cls) ? 1 : 0;
                P.pair_seg[off + i] = k;
                P.pair_leaf[off + i] = cand[i];
                P.pair_cls[off + i] = cls;
            }
            P.seg_off[k] = off;
            P.seg_cnt[k] = nc;
        } else if (k < nb) {
            if (k < P.seg_cap) P.seg_cnt[k] = -1;
        }
        // the undecided pairs, listed for step 2 (one reservation for the warp)
        int uincl = n_undec;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, uincl, o);
            if (lane >= o) uincl += v;
        }
        const int utotal = __shfl_sync(kFull, uincl, 31);
        if (utotal > 0) {
            int ubase = 0;
            if (lane == 0) ubase = atomicAdd(&A.ctr->todo_count, utotal);
            ubase = __shfl_sync(kFull, ubase, 0) + uincl - n_undec;
            if (placed) {
                const int off = base + incl - nc;
                for (int i = 0; i < nc; ++i)
                    if (!(P.fp32_hits && ((hits >> i) & 1u))) P.todo[ubase++] = off + i;
            }
        }
        warp_append(k < nb && !placed, k < nb ? A.band_ids[k] : 0, P.fb_ids, &A.ctr->fb_count);
    }
}

// Step 2a: the certain FP64 test of every listed pair (no division or square
// root unless the nearest mode needs the t of a certain hit; the count mode
// computes it in step 3 where needed).  The pairs this test leaves undecided
// are listed for step 2b, so that the long evaluation of the definition runs
// apart (k_band_classify_hard): a few of them one warp each, whose lanes
// share the work of one pair, many of them one thread each.
constexpr int kHardWarpMax = 2048;   // undecided pairs up to which each gets a warp
template <int MODE, bool BATCHED>
__global__ void __launch_bounds__(256) k_band_classify(QueryArgs A, BatchArgs B, PairScratch P) {
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int np = min(*(volatile int*)&A.ctr->todo_count, P.pair_cap);
    const int stride = gridDim.x * blockDim.x;
    for (int j0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); j0 < np; j0 += stride) {
        const int i = j0 + lane < np ? P.todo[j0 + lane] : -1;
        bool hard = false;
        if (i >= 0) {
            const int k = P.pair_seg[i];
            if (k >= 0) {
                int64_t r;
                const QueryArgs Q = band_segment<BATCHED>(A, B, A.band_ids[k], r);
                const D3 sd = {(double)Q.from[3 * r], (double)Q.from[3 * r + 1], (double)Q.from[3 * r + 2]};
                const D3 ed = {(double)Q.to[3 * r], (double)Q.to[3 * r + 1], (double)Q.to[3 * r + 2]};
                const Tri tr = load_tri(Q.tris, P.pair_leaf[i]);
                const D3 a = d3of(tr.v0), b = d3of(tr.v1), c = d3of(tr.v2);
                int cls = tri_certain64(sd, ed, a, b, c);
                double t = 0.0;
                bool incl = cls == kHit;
                if (cls == kHit && MODE == RSI_NEAREST) t = t_of_definition(sd, ed, a, b, c);
                hard = cls == kBand;   // settled by the definition in step 2b
                const bool pending = incl && MODE == RSI_COUNT;   // t of a certain hit: step 3, if needed
                P.pair_cls[i] = (uint8_t)(cls | (incl ? 4 : 0) | (pending ? kTPending : 0));
                P.pair_t[i] = t;
            }
        }
        const unsigned m = __ballot_sync(kFull, hard);
        if (m) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&A.ctr->hard_count, __popc(m));
            base = __shfl_sync(kFull, base, 0);
            if (hard) P.hard[base + __popc(m & ((1u << lane) - 1u))] = i;
        }
    }
}

// Step 2b: the definition itself (classify_fp64) for the undecided pairs:
// one warp per pair for short lists (the lanes share the pair's work), one
// thread per pair for long ones.
template <bool BATCHED>
__global__ void __launch_bounds__(128) k_band_classify_hard(QueryArgs A, BatchArgs B, PairScratch P) {
    const int nh = *(volatile int*)&A.ctr->hard_count;
    if (nh < kHardWarpMax) {
        const int lane = threadIdx.x & 31;
        const int warps = (gridDim.x * blockDim.x) >> 5;
        for (int h = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < nh; h += warps) {
            const int i = P.hard[h];
            int64_t r;
            const QueryArgs Q = band_segment<BATCHED>(A, B, A.band_ids[P.pair_seg[i]], r);
            const D3 sd = {(double)Q.from[3 * r], (double)Q.from[3 * r + 1], (double)Q.from[3 * r + 2]};
            const D3 ed = {(double)Q.to[3 * r], (double)Q.to[3 * r + 1], (double)Q.to[3 * r + 2]};
            const Tri tr = load_tri(Q.tris, P.pair_leaf[i]);
            double t = 0.0;
            bool incl = false;
            const int cls = classify_fp64_warp(sd, ed, d3of(tr.v0), d3of(tr.v1), d3of(tr.v2), t, incl);
            if (lane == 0) {
                P.pair_cls[i] = (uint8_t)(cls | (incl ? 4 : 0));
                P.pair_t[i] = t;
            }
        }
        return;
    }
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        const int i = P.hard[h];
        int64_t r;
        const QueryArgs Q = band_segment<BATCHED>(A, B, A.band_ids[P.pair_seg[i]], r);
        const D3 sd = {(double)Q.from[3 * r], (double)Q.from[3 * r + 1], (double)Q.from[3 * r + 2]};
        const D3 ed = {(double)Q.to[3 * r], (double)Q.to[3 * r + 1], (double)Q.to[3 * r + 2]};
        const Tri tr = load_tri(Q.tris, P.pair_leaf[i]);
        double t = 0.0;
        bool incl = false;
        const int cls = classify_fp64(sd, ed, d3of(tr.v0), d3of(tr.v1), d3of(tr.v2), t, incl);
        P.pair_cls[i] = (uint8_t)(cls | (incl ? 4 : 0));
        P.pair_t[i] = t;
    }
}

// Step 3, one thread per queued segment.  In the count mode an ambiguous
// segment (its distinct crossings need every crossing's t) is listed, and
// so are its certain hits whose t is not computed yet; k_band_tfix and
// k_band_crossings finish it.
template <int MODE, bool BATCHED>
__global__ void __launch_bounds__(128) k_band_reduce(QueryArgs A, BatchArgs B, PairScratch P) {
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nb = min(*(volatile int*)&A.ctr->band_count, P.seg_cap);
    const int stride = gridDim.x * blockDim.x;
    for (int k0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); k0 < nb; k0 += stride) {   // warp-uniform
        const int k = k0 + lane;
        const int cnt = k < nb ? P.seg_cnt[k] : -1;
        bool amb_count = false;   // an ambiguous count-mode segment, finished below
        if (cnt >= 0) {
            const int off = P.seg_off[k];
            int64_t r;
            const QueryArgs Q = band_segment<BATCHED>(A, B, A.band_ids[k], r);
            int n_hit = 0, n_amb = 0, n_incl = 0;
            double best_t = __longlong_as_double(0x7ff0000000000000ll);
            int best_id = 0x7FFFFFFF, best_leaf = -1;
            for (int j = 0; j < cnt; ++j) {
                const int c = P.pair_cls[off + j];
                n_hit += (c & 3) == kHit;
                n_amb += (c & 3) == kBand;
                if (c & 4) {
                    if (MODE == RSI_NEAREST) {
                        const double t = P.pair_t[off + j];
                        const int leaf = P.pair_leaf[off + j];
                        const int id = __float_as_int(Q.tris[leaf].v0.w);
                        if (t < best_t || (t == best_t && id < best_id)) {
                            best_t = t;
                            best_id = id;
                            best_leaf = leaf;
                        }
                    }
                    ++n_incl;
                }
            }
            if (MODE == RSI_ANY_HIT) {
                const bool amb = n_hit == 0 && n_amb > 0;
                Q.hit[r] = (uint8_t)(n_hit > 0 || (amb && n_incl > 0));
                if (Q.amb) Q.amb[r] = (uint8_t)amb;
                if (amb) atomicAdd(&A.ctr->ambiguous, 1ull);
            } else if (MODE == RSI_NEAREST) {
                Q.near[r] = best_leaf;
                if (Q.amb) Q.amb[r] = (uint8_t)(n_amb > 0);
                if (n_amb > 0) atomicAdd(&A.ctr->ambiguous, 1ull);
            } else if (n_amb > 0) {
                amb_count = true;
            } else {
                Q.count[r] = n_hit;
                if (Q.hit) Q.hit[r] = (uint8_t)(n_hit > 0);
                if (Q.amb) Q.amb[r] = both_modes_amb(A.amb_bits, false, n_hit);
            }
        }
        if (MODE != RSI_COUNT) continue;
        // the ambiguous segments and their pending t's, one reservation per warp each
        int npend = 0;
        if (amb_count)
            for (int j = 0; j < cnt; ++j) npend += (P.pair_cls[P.seg_off[k] + j] & kTPending) ? 1 : 0;
        int incl = npend;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        if (total > 0) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&A.ctr->tpend_count, total);
            base = __shfl_sync(kFull, base, 0) + incl - npend;
            if (npend > 0) {
                const int off = P.seg_off[k];
                for (int j = 0; j < cnt; ++j)
                    if (P.pair_cls[off + j] & kTPending) P.hard[base++] = off + j;
            }
        }
        warp_append(amb_count, k, P.todo, &A.ctr->amb_seg_count);
    }
}

// The t of the listed certain hits, one thread each, by the definition's operations.
template <bool BATCHED>
__global__ void __launch_bounds__(128) k_band_tfix(QueryArgs A, BatchArgs B, PairScratch P) {
    const int np = *(volatile int*)&A.ctr->tpend_count;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < np; j += gridDim.x * blockDim.x) {
        const int i = P.hard[j];
        int64_t r;
        const QueryArgs Q = band_segment<BATCHED>(A, B, A.band_ids[P.pair_seg[i]], r);
        const D3 sd = {(double)Q.from[3 * r], (double)Q.from[3 * r + 1], (double)Q.from[3 * r + 2]};
        const D3 ed = {(double)Q.to[3 * r], (double)Q.to[3 * r + 1], (double)Q.to[3 * r + 2]};
        const Tri tr = load_tri(Q.tris, P.pair_leaf[i]);
        P.pair_t[i] = t_of_definition(sd, ed, d3of(tr.v0), d3of(tr.v1), d3of(tr.v2));
    }
}

// The distinct crossings of each listed ambiguous segment (closed-interval
// reading: inclusive crossings whose t differ by more than 1e-9 count apart).
template <bool BATCHED>
__global__ void __launch_bounds__(128) k_band_crossings(QueryArgs A, BatchArgs B, PairScratch P) {
    const int na = *(volatile int*)&A.ctr->amb_seg_count;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < na; j += gridDim.x * blockDim.x) {
        const int k = P.todo[j];
        const int cnt = P.seg_cnt[k], off = P.seg_off[k];
        int64_t r;
        const QueryArgs Q = band_segment<BATCHED>(A, B, A.band_ids[k], r);
        // an inclusive crossing's t lies in [0, 1] (-0.0 included), where the
        // order of the bit patterns as integers is the order of the values
        // (-0.0 first, then equal to +0.0, which the merge below treats alike):
        // the sort compares integers, not FP64 values
        long long ts[kCandMax];
        int n_incl = 0, n_hit = 0;
        for (int i = 0; i < cnt; ++i) {
            const int c = P.pair_cls[off + i];
            n_hit += (c & 3) == kHit;
            if (c & 4) ts[n_incl++] = __double_as_longlong(P.pair_t[off + i]);
        }
        for (int i = 1; i < n_incl; ++i) {
            const long long x = ts[i];
            int k2 = i - 1;
            while (k2 >= 0 && ts[k2] > x) {
                ts[k2 + 1] = ts[k2];
                --k2;
            }
            ts[k2 + 1] = x;
        }
        int count = 0;
        for (int i = 0; i < n_incl; ++i)
            if (i == 0 || __dsub_rn(__longlong_as_double(ts[i]), __longlong_as_double(ts[i - 1])) > kTMerge) ++count;
        atomicAdd(&A.ctr->ambiguous, 1ull);
        Q.count[r] = count;
        if (Q.hit) Q.hit[r] = (uint8_t)(count > 0);
        if (Q.amb) Q.amb[r] = both_modes_amb(A.amb_bits, true, n_hit);
    }
}


// Barycentric-mode results (Sec. 1: the intersecting triangle, the distance
// to and the location of the nearest intersecting point) from the leaf the
// passes chose: t by the definition's own FP64 operations, the point
// s + t (e - s) and the distance t |e - s| from the start point, each rounded
// once to FP32; the leaf is replaced by the caller's triangle index.  No hit:
// triangle -1, t -1, distance -1, point NaN.  Two kernels: the first writes
// the segments without a hit and lists the hitting ones (in A.band_ids, free
// once the FP64 pass is over); the second evaluates the listed segments in
// full warps -- GB300 charges a warp's FP64 instruction the same for 1 or 32
// active lanes, and the hits are spread over the batch.
__global__ void __launch_bounds__(256) k_nearest_list(QueryArgs A, float* __restrict__ t_out,
                                                      float* __restrict__ point, float* __restrict__ dist) {
    __shared__ int s_warp[8];   // hits per warp, then the warp's first list slot
    __shared__ int s_base;
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the block's 256 segments per round (block-uniform loop: one list
    // reservation per block and round, so the counter is not a hot spot)
    for (int64_t b0 = blockIdx.x * (int64_t)blockDim.x; b0 < A.n_rays; b0 += stride) {
        const int64_t r = b0 + threadIdx.x;
        bool hit = false;
        if (r < A.n_rays) {
            int j = A.near[r];
            if (j >= A.n_tri) {   // no pass wrote this segment: reported, never dereferenced
                raise_error(A.ctr, RSI_ERR_INDEX);
                A.near[r] = j = -1;
            }
            hit = j >= 0;
            if (!hit) {
                const float qnan = __int_as_float(0x7fc00000);
                if (t_out) t_out[r] = -1.0f;
                if (dist) dist[r] = -1.0f;
                if (point) {
                    point[3 * r] = qnan;
                    point[3 * r + 1] = qnan;
                    point[3 * r + 2] = qnan;
                }
            }
        }
        const unsigned m = __ballot_sync(kFull, hit);
        if (lane == 0) s_warp[w] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                const int c = s_warp[k];
                s_warp[k] = tot;
                tot += c;
            }
            s_base = tot ? atomicAdd(&A.ctr->n_finish, tot) : 0;
        }
        __syncthreads();
        if (hit) A.band_ids[s_base + s_warp[w] + __popc(m & ((1u << lane) - 1u))] = (int32_t)r;
        __syncthreads();
    }
}

// ---- double-float arithmetic (a value is hi + lo, two FP32 numbers) with
// the error-free transformations of Knuth (two-sum), Dekker (fast two-sum)
// and the FMA product; explicit round-to-nearest operations keep the
// compiler from contracting or reassociating them.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_fast(float a, float b) {   // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
    const FF s = ff_two_sum(x.hi, y.hi);
    return ff_fast(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ FF ff_neg(FF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return ff_fast(p, e);
}
__device__ __forceinline__ FF ff_div(FF x, FF y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const FF r = ff_add(x, ff_neg(ff_mul({q1, 0.0f}, y)));
    return ff_fast(q1, __fdiv_rn(r.hi, y.hi));
}
__device__ __forceinline__ FF ff_sqrt(FF x) {
    const float s = __fsqrt_rn(x.hi);
    const FF r = ff_add(x, ff_neg(ff_mul({s, 0.0f}, {s, 0.0f})));
    return ff_fast(s, __fdiv_rn(r.hi, __fmul_rn(2.0f, s)));
}
__device__ __forceinline__ FF ff_diff(float a, float b) { return ff_two_sum(a, -b); }   // exact a - b

// Round-to-nearest FP32 of every real within r of v, when they all agree:
// v.hi (the FP32 nearest to v) provided |v.lo| + r stays below half the gap
// to v.hi's neighbours.
__device__ __forceinline__ bool ff_round_certain(FF v, float r, float& out) {
    const float h = v.hi;
    if (!(fabsf(h) >= 1.17549435e-38f) || !(fabsf(h) < 1e30f)) return false;   // zero, subnormal, huge
    const float up = fabsf(__int_as_float(__float_as_int(fabsf(h)) + 1) - fabsf(h));
    const float dn = fabsf(fabsf(h) - __int_as_float(__float_as_int(fabsf(h)) - 1));
    const float gap = fminf(up, dn);   // the smaller neighbour spacing
    if (!(__fadd_ru(fabsf(v.lo), r) < 0.5f * gap)) return false;
    out = h;
    return true;
}

// t, point and distance of a hitting segment in double-float, with a bound
// on their distance from the FP64 evaluation of the definition (t by the
// definition's operations, s + t d, t |d|): each of the FP64 and the
// double-float evaluations of T = e2.(sv x e1) and det = e1.(d x e2) is
// within c u M of the exact value, M the same expression in magnitudes and
// c u = 8 x 2^-53 (FP64: each elementary term at most eight roundings deep, the
// 2 % slack covering gamma_8) or 2^-40 (double-float:
// each operation within 2^-44 of its operands' magnitudes); the quotient
// and the point and distance formulas add their own rounding terms.  When
// every rounding is certain the FP32 results are written; false otherwise.
__device__ __forceinline__ bool nearest_ff(float3 s, float3 e, float3 a, float3 b, float3 c, float& t32, float& px,
                                           float& py, float& pz, float& d32) {
    const FF dx = ff_diff(e.x, s.x), dy = ff_diff(e.y, s.y), dz = ff_diff(e.z, s.z);
    const FF e1x = ff_diff(b.x, a.x), e1y = ff_diff(b.y, a.y), e1z = ff_diff(b.z, a.z);
    const FF e2x = ff_diff(c.x, a.x), e2y = ff_diff(c.y, a.y), e2z = ff_diff(c.z, a.z);
    const FF svx = ff_diff(s.x, a.x), svy = ff_diff(s.y, a.y), svz = ff_diff(s.z, a.z);
    // p = d x e2, det = e1 . p, q = sv x e1, T = e2 . q
    const FF p0 = ff_add(ff_mul(dy, e2z), ff_neg(ff_mul(dz, e2y)));
    const FF p1 = ff_add(ff_mul(dz, e2x), ff_neg(ff_mul(dx, e2z)));
    const FF p2 = ff_add(ff_mul(dx, e2y), ff_neg(ff_mul(dy, e2x)));
    const FF det = ff_add(ff_add(ff_mul(e1x, p0), ff_mul(e1y, p1)), ff_mul(e1z, p2));
    const FF q0 = ff_add(ff_mul(svy, e1z), ff_neg(ff_mul(svz, e1y)));
    const FF q1 = ff_add(ff_mul(svz, e1x), ff_neg(ff_mul(svx, e1z)));
    const FF q2 = ff_add(ff_mul(svx, e1y), ff_neg(ff_mul(svy, e1x)));
    const FF T = ff_add(ff_add(ff_mul(e2x, q0), ff_mul(e2y, q1)), ff_mul(e2z, q2));
    // magnitudes (FP32 from the leading parts, with slack for their own rounding)
    const float adx = fabsf(dx.hi), ady = fabsf(dy.hi), adz = fabsf(dz.hi);
    const float a1x = fabsf(e1x.hi), a1y = fabsf(e1y.hi), a1z = fabsf(e1z.hi);
    const float a2x = fabsf(e2x.hi), a2y = fabsf(e2y.hi), a2z = fabsf(e2z.hi);
    const float asx = fabsf(svx.hi), asy = fabsf(svy.hi), asz = fabsf(svz.hi);
    const float Md = 1.001f * (a1x * (ady * a2z + adz * a2y) + a1y * (adz * a2x + adx * a2z) + a1z * (adx * a2y + ady * a2x));
    const float MT = 1.001f * (a2x * (asy * a1z + asz * a1y) + a2y * (asz * a1x + asx * a1z) + a2z * (asx * a1y + asy * a1x));
    const float cu = 8.0f * 1.1102230e-16f + 9.0949470e-13f;   // 8 x 2^-53 + 2^-40
    const float D = fabsf(det.hi);
    if (!(cu * Md < 0.01f * D)) return false;
    const FF t = ff_div(T, det);
    const float at = fabsf(t.hi);
    const float rt = 1.02f * (cu * (MT + at * Md) / D + (1.1102230e-16f + 9.0949470e-13f) * at);
    const FF px_ = ff_add({s.x, 0.0f}, ff_mul(dx, t));
    const FF py_ = ff_add({s.y, 0.0f}, ff_mul(dy, t));
    const FF pz_ = ff_add({s.z, 0.0f}, ff_mul(dz, t));
    const FF nrm = ff_sqrt(ff_add(ff_add(ff_mul(dx, dx), ff_mul(dy, dy)), ff_mul(dz, dz)));
    const FF dist = ff_mul(t, nrm);
    const float cp = 1.8189894e-12f;   // 2^-39: the FP64 and double-float rounding of s + t d and of t |d|
    const float rpx = 1.02f * (adx * rt + cp * (fabsf(s.x) + adx * at));
    const float rpy = 1.02f * (ady * rt + cp * (fabsf(s.y) + ady * at));
    const float rpz = 1.02f * (adz * rt + cp * (fabsf(s.z) + adz * at));
    const float rd = 1.02f * (fabsf(nrm.hi) * rt + cp * fabsf(dist.hi));
    return ff_round_certain(t, rt, t32) && ff_round_certain(px_, rpx, px) && ff_round_certain(py_, rpy, py) &&
           ff_round_certain(pz_, rpz, pz) && ff_round_certain(dist, rd, d32);
}

// The listed hitting segments: double-float with certified rounding, the
// rest (rare) listed for the FP64 evaluation.
__global__ void __launch_bounds__(256) k_nearest_finish_ff(QueryArgs A, float* __restrict__ t_out,
                                                           float* __restrict__ point, float* __restrict__ dist,
                                                           int32_t* __restrict__ list64) {
    const int nf = *(volatile int*)&A.ctr->n_finish;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
        const int64_t r = A.band_ids[i];
        const int j = A.near[r];
        const Tri tr = load_tri(A.tris, j);
        const float3 s = make_float3(A.from[3 * r], A.from[3 * r + 1], A.from[3 * r + 2]);
        const float3 e = make_float3(A.to[3 * r], A.to[3 * r + 1], A.to[3 * r + 2]);
        float t32, px, py, pz, d32;
        if (nearest_ff(s, e, f3(tr.v0), f3(tr.v1), f3(tr.v2), t32, px, py, pz, d32)) {
            if (t_out) t_out[r] = t32;
            if (dist) dist[r] = d32;
            if (point) {
                point[3 * r] = px;
                point[3 * r + 1] = py;
                point[3 * r + 2] = pz;
            }
            A.near[r] = __float_as_int(tr.v0.w);
        } else {
            list64[atomicAdd(&A.ctr->n_finish64, 1)] = (int32_t)r;
        }
    }
}

// FP64 evaluation of the definition for the listed segments (list, *n_list).
__global__ void __launch_bounds__(256) k_nearest_finish(QueryArgs A, float* __restrict__ t_out,
                                                        float* __restrict__ point, float* __restrict__ dist,
                                                        const int32_t* __restrict__ list,
                                                        const int* __restrict__ n_list) {
    const int nf = *(volatile const int*)n_list;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
        const int64_t r = list[i];
        const int j = A.near[r];
        const Tri tr = load_tri(A.tris, j);
        const D3 sd = {(double)A.from[3 * r], (double)A.from[3 * r + 1], (double)A.from[3 * r + 2]};
        const D3 ed = {(double)A.to[3 * r], (double)A.to[3 * r + 1], (double)A.to[3 * r + 2]};
        const double t = t_of_definition(sd, ed, d3of(tr.v0), d3of(tr.v1), d3of(tr.v2));
        const D3 d = dsub(ed, sd);
        const D3 p = dadd(sd, dscale(d, t));
        if (t_out) t_out[r] = __double2float_rn(t);
        if (dist) dist[r] = __double2float_rn(__dmul_rn(t, dnorm(d)));
        if (point) {
            point[3 * r] = __double2float_rn(p.x);
            point[3 * r + 1] = __double2float_rn(p.y);
            point[3 * r + 2] = __double2float_rn(p.z);
        }
        A.near[r] = __float_as_int(tr.v0.w);
    }
}

// Stream compaction of the hitting segments in index order (the paper's
// barycentric result lists only the intersecting rays): per-tile counts, one
// exclusive scan, and an ordered scatter.  A block takes a 4096-segment tile
// in 16 rounds of 256 consecutive segments.
constexpr int kCompactPer = 16;
constexpr int kCompactTile = 256 * kCompactPer;

__device__ __forceinline__ int block_exclusive_scan256(int v, int* wsum, int& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = v;
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int pre = 0;
    total = 0;
    for (int k = 0; k < 8; ++k) {
        if (k < w) pre += wsum[k];
        total += wsum[k];
    }
    __syncthreads();
    return pre + inc - v;
}

// Segment r of a tile is t0 + k * 256 + thread (k < kCompactPer): each
// round of the block reads 256 consecutive entries (coalesced).
__global__ void __launch_bounds__(256) k_compact_count(const int32_t* __restrict__ tri, int64_t n,
                                                       int* __restrict__ tile_count) {
    __shared__ int wsum[8];
    const int64_t t0 = (int64_t)blockIdx.x * kCompactTile;
    int c = 0;
    for (int k = 0; k < kCompactPer; ++k) {
        const int64_t r = t0 + k * 256 + threadIdx.x;
        if (r < n && tri[r] >= 0) ++c;
    }
    int total;
    block_exclusive_scan256(c, wsum, total);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = total;
}

// One block: tile counts -> exclusive offsets (in place), total in *n_out.
__global__ void __launch_bounds__(256) k_compact_scan(int* __restrict__ tile_count, int n_tiles,
                                                      long long* __restrict__ n_out) {
    __shared__ int wsum[8];
    int carry = 0;
    for (int base = 0; base < n_tiles; base += 256) {
        const int i = base + threadIdx.x;
        const int v = i < n_tiles ? tile_count[i] : 0;
        int total;
        const int ex = block_exclusive_scan256(v, wsum, total);
        if (i < n_tiles) tile_count[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *n_out = carry;
}

__global__ void __launch_bounds__(256) k_compact_scatter(const int32_t* __restrict__ tri, const float* __restrict__ dist,
                                                         const float* __restrict__ point, int64_t n,
                                                         const int* __restrict__ tile_off, int32_t* __restrict__ rays,
                                                         int32_t* __restrict__ tri_out, float* __restrict__ dist_out,
                                                         float* __restrict__ point_out) {
    __shared__ int wcnt[8];
    const unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t t0 = (int64_t)blockIdx.x * kCompactTile;
    int base = tile_off[blockIdx.x];
    for (int k = 0; k < kCompactPer; ++k) {   // rounds of 256 consecutive segments, in index order
        const int64_t r = t0 + k * 256 + threadIdx.x;
        const bool hit = r < n && tri[r] >= 0;
        const unsigned m = __ballot_sync(kFull, hit);
        if (lane == 0) wcnt[w] = __popc(m);
        __syncthreads();
        int pre = 0, tot = 0;
        for (int q = 0; q < 8; ++q) {
            const int c = wcnt[q];
            if (q < w) pre += c;
            tot += c;
        }
        if (hit) {
            const int64_t pos = base + pre + __popc(m & lt);
            if (rays) rays[pos] = (int32_t)r;
            if (tri_out) tri_out[pos] = tri[r];
            if (dist_out) dist_out[pos] = dist[r];
            if (point_out) {
                point_out[3 * pos] = point[3 * r];
                point_out[3 * pos + 1] = point[3 * r + 1];
                point_out[3 * pos + 2] = point[3 * r + 2];
            }
        }
        base += tot;
        __syncthreads();
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

// Traversal order of a whole batch: a counting sort of the segments by the
// Morton cell of their midpoint on a 32 x 32 x 32 grid over the mesh extent
// (15-bit keys, z the most significant of each 3-bit group, as the build's
// codes).  Neighbours in this order cross the same part of the hierarchy, so
// the warps of an SM share node fetches.  Order inside a cell is arbitrary:
// answers do not depend on the order.
constexpr int kOrderBins = 1 << 15;

__device__ __forceinline__ uint32_t order_key(const float* __restrict__ from, const float* __restrict__ to, int64_t r,
                                              float lox, float loy, float loz, float sx, float sy, float sz) {
    const float mx = 0.5f * (__ldg(from + 3 * r) + __ldg(to + 3 * r));
    const float my = 0.5f * (__ldg(from + 3 * r + 1) + __ldg(to + 3 * r + 1));
    const float mz = 0.5f * (__ldg(from + 3 * r + 2) + __ldg(to + 3 * r + 2));
    const uint32_t qx = (uint32_t)fminf(fmaxf((mx - lox) * sx, 0.0f), 31.0f);   // NaN -> 0
    const uint32_t qy = (uint32_t)fminf(fmaxf((my - loy) * sy, 0.0f), 31.0f);
    const uint32_t qz = (uint32_t)fminf(fmaxf((mz - loz) * sz, 0.0f), 31.0f);
    return spread10q(qx) | (spread10q(qy) << 1) | (spread10q(qz) << 2);
}

// Per-block histogram in shared memory (128 KB), added to the global one.
__global__ void __launch_bounds__(1024) k_order_hist(const float* __restrict__ from, const float* __restrict__ to,
                                                     int64_t n, float lox, float loy, float loz, float sx, float sy,
                                                     float sz, unsigned int* __restrict__ hist) {
    extern __shared__ unsigned int sh_hist[];
    for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x) sh_hist[i] = 0u;
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&sh_hist[order_key(from, to, r, lox, loy, loz, sx, sy, sz)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x) {
        const unsigned int c = sh_hist[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// Exclusive scan of the 2^15 bins by one block of 1024 threads (32 each).
__global__ void __launch_bounds__(1024) k_order_scan(unsigned int* __restrict__ hist) {
    __shared__ unsigned int part[1024];
    const int t = threadIdx.x;
    unsigned int v[32], sum = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        v[k] = hist[32 * t + k];
        sum += v[k];
    }
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned int x = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += x;
        __syncthreads();
    }
    unsigned int run = part[t] - sum;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        hist[32 * t + k] = run;
        run += v[k];
    }
}

// Scatter: each segment takes the next slot of its cell (lanes of a warp
// with the same cell share one atomic).
__global__ void __launch_bounds__(256) k_order_scatter(const float* __restrict__ from, const float* __restrict__ to,
                                                       int64_t n, float lox, float loy, float loz, float sx, float sy,
                                                       float sz, unsigned int* __restrict__ cursor,
                                                       int32_t* __restrict__ order) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31u); base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = base + lane;
        const bool ok = r < n;
        const uint32_t key = ok ? order_key(from, to, r, lox, loy, loz, sx, sy, sz) : 0xFFFFFFFFu - lane;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        unsigned int pos = 0;
        if (ok && lane == leader) pos = atomicAdd(&cursor[key], (unsigned int)__popc(peers));
        pos = __shfl_sync(0xffffffffu, pos, leader);
        if (ok) order[pos + __popc(peers & ((1u << lane) - 1u))] = (int32_t)r;
    }
}

// Cluster of leaf j: 256 equal ranges of the Morton-ordered leaves.
__device__ __forceinline__ int leaf_cluster(int j, int64_t n_tri) { return (int)(((int64_t)j * 256) / n_tri); }

// Multi-hot training labels: every leaf the segment's padded box search
// reaches, tested in FP32 (certain hit, or the plain decision in the band).
template <int STACK>
__global__ void __launch_bounds__(128) k_cluster_labels(QueryArgs A, uint32_t* __restrict__ labels) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        uint32_t bits[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const float3 s = make_float3(A.from[3 * r], A.from[3 * r + 1], A.from[3 * r + 2]);
        const float3 e = make_float3(A.to[3 * r], A.to[3 * r + 1], A.to[3 * r + 2]);
        if (!(bad3(s) || bad3(e))) {
            const SegF g = make_seg(s, e, A.dmax0, A.dmax1, A.dmax2);
            auto leaf = [&](int j) {
                bool plain;
                const int c = tri_fp32(g, load_tri(A.tris, j), true, plain);
                if (c == kHit || (c == kBand && plain)) {
                    const int k = leaf_cluster(j, A.n_tri);
                    bits[k >> 5] |= 1u << (k & 31);
                }
            };
            if (A.n_tri == 1) {
                leaf(0);
            } else {
                int stack[STACK];
                int sp = 0, node = 0;
                while (true) {
                    float4 lmin, lmax, rmin, rmax;
                    load_node(A.nodes, node, lmin, lmax, rmin, rmax);
                    const int lref = __float_as_int(lmin.w), rref = __float_as_int(lmax.w);
                    bool hl = slab(lmin, lmax, g), hr = slab(rmin, rmax, g);
                    if (hl && lref < 0) {
                        leaf(~lref);
                        hl = false;
                    }
                    if (hr && rref < 0) {
                        leaf(~rref);
                        hr = false;
                    }
                    if (hl && hr && sp < STACK) {
                        stack[sp++] = rref;
                        node = lref;
                    } else if (hl) {
                        node = lref;
                    } else if (hr) {
                        node = rref;
                    } else if (sp > 0) {
                        node = stack[--sp];
                    } else {
                        break;
                    }
                }
            }
        }
#pragma unroll
        for (int w = 0; w < 8; ++w) labels[r * 8 + w] = bits[w];
    }
}

// After a rebuild in the graph: each descriptor's padding extent (the largest
// triangle box side per axis) from its mesh's new build counters.
__global__ void k_desc_dmax(BatchDesc* __restrict__ desc, const DevCounters* __restrict__ ctr, int M) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) {
        desc[m].dmax0 = __uint_as_float(ctr[m].dmax_bits[0]);
        desc[m].dmax1 = __uint_as_float(ctr[m].dmax_bits[1]);
        desc[m].dmax2 = __uint_as_float(ctr[m].dmax_bits[2]);
    }
}

// Validation mode (rsi_options.fp64_all): every segment is queued for the
// FP64 re-test, none is settled by the FP32 traversal.
__global__ void k_queue_all(int32_t* __restrict__ band_ids, int64_t n, DevCounters* c) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) band_ids[i] = (int32_t)i;
    if (i == 0) c->band_count = (int)n;
}

__global__ void k_reset_query(DevCounters* c, unsigned long long ready) {
    c->band_count = 0;
    c->next_ray = 0;
    c->n_fallback = 0;
    c->n_confirmed = 0;
    c->pair_count = 0;
    c->fb_count = 0;
    c->hard_count = 0;
    c->todo_count = 0;
    c->amb_seg_count = 0;
    c->tpend_count = 0;
    c->n_finish = 0;
    c->n_finish64 = 0;
    if (ready != ~0ull) c->ready = ready;   // ~0: a streaming plan, fed by posts
    c->error = 0;
    c->node_visits = c->tri_tests = c->ambiguous = 0;
}

template <int MODE, bool STATS, int STACK, bool BATCHED, int NW>
void launch_fp32(const QueryArgs& A, const BatchArgs& B, int grid, int block, cudaStream_t s) {
    k_query_fp32<MODE, STATS, STACK, BATCHED, NW><<<grid, block, trav_smem_bytes(STACK, block), s>>>(A, B);
}

// The host-buffer traversal that counts its finished segments per output
// chunk (child-pair nodes, no statistics).
template <int MODE>
void launch_fp32_done(const QueryArgs& A, int height, int grid, int block, cudaStream_t s, const BatchArgs& B,
                      int stack_min) {
    const int need = std::max(height + 1, stack_min);
    if (need <= 32) k_query_fp32<MODE, false, 32, false, 0, true><<<grid, block, trav_smem_bytes(32, block), s>>>(A, B);
    else if (need <= 64) k_query_fp32<MODE, false, 64, false, 0, true><<<grid, block, trav_smem_bytes(64, block), s>>>(A, B);
    else k_query_fp32<MODE, false, 128, false, 0, true><<<grid, block, trav_smem_bytes(128, block), s>>>(A, B);
}

// Stack entries a traversal needs: the binary walk pushes at most one entry
// per level (height < STACK); the four-wide walk at most three per four-wide
// level, and a binary tree of height h has ceil((h + 1) / 2) such levels.
inline int wide_stack_need(int height) { return 3 * ((height + 2) / 2); }
inline bool wide_ok(int height) { return wide_stack_need(height) <= 128; }

// nw: 0 child-pair nodes, 1 four-wide nodes, 2 compressed child-pair nodes
// (single queries only; batched plans pass 0 or 1).  The stack is the
// smallest of 32 / 64 / 128 entries that holds the walk and `stack_min`.
template <int MODE, bool STATS, bool BATCHED = false>
void launch_fp32_stack(const QueryArgs& A, int height, int nw, int grid, int block, cudaStream_t s,
                       const BatchArgs& B = BatchArgs{}, int stack_min = 0) {
    const bool wide = nw == 1 && wide_ok(height);
    const int need = std::max(wide ? wide_stack_need(height) : height + 1, stack_min);
    const int st = need <= 32 ? 32 : (need <= 64 ? 64 : 128);
    if (wide) {
        if (st == 32) launch_fp32<MODE, STATS, 32, BATCHED, 1>(A, B, grid, block, s);
        else if (st == 64) launch_fp32<MODE, STATS, 64, BATCHED, 1>(A, B, grid, block, s);
        else launch_fp32<MODE, STATS, 128, BATCHED, 1>(A, B, grid, block, s);
    } else if (!BATCHED && nw == 2) {
        if (st == 32) launch_fp32<MODE, STATS, 32, false, 2>(A, B, grid, block, s);
        else if (st == 64) launch_fp32<MODE, STATS, 64, false, 2>(A, B, grid, block, s);
        else launch_fp32<MODE, STATS, 128, false, 2>(A, B, grid, block, s);
    } else if (st == 32) launch_fp32<MODE, STATS, 32, BATCHED, 0>(A, B, grid, block, s);
    else if (st == 64) launch_fp32<MODE, STATS, 64, BATCHED, 0>(A, B, grid, block, s);
    else launch_fp32<MODE, STATS, 128, BATCHED, 0>(A, B, grid, block, s);
}

// k_query_fp64 over the first *n_list entries of A.band_ids.
template <int MODE, bool BATCHED = false>
void launch_fp64(const QueryArgs& A, int height, int grid, cudaStream_t s, const int* n_list,
                 const BatchArgs& B = BatchArgs{}) {
    if (height < 32) k_query_fp64<MODE, 32, BATCHED><<<grid, 128, 0, s>>>(A, B, n_list);
    else if (height < 64) k_query_fp64<MODE, 64, BATCHED><<<grid, 128, 0, s>>>(A, B, n_list);
    else k_query_fp64<MODE, 128, BATCHED><<<grid, 128, 0, s>>>(A, B, n_list);
    note_launches(1);
}

// The FP64 pass over the queued segments: pair-parallel when scratch P is
// given (collect, classify, combine, then k_query_fp64 for the fallback
// list), else k_query_fp64 for every queued segment.  The pair path serves
// queues of every length and all three modes (c2 boolean mode, 1,330
// queued: 0.072 ms against 0.137 ms with k_query_fp64 for the whole queue).
template <int MODE, bool BATCHED = false>
void launch_fp64_pass(const QueryArgs& A, int height, const PairScratch* P0, cudaStream_t s,
                      const BatchArgs& B = BatchArgs{}) {
    const int grid = device_sm_count() * 4;
    if (!P0) {
        launch_fp64<MODE, BATCHED>(A, height, grid, s, &A.ctr->band_count, B);
        return;
    }
    PairScratch Pm = *P0;
    Pm.fp32_hits = MODE != RSI_NEAREST;   // the nearest mode needs every hit's t
    const PairScratch* P = &Pm;
    // step 1: both collect kernels are launched; the queue length (on the
    // device) lets exactly one of them work
    const int cgrid = device_sm_count() * 16;   // one warp per queued segment, 4 per block
    k_band_collect<BATCHED><<<cgrid, 128, 0, s>>>(A, B, *P);
    if (height < 32) k_band_collect_threads<32, BATCHED><<<cgrid, 128, 0, s>>>(A, B, *P);
    else if (height < 64) k_band_collect_threads<64, BATCHED><<<cgrid, 128, 0, s>>>(A, B, *P);
    else k_band_collect_threads<128, BATCHED><<<cgrid, 128, 0, s>>>(A, B, *P);
    k_band_classify<MODE, BATCHED><<<device_sm_count() * 8, 256, 0, s>>>(A, B, *P);
    k_band_classify_hard<BATCHED><<<device_sm_count() * 8, 128, 0, s>>>(A, B, *P);
    k_band_reduce<MODE, BATCHED><<<grid, 128, 0, s>>>(A, B, *P);
    note_launches(5);
    if (MODE == RSI_COUNT) {   // the ambiguous segments' crossings
        k_band_tfix<BATCHED><<<grid, 128, 0, s>>>(A, B, *P);
        k_band_crossings<BATCHED><<<grid, 128, 0, s>>>(A, B, *P);
        note_launches(2);
    }
    QueryArgs F = A;
    F.band_ids = P->fb_ids;
    launch_fp64<MODE, BATCHED>(F, height, grid, s, &A.ctr->fb_count, B);
}

}  // namespace

// Launch the two passes for one batch of segments already on the device.
struct NearestOut {
    int32_t* tri;
    float* t;
    float* point;
    float* dist;
};

int query_device(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n, int mode, const rsi_options* opt,
                 uint8_t* d_hit, int32_t* d_count, uint8_t* d_amb, int32_t* band_ids, int32_t* perm_scratch,
                 DevCounters* ctr, cudaStream_t s, const int32_t* order = nullptr, const int* n_dev = nullptr,
                 const NearestOut* nearest = nullptr, const PairScratch* pairs = nullptr) {
    rsi_options o = {};
    if (opt) o = *opt;
    if (h->height >= 127) return fail(RSI_ERR_STACK, "rsi_query: tree height exceeds the 128-entry traversal stack");
    const bool both = mode == RSI_BOTH;   // the count pass, which also answers the boolean mode
    if (both) mode = RSI_COUNT;
    QueryArgs A{};
    A.nodes = h->nodes;
    A.nodes4 = h->nodes4;
    A.nodesq = h->nodesq;
    A.tris = h->tris;
    A.n_tri = h->n_tri;
    A.from = d_from;
    A.to = d_to;
    A.n_rays = n;
    A.hit = d_hit;
    A.count = d_count;
    A.amb = d_amb;
    A.near = nearest ? nearest->tri : nullptr;
    A.band_ids = band_ids;
    A.perm = nullptr;
    A.n_dev = nullptr;
    A.ctr = ctr;
    A.dmax0 = h->dmax[0];
    A.dmax1 = h->dmax[1];
    A.dmax2 = h->dmax[2];
    A.fp32_only = o.fp32_only;
    A.amb_bits = both ? 1 : 0;
    if (o.block != 0 && (o.block < 32 || o.block > 256 || o.block % 32 != 0))
        return fail(RSI_ERR_INVALID_ARG, "rsi_query: block must be a multiple of 32 in [32, 256]");
    if (o.blocks_per_sm < 0) return fail(RSI_ERR_INVALID_ARG, "rsi_query: blocks_per_sm < 0");
    if (o.node_width != 0 && o.node_width != 2 && o.node_width != 3 && o.node_width != 4)
        return fail(RSI_ERR_INVALID_ARG, "rsi_query: node_width must be 0, 2, 3 or 4");
    if (o.fp64_all && (o.fp32_only || order))
        return fail(RSI_ERR_INVALID_ARG, "rsi_query: fp64_all excludes fp32_only and the learned query");
    if (o.stack != 0 && o.stack != 32 && o.stack != 64 && o.stack != 128)
        return fail(RSI_ERR_INVALID_ARG, "rsi_query: stack must be 0, 32, 64 or 128");
    const int nw = o.node_width == 4 ? 1 : (o.node_width == 3 && h->has_q ? 2 : 0);
    const int block = o.block > 0 ? o.block : 256;
    const int bps = o.blocks_per_sm > 0 ? o.blocks_per_sm : 8;
    int64_t want = (n + block - 1) / block;
    int64_t cap = (int64_t)device_sm_count() * bps;
    int grid = (int)std::max<int64_t>(1, std::min(want, cap));
    if (o.time_kernels && !h->ev[0]) {
        for (auto& e : h->ev) RSI_CUDA_TRY(cudaEventCreate(&e));
    }
    h->timed = o.time_kernels != 0;
    if (o.order && (o.ray_sort_tile != 0 || order))
        return fail(RSI_ERR_INVALID_ARG, "rsi_query: order excludes ray_sort_tile and the learned query");
    if (o.order) A.perm = o.order;   // the caller's traversal order (rsi_segment_order)
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
    if (order) {   // learned path: the segments left by the proposal, counted on the device
        A.perm = order;
        A.n_dev = n_dev;
    } else {
        k_reset_query<<<1, 1, 0, s>>>(ctr, (unsigned long long)n);
    }
    if (h->timed) RSI_CUDA_TRY(cudaEventRecord(h->ev[0], s));
    if (o.fp64_all) {
        k_queue_all<<<grid_for(n, 256), 256, 0, s>>>(band_ids, n, ctr);
    } else if (mode == RSI_ANY_HIT) {
        if (o.collect_stats) launch_fp32_stack<RSI_ANY_HIT, true>(A, h->height, nw, grid, block, s, {}, o.stack);
        else launch_fp32_stack<RSI_ANY_HIT, false>(A, h->height, nw, grid, block, s, {}, o.stack);
    } else if (mode == RSI_COUNT) {
        if (o.collect_stats) launch_fp32_stack<RSI_COUNT, true>(A, h->height, nw, grid, block, s, {}, o.stack);
        else launch_fp32_stack<RSI_COUNT, false>(A, h->height, nw, grid, block, s, {}, o.stack);
    } else {
        if (o.collect_stats) launch_fp32_stack<RSI_NEAREST, true>(A, h->height, nw, grid, block, s, {}, o.stack);
        else launch_fp32_stack<RSI_NEAREST, false>(A, h->height, nw, grid, block, s, {}, o.stack);
    }
    if (h->timed) RSI_CUDA_TRY(cudaEventRecord(h->ev[1], s));
    if (!o.fp32_only) {
        if (mode == RSI_ANY_HIT) launch_fp64_pass<RSI_ANY_HIT>(A, h->height, pairs, s);
        else if (mode == RSI_COUNT) launch_fp64_pass<RSI_COUNT>(A, h->height, pairs, s);
        else launch_fp64_pass<RSI_NEAREST>(A, h->height, pairs, s);
    }
    if (mode == RSI_NEAREST) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count() * 8));
        k_nearest_list<<<g, 256, 0, s>>>(A, nearest->t, nearest->point, nearest->dist);
        if (perm_scratch) {   // double-float first, FP64 for the segments it leaves
            k_nearest_finish_ff<<<g, 256, 0, s>>>(A, nearest->t, nearest->point, nearest->dist, perm_scratch);
            k_nearest_finish<<<g, 256, 0, s>>>(A, nearest->t, nearest->point, nearest->dist, perm_scratch,
                                               &ctr->n_finish64);
            note_launches(3);
        } else {
            k_nearest_finish<<<g, 256, 0, s>>>(A, nearest->t, nearest->point, nearest->dist, A.band_ids,
                                               &ctr->n_finish);
            note_launches(2);
        }
    }
    if (h->timed) RSI_CUDA_TRY(cudaEventRecord(h->ev[2], s));
    note_launches(2);   // k_reset_query, k_query_fp32 (the FP64 pass counts its own)
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rsi_query launch");
    return RSI_OK;
}

// Pair scratch of the FP64 pass for a queue of up to q segments: room for
// q / 16 queued segments (at least 4096) and 4 pairs each on average; the
// rest goes to the fallback list.
void pair_sizes(int64_t q, int64_t& seg_cap, int64_t& pair_cap, size_t& bytes) {
    seg_cap = std::min<int64_t>(std::max<int64_t>(q / 16, 4096), 1 << 24);
    pair_cap = 4 * seg_cap;
    bytes = 8 * (size_t)seg_cap + 25 * (size_t)pair_cap + 8 * 256;   // + alignment of the pieces
}

PairScratch carve_pairs(char* mem, int64_t seg_cap, int64_t pair_cap, int32_t* fb_ids) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    PairScratch P;
    size_t o = 0;
    P.pair_t = reinterpret_cast<double*>(mem + o);
    o += al(8 * (size_t)pair_cap);
    P.seg_off = reinterpret_cast<int32_t*>(mem + o);
    o += al(4 * (size_t)seg_cap);
    P.seg_cnt = reinterpret_cast<int32_t*>(mem + o);
    o += al(4 * (size_t)seg_cap);
    P.pair_seg = reinterpret_cast<int32_t*>(mem + o);
    o += al(4 * (size_t)pair_cap);
    P.pair_leaf = reinterpret_cast<int32_t*>(mem + o);
    o += al(4 * (size_t)pair_cap);
    P.hard = reinterpret_cast<int32_t*>(mem + o);
    o += al(4 * (size_t)pair_cap);
    P.todo = reinterpret_cast<int32_t*>(mem + o);
    o += al(4 * (size_t)pair_cap);
    P.pair_cls = reinterpret_cast<uint8_t*>(mem + o);
    P.fb_ids = fb_ids;
    P.seg_cap = (int)seg_cap;
    P.pair_cap = (int)pair_cap;
    P.fp32_hits = 0;
    return P;
}

int ensure_band_capacity(rsi_bvh_t h, int64_t n, cudaStream_t s) {
    if (h->band_cap >= n) return RSI_OK;
    int64_t cap = std::max<int64_t>(n, 1 << 16);
    if (h->band_ids) {   // stream-ordered: after the queries that used it on s
        pool_free(h->band_ids, s);
        pool_free(h->pair_mem, s);
        h->band_ids = nullptr;
        h->pair_mem = nullptr;
        h->band_cap = 0;
        h->pair_bytes = 0;
    }
    // band | order (in-tile reordering, the learned query's leftovers, the nearest mode's list) | FP64 fallback list
    if (pool_alloc(reinterpret_cast<void**>(&h->band_ids), 12 * (size_t)cap, s) != RSI_OK) return RSI_ERR_OOM;
    int64_t seg_cap, pair_cap;
    size_t bytes;
    pair_sizes(cap, seg_cap, pair_cap, bytes);
    if (pool_alloc(reinterpret_cast<void**>(&h->pair_mem), bytes, s) != RSI_OK) {
        pool_free(h->band_ids, s);
        h->band_ids = nullptr;
        return RSI_ERR_OOM;
    }
    h->band_cap = cap;
    h->pair_seg_cap = seg_cap;
    h->pair_cap = pair_cap;
    h->pair_bytes = (int64_t)bytes;
    return RSI_OK;
}

PairScratch handle_pairs(rsi_bvh_t h) {
    return carve_pairs(h->pair_mem, h->pair_seg_cap, h->pair_cap, h->band_ids + 2 * h->band_cap);
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
        st->proposal_confirmed = c.n_confirmed;
        st->fallback_rays = c.n_fallback;
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

// Argument checks shared by the boolean / intercept_count entry points; `fn`
// names the caller in the error message.
static int check_query_args(const char* fn, rsi_bvh_t h, const void* from, const void* to, int64_t n, int mode,
                            const void* hit, const void* count) {
    const std::string f(fn);
    if (!h) return rsi::fail(RSI_ERR_INVALID_ARG, f + ": NULL handle");
    if (n < 0 || n > 0x7FFFFFFFll) return rsi::fail(RSI_ERR_INVALID_ARG, f + ": need 0 <= n_rays < 2^31");
    if (mode != RSI_ANY_HIT && mode != RSI_COUNT && mode != RSI_BOTH)
        return rsi::fail(RSI_ERR_INVALID_ARG, f + ": bad mode");
    if (n > 0 && (!from || !to)) return rsi::fail(RSI_ERR_INVALID_ARG, f + ": NULL segment pointer");
    if (n > 0 && mode != RSI_COUNT && !hit) return rsi::fail(RSI_ERR_INVALID_ARG, f + ": any-hit needs hit");
    if (n > 0 && mode != RSI_ANY_HIT && !count) return rsi::fail(RSI_ERR_INVALID_ARG, f + ": count needs count");
    return RSI_OK;
}

extern "C" int rsi_query(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays, int mode,
                         const rsi_options* opt, uint8_t* d_hit, int32_t* d_count, uint8_t* d_ambiguous,
                         rsi_stats* stats, void* stream) {
    int rc = check_query_args("rsi_query", h, d_from, d_to, n_rays, mode, d_hit, d_count);
    if (rc) return rc;
    if (mode == RSI_ANY_HIT && h->mlp && !(opt && opt->fp64_all))   // attached proposal network
        return rsi_query_learned(h, h->mlp, d_from, d_to, n_rays, opt, d_hit, d_ambiguous, stats, stream);
    cudaStream_t s = (cudaStream_t)stream;
    if (n_rays == 0) {
        if (stats) *stats = rsi_stats{};
        return RSI_OK;
    }
    rc = rsi::ensure_band_capacity(h, n_rays, s);
    if (rc) return rc;
    const rsi::PairScratch P = rsi::handle_pairs(h);
    rc = rsi::query_device(h, d_from, d_to, n_rays, mode, opt, d_hit, d_count, d_ambiguous, h->band_ids,
                           h->band_ids + h->band_cap, h->ctr, s, nullptr, nullptr, nullptr, &P);
    if (rc) return rc;
    if (stats) return rsi::read_stats(h, h->ctr, n_rays, stats, s);
    return RSI_OK;
}

extern "C" int rsi_query_nearest(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays,
                                 const rsi_options* opt, int32_t* d_tri, float* d_t, float* d_point, float* d_dist,
                                 uint8_t* d_ambiguous, rsi_stats* stats, void* stream) {
    if (!h) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_nearest: NULL handle");
    if (n_rays < 0 || n_rays > 0x7FFFFFFFll)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_nearest: need 0 <= n_rays < 2^31");
    if (n_rays > 0 && (!d_from || !d_to || !d_tri))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_nearest: NULL segment or triangle pointer");
    cudaStream_t s = (cudaStream_t)stream;
    if (n_rays == 0) {
        if (stats) *stats = rsi_stats{};
        return RSI_OK;
    }
    int rc = rsi::ensure_band_capacity(h, n_rays, s);
    if (rc) return rc;
    const rsi::NearestOut no = {d_tri, d_t, d_point, d_dist};
    const rsi::PairScratch P = rsi::handle_pairs(h);
    rc = rsi::query_device(h, d_from, d_to, n_rays, RSI_NEAREST, opt, nullptr, nullptr, d_ambiguous, h->band_ids,
                           h->band_ids + h->band_cap, h->ctr, s, nullptr, nullptr, &no, &P);
    if (rc) return rc;
    if (stats) return rsi::read_stats(h, h->ctr, n_rays, stats, s);
    return RSI_OK;
}

extern "C" int rsi_nearest_compact(const int32_t* d_tri, const float* d_dist, const float* d_point, int64_t n_rays,
                                   int32_t* d_rays, int32_t* d_tri_out, float* d_dist_out, float* d_point_out,
                                   int64_t* n_hits, void* stream) {
    if (!n_hits || n_rays < 0 || n_rays > 0x7FFFFFFFll || (n_rays > 0 && !d_tri) || (d_dist_out && !d_dist) ||
        (d_point_out && !d_point))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_nearest_compact: bad arguments");
    *n_hits = 0;
    if (n_rays == 0) return RSI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_tiles = (n_rays + rsi::kCompactTile - 1) / rsi::kCompactTile;
    void* scratch = nullptr;   // [total (8 B)] [tile offsets]
    if (rsi::pool_alloc(&scratch, 8 + 4 * (size_t)n_tiles, s) != RSI_OK) return RSI_ERR_OOM;
    long long* d_total = reinterpret_cast<long long*>(scratch);
    int* tiles = reinterpret_cast<int*>(d_total + 1);
    rsi::k_compact_count<<<(int)n_tiles, 256, 0, s>>>(d_tri, n_rays, tiles);
    rsi::k_compact_scan<<<1, 256, 0, s>>>(tiles, (int)n_tiles, d_total);
    rsi::k_compact_scatter<<<(int)n_tiles, 256, 0, s>>>(d_tri, d_dist, d_point, n_rays, tiles, d_rays, d_tri_out,
                                                        d_dist_out, d_point_out);
    rsi::note_launches(3);
    long long total = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, d_total, sizeof(total), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    rsi::pool_free(scratch, s);
    if (e != cudaSuccess) return rsi::cuda_fail(e, "rsi_nearest_compact");
    *n_hits = total;
    return RSI_OK;
}

// Host-buffer query: segments streamed in chunks through two device staging
// slots of the device context.  Copies in run on its st_in, the traversal on
// the caller's stream, copies out on its st_out; events chain them so that chunk k's traversal
// overlaps chunk k+1's copy in and chunk k-1's copy out, and a slot is
// reused only after its previous chunk has left it.
namespace {
constexpr int64_t kHostChunk = 1 << 21;

// The copy streams and events of host-buffer queries (each made once).
int host_streams(rsi::DeviceCtx* c) {
    if (!c->st_in) RSI_CUDA_TRY(cudaStreamCreateWithFlags(&c->st_in, cudaStreamNonBlocking));
    if (!c->st_out) RSI_CUDA_TRY(cudaStreamCreateWithFlags(&c->st_out, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
        if (!c->ev_in[i]) RSI_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_in[i], cudaEventDisableTiming));
        if (!c->ev_q[i]) RSI_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_q[i], cudaEventDisableTiming));
        if (!c->ev_out[i]) RSI_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_out[i], cudaEventDisableTiming));
    }
    for (cudaEvent_t& e : c->ev_chunk)
        if (!e) RSI_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return RSI_OK;
}

int host_setup(rsi::DeviceCtx* c, int64_t chunk, int64_t n_chunks) {
    int rc = host_streams(c);
    if (rc) return rc;
    if (c->stage_chunk < chunk) {
        if (c->stage) {
            RSI_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(c->stage);
            c->stage = nullptr;
            c->stage_chunk = 0;
        }
        if (rsi::dev_malloc(&c->stage, 2 * 32 * (size_t)chunk) != cudaSuccess) {   // 2 slots x (24 + 1 + 4 + 1) B
            cudaGetLastError();
            return rsi::fail(RSI_ERR_OOM, "rsi_query_host: staging allocation failed");
        }
        c->stage_chunk = chunk;
    }
    if (c->h_chunk_cap < n_chunks) {
        if (c->h_chunk_ctr) {
            RSI_CUDA_TRY(cudaDeviceSynchronize());
            cudaFreeHost(c->h_chunk_ctr);
            c->h_chunk_ctr = nullptr;
        }
        const int64_t cap = std::max<int64_t>(n_chunks, 64);
        if (rsi::host_malloc_pinned(&c->h_chunk_ctr, sizeof(rsi::DevCounters) * (size_t)cap) != cudaSuccess) {
            cudaGetLastError();
            c->h_chunk_cap = 0;
            return rsi::fail(RSI_ERR_OOM, "rsi_query_host: counter allocation failed");
        }
        c->h_chunk_cap = cap;
    }
    return RSI_OK;
}
}  // namespace

namespace {
using namespace rsi;   // the kernels and launchers above
// Whole-batch host-buffer query (batches of up to kHostWhole segments): the
// segments are copied in chunks on st_in, each chunk followed by a post of
// the number of segments now on the device; one persistent FP32 traversal
// on the caller's stream takes segments as they are posted (a device work
// queue with bounded waits, as in streaming batched plans), so copies and
// traversal overlap without a kernel tail per chunk (the first chunk is
// small so that the traversal starts early); one FP64 pass then settles the
// whole queue and the results are copied out.  With page-locked outputs the
// traversal counts its finished segments per output chunk of 2^21 segments
// into page-locked counters, and the host copies each chunk out as soon as
// it is answered, while the traversal goes on; the queued segments' answers
// are written into the host arrays after the FP64 pass.  Up to 2^28 segments
// (8 GB of staging); a batch whose staging does not fit goes through the two
// slots.
constexpr int64_t kHostWhole = (int64_t)1 << 28;
constexpr int kOutShift = 21;
constexpr int kOutChunks = (int)(kHostWhole >> kOutShift);
}  // namespace

namespace rsi {
namespace {
// After the FP64 pass: the queued segments' answers, from the device arrays
// into the caller's page-locked host arrays through their mapped addresses
// (launched once the bulk copy of the FP32 answers has landed there).
__global__ void k_patch_host(const int32_t* __restrict__ band_ids, const int* __restrict__ n_band,
                             const uint8_t* __restrict__ dh, const int32_t* __restrict__ dc,
                             const uint8_t* __restrict__ da, uint8_t* hh, int32_t* hc, uint8_t* ha) {
    const int nb = *n_band;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
        const int i = band_ids[k];
        if (hh) hh[i] = dh[i];
        if (hc) hc[i] = dc[i];
        if (ha) ha[i] = da[i];
    }
}
}  // namespace
}  // namespace rsi

namespace {
using namespace rsi;

// The device address of a page-locked host buffer (NULL stays NULL); false
// for pageable memory.
template <typename T>
bool mapped_host(T* p, T** dev) {
    *dev = nullptr;
    if (!p) return true;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return false;
    *dev = static_cast<T*>(at.devicePointer);
    return true;
}

int host_whole(rsi_bvh_t h, const float* h_from, const float* h_to, int64_t n, int mode, const rsi_options& o,
               uint8_t* h_hit, int32_t* h_count, uint8_t* h_amb, rsi_stats* stats, cudaStream_t s,
               rsi::DeviceCtx* c) {
    if (o.block != 0 && (o.block < 32 || o.block > 256 || o.block % 32 != 0))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query: block must be a multiple of 32 in [32, 256]");
    if (o.blocks_per_sm < 0) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query: blocks_per_sm < 0");
    if (o.node_width != 0 && o.node_width != 2 && o.node_width != 3 && o.node_width != 4)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query: node_width must be 0, 2, 3 or 4");
    if (o.stack != 0 && o.stack != 32 && o.stack != 64 && o.stack != 128)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query: stack must be 0, 32, 64 or 128");
    if (h->height >= 127) return rsi::fail(RSI_ERR_STACK, "rsi_query: tree height exceeds the 128-entry traversal stack");
    int rc = rsi::ensure_band_capacity(h, n, s);
    if (rc) return rc;
    if (c->whole_cap < n) {
        if (c->whole) {
            RSI_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(c->whole);
            c->whole = nullptr;
            c->whole_cap = 0;
        }
        if (rsi::dev_malloc(&c->whole, 30 * (size_t)n + 1024) != cudaSuccess) {
            cudaGetLastError();
            return rsi::fail(RSI_ERR_OOM, "rsi_query_host: staging allocation failed");
        }
        c->whole_cap = n;
    }
    rc = host_streams(c);
    if (rc) return rc;
    if (!c->h_chunk_ctr) {
        if (rsi::host_malloc_pinned(&c->h_chunk_ctr, sizeof(rsi::DevCounters) * 64) != cudaSuccess) {
            cudaGetLastError();
            return rsi::fail(RSI_ERR_OOM, "rsi_query_host: counter allocation failed");
        }
        c->h_chunk_cap = 64;
    }
    if (!c->h_ready && rsi::host_malloc_pinned(&c->h_ready, 64 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        c->h_ready = nullptr;
        return rsi::fail(RSI_ERR_OOM, "rsi_query_host: counter allocation failed");
    }
    if (!c->h_done && rsi::host_malloc_pinned(&c->h_done, kOutChunks * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        c->h_done = nullptr;
        return rsi::fail(RSI_ERR_OOM, "rsi_query_host: counter allocation failed");
    }
    if (!c->d_done && rsi::dev_malloc(&c->d_done, kOutChunks * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        c->d_done = nullptr;
        return rsi::fail(RSI_ERR_OOM, "rsi_query_host: counter allocation failed");
    }
    if (!c->st_poll) RSI_CUDA_TRY(cudaStreamCreateWithFlags(&c->st_poll, cudaStreamNonBlocking));
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    float* df = reinterpret_cast<float*>(c->whole);
    float* dt = reinterpret_cast<float*>(c->whole + al(12 * (size_t)n));
    int32_t* dc = reinterpret_cast<int32_t*>(c->whole + 2 * al(12 * (size_t)n));
    uint8_t* dh = reinterpret_cast<uint8_t*>(c->whole + 2 * al(12 * (size_t)n) + al(4 * (size_t)n));
    uint8_t* da = dh + al((size_t)n);
    // chunk k covers [bounds[k], bounds[k + 1]): 2^16, 2^17, ..., 2^20
    // segments (the copies run ~2.7x faster than the traversal consumes
    // segments, so each of these lands before the traversal has used up the
    // ones before it), then equal chunks of at least 2^21 (at most 64 in all)
    std::vector<int64_t> bounds{0};
    for (int e = 16; e <= 20 && bounds.back() < n; ++e)
        bounds.push_back(std::min<int64_t>(n, bounds.back() + ((int64_t)1 << e)));
    const int64_t rest = n - bounds.back();
    const int64_t chunk = std::max<int64_t>(kHostChunk, (rest + 58) / 59);
    while (bounds.back() < n) bounds.push_back(std::min<int64_t>(n, bounds.back() + chunk));
    const int n_chunks = (int)bounds.size() - 1;
    auto first = [&](int k) { return bounds[(size_t)k]; };
    // empty the work queue, then start the copies once the caller's stream
    // is done with the previous call's staging
    RSI_CUDA_TRY(cudaMemsetAsync(&h->ctr->ready, 0, sizeof(unsigned long long), s));
    RSI_CUDA_TRY(cudaEventRecord(c->ev_chunk[0], s));
    RSI_CUDA_TRY(cudaStreamWaitEvent(c->st_in, c->ev_chunk[0], 0));
    for (int k = 0; k < n_chunks; ++k) {
        const int64_t r0 = first(k), m = first(k + 1) - r0;
        RSI_CUDA_TRY(cudaMemcpyAsync(df + 3 * r0, h_from + 3 * r0, 12 * (size_t)m, cudaMemcpyHostToDevice, c->st_in));
        RSI_CUDA_TRY(cudaMemcpyAsync(dt + 3 * r0, h_to + 3 * r0, 12 * (size_t)m, cudaMemcpyHostToDevice, c->st_in));
        c->h_ready[k] = (unsigned long long)(r0 + m);   // read by the copy below when it runs
        RSI_CUDA_TRY(cudaMemcpyAsync(&h->ctr->ready, &c->h_ready[k], sizeof(unsigned long long),
                                     cudaMemcpyHostToDevice, c->st_in));
        RSI_CUDA_TRY(cudaEventRecord(c->ev_chunk[k], c->st_in));
    }
    QueryArgs A{};
    A.nodes = h->nodes;
    A.nodes4 = h->nodes4;
    A.nodesq = h->nodesq;
    A.tris = h->tris;
    A.n_tri = h->n_tri;
    A.from = df;
    A.to = dt;
    const bool both = mode == RSI_BOTH;   // the count pass, which also answers the boolean mode
    if (both) mode = RSI_COUNT;
    A.amb_bits = both ? 1 : 0;
    A.hit = h_hit ? dh : nullptr;
    A.count = mode == RSI_COUNT ? dc : nullptr;
    A.amb = h_amb ? da : nullptr;
    A.band_ids = h->band_ids;
    A.ctr = h->ctr;
    A.dmax0 = h->dmax[0];
    A.dmax1 = h->dmax[1];
    A.dmax2 = h->dmax[2];
    A.fp32_only = o.fp32_only;
    const int block = o.block > 0 ? o.block : 256;
    const int bps = o.blocks_per_sm > 0 ? o.blocks_per_sm : 8;
    const int nw = o.node_width == 4 ? 1 : (o.node_width == 3 && h->has_q ? 2 : 0);
    // page-locked outputs: the FP32 answers are copied out chunk by chunk as
    // the traversal finishes them, then the queued segments' answers are
    // written into them after the FP64 pass
    uint8_t *mh = nullptr, *ma = nullptr;
    int32_t* mc = nullptr;
    const bool overlap = !o.fp32_only && mapped_host(h_hit, &mh) && mapped_host(h_amb, &ma) &&
                         mapped_host(mode == RSI_COUNT ? h_count : (int32_t*)nullptr, &mc);
    const int n_out = (int)((n + ((int64_t)1 << kOutShift) - 1) >> kOutShift);
    // the counting traversal: child-pair nodes without statistics; otherwise
    // the answers are copied out once the traversal has ended
    const bool counted = overlap && nw == 0 && !o.collect_stats;
    if (counted) {
        RSI_CUDA_TRY(cudaMemsetAsync(c->d_done, 0, sizeof(unsigned int) * (size_t)n_out, s));
        RSI_CUDA_TRY(cudaEventRecord(c->ev_q[1], s));   // the polls read the counters after this
        RSI_CUDA_TRY(cudaStreamWaitEvent(c->st_poll, c->ev_q[1], 0));
        A.done = c->d_done;
        A.done_shift = kOutShift;
    }
    k_reset_query<<<1, 1, 0, s>>>(h->ctr, ~0ull);   // ~0: the queue is fed by the posts above
    A.n_rays = n;
    BatchArgs Bs{};
    Bs.streamed = 1;
    Bs.timeout_ns = 10000000000ll;   // a post may wait behind pageable-memory copies
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + block - 1) / block,
                                                                   (int64_t)rsi::device_sm_count() * bps));
    if (counted) {
        if (mode == RSI_ANY_HIT) launch_fp32_done<RSI_ANY_HIT>(A, h->height, grid, block, s, Bs, o.stack);
        else launch_fp32_done<RSI_COUNT>(A, h->height, grid, block, s, Bs, o.stack);
    } else if (mode == RSI_ANY_HIT) {
        if (o.collect_stats) launch_fp32_stack<RSI_ANY_HIT, true>(A, h->height, nw, grid, block, s, Bs, o.stack);
        else launch_fp32_stack<RSI_ANY_HIT, false>(A, h->height, nw, grid, block, s, Bs, o.stack);
    } else {
        if (o.collect_stats) launch_fp32_stack<RSI_COUNT, true>(A, h->height, nw, grid, block, s, Bs, o.stack);
        else launch_fp32_stack<RSI_COUNT, false>(A, h->height, nw, grid, block, s, Bs, o.stack);
    }
    rsi::note_launches(2);
    RSI_CUDA_TRY(cudaEventRecord(c->ev_q[0], s));   // the traversal has ended
    // every copy has landed once the traversal ends; the wait orders the FP64 pass after them
    RSI_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_chunk[n_chunks - 1], 0));
    if (!o.fp32_only) {
        const rsi::PairScratch P = rsi::handle_pairs(h);
        if (mode == RSI_ANY_HIT) launch_fp64_pass<RSI_ANY_HIT>(A, h->height, &P, s);
        else launch_fp64_pass<RSI_COUNT>(A, h->height, &P, s);
    }
    RSI_CUDA_TRY(cudaGetLastError());
    if (overlap) {
        // copy out each output chunk once the traversal has finished all its
        // segments (or, for whatever is left, once the traversal has ended)
        auto copy_out = [&](int k) -> int {
            const int64_t a = (int64_t)k << kOutShift, m = std::min<int64_t>(n, a + ((int64_t)1 << kOutShift)) - a;
            if (h_hit) RSI_CUDA_TRY(cudaMemcpyAsync(h_hit + a, dh + a, (size_t)m, cudaMemcpyDeviceToHost, c->st_out));
            if (h_amb) RSI_CUDA_TRY(cudaMemcpyAsync(h_amb + a, da + a, (size_t)m, cudaMemcpyDeviceToHost, c->st_out));
            if (mode == RSI_COUNT)
                RSI_CUDA_TRY(cudaMemcpyAsync(h_count + a, dc + a, 4 * (size_t)m, cudaMemcpyDeviceToHost, c->st_out));
            return RSI_OK;
        };
        std::vector<char> out_done((size_t)n_out, 0);
        int left = n_out;
        const unsigned int* hd = c->h_done;
        while (counted && left > 0) {
            const bool ended = cudaEventQuery(c->ev_q[0]) == cudaSuccess;
            if (ended) break;
            RSI_CUDA_TRY(cudaMemcpyAsync(c->h_done, c->d_done, sizeof(unsigned int) * (size_t)n_out,
                                         cudaMemcpyDeviceToHost, c->st_poll));
            RSI_CUDA_TRY(cudaStreamSynchronize(c->st_poll));
            for (int k = 0; k < n_out; ++k) {
                const int64_t a = (int64_t)k << kOutShift;
                const int64_t m = std::min<int64_t>(n, a + ((int64_t)1 << kOutShift)) - a;
                if (!out_done[k] && (int64_t)hd[k] >= m) {
                    rc = copy_out(k);
                    if (rc) return rc;
                    out_done[k] = 1;
                    --left;
                }
            }
        }
        cudaGetLastError();   // cudaErrorNotReady of the event queries
        if (left > 0) {
            RSI_CUDA_TRY(cudaStreamWaitEvent(c->st_out, c->ev_q[0], 0));
            for (int k = 0; k < n_out; ++k)
                if (!out_done[k]) {
                    rc = copy_out(k);
                    if (rc) return rc;
                }
        }
        RSI_CUDA_TRY(cudaEventRecord(c->ev_out[0], c->st_out));
        RSI_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_out[0], 0));
        rsi::k_patch_host<<<rsi::device_sm_count() * 4, 256, 0, s>>>(h->band_ids, &h->ctr->band_count, dh,
                                                                mode == RSI_COUNT ? dc : nullptr, da, mh, mc, ma);
        rsi::note_launches(1);
        RSI_CUDA_TRY(cudaGetLastError());
    } else {
        if (h_hit) RSI_CUDA_TRY(cudaMemcpyAsync(h_hit, dh, (size_t)n, cudaMemcpyDeviceToHost, s));
        if (h_amb) RSI_CUDA_TRY(cudaMemcpyAsync(h_amb, da, (size_t)n, cudaMemcpyDeviceToHost, s));
        if (mode == RSI_COUNT) RSI_CUDA_TRY(cudaMemcpyAsync(h_count, dc, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
    }
    RSI_CUDA_TRY(cudaMemcpyAsync(c->h_chunk_ctr, h->ctr, sizeof(rsi::DevCounters), cudaMemcpyDeviceToHost, s));
    RSI_CUDA_TRY(cudaStreamSynchronize(s));
    const rsi::DevCounters& kc = c->h_chunk_ctr[0];
    if (stats) {
        rsi_stats acc{};
        acc.n_rays = n;
        acc.tree_height = h->height;
        acc.node_visits = (int64_t)kc.node_visits;
        acc.tri_tests = (int64_t)kc.tri_tests;
        acc.band_rays = kc.band_count;
        acc.ambiguous = (int64_t)kc.ambiguous;
        acc.device_error = kc.error;
        *stats = acc;
    }
    if (kc.error) return rsi::fail(kc.error, "rsi_query_host: device error " + std::to_string(kc.error));
    return RSI_OK;
}
}  // namespace

extern "C" int rsi_query_host(rsi_bvh_t h, const float* h_from, const float* h_to, int64_t n_rays, int mode,
                              const rsi_options* opt, uint8_t* h_hit, int32_t* h_count, uint8_t* h_ambiguous,
                              rsi_stats* stats, void* stream) {
    int rc = check_query_args("rsi_query_host", h, h_from, h_to, n_rays, mode, h_hit, h_count);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_rays == 0) {
        if (stats) *stats = rsi_stats{};
        return RSI_OK;
    }
    rsi_options o = {};
    if (opt) o = *opt;
    if (o.fp64_all) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_host: fp64_all is for device-buffer queries");
    if (n_rays <= kHostWhole && o.ray_sort_tile == 0) {
        rsi::DeviceCtx* c = rsi::device_ctx();
        if (!c) return rsi::fail(RSI_ERR_CUDA, "rsi_query_host: no device context");
        std::lock_guard<std::mutex> lock(c->host_mu);   // one host-buffer query per device at a time
        rc = host_whole(h, h_from, h_to, n_rays, mode, o, h_hit, h_count, h_ambiguous, stats, s, c);
        // no room to stage the whole batch (nothing was enqueued): stream it through the slots
        if (rc != RSI_ERR_OOM) return rc;
    }
    const int64_t chunk = std::min<int64_t>(n_rays, kHostChunk);
    const int64_t n_chunks = (n_rays + chunk - 1) / chunk;
    rc = rsi::ensure_band_capacity(h, chunk, s);
    if (rc) return rc;
    rsi::DeviceCtx* c = rsi::device_ctx();
    if (!c) return rsi::fail(RSI_ERR_CUDA, "rsi_query_host: no device context");
    std::lock_guard<std::mutex> lock(c->host_mu);   // one host-buffer query per device at a time
    rc = host_setup(c, chunk, n_chunks);
    if (rc) return rc;
    for (int64_t k = 0; k < n_chunks && rc == RSI_OK; ++k) {
        const int b = (int)(k & 1);
        const int64_t r0 = k * chunk, m = std::min(chunk, n_rays - r0);
        char* slot = c->stage + (size_t)b * 32 * (size_t)chunk;
        float* df = reinterpret_cast<float*>(slot);
        float* dt = df + 3 * chunk;
        int32_t* dc = reinterpret_cast<int32_t*>(dt + 3 * chunk);
        uint8_t* dh = reinterpret_cast<uint8_t*>(dc + chunk);
        uint8_t* da = dh + chunk;
        cudaError_t e = cudaStreamWaitEvent(c->st_in, c->ev_q[b], 0);   // slot's inputs no longer read
        if (e == cudaSuccess) e = cudaMemcpyAsync(df, h_from + 3 * r0, 12 * (size_t)m, cudaMemcpyHostToDevice, c->st_in);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dt, h_to + 3 * r0, 12 * (size_t)m, cudaMemcpyHostToDevice, c->st_in);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_in[b], c->st_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_in[b], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_out[b], 0);   // slot's outputs copied out
        if (e != cudaSuccess) {
            rc = rsi::cuda_fail(e, "rsi_query_host copy in");
            break;
        }
        const rsi::PairScratch P = rsi::handle_pairs(h);
        rc = rsi::query_device(h, df, dt, m, mode, opt, h_hit ? dh : nullptr, mode != RSI_ANY_HIT ? dc : nullptr,
                               h_ambiguous ? da : nullptr, h->band_ids, h->band_ids + h->band_cap, h->ctr, s, nullptr,
                               nullptr, nullptr, &P);
        if (rc) break;
        e = cudaMemcpyAsync(c->h_chunk_ctr + k, h->ctr, sizeof(rsi::DevCounters), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_q[b], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->st_out, c->ev_q[b], 0);
        if (e == cudaSuccess && h_hit) e = cudaMemcpyAsync(h_hit + r0, dh, (size_t)m, cudaMemcpyDeviceToHost, c->st_out);
        if (e == cudaSuccess && h_ambiguous)
            e = cudaMemcpyAsync(h_ambiguous + r0, da, (size_t)m, cudaMemcpyDeviceToHost, c->st_out);
        if (e == cudaSuccess && mode != RSI_ANY_HIT)
            e = cudaMemcpyAsync(h_count + r0, dc, 4 * (size_t)m, cudaMemcpyDeviceToHost, c->st_out);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_out[b], c->st_out);
        if (e != cudaSuccess) rc = rsi::cuda_fail(e, "rsi_query_host copy out");
    }
    cudaError_t e1 = cudaStreamSynchronize(c->st_out);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (rc) return rc;
    if (e1 != cudaSuccess || e2 != cudaSuccess) return rsi::cuda_fail(e1 != cudaSuccess ? e1 : e2, "rsi_query_host");
    rsi_stats acc{};
    acc.n_rays = n_rays;
    acc.tree_height = h->height;
    for (int64_t k = 0; k < n_chunks; ++k) {
        const rsi::DevCounters& kc = c->h_chunk_ctr[k];
        acc.node_visits += (int64_t)kc.node_visits;
        acc.tri_tests += (int64_t)kc.tri_tests;
        acc.band_rays += kc.band_count;
        acc.ambiguous += (int64_t)kc.ambiguous;
        if (kc.error && !acc.device_error) acc.device_error = kc.error;
    }
    if (stats) *stats = acc;
    if (acc.device_error) return rsi::fail(acc.device_error, "rsi_query_host: device error " + std::to_string(acc.device_error));
    return RSI_OK;
}

// ---------------------------------------------------------------- traversal order
extern "C" int rsi_segment_order(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays,
                                 int32_t* d_order, void* stream) {
    if (!h) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_segment_order: NULL handle");
    if (n_rays < 0 || n_rays > 0x7FFFFFFFll)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_segment_order: need 0 <= n_rays < 2^31");
    if (n_rays > 0 && (!d_from || !d_to || !d_order))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_segment_order: NULL segment or order pointer");
    if (n_rays == 0) return RSI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->order_hist) {
        if (rsi::pool_alloc(reinterpret_cast<void**>(&h->order_hist), sizeof(unsigned int) * rsi::kOrderBins, s) !=
            RSI_OK)
            return RSI_ERR_OOM;
    }
    // 128 KB of shared memory per block for the histogram (set on every call:
    // the attribute belongs to the current device's context)
    RSI_CUDA_TRY(cudaFuncSetAttribute(rsi::k_order_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(unsigned int) * rsi::kOrderBins)));
    float sc[3];
    for (int a = 0; a < 3; ++a) sc[a] = h->hi[a] > h->lo[a] ? 32.0f / (h->hi[a] - h->lo[a]) : 0.0f;
    RSI_CUDA_TRY(cudaMemsetAsync(h->order_hist, 0, sizeof(unsigned int) * rsi::kOrderBins, s));
    const int sms = rsi::device_sm_count();
    rsi::k_order_hist<<<sms, 1024, sizeof(unsigned int) * rsi::kOrderBins, s>>>(
        d_from, d_to, n_rays, h->lo[0], h->lo[1], h->lo[2], sc[0], sc[1], sc[2], h->order_hist);
    rsi::k_order_scan<<<1, 1024, 0, s>>>(h->order_hist);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n_rays + 255) / 256, (int64_t)sms * 8));
    rsi::k_order_scatter<<<g, 256, 0, s>>>(d_from, d_to, n_rays, h->lo[0], h->lo[1], h->lo[2], sc[0], sc[1], sc[2],
                                           h->order_hist, d_order);
    rsi::note_launches(3);
    RSI_CUDA_TRY(cudaGetLastError());
    return RSI_OK;
}

// ---------------------------------------------------------------- learned
using namespace rsi;   // the kernels and launchers above

extern "C" int rsi_cluster_labels(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n, uint32_t* d_labels,
                                  void* stream) {
    if (!h || n < 0 || n > 0x7FFFFFFFll || (n > 0 && (!d_from || !d_to || !d_labels)))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_cluster_labels: bad arguments");
    if (n == 0) return RSI_OK;
    if (h->height >= 127) return rsi::fail(RSI_ERR_STACK, "rsi_cluster_labels: tree too deep");
    QueryArgs A{};
    A.nodes = h->nodes;
    A.tris = h->tris;
    A.n_tri = h->n_tri;
    A.from = d_from;
    A.to = d_to;
    A.n_rays = n;
    A.dmax0 = h->dmax[0];
    A.dmax1 = h->dmax[1];
    A.dmax2 = h->dmax[2];
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = rsi::device_sm_count() * 8;
    if (h->height < 32) k_cluster_labels<32><<<grid, 128, 0, s>>>(A, d_labels);
    else if (h->height < 64) k_cluster_labels<64><<<grid, 128, 0, s>>>(A, d_labels);
    else k_cluster_labels<128><<<grid, 128, 0, s>>>(A, d_labels);
    rsi::note_launches(1);
    RSI_CUDA_TRY(cudaGetLastError());
    return RSI_OK;
}

extern "C" int rsi_query_learned(rsi_bvh_t h, rsi_mlp_t m, const float* d_from, const float* d_to, int64_t n_rays,
                                 const rsi_options* opt, uint8_t* d_hit, uint8_t* d_ambiguous, rsi_stats* stats,
                                 void* stream) {
    int rc = check_query_args("rsi_query_learned", h, d_from, d_to, n_rays, RSI_ANY_HIT, d_hit, nullptr);
    if (rc) return rc;
    if (!m) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_learned: NULL network");
    if (n_rays > 0x7FFFFF00ll) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_learned: too many segments");
    if (opt && opt->fp64_all)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_learned: fp64_all excludes the learned query");
    cudaStream_t s = (cudaStream_t)stream;
    if (n_rays == 0) {
        if (stats) *stats = rsi_stats{};
        return RSI_OK;
    }
    rc = rsi::ensure_band_capacity(h, n_rays, s);
    if (rc) return rc;
    rsi_options o = {};
    if (opt) o = *opt;
    o.ray_sort_tile = 0;
    o.order = nullptr;   // the fallback walks the proposal's leftovers in its own order
    int32_t* order = h->band_ids + h->band_cap;
    // proposal + verification in one tensor-core kernel (the top-4 stay in
    // registers), then the tree search over the segments it left
    k_reset_query<<<1, 1, 0, s>>>(h->ctr, (unsigned long long)n_rays);
    rsi::note_launches(1);
    rc = rsi::mlpk::propose_verify(m, h, d_from, d_to, n_rays, d_hit, d_ambiguous, order, h->ctr, o.collect_stats, s);
    if (rc) return rc;
    const rsi::PairScratch P = rsi::handle_pairs(h);
    rc = rsi::query_device(h, d_from, d_to, n_rays, RSI_ANY_HIT, &o, d_hit, nullptr, d_ambiguous, h->band_ids, nullptr,
                           h->ctr, s, order, &h->ctr->n_fallback, nullptr, &P);
    if (rc) return rc;
    if (stats) return rsi::read_stats(h, h->ctr, n_rays, stats, s);
    return RSI_OK;
}

// ---------------------------------------------------------------- batched

// Many independent (hierarchy, segment batch) pairs answered by one
// persistent traversal launch over the concatenated segment index space,
// followed by one FP64 pass; the three kernels are captured once into a CUDA
// graph and replayed by rsi_query_batched.
struct rsi_batch_s {
    int mode = 0;
    rsi_options opt{};
    int n_batches = 0;
    int total = 0;
    int height = 0;
    char* dev = nullptr;
    rsi::DevCounters* ctr = nullptr;
    int* begins = nullptr;
    rsi::BatchDesc* desc = nullptr;
    int32_t* band = nullptr;
    int32_t* fb = nullptr;        // FP64 fallback list [total]
    char* pairs = nullptr;        // pair scratch of the FP64 pass
    int64_t seg_cap = 0, pair_cap = 0;
    rsi::DevCounters* h_ctr = nullptr;
    unsigned long long* h_post = nullptr;   // pinned ring of posted counts
    cudaEvent_t post_ev[256] = {};
    cudaEvent_t reset_ev = nullptr;   // streaming: the queue was emptied on the launch stream
    bool streamed = false;
    int post_idx = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int sort_launches = 0;        // in-tile reorderings captured in the graph
    int64_t graph_kernels = 0;    // kernel nodes of the graph (launches per replay)
    rsi::RebuildSpec rebuild;     // rebuilding plans: the in-place rebuild that precedes the query
    bool rebuilds = false;
};

namespace {

void batch_destroy(rsi_batch_s* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaEvent_t e : b->post_ev)
        if (e) cudaEventDestroy(e);
    if (b->reset_ev) cudaEventDestroy(b->reset_ev);
    if (b->dev) cudaFree(b->dev);
    if (b->h_ctr) cudaFreeHost(b->h_ctr);
    if (b->h_post) cudaFreeHost(b->h_post);
    if (b->rebuilds) rsi::rebuild_release(b->rebuild);
    delete b;
}


template <int MODE>
void launch_batched(rsi_batch_s* b, const QueryArgs& A, const BatchArgs& B, cudaStream_t s) {
    const int block = b->opt.block > 0 ? b->opt.block : 256;
    const int bps = b->opt.blocks_per_sm > 0 ? b->opt.blocks_per_sm : 3;
    int64_t want = ((int64_t)b->total + block - 1) / block;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)rsi::device_sm_count() * bps));
    const int nw = b->opt.node_width == 4 ? 1 : 0;
    if (b->opt.collect_stats) launch_fp32_stack<MODE, true, true>(A, b->height, nw, grid, block, s, B, b->opt.stack);
    else launch_fp32_stack<MODE, false, true>(A, b->height, nw, grid, block, s, B, b->opt.stack);
    if (!b->opt.fp32_only) {
        const rsi::PairScratch P = rsi::carve_pairs(b->pairs, b->seg_cap, b->pair_cap, b->fb);
        launch_fp64_pass<MODE, true>(A, b->height, &P, s, B);
    }
}

}  // namespace

namespace {
int batch_create_impl(const rsi_ray_batch* batches, int n_batches, int mode, const rsi_options* opt, void* stream,
                      rsi_batch_t* out, const float* const* rebuild_V, const int32_t* const* rebuild_T) {
    if (!out) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: out is NULL");
    *out = nullptr;
    if (!batches || n_batches < 1) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: need >= 1 batch");
    if (mode != RSI_ANY_HIT && mode != RSI_COUNT) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: bad mode");
    rsi_options o = {};
    if (opt) o = *opt;
    if (o.block != 0 && (o.block < 32 || o.block > 256 || o.block % 32 != 0))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: block must be a multiple of 32 in [32, 256]");
    if (o.blocks_per_sm < 0) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: blocks_per_sm < 0");
    if (o.node_width != 0 && o.node_width != 2 && o.node_width != 3 && o.node_width != 4)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: node_width must be 0, 2, 3 or 4");
    if (o.stack != 0 && o.stack != 32 && o.stack != 64 && o.stack != 128)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: stack must be 0, 32, 64 or 128");
    if (o.timeout_ns < 0) o.ray_sort_tile = 0;   // streaming: segments arrive while the plan runs
    if (o.ray_sort_tile != 0 && (o.ray_sort_tile < 256 || o.ray_sort_tile > kMaxSortTile))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: ray_sort_tile must be 0 or in [256, 8192]");
    std::vector<int> begins(n_batches + 1, 0);
    std::vector<rsi::BatchDesc> desc(n_batches);
    int height = 0;
    int64_t total = 0;
    for (int i = 0; i < n_batches; ++i) {
        const rsi_ray_batch& rb = batches[i];
        if (!rb.bvh) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: batch " + std::to_string(i) + " has no hierarchy");
        if (rb.n_rays < 0) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: negative n_rays");
        if (rb.n_rays > 0 && (!rb.d_from || !rb.d_to || (mode == RSI_ANY_HIT && !rb.d_hit) ||
                              (mode == RSI_COUNT && !rb.d_count)))
            return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: batch " + std::to_string(i) + " lacks a buffer");
        if (rb.bvh->height >= 127) return rsi::fail(RSI_ERR_STACK, "rsi_batch_create: tree too deep");
        begins[i] = (int)total;
        total += rb.n_rays;
        if (total > 0x7FFFFFFFll) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create: more than 2^31 segments");
        height = std::max(height, rb.bvh->height);
        rsi::BatchDesc& d = desc[i];
        d.nodes = rb.bvh->nodes;
        d.nodes4 = rb.bvh->nodes4;
        d.tris = rb.bvh->tris;
        d.from = rb.d_from;
        d.to = rb.d_to;
        d.hit = rb.d_hit;
        d.count = rb.d_count;
        d.amb = rb.d_ambiguous;
        d.n_tri = (int)rb.bvh->n_tri;
        d.n_rays = (int)rb.n_rays;
        d.ray_begin = begins[i];
        d.dmax0 = rb.bvh->dmax[0];
        d.dmax1 = rb.bvh->dmax[1];
        d.dmax2 = rb.bvh->dmax[2];
    }
    begins[n_batches] = (int)total;
    if (rebuild_V) {
        // the trees are rebuilt inside the graph: their heights are not known
        // when it is captured, so every walk gets the deepest stack
        for (int i = 0; i < n_batches; ++i)
            for (int j = 0; j < i; ++j)
                if (batches[i].bvh == batches[j].bvh)
                    return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create_rebuild: hierarchy of batch " +
                                                              std::to_string(i) + " appears twice");
        height = 126;
        o.stack = 128;
        if (o.node_width == 4) o.node_width = 0;
    }
    int64_t b_seg_cap = 0, b_pair_cap = 0;
    auto* b = new rsi_batch_s();
    b->mode = mode;
    b->opt = o;
    b->n_batches = n_batches;
    b->total = (int)total;
    b->height = height;
    const size_t off_begins = 256, off_desc = off_begins + ((4 * (size_t)(n_batches + 1) + 255) & ~(size_t)255);
    const size_t off_band = off_desc + ((sizeof(rsi::BatchDesc) * (size_t)n_batches + 255) & ~(size_t)255);
    const size_t off_fb = off_band + ((4 * (size_t)std::max<int64_t>(total, 1) + 255) & ~(size_t)255);
    const size_t off_pairs = off_fb + ((4 * (size_t)std::max<int64_t>(total, 1) + 255) & ~(size_t)255);
    size_t pair_bytes;
    rsi::pair_sizes(std::max<int64_t>(total, 1), b_seg_cap, b_pair_cap, pair_bytes);
    const size_t off_perm = off_pairs + ((pair_bytes + 255) & ~(size_t)255);
    const size_t bytes = off_perm + (o.ray_sort_tile ? 4 * (size_t)std::max<int64_t>(total, 1) : 0);
    if (rsi::dev_malloc(&b->dev, bytes) != cudaSuccess || rsi::host_malloc_pinned(&b->h_ctr, sizeof(rsi::DevCounters)) != cudaSuccess ||
        rsi::host_malloc_pinned(&b->h_post, 256 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        batch_destroy(b);
        return rsi::fail(RSI_ERR_OOM, "rsi_batch_create: allocation failed");
    }
    b->ctr = reinterpret_cast<rsi::DevCounters*>(b->dev);
    b->begins = reinterpret_cast<int*>(b->dev + off_begins);
    b->desc = reinterpret_cast<rsi::BatchDesc*>(b->dev + off_desc);
    b->band = reinterpret_cast<int32_t*>(b->dev + off_band);
    b->fb = reinterpret_cast<int32_t*>(b->dev + off_fb);
    b->pairs = b->dev + off_pairs;
    int32_t* perm = o.ray_sort_tile ? reinterpret_cast<int32_t*>(b->dev + off_perm) : nullptr;
    b->seg_cap = b_seg_cap;
    b->pair_cap = b_pair_cap;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(b->begins, begins.data(), 4 * begins.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->desc, desc.data(), sizeof(rsi::BatchDesc) * desc.size(),
                                              cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ctr, 0, sizeof(rsi::DevCounters), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int i = 0; e == cudaSuccess && i < 256; ++i) e = cudaEventCreateWithFlags(&b->post_ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->reset_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        int rc = rsi::cuda_fail(e, "rsi_batch_create");
        batch_destroy(b);
        return rc;
    }
    if (rebuild_V) {
        std::vector<rsi_bvh_t> hs(n_batches);
        for (int i = 0; i < n_batches; ++i) hs[i] = batches[i].bvh;
        int rc = rsi::rebuild_prepare(hs.data(), n_batches, rebuild_V, rebuild_T, s, &b->rebuild);
        if (rc) {
            batch_destroy(b);
            return rc;
        }
        b->rebuilds = true;
    }
    // capture [rebuild ->] reset -> traversal -> FP64 pass into a graph
    QueryArgs A{};
    A.band_ids = b->band;
    A.ctr = b->ctr;
    A.fp32_only = o.fp32_only;
    BatchArgs B{b->desc, b->begins, n_batches, (int)total, o.timeout_ns > 0 ? (long long)o.timeout_ns : 2000000000ll,
                0};
    const bool streamed = o.timeout_ns < 0;
    if (streamed) B.timeout_ns = -(long long)o.timeout_ns;
    B.streamed = streamed ? 1 : 0;
    B.perm = perm;
    b->streamed = streamed;
    const uint64_t noted0 = rsi_kernel_launches();
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (b->rebuilds) {
            rsi::rebuild_enqueue(b->rebuild, b->cap);
            rsi::k_desc_dmax<<<rsi::grid_for(n_batches, 128), 128, 0, b->cap>>>(b->desc, b->rebuild.d_ctr, n_batches);
        }
        k_reset_query<<<1, 1, 0, b->cap>>>(b->ctr, streamed ? ~0ull : (unsigned long long)total);
        if (perm) {   // in-tile reordering of every batch, into the global index space
            for (int i = 0; i < n_batches; ++i) {
                const rsi_ray_batch& rb = batches[i];
                if (rb.n_rays == 0) continue;
                float sc[3];
                for (int a = 0; a < 3; ++a)
                    sc[a] = rb.bvh->hi[a] > rb.bvh->lo[a] ? 1024.0f / (rb.bvh->hi[a] - rb.bvh->lo[a]) : 0.0f;
                k_ray_tile_sort<<<rsi::grid_for(rb.n_rays, o.ray_sort_tile), 256, 0, b->cap>>>(
                    rb.d_from, rb.d_to, (int)rb.n_rays, o.ray_sort_tile, rb.bvh->lo[0], rb.bvh->lo[1], rb.bvh->lo[2],
                    sc[0], sc[1], sc[2], perm + begins[i]);
                ++b->sort_launches;
            }
        }
        if (mode == RSI_ANY_HIT) launch_batched<RSI_ANY_HIT>(b, A, B, b->cap);
        else launch_batched<RSI_COUNT>(b, A, B, b->cap);
        cudaError_t le = cudaGetLastError();
        e = cudaStreamEndCapture(b->cap, &b->graph);
        if (e == cudaSuccess) e = le;
    }
    // launches noted while capturing run on every replay instead: count the
    // graph's kernel nodes once and note that many per launch
    rsi::note_launches(-(int)(rsi_kernel_launches() - noted0));
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e == cudaSuccess) {
        size_t n_nodes = 0;
        e = cudaGraphGetNodes(b->graph, nullptr, &n_nodes);
        std::vector<cudaGraphNode_t> nodes(n_nodes);
        if (e == cudaSuccess && n_nodes) e = cudaGraphGetNodes(b->graph, nodes.data(), &n_nodes);
        for (size_t i = 0; e == cudaSuccess && i < n_nodes; ++i) {
            cudaGraphNodeType t;
            e = cudaGraphNodeGetType(nodes[i], &t);
            if (t == cudaGraphNodeTypeKernel) ++b->graph_kernels;
        }
    }
    if (e != cudaSuccess) {
        int rc = rsi::cuda_fail(e, "rsi_batch_create: graph capture");
        batch_destroy(b);
        return rc;
    }
    *out = b;
    return RSI_OK;
}
}  // namespace

extern "C" int rsi_batch_create(const rsi_ray_batch* batches, int n_batches, int mode, const rsi_options* opt,
                                void* stream, rsi_batch_t* out) {
    return batch_create_impl(batches, n_batches, mode, opt, stream, out, nullptr, nullptr);
}

extern "C" int rsi_batch_create_rebuild(const rsi_ray_batch* batches, int n_batches, const float* const* d_vertices,
                                        const int32_t* const* d_triangles, int mode, const rsi_options* opt,
                                        void* stream, rsi_batch_t* out) {
    if (!d_vertices || !d_triangles)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create_rebuild: NULL mesh arrays");
    if (opt && opt->timeout_ns < 0)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_create_rebuild: streaming plans cannot rebuild");
    return batch_create_impl(batches, n_batches, mode, opt, stream, out, d_vertices, d_triangles);
}

extern "C" int rsi_batch_launch(rsi_batch_t b, void* stream) {
    if (!b) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_launch: NULL plan");
    if (b->streamed) {   // empty the queue before any post of this run can land
        RSI_CUDA_TRY(cudaMemsetAsync(&b->ctr->ready, 0, sizeof(unsigned long long), (cudaStream_t)stream));
        RSI_CUDA_TRY(cudaEventRecord(b->reset_ev, (cudaStream_t)stream));
    }
    RSI_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    rsi::note_launches((int)b->graph_kernels);
    return RSI_OK;
}

extern "C" int rsi_batch_post(rsi_batch_t b, int64_t n_ready, void* stream) {
    if (!b) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_post: NULL plan");
    if (!b->streamed) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_post: the plan is not streaming");
    if (n_ready < 0 || n_ready > b->total) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_post: n_ready out of range");
    const int k = b->post_idx++ & 255;
    RSI_CUDA_TRY(cudaStreamWaitEvent((cudaStream_t)stream, b->reset_ev, 0));
    RSI_CUDA_TRY(cudaEventSynchronize(b->post_ev[k]));   // the slot's previous copy has run
    b->h_post[k] = (unsigned long long)n_ready;
    RSI_CUDA_TRY(cudaMemcpyAsync(&b->ctr->ready, &b->h_post[k], sizeof(unsigned long long), cudaMemcpyHostToDevice,
                                 (cudaStream_t)stream));
    RSI_CUDA_TRY(cudaEventRecord(b->post_ev[k], (cudaStream_t)stream));
    return RSI_OK;
}

extern "C" int rsi_batch_stats(rsi_batch_t b, rsi_stats* st, void* stream) {
    if (!b || !st) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_stats: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    RSI_CUDA_TRY(cudaMemcpyAsync(b->h_ctr, b->ctr, sizeof(rsi::DevCounters), cudaMemcpyDeviceToHost, s));
    RSI_CUDA_TRY(cudaStreamSynchronize(s));
    if (b->rebuilds) {   // the rebuilt hierarchies' host-side extent, padding and height
        const int rc = rsi::refresh_handles(b->rebuild, s);
        if (rc) return rc;
    }
    const rsi::DevCounters& c = *b->h_ctr;
    st->n_rays = b->total;
    st->node_visits = (int64_t)c.node_visits;
    st->tri_tests = (int64_t)c.tri_tests;
    st->band_rays = c.band_count;
    st->ambiguous = (int64_t)c.ambiguous;
    st->tree_height = b->height;
    st->device_error = c.error;
    if (c.error) return rsi::fail(c.error, "rsi_query_batched: device error " + std::to_string(c.error));
    return RSI_OK;
}

extern "C" int rsi_batch_free(rsi_batch_t b) {
    if (!b) return RSI_OK;
    cudaDeviceSynchronize();
    batch_destroy(b);
    return RSI_OK;
}

// ---------------------------------------------------------------- one-call batched query
// rsi_query_batched plans a call once and replays the plan when the same
// arguments come back: the key holds each hierarchy's process-unique id (an
// address can be reused by a later handle, an id cannot), the device, every
// batch's buffers and sizes, the mode and the options.
namespace {

struct PlanKey {
    int device = 0, mode = 0;
    rsi_options opt{};
    std::vector<uint64_t> gens;
    std::vector<rsi_ray_batch> batches;   // .bvh as given by hs
    bool operator==(const PlanKey& o) const {
        if (device != o.device || mode != o.mode || gens != o.gens || batches.size() != o.batches.size()) return false;
        // the fields a plan depends on (compared one by one: the struct has padding)
        if (opt.fp32_only != o.opt.fp32_only || opt.block != o.opt.block || opt.blocks_per_sm != o.opt.blocks_per_sm ||
            opt.collect_stats != o.opt.collect_stats || opt.timeout_ns != o.opt.timeout_ns ||
            opt.ray_sort_tile != o.opt.ray_sort_tile || opt.node_width != o.opt.node_width || opt.stack != o.opt.stack)
            return false;
        for (size_t i = 0; i < batches.size(); ++i) {
            const rsi_ray_batch &a = batches[i], &b = o.batches[i];
            if (a.bvh != b.bvh || a.d_from != b.d_from || a.d_to != b.d_to || a.n_rays != b.n_rays ||
                a.d_hit != b.d_hit || a.d_count != b.d_count || a.d_ambiguous != b.d_ambiguous)
                return false;
        }
        return true;
    }
};

constexpr size_t kPlanCacheSize = 4;
std::mutex g_plan_mu;
std::vector<std::pair<PlanKey, rsi_batch_t>> g_plans;   // most recently used last

}  // namespace

namespace rsi {
void drop_plans_of(uint64_t gen) {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    for (size_t i = 0; i < g_plans.size();) {
        const std::vector<uint64_t>& g = g_plans[i].first.gens;
        if (std::find(g.begin(), g.end(), gen) != g.end()) {
            batch_destroy(g_plans[i].second);   // the caller (lbvh_free) has synchronized the device
            g_plans.erase(g_plans.begin() + (long)i);
        } else {
            ++i;
        }
    }
}
}  // namespace rsi

extern "C" int rsi_query_batched(const rsi_bvh_t* hs, int n_meshes, const rsi_ray_batch* batches, int mode,
                                 const rsi_options* opt, void* stream) {
    if (!hs || !batches || n_meshes < 1)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_batched: need n_meshes >= 1 hierarchies and batches");
    if (opt && opt->timeout_ns < 0)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_batched: streaming plans need rsi_batch_create");
    PlanKey key;
    RSI_CUDA_TRY(cudaGetDevice(&key.device));
    key.mode = mode;
    if (opt) key.opt = *opt;
    key.gens.resize(n_meshes);
    key.batches.assign(batches, batches + n_meshes);
    for (int i = 0; i < n_meshes; ++i) {
        if (!hs[i]) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_batched: hierarchy " + std::to_string(i) + " is NULL");
        if (batches[i].bvh && batches[i].bvh != hs[i])
            return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_query_batched: batches[" + std::to_string(i) +
                                                      "].bvh is neither NULL nor hs[" + std::to_string(i) + "]");
        key.batches[i].bvh = hs[i];
        key.gens[i] = hs[i]->gen;
    }
    std::lock_guard<std::mutex> lock(g_plan_mu);
    for (size_t i = 0; i < g_plans.size(); ++i) {
        if (g_plans[i].first == key) {
            rsi_batch_t b = g_plans[i].second;
            std::rotate(g_plans.begin() + (long)i, g_plans.begin() + (long)i + 1, g_plans.end());
            return rsi_batch_launch(b, stream);
        }
    }
    rsi_batch_t b = nullptr;
    int rc = rsi_batch_create(key.batches.data(), n_meshes, mode, opt, stream, &b);
    if (rc) return rc;
    if (g_plans.size() >= kPlanCacheSize) {   // the oldest plan may still run: wait before releasing it
        cudaDeviceSynchronize();
        batch_destroy(g_plans.front().second);
        g_plans.erase(g_plans.begin());
    }
    g_plans.emplace_back(std::move(key), b);
    return rsi_batch_launch(b, stream);
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
    int rc = check_query_args("rsi_query_noalloc", h, d_from, d_to, n_rays, mode, d_hit, d_count);
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
