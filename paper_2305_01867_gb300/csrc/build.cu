// build.cu -- GPU construction of the linear BVH (Sec. 3.2, 3.3, 4.1, 4.2):
//   k_extent   surface extent (Sec. 3.3, get_min_max_extent_of_surface)
//   k_morton   30/63-bit Morton codes of triangle centroids (Sec. 3.2; the
//              paper turned the host createMortonCode into a kernel)
//   radix sort stable LSD sort of (code, triangle id), 8-bit digits (the
//              paper sorted on the host with argsort, Sec. 3.2)
//   k_karras   binary radix tree, one thread per internal node (Karras 2012,
//              cited in Sec. 1)
//   k_refit    bottom-up boxes: the second child to arrive at a node (atomic
//              counter) unions the children and climbs on (Sec. 4.2: a node
//              left with counter 1 is "half-filled")
//   k_apetrei  the alternative single pass that builds the same tree and its
//              boxes bottom-up at once (Apetrei 2014, the agglomerative build
//              the paper's Sec. 4.2 follows), replacing k_karras + k_refit
// Every grid is sized from its own element count (the grid-size error of
// Sec. 4.2.3 is the lesson) and all steps run on the caller's stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

#include "rsi_internal.cuh"

namespace rsi {
namespace {

constexpr int kBlock = 256;

// Atomic add at GPU scope with acquire-release ordering: this thread's earlier
// writes are visible to a thread that reads the result, and that thread's
// later loads see the writes released before it.
__device__ __forceinline__ int atomic_add_acq_rel(int32_t* p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ int32_t atomic_exch_acq_rel(int32_t* p, int32_t v) {
    int32_t old;
    asm volatile("atom.acq_rel.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned int f2ord(float f) {
    unsigned int b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __host__ __forceinline__ float ord2f(unsigned int o) {
    unsigned int b = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    std::memcpy(&f, &b, 4);
    return f;
#endif
}

__device__ __forceinline__ void raise_error(DevCounters* c, int code) { atomicCAS(&c->error, 0, code); }

__device__ __forceinline__ void init_counters(DevCounters* c) {
    c->error = 0;
    c->band_count = 0;
    c->height = 0;
    c->node_visits = c->tri_tests = c->ambiguous = 0;
    for (int a = 0; a < 3; ++a) {
        c->ext_bits[a] = 0xFFFFFFFFu;   // running min
        c->ext_bits[3 + a] = 0u;        // running max
        c->dmax_bits[a] = 0u;
    }
}

__global__ void k_init(DevCounters* c) {
    if (threadIdx.x == 0) init_counters(c);
}

// Per-axis min / max over all vertices; NaN raises RSI_ERR_NAN.  The
// calling threads take vertices i0, i0 + stride, ...; every lane of each
// warp must call it (warp reduction).
__device__ __forceinline__ void extent_body(const float* __restrict__ V, int64_t nv, DevCounters* c, int64_t i0,
                                            int64_t stride) {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool nan = false;
    for (int64_t i = i0; i < nv; i += stride) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float x = __ldg(V + 3 * i + a);
            nan |= (x != x);
            mn[a] = fminf(mn[a], x);
            mx[a] = fmaxf(mx[a], x);
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], off));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], off));
        }
    if (__any_sync(0xffffffffu, nan) && (threadIdx.x & 31) == 0) raise_error(c, RSI_ERR_NAN);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (mn[a] <= mx[a]) {
                atomicMin(&c->ext_bits[a], f2ord(mn[a]));
                atomicMax(&c->ext_bits[3 + a], f2ord(mx[a]));
            }
        }
    }
}

__global__ void k_extent(const float* __restrict__ V, int64_t nv, DevCounters* c) {
    extent_body(V, nv, c, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Spread the low bits of q so that bit i lands on bit 3i.
__device__ __forceinline__ uint32_t spread10(uint32_t x) {
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}
__device__ __forceinline__ uint64_t spread21(uint64_t x) {
    x &= 0x1FFFFFull;
    x = (x | (x << 32)) & 0x001F00000000FFFFull;
    x = (x | (x << 16)) & 0x001F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

template <typename K>
struct MortonTraits;
template <>
struct MortonTraits<uint32_t> {
    static constexpr int kBitsPerAxis = 10;
    static __device__ __forceinline__ uint32_t encode(uint32_t x, uint32_t y, uint32_t z) {
        return spread10(x) | (spread10(y) << 1) | (spread10(z) << 2);
    }
};
template <>
struct MortonTraits<uint64_t> {
    static constexpr int kBitsPerAxis = 21;
    static __device__ __forceinline__ uint64_t encode(uint32_t x, uint32_t y, uint32_t z) {
        return spread21(x) | (spread21(y) << 1) | (spread21(z) << 2);
    }
};

// Morton code of triangle j: centroid ((v0 + v1) + v2) / 3, normalised per
// axis by the extent, clamped to [0, 1], truncated to b bits; z is the high
// bit of every 3-bit group.  Explicit round-to-nearest intrinsics keep the
// compiler from fusing any multiply-add, so the code is the same on any host
// that evaluates the same IEEE operations.
template <typename K>
__device__ __forceinline__ K morton_key(const float* __restrict__ V, int64_t nv, const int32_t* __restrict__ T,
                                        int64_t j, DevCounters* c) {
    const int b = MortonTraits<K>::kBitsPerAxis;
    const float scale = (float)(1u << b);
    const uint32_t qmax = (1u << b) - 1u;
    int32_t i0 = __ldg(T + 3 * j), i1 = __ldg(T + 3 * j + 1), i2 = __ldg(T + 3 * j + 2);
    if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {
        raise_error(c, RSI_ERR_INDEX);
        return K(0);
    }
    uint32_t q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float lo = ord2f(c->ext_bits[a]), hi = ord2f(c->ext_bits[3 + a]);
        float x0 = __ldg(V + 3 * (int64_t)i0 + a), x1 = __ldg(V + 3 * (int64_t)i1 + a), x2 = __ldg(V + 3 * (int64_t)i2 + a);
        float cen = __fdiv_rn(__fadd_rn(__fadd_rn(x0, x1), x2), 3.0f);
        float u = (hi != lo) ? __fdiv_rn(__fsub_rn(cen, lo), __fsub_rn(hi, lo)) : 0.0f;
        u = fminf(fmaxf(u, 0.0f), 1.0f);
        uint32_t qq = __float2uint_rz(__fmul_rn(u, scale));
        q[a] = qq > qmax ? qmax : qq;
    }
    return MortonTraits<K>::encode(q[0], q[1], q[2]);
}

// With `hist0`, also the count of every lowest 8-bit digit per sort tile of
// `tile` keys (tile-major, 256 counters per tile): the first pass's histogram.
template <typename K>
__global__ void k_morton(const float* __restrict__ V, int64_t nv, const int32_t* __restrict__ T, int64_t nt,
                         DevCounters* c, K* __restrict__ keys, int32_t* __restrict__ ids, uint32_t* __restrict__ hist0,
                         int tile) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= nt) return;
    ids[j] = (int32_t)j;
    const K key = morton_key<K>(V, nv, T, j, c);
    keys[j] = key;
    if (hist0) atomicAdd(&hist0[(j / tile) * 256 + (uint32_t)(key & 255u)], 1u);
}

// ---------------------------------------------------------------- radix sort
// One LSD pass over 8-bit digit `shift`: per-tile histograms (digit-major so
// a single exclusive scan yields every tile's scatter base), then a stable
// scatter that ranks keys inside the tile in index order.
constexpr int kSortTile = 4096;   // keys per block (16 rounds of 256)

template <typename K>
__global__ void k_rs_hist(const K* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist, int ntiles) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    int64_t end = min(base + (int64_t)kSortTile, n);
    for (int64_t i = base + threadIdx.x; i < end; i += blockDim.x)
        atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of m words by one block of 1024 threads.
__global__ void k_rs_scan(uint32_t* __restrict__ h, int64_t m) {
    __shared__ uint32_t part[1024];
    int64_t per = (m + blockDim.x - 1) / blockDim.x;
    int64_t b = threadIdx.x * per, e = min(b + per, m);
    uint32_t s = 0;
    for (int64_t i = b; i < e; ++i) s += h[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;
    for (int64_t i = b; i < e; ++i) {
        uint32_t v = h[i];
        h[i] = run;
        run += v;
    }
}

// Stable scatter of `rounds` rounds of 256 keys from tile0 on: keys are
// ranked inside each round in index order (warp match, then the warps in
// order) and go to base[digit] + rank; base[] advances by each round's
// counts.  With `hist_next`, every written key is also counted under its next
// digit in the histogram of the output tile (tsize keys) it lands in.
template <typename K>
__device__ __forceinline__ void scatter_rounds(const K* __restrict__ kin, const int32_t* __restrict__ vin,
                                               K* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
                                               int shift, int64_t tile0, int rounds, uint32_t* base,
                                               uint32_t (*wcnt)[256], uint32_t* __restrict__ hist_next,
                                               int64_t tsize) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r < rounds; ++r) {
        int64_t i = tile0 + r * 256 + threadIdx.x;
        bool valid = i < n;
        K key = valid ? kin[i] : K(0);
        uint32_t dig = valid ? ((uint32_t)(key >> shift) & 255u) : 256u + lane;   // invalid lanes never match
#pragma unroll
        for (int w = 0; w < 8; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        uint32_t peers = __match_any_sync(0xffffffffu, dig);
        uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[warp][dig] = __popc(peers);
        __syncthreads();
        // exclusive prefix over warps for digit threadIdx.x; total goes to base
        {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                uint32_t v = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = run;
                run += v;
            }
            __syncthreads();
            if (valid) {
                uint32_t pos = base[dig] + wcnt[warp][dig] + rank;
                kout[pos] = key;
                vout[pos] = vin[i];
                if (hist_next) atomicAdd(&hist_next[(pos / tsize) * 256 + ((uint32_t)(key >> (shift + 8)) & 255u)], 1u);
            }
            __syncthreads();
            base[threadIdx.x] += run;
        }
        __syncthreads();
    }
}

template <typename K>
__global__ void __launch_bounds__(256) k_rs_scatter(const K* __restrict__ kin, const int32_t* __restrict__ vin,
                                                    K* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
                                                    int shift, const uint32_t* __restrict__ hist, int ntiles) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[8][256];
    base[threadIdx.x] = hist[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    scatter_rounds<K>(kin, vin, kout, vout, n, shift, (int64_t)blockIdx.x * kSortTile, kSortTile / 256, base, wcnt,
                      nullptr, 1);
}

// One pass of the single-mesh sort (at most kScanTiles tiles of 256 * rounds
// keys): the block sums the tile histograms itself -- digit d of tile b
// starts after every key of a smaller digit and the keys of digit d in tiles
// before b -- then scatters its tile stably and counts the next digit of the
// written keys per output tile (hist_next, null in the last pass).
constexpr int kScanTiles = 128;
template <typename K>
__global__ void __launch_bounds__(256) k_rs_pass(const K* __restrict__ kin, const int32_t* __restrict__ vin,
                                                 K* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
                                                 int shift, int rounds, int ntiles, const uint32_t* __restrict__ hist,
                                                 uint32_t* __restrict__ hist_next) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[8][256];
    __shared__ uint32_t wsum[8];
    const int d = threadIdx.x, lane = d & 31, warp = d >> 5;
    uint32_t before = 0, total = 0;
    for (int t0 = 0; t0 < ntiles; t0 += 32) {   // 32 independent loads in flight per thread
        uint32_t c[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) c[u] = t0 + u < ntiles ? __ldcg(hist + (int64_t)(t0 + u) * 256 + d) : 0u;
#pragma unroll
        for (int u = 0; u < 32; ++u) {
            before += t0 + u < (int)blockIdx.x ? c[u] : 0u;
            total += c[u];
        }
    }
    uint32_t incl = total;   // inclusive scan of the digit totals: warps, then across warps
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += wsum[w];
    base[d] = wpre + incl - total + before;
    const int64_t tsize = (int64_t)rounds * 256;
    scatter_rounds<K>(kin, vin, kout, vout, n, shift, (int64_t)blockIdx.x * tsize, rounds, base, wcnt, hist_next,
                      tsize);
}

// How a single mesh's keys are sorted: up to kScanTiles * kSortTile keys in
// tiles of 256 * rounds keys (rounds as small as the tile limit allows, so
// that small meshes get many short blocks), one launch per pass; more keys
// take the three-launch passes over tiles of kSortTile keys.
struct SortPlan {
    int rounds, ntiles;
    bool fused;
};
inline SortPlan sort_plan(int64_t n) {
    if (n > (int64_t)kScanTiles * kSortTile) return {kSortTile / 256, grid_for(n, kSortTile), false};
    int64_t rounds = (n + 256LL * kScanTiles - 1) / (256LL * kScanTiles);
    if (rounds < 1) rounds = 1;
    return {(int)rounds, grid_for(n, 256 * (int)rounds), true};
}
inline size_t sort_hist_bytes(int64_t n, int passes) {
    const SortPlan sp = sort_plan(n);
    const size_t three = 4 * 256 * (size_t)grid_for(n, kSortTile);
    return sp.fused ? std::max(three, 4 * 256 * (size_t)sp.ntiles * passes) : three;
}

// ---------------------------------------------------------------- radix tree
template <typename K>
struct KeyBits;
template <>
struct KeyBits<uint32_t> {
    static __device__ __forceinline__ int clz(uint32_t x) { return __clz(x); }
    static constexpr int kWidth = 32;
};
template <>
struct KeyBits<uint64_t> {
    static __device__ __forceinline__ int clz(uint64_t x) { return __clzll(x); }
    static constexpr int kWidth = 64;
};

// Length of the common prefix of the keys at i and j, with the index appended
// below the key so that equal keys still differ; -1 outside [0, n).
template <typename K>
__device__ __forceinline__ int delta(const K* __restrict__ k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    K a = k[i], b = k[j];
    if (a == b) return KeyBits<K>::kWidth + __clz((uint32_t)i ^ (uint32_t)j);
    return KeyBits<K>::clz(a ^ b);
}

// Internal node i (Karras 2012): find the direction of its range, the other
// end j by an exponential then binary search on the common-prefix length,
// and the split gamma by a binary search; children are gamma and gamma + 1,
// leaves when they coincide with an end of the range.
template <typename K>
__device__ __forceinline__ void karras_node(const K* __restrict__ k, int64_t n, int64_t i, int32_t* __restrict__ left,
                                            int32_t* __restrict__ right, int32_t* __restrict__ parent) {
    int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) > 0 ? 1 : -1;
    int dmin = delta(k, n, i, i - d);
    int64_t lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    int64_t j = i + l * d;
    int dnode = delta(k, n, i, j);
    int64_t s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int64_t g = i + s * d + (d < 0 ? -1 : 0);
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    int32_t lc, rc;
    if (lo == g) { lc = (int32_t)(kLeafTag | (uint32_t)g); parent[n - 1 + g] = (int32_t)i; }
    else { lc = (int32_t)g; parent[g] = (int32_t)i; }
    if (hi == g + 1) { rc = (int32_t)(kLeafTag | (uint32_t)(g + 1)); parent[n - 1 + g + 1] = (int32_t)i; }
    else { rc = (int32_t)(g + 1); parent[g + 1] = (int32_t)i; }
    left[i] = lc;
    right[i] = rc;
    if (i == 0) parent[0] = -1;
}

template <typename K>
__global__ void k_karras(const K* __restrict__ k, int64_t n, int32_t* __restrict__ left, int32_t* __restrict__ right,
                         int32_t* __restrict__ parent) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n - 1) karras_node<K>(k, n, i, left, right, parent);
}

// ---------------------------------------------------------------- refit
__device__ __forceinline__ int64_t box_slot(int32_t ref, int64_t n) {
    return ((uint32_t)ref & kLeafTag) ? (n - 1 + (int64_t)((uint32_t)ref & ~kLeafTag)) : (int64_t)ref;
}
__device__ __forceinline__ int packed_ref(int32_t ref) {
    return ((uint32_t)ref & kLeafTag) ? ~(int)((uint32_t)ref & ~kLeafTag) : (int)ref;
}

// Leaf j: pack triangle perm[j] and its box, then climb: the first thread to
// reach a node stops, the second (both child boxes final) writes the node.
__global__ void k_refit(const float* __restrict__ V, int64_t nv, const int32_t* __restrict__ T,
                        const int32_t* __restrict__ perm, int64_t n, const int32_t* __restrict__ left,
                        const int32_t* __restrict__ right, const int32_t* __restrict__ parent,
                        float* __restrict__ box, int32_t* __restrict__ hgt, int32_t* __restrict__ flag,
                        Node* __restrict__ nodes, Tri* __restrict__ tris, DevCounters* c) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    int32_t t = perm[j];
    int32_t i0 = T[3 * (int64_t)t], i1 = T[3 * (int64_t)t + 1], i2 = T[3 * (int64_t)t + 2];
    float v[3][3];
    if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {
        raise_error(c, RSI_ERR_INDEX);
#pragma unroll
        for (int a = 0; a < 3; ++a) v[0][a] = v[1][a] = v[2][a] = 0.0f;
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            v[0][a] = V[3 * (int64_t)i0 + a];
            v[1][a] = V[3 * (int64_t)i1 + a];
            v[2][a] = V[3 * (int64_t)i2 + a];
        }
    }
    Tri tr;
    tr.v0 = make_float4(v[0][0], v[0][1], v[0][2], __int_as_float(t));
    tr.v1 = make_float4(v[1][0], v[1][1], v[1][2], 0.0f);
    tr.v2 = make_float4(v[2][0], v[2][1], v[2][2], 0.0f);
    tr.pad = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    tris[j] = tr;
    float* bx = box + 6 * (n - 1 + j);
    float cb[6];   // the box and height of the subtree this thread climbs from
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float mn = fminf(fminf(v[0][a], v[1][a]), v[2][a]);
        float mx = fmaxf(fmaxf(v[0][a], v[1][a]), v[2][a]);
        bx[a] = cb[a] = mn;
        bx[3 + a] = cb[3 + a] = mx;
        atomicMax(&c->dmax_bits[a], __float_as_uint(mx - mn));   // >= 0: uint order = float order
    }
    hgt[n - 1 + j] = 0;
    if (n == 1) return;
    int ch = 0;
    int64_t from = n - 1 + j;
    int32_t node = parent[n - 1 + j];
    while (node >= 0) {
        // the node's links are fixed during the pass: read them before arriving
        const int32_t lc = left[node], rc = right[node], up = parent[node];
        // release this thread's box writes and acquire the sibling's: the
        // first arrival stops, the second unions the two children
        if (atomic_add_acq_rel(&flag[node], 1) == 0) return;
        const int64_t sl = box_slot(lc, n), sr = box_slot(rc, n);
        const bool from_left = sl == from;
        const int64_t sib = from_left ? sr : sl;
        float sb[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) sb[a] = __ldcg(box + 6 * sib + a);
        const int h = 1 + max(ch, __ldcg(hgt + sib));
        float bl[6], br[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            bl[a] = from_left ? cb[a] : sb[a];
            br[a] = from_left ? sb[a] : cb[a];
        }
        float* bn = box + 6 * (int64_t)node;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bn[a] = cb[a] = fminf(bl[a], br[a]);
            bn[3 + a] = cb[3 + a] = fmaxf(bl[3 + a], br[3 + a]);
        }
        hgt[node] = h;
        ch = h;
        from = node;
        Node nd;
        nd.lmin = make_float4(bl[0], bl[1], bl[2], __int_as_float(packed_ref(lc)));
        nd.lmax = make_float4(bl[3], bl[4], bl[5], __int_as_float(packed_ref(rc)));
        nd.rmin = make_float4(br[0], br[1], br[2], 0.0f);
        nd.rmax = make_float4(br[3], br[4], br[5], 0.0f);
        nodes[node] = nd;
        if (node == 0) c->height = h;
        node = up;
    }
}

// ---------------------------------------------------------------- 4-wide nodes
// Binary node i at even depth becomes a four-wide node holding its children,
// an internal child being replaced by that child's two children.  Child order
// is leaf order (Morton order).  Odd-depth nodes get no four-wide node.
__device__ __forceinline__ void collapse_node(const Node* __restrict__ nodes, const int32_t* __restrict__ parent,
                                              int64_t i, Node4* __restrict__ out) {
    int depth = 0;
    for (int32_t p = (int32_t)i; p != 0; p = parent[p]) ++depth;
    if (depth & 1) return;
    float bx[6][4];
    int rf[4];
    int m = 0;
    const Node nd = nodes[i];
    const float4 side[2][2] = {{nd.lmin, nd.lmax}, {nd.rmin, nd.rmax}};
    const int refs[2] = {__float_as_int(nd.lmin.w), __float_as_int(nd.lmax.w)};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (refs[c] < 0) {   // a leaf: kept as it is
            bx[0][m] = side[c][0].x; bx[1][m] = side[c][1].x;
            bx[2][m] = side[c][0].y; bx[3][m] = side[c][1].y;
            bx[4][m] = side[c][0].z; bx[5][m] = side[c][1].z;
            rf[m++] = refs[c];
        } else {             // an internal node: its two children instead
            const Node k = nodes[refs[c]];
            const float4 ks[2][2] = {{k.lmin, k.lmax}, {k.rmin, k.rmax}};
            const int krefs[2] = {__float_as_int(k.lmin.w), __float_as_int(k.lmax.w)};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                bx[0][m] = ks[e][0].x; bx[1][m] = ks[e][1].x;
                bx[2][m] = ks[e][0].y; bx[3][m] = ks[e][1].y;
                bx[4][m] = ks[e][0].z; bx[5][m] = ks[e][1].z;
                rf[m++] = krefs[e];
            }
        }
    }
    for (int c = m; c < 4; ++c) {   // empty lanes: a NaN box (never passes a slab test) and kEmpty4
        for (int a = 0; a < 6; ++a) bx[a][c] = __int_as_float(0x7fc00000);
        rf[c] = kEmpty4;
    }
    Node4 o;
    o.xlo = make_float4(bx[0][0], bx[0][1], bx[0][2], bx[0][3]);
    o.xhi = make_float4(bx[1][0], bx[1][1], bx[1][2], bx[1][3]);
    o.ylo = make_float4(bx[2][0], bx[2][1], bx[2][2], bx[2][3]);
    o.yhi = make_float4(bx[3][0], bx[3][1], bx[3][2], bx[3][3]);
    o.zlo = make_float4(bx[4][0], bx[4][1], bx[4][2], bx[4][3]);
    o.zhi = make_float4(bx[5][0], bx[5][1], bx[5][2], bx[5][3]);
    o.ref = make_int4(rf[0], rf[1], rf[2], rf[3]);
    o.pad = make_int4(m, 0, 0, 0);
    out[i] = o;
}

__global__ void k_collapse4(const Node* __restrict__ nodes, const int32_t* __restrict__ parent, int64_t n,
                            Node4* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n - 1) collapse_node(nodes, parent, i, out);
}

// ---------------------------------------------------------------- compressed nodes
// Smallest power of two 2^k (k >= -126, a normal float) whose 255 multiples
// reach `ext` with a little to spare.
__device__ __forceinline__ int grid_exponent(double ext) {
    int k = -126;
    if (ext > 0.0) {
        const double need = ext * (1.0 + 0x1p-40);
        k = ilogb(need / 255.0);
        while (ldexp(255.0, k) < need) ++k;
        while (k > -126 && ldexp(255.0, k - 1) >= need) --k;
        if (k < -126) k = -126;
    }
    return k;
}

// Grid coordinate of a lower plane: the largest q whose rebuilt value
// fma_rd(q, step, o) does not exceed x (q = 0 gives o <= x).
__device__ __forceinline__ unsigned quant_lo(float x, float o, float step) {
    double q = floor(((double)x - (double)o) / (double)step);
    unsigned u = q < 0.0 ? 0u : (q > 255.0 ? 255u : (unsigned)q);
    while (u > 0 && __fmaf_rd((float)u, step, o) > x) --u;
    while (u < 255 && __fmaf_rd((float)(u + 1), step, o) <= x) ++u;
    return u;
}

// Grid coordinate of an upper plane: the smallest q whose rebuilt value
// fma_ru(q, step, o) is at least x (255 always is, by the choice of step).
__device__ __forceinline__ unsigned quant_hi(float x, float o, float step) {
    double q = ceil(((double)x - (double)o) / (double)step);
    unsigned u = q < 0.0 ? 0u : (q > 255.0 ? 255u : (unsigned)q);
    while (u < 255 && __fmaf_ru((float)u, step, o) < x) ++u;
    while (u > 0 && __fmaf_ru((float)(u - 1), step, o) >= x) --u;
    return u;
}

// One compressed node per internal node.  The right child must be the left
// one + 1 (Karras numbering); anything else raises RSI_ERR_INDEX.
__global__ void k_quantize(const Node* __restrict__ nodes, int64_t n, NodeQ* __restrict__ out,
                           DevCounters* __restrict__ ctr) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const Node nd = nodes[i];
    const float lo[3] = {fminf(nd.lmin.x, nd.rmin.x), fminf(nd.lmin.y, nd.rmin.y), fminf(nd.lmin.z, nd.rmin.z)};
    const float hi[3] = {fmaxf(nd.lmax.x, nd.rmax.x), fmaxf(nd.lmax.y, nd.rmax.y), fmaxf(nd.lmax.z, nd.rmax.z)};
    float step[3];
    unsigned meta = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int k = grid_exponent((double)hi[a] - (double)lo[a]);
        step[a] = __int_as_float((k + 127) << 23);
        meta |= (unsigned)(k + 127) << (8 * a);
    }
    const float clo[2][3] = {{nd.lmin.x, nd.lmin.y, nd.lmin.z}, {nd.rmin.x, nd.rmin.y, nd.rmin.z}};
    const float chi[2][3] = {{nd.lmax.x, nd.lmax.y, nd.lmax.z}, {nd.rmax.x, nd.rmax.y, nd.rmax.z}};
    unsigned b[12];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            b[6 * c + a] = quant_lo(clo[c][a], lo[a], step[a]);
            b[6 * c + 3 + a] = quant_hi(chi[c][a], lo[a], step[a]);
        }
    }
    const int lref = __float_as_int(nd.lmin.w), rref = __float_as_int(nd.lmax.w);
    const int split = lref >= 0 ? lref : ~lref;
    const int right = rref >= 0 ? rref : ~rref;
    if (right != split + 1) atomicCAS(&ctr->error, 0, RSI_ERR_INDEX);
    meta |= (lref < 0 ? 1u : 0u) << 24 | (rref < 0 ? 1u : 0u) << 25;
    NodeQ q;
    q.ox = lo[0];
    q.oy = lo[1];
    q.oz = lo[2];
    q.meta = meta;
    q.w0 = b[0] | b[1] << 8 | b[2] << 16 | b[3] << 24;
    q.w1 = b[4] | b[5] << 8 | b[6] << 16 | b[7] << 24;
    q.w2 = b[8] | b[9] << 8 | b[10] << 16 | b[11] << 24;
    q.split = split;
    out[i] = q;
}

// ---------------------------------------------------------------- single pass
// Agglomerative build (Apetrei 2014; the bottom-up construction of Sec. 4.2):
// one thread per leaf climbs the tree.  A node covering leaves [lo, hi] is
// the left child of the node split between hi and hi + 1 if the keys there
// share a longer prefix than the keys at lo - 1, lo (delta() with the index
// appended, -1 past either end); otherwise it is the right child of the node
// split between lo - 1 and lo.  Both children post their outer range end to
// the parent's split slot with one atomic exchange; the second to arrive
// learns the parent's full range, unions the boxes and climbs on.
//
// The radix tree over distinct (key, index) pairs is unique, so this is the
// tree k_karras builds; it is written in the same Karras numbering (the root
// is 0, a left child is numbered by its last leaf, a right child by its
// first), which a node learns only when it knows which side of its parent it
// is on -- so a node's arrays are written one step up the climb.
template <typename K>
__device__ __forceinline__ void apetrei_leaf(const float* __restrict__ V, int64_t nv, const int32_t* __restrict__ T,
                                             const int32_t* __restrict__ perm, const K* __restrict__ keys, int64_t n,
                                             int64_t j, int32_t* __restrict__ left, int32_t* __restrict__ right,
                                             int32_t* __restrict__ parent, float* __restrict__ box,
                                             int32_t* __restrict__ hgt, int32_t* __restrict__ ends,
                                             Node* __restrict__ nodes, Tri* __restrict__ tris, DevCounters* c) {
    int32_t t = perm[j];
    int32_t i0 = T[3 * (int64_t)t], i1 = T[3 * (int64_t)t + 1], i2 = T[3 * (int64_t)t + 2];
    float v[3][3];
    if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {
        raise_error(c, RSI_ERR_INDEX);
#pragma unroll
        for (int a = 0; a < 3; ++a) v[0][a] = v[1][a] = v[2][a] = 0.0f;
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            v[0][a] = V[3 * (int64_t)i0 + a];
            v[1][a] = V[3 * (int64_t)i1 + a];
            v[2][a] = V[3 * (int64_t)i2 + a];
        }
    }
    Tri tr;
    tr.v0 = make_float4(v[0][0], v[0][1], v[0][2], __int_as_float(t));
    tr.v1 = make_float4(v[1][0], v[1][1], v[1][2], 0.0f);
    tr.v2 = make_float4(v[2][0], v[2][1], v[2][2], 0.0f);
    tr.pad = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    tris[j] = tr;
    float b[6];   // box of the current node: min xyz, max xyz
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b[a] = fminf(fminf(v[0][a], v[1][a]), v[2][a]);
        b[3 + a] = fmaxf(fmaxf(v[0][a], v[1][a]), v[2][a]);
        box[6 * (n - 1 + j) + a] = b[a];
        box[6 * (n - 1 + j) + 3 + a] = b[3 + a];
        atomicMax(&c->dmax_bits[a], __float_as_uint(b[3 + a] - b[a]));
    }
    hgt[n - 1 + j] = 0;
    if (n == 1) {
        parent[0] = -1;
        return;
    }
    int64_t lo = j, hi = j;
    int h = 0;
    int64_t split = -1;   // split of the current node (-1: it is the leaf j)
    float bl[6], br[6];   // its children's boxes (internal nodes only)
    for (;;) {
        const bool root = lo == 0 && hi == n - 1;
        const bool is_left = !root && delta(keys, n, hi, hi + 1) > delta(keys, n, lo, lo - 1);
        if (split >= 0) {
            // the current internal node learns its number and writes itself
            const int64_t k = root ? 0 : (is_left ? hi : lo);
            const int32_t lc = lo == split ? (int32_t)(kLeafTag | (uint32_t)split) : (int32_t)split;
            const int32_t rc = hi == split + 1 ? (int32_t)(kLeafTag | (uint32_t)(split + 1)) : (int32_t)(split + 1);
            left[k] = lc;
            right[k] = rc;
            parent[box_slot(lc, n)] = (int32_t)k;
            parent[box_slot(rc, n)] = (int32_t)k;
#pragma unroll
            for (int a = 0; a < 6; ++a) box[6 * k + a] = b[a];
            hgt[k] = h;
            Node nd;
            nd.lmin = make_float4(bl[0], bl[1], bl[2], __int_as_float(packed_ref(lc)));
            nd.lmax = make_float4(bl[3], bl[4], bl[5], __int_as_float(packed_ref(rc)));
            nd.rmin = make_float4(br[0], br[1], br[2], 0.0f);
            nd.rmax = make_float4(br[3], br[4], br[5], 0.0f);
            nodes[k] = nd;
            if (root) {
                parent[0] = -1;
                c->height = h;
            }
        }
        if (root) return;
        const int64_t g = is_left ? hi : lo - 1;   // the parent's split
        // released with this thread's writes; acquires the sibling's
        const int32_t other = atomic_exch_acq_rel(&ends[g], (int32_t)(is_left ? lo : hi));
        if (other < 0) return;   // first to arrive: the sibling carries on
        const int64_t plo = is_left ? lo : (int64_t)other, phi = is_left ? (int64_t)other : hi;
        // the sibling's number (as in the Karras numbering) and its box
        const int64_t sib = is_left ? (phi == g + 1 ? n - 1 + g + 1 : g + 1) : (plo == g ? n - 1 + g : g);
        float s[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) s[a] = __ldcg(box + 6 * sib + a);
        h = 1 + max(h, __ldcg(hgt + sib));
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            bl[a] = is_left ? b[a] : s[a];
            br[a] = is_left ? s[a] : b[a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            b[a] = fminf(bl[a], br[a]);
            b[3 + a] = fmaxf(bl[3 + a], br[3 + a]);
        }
        lo = plo;
        hi = phi;
        split = g;
    }
}

template <typename K>
__global__ void k_apetrei(const float* __restrict__ V, int64_t nv, const int32_t* __restrict__ T,
                          const int32_t* __restrict__ perm, const K* __restrict__ keys, int64_t n,
                          int32_t* __restrict__ left, int32_t* __restrict__ right, int32_t* __restrict__ parent,
                          float* __restrict__ box, int32_t* __restrict__ hgt, int32_t* __restrict__ ends,
                          Node* __restrict__ nodes, Tri* __restrict__ tris, DevCounters* c) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < n) apetrei_leaf<K>(V, nv, T, perm, keys, n, j, left, right, parent, box, hgt, ends, nodes, tris, c);
}

template <typename K>
int sort_pairs(K* ka, int32_t* va, K* kb, int32_t* vb, int64_t n, int passes, uint32_t* hist, cudaStream_t s,
               K** out_k, int32_t** out_v) {
    int ntiles = grid_for(n, kSortTile);
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_hist<K><<<ntiles, 256, 0, s>>>(ka, n, shift, hist, ntiles);
        k_rs_scan<<<1, 1024, 0, s>>>(hist, (int64_t)256 * ntiles);
        k_rs_scatter<K><<<ntiles, 256, 0, s>>>(ka, va, kb, vb, n, shift, hist, ntiles);
        note_launches(3);
        K* tk = ka; ka = kb; kb = tk;
        int32_t* tv = va; va = vb; vb = tv;
    }
    *out_k = ka;
    *out_v = va;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RSI_OK : rsi::cuda_fail(e, "radix sort launch");
}

// The fused passes (sort_plan(n).fused): hist holds one tile-major
// histogram per pass, zeroed, the first filled by k_morton; the last pass
// writes the sorted keys and values to out_k / out_v.
template <typename K>
int sort_pairs_fused(K* ka, int32_t* va, K* kb, int32_t* vb, int64_t n, int passes, const SortPlan& sp,
                     uint32_t* hist, K* out_k, int32_t* out_v, cudaStream_t s) {
    const size_t per = (size_t)256 * sp.ntiles;
    for (int p = 0; p < passes; ++p) {
        const bool last = p + 1 == passes;
        k_rs_pass<K><<<sp.ntiles, 256, 0, s>>>(ka, va, last ? out_k : kb, last ? out_v : vb, n, 8 * p, sp.rounds,
                                                sp.ntiles, hist + per * p, last ? nullptr : hist + per * (p + 1));
        K* tk = ka;
        ka = kb;
        kb = tk;
        int32_t* tv = va;
        va = vb;
        vb = tv;
    }
    note_launches(passes);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RSI_OK : rsi::cuda_fail(e, "radix sort launch");
}

template <typename K>
int build_impl(rsi_bvh_s* h, const float* V, const int32_t* T, int builder, cudaStream_t s, char* scratch,
               float* box, int32_t* hgt, int32_t* flag) {
    const int64_t n = h->n_tri;
    K* ka = (K*)scratch;
    K* kb = ka + n;
    int32_t* va = (int32_t*)(kb + n);
    int32_t* vb = va + n;
    uint32_t* hist = (uint32_t*)(vb + n);
    const int passes = sizeof(K) == 4 ? 4 : 8;   // 30-bit codes: 4 digits; 63-bit: 8
    const SortPlan sp = sort_plan(n);
    if (sp.fused) RSI_CUDA_TRY(cudaMemsetAsync(hist, 0, (size_t)4 * 256 * sp.ntiles * passes, s));
    k_morton<K><<<grid_for(n, kBlock), kBlock, 0, s>>>(V, h->n_vert, T, n, h->ctr, ka, va, sp.fused ? hist : nullptr,
                                                       256 * sp.rounds);
    note_launches(1);
    if (sp.fused) {
        const int rc = sort_pairs_fused<K>(ka, va, kb, vb, n, passes, sp, hist, (K*)h->sorted_keys, h->perm, s);
        if (rc) return rc;
    } else {
        K* sk;
        int32_t* sv;
        const int rc = sort_pairs<K>(ka, va, kb, vb, n, passes, hist, s, &sk, &sv);
        if (rc) return rc;
        RSI_CUDA_TRY(cudaMemcpyAsync(h->sorted_keys, sk, n * sizeof(K), cudaMemcpyDeviceToDevice, s));
        RSI_CUDA_TRY(cudaMemcpyAsync(h->perm, sv, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    if (builder == RSI_TREE_APETREI) {
        k_apetrei<K><<<grid_for(n, kBlock), kBlock, 0, s>>>(V, h->n_vert, T, h->perm, (const K*)h->sorted_keys, n,
                                                             h->left, h->right, h->parent, box, hgt, flag, h->nodes,
                                                             h->tris, h->ctr);
        note_launches(1);
        return RSI_OK;
    }
    if (n > 1) {
        k_karras<K><<<grid_for(n - 1, kBlock), kBlock, 0, s>>>((const K*)h->sorted_keys, n, h->left, h->right,
                                                                h->parent);
        note_launches(1);
    } else
        RSI_CUDA_TRY(cudaMemsetAsync(h->parent, 0xFF, sizeof(int32_t), s));
    k_refit<<<grid_for(n, kBlock), kBlock, 0, s>>>(V, h->n_vert, T, h->perm, n, h->left, h->right, h->parent, box,
                                                   hgt, flag, h->nodes, h->tris, h->ctr);
    note_launches(1);
    return RSI_OK;
}

// ---------------------------------------------------------------- many meshes
// One build of many meshes (lbvh_build_batched): every stage is one launch
// over all meshes' vertices, triangles or nodes; a thread finds its mesh by
// a binary search over the prefix of the per-mesh counts and then runs the
// single-mesh code on that mesh's arrays.
// The mesh m with pre[m] <= g < pre[m + 1] (pre: M + 1 prefix entries).
__device__ __forceinline__ int mesh_of(const int64_t* __restrict__ pre, int M, int64_t g) {
    int lo = 0, hi = M - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(pre + mid) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_init_seg(const MeshBuild* __restrict__ d, int M) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) init_counters(d[m].ctr);
}

__global__ void k_extent_seg(const MeshBuild* __restrict__ d) {   // one block per mesh
    const MeshBuild& mb = d[blockIdx.x];
    extent_body(mb.V, mb.nv, mb.ctr, threadIdx.x, blockDim.x);
}

// Morton code of every triangle (global index g, tri_pre = triangle prefix),
// a copy of it by triangle, the identity as values, and the range-end slots
// of the bottom-up pass set to -1.
template <typename K>
__global__ void k_morton_seg(const MeshBuild* __restrict__ d, const int64_t* __restrict__ tri_pre, int M, int64_t total,
                             K* __restrict__ keys, K* __restrict__ codes, int32_t* __restrict__ vals) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int m = mesh_of(tri_pre, M, g);
    const MeshBuild& mb = d[m];
    const int64_t j = g - tri_pre[m];
    const K key = morton_key<K>(mb.V, mb.nv, mb.T, j, mb.ctr);
    keys[g] = key;
    codes[g] = key;
    vals[g] = (int32_t)g;
    if (j < mb.nt - 1) mb.ends[j] = -1;
}

// The mesh of each entry (values are global triangle indices), as a sort key.
__global__ void k_mesh_keys(const int32_t* __restrict__ vals, const int64_t* __restrict__ tri_pre, int M, int64_t total,
                            uint32_t* __restrict__ mk) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < total) mk[g] = (uint32_t)mesh_of(tri_pre, M, vals[g]);
}

// After the sorts entries are grouped by mesh, in (code, triangle) order
// within each: give every mesh its sorted keys and leaf order.
template <typename K>
__global__ void k_scatter_seg(const MeshBuild* __restrict__ d, const int64_t* __restrict__ tri_pre, int M,
                              int64_t total, const int32_t* __restrict__ vals, const K* __restrict__ codes) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int m = mesh_of(tri_pre, M, g);
    const int64_t i = g - tri_pre[m];
    const int32_t gid = vals[g];
    d[m].perm[i] = (int32_t)(gid - tri_pre[m]);
    reinterpret_cast<K*>(d[m].keys)[i] = codes[gid];
}

template <typename K>
__global__ void k_apetrei_seg(const MeshBuild* __restrict__ d, const int64_t* __restrict__ tri_pre, int M,
                              int64_t total) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int m = mesh_of(tri_pre, M, g);
    const MeshBuild& mb = d[m];
    apetrei_leaf<K>(mb.V, mb.nv, mb.T, mb.perm, reinterpret_cast<const K*>(mb.keys), mb.nt, g - tri_pre[m], mb.left,
                    mb.right, mb.parent, mb.box, mb.hgt, mb.ends, mb.nodes, mb.tris, mb.ctr);
}

// int_pre: prefix of the internal node counts max(nt - 1, 0).
__global__ void k_collapse4_seg(const MeshBuild* __restrict__ d, const int64_t* __restrict__ int_pre, int M,
                                int64_t total) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int m = mesh_of(int_pre, M, g);
    collapse_node(d[m].nodes, d[m].parent, g - int_pre[m], d[m].nodes4);
}

__global__ void k_gather_ctr(const MeshBuild* __restrict__ d, int M, DevCounters* __restrict__ out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) out[m] = *d[m].ctr;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// A handle with its device arrays in one pool allocation (256-byte aligned
// pieces); sort scratch for a single-mesh build when `sort_scratch`.
// Returns nullptr (error set) when the allocation fails.
rsi_bvh_s* alloc_handle(int64_t nv, int64_t nt, int morton_bits, bool sort_scratch, cudaStream_t s, char** base_out,
                        int32_t** hgt, int32_t** flag, char** scratch) {
    rsi_bvh_s* h = new rsi_bvh_s();
    h->gen = next_handle_gen();
    h->n_tri = nt;
    h->n_vert = nv;
    h->morton_bits = morton_bits;
    const int64_t n = nt, ni = n > 1 ? n - 1 : 1;
    const size_t ksz = morton_bits == 30 ? 4 : 8;
    // one allocation, carved into the handle's arrays (256-byte aligned)
    size_t off[14], total = 0;
    size_t sizes[14] = {
        sizeof(Node) * (size_t)ni,                 // 0 nodes
        sizeof(Tri) * (size_t)n,                   // 1 tris
        ksz * (size_t)n,                           // 2 sorted keys
        4 * (size_t)n,                             // 3 perm
        4 * (size_t)ni,                            // 4 left
        4 * (size_t)ni,                            // 5 right
        4 * (size_t)(2 * n - 1),                   // 6 parent
        24 * (size_t)(2 * n - 1),                  // 7 box
        4 * (size_t)(2 * n - 1),                   // 8 heights
        4 * (size_t)ni,                            // 9 flags
        sizeof(DevCounters),                       // 10 counters
        sort_scratch ? 2 * ksz * (size_t)n + 8 * (size_t)n + sort_hist_bytes(n, ksz == 4 ? 4 : 8) : 0,  // 11 sort scratch
        sizeof(Node4) * (size_t)ni,                // 12 four-wide nodes
        sizeof(NodeQ) * (size_t)ni                 // 13 compressed nodes
    };
    for (int i = 0; i < 14; ++i) {
        off[i] = total;
        total += align_up(sizes[i]);
    }
    char* base = nullptr;
    if (pool_alloc(reinterpret_cast<void**>(&base), total, s) != RSI_OK) {
        delete h;
        return nullptr;
    }
    h->device_bytes = (int64_t)total;
    h->nodes = (Node*)(base + off[0]);
    h->tris = (Tri*)(base + off[1]);
    h->sorted_keys = base + off[2];
    h->perm = (int32_t*)(base + off[3]);
    h->left = (int32_t*)(base + off[4]);
    h->right = (int32_t*)(base + off[5]);
    h->parent = (int32_t*)(base + off[6]);
    h->box = (float*)(base + off[7]);
    *hgt = (int32_t*)(base + off[8]);
    *flag = (int32_t*)(base + off[9]);
    h->hgt = *hgt;
    h->flags = *flag;
    h->ctr = (DevCounters*)(base + off[10]);
    *scratch = base + off[11];
    h->nodes4 = (Node4*)(base + off[12]);
    h->nodesq = (NodeQ*)(base + off[13]);
    *base_out = base;
    return h;
}

// Extent, padding and height of a finished build from its counters.
void finish_handle(rsi_bvh_s* h, const DevCounters& hc) {
    h->height = hc.height;
    for (int a = 0; a < 3; ++a) {
        h->lo[a] = ord2f(hc.ext_bits[a]);
        h->hi[a] = ord2f(hc.ext_bits[3 + a]);
        float f;
        std::memcpy(&f, &hc.dmax_bits[a], 4);
        h->dmax[a] = f;
    }
}

int build_from_device(const float* V, int64_t nv, const int32_t* T, int64_t nt, int morton_bits, int tree_builder,
                      cudaStream_t s, rsi_bvh_t* out) {
    const int64_t n = nt, ni = n > 1 ? n - 1 : 1;
    const int builder = tree_builder & 0xFF, passes = tree_builder >> 8;   // RSI_TREE_TREELETS(passes)
    char* base = nullptr;
    int32_t *hgt = nullptr, *flag = nullptr;
    char* scratch = nullptr;
    rsi_bvh_s* h = alloc_handle(nv, nt, morton_bits, true, s, &base, &hgt, &flag, &scratch);
    if (!h) return RSI_ERR_OOM;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&](int code) {
        cudaStreamSynchronize(s);
        pool_free(base, s);
        delete h;
        return code;
    };
    k_init<<<1, 32, 0, s>>>(h->ctr);
    note_launches(2);   // k_init, k_extent
    k_extent<<<grid_for(nv, kBlock) < 4 * 152 ? grid_for(nv, kBlock) : 4 * 152, kBlock, 0, s>>>(V, nv, h->ctr);
    // arrival counters of k_refit start at 0; range-end slots of k_apetrei at -1
    if (cudaMemsetAsync(flag, builder == RSI_TREE_APETREI ? 0xFF : 0, 4 * (size_t)ni, s) != cudaSuccess)
        return cleanup(cuda_fail(cudaGetLastError(), "memset"));
    int rc = morton_bits == 30 ? build_impl<uint32_t>(h, V, T, builder, s, scratch, h->box, hgt, flag)
                               : build_impl<uint64_t>(h, V, T, builder, s, scratch, h->box, hgt, flag);
    if (rc) return cleanup(rc);
    rc = enqueue_treelets(h, passes, hgt, reinterpret_cast<int32_t*>(scratch), s);   // the sort scratch is free now
    if (rc) return cleanup(rc);
    if (n > 1) {
        k_collapse4<<<grid_for(n - 1, kBlock), kBlock, 0, s>>>(h->nodes, h->parent, n, h->nodes4);
        note_launches(1);
        if (passes == 0) {   // compressed nodes name both children by one index (Karras numbering)
            k_quantize<<<grid_for(n - 1, kBlock), kBlock, 0, s>>>(h->nodes, n, h->nodesq, h->ctr);
            note_launches(1);
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "lbvh_build kernels"));
    e = cudaMemcpyAsync(h->h_ctr, h->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "lbvh_build"));
    const DevCounters& hc = *h->h_ctr;
    if (hc.error) {
        return cleanup(fail(hc.error, hc.error == RSI_ERR_NAN ? "lbvh_build: NaN vertex coordinate"
                                                             : "lbvh_build: triangle vertex index out of range"));
    }
    finish_handle(h, hc);
    h->has_q = n > 1 && passes == 0;
    h->treelet_passes = passes;
    *out = h;
    return RSI_OK;
}

// The kernels of a batched build, in stream order and without any host
// synchronization (so that a CUDA graph can capture them): counters reset,
// extents, Morton codes, the stable sort by code and then by mesh, leaf
// scatter, the bottom-up tree and boxes, four-wide nodes, and a copy of
// every mesh's counters into d_ctr.
template <typename K>
int enqueue_batched_build(const MeshBuild* d_mb, const int64_t* d_tri_pre, const int64_t* d_int_pre, int M,
                          int64_t total, int64_t total_int, K* ka, K* kb, K* codes, int32_t* va, int32_t* vb,
                          uint32_t* mka, uint32_t* mkb, uint32_t* hist, DevCounters* d_ctr, cudaStream_t s,
                          int treelet_passes = 0) {
    k_init_seg<<<grid_for(M, 128), 128, 0, s>>>(d_mb, M);
    k_extent_seg<<<M, kBlock, 0, s>>>(d_mb);
    k_morton_seg<K><<<grid_for(total, kBlock), kBlock, 0, s>>>(d_mb, d_tri_pre, M, total, ka, codes, va);
    note_launches(3);
    // stable sort by code, then stably by mesh: (mesh, code, triangle) order
    K* sk;
    int32_t* sv;
    int rc = sort_pairs<K>(ka, va, kb, vb, total, sizeof(K) == 4 ? 4 : 8, hist, s, &sk, &sv);
    if (rc) return rc;
    int32_t* sv2 = sv == va ? vb : va;   // the other value buffer
    k_mesh_keys<<<grid_for(total, kBlock), kBlock, 0, s>>>(sv, d_tri_pre, M, total, mka);
    note_launches(1);
    uint32_t* smk;
    int32_t* fv;
    rc = sort_pairs<uint32_t>(mka, sv, mkb, sv2, total, M <= 256 ? 1 : (M <= 65536 ? 2 : 4), hist, s, &smk, &fv);
    if (rc) return rc;
    k_scatter_seg<K><<<grid_for(total, kBlock), kBlock, 0, s>>>(d_mb, d_tri_pre, M, total, fv, codes);
    k_apetrei_seg<K><<<grid_for(total, kBlock), kBlock, 0, s>>>(d_mb, d_tri_pre, M, total);
    note_launches(2);
    if (treelet_passes > 0 && total_int > 0) {   // the sort buffers are free now: root lists and their counts
        rc = enqueue_treelets_batched(d_mb, d_tri_pre, d_int_pre, M, total, total_int, treelet_passes, va, vb,
                                      reinterpret_cast<int*>(hist), s);
        if (rc) return rc;
    }
    if (total_int > 0) {
        k_collapse4_seg<<<grid_for(total_int, kBlock), kBlock, 0, s>>>(d_mb, d_int_pre, M, total_int);
        note_launches(1);
    }
    k_gather_ctr<<<grid_for(M, 128), 128, 0, s>>>(d_mb, M, d_ctr);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RSI_OK : cuda_fail(e, "batched build launch");
}

// Many meshes in one build: ~20 launches in all, one synchronization.
template <typename K>
int build_batched_impl(int M, const float* const* V, const int64_t* nv, const int32_t* const* T, const int64_t* nt,
                       int morton_bits, int treelet_passes, cudaStream_t s, rsi_bvh_t* out) {
    std::vector<MeshBuild> mb(M);
    std::vector<int64_t> tri_pre(M + 1, 0), int_pre(M + 1, 0);
    std::vector<rsi_bvh_s*> hs(M, nullptr);
    std::vector<char*> bases(M, nullptr);
    auto free_all = [&]() {
        for (int m = 0; m < M; ++m) {
            if (bases[m]) pool_free(bases[m], s);
            delete hs[m];
        }
    };
    for (int m = 0; m < M; ++m) {
        char* scratch = nullptr;
        int32_t *hgt = nullptr, *ends = nullptr;
        hs[m] = alloc_handle(nv[m], nt[m], morton_bits, false, s, &bases[m], &hgt, &ends, &scratch);
        if (!hs[m]) {
            free_all();
            return RSI_ERR_OOM;
        }
        rsi_bvh_s* h = hs[m];
        mb[m] = MeshBuild{V[m], T[m], nv[m], nt[m], h->nodes, h->nodes4, h->tris, h->sorted_keys, h->perm,
                          h->left, h->right, h->parent, hgt, ends, h->box, h->ctr};
        tri_pre[m + 1] = tri_pre[m] + nt[m];
        int_pre[m + 1] = int_pre[m] + (nt[m] > 1 ? nt[m] - 1 : 0);
    }
    const int64_t total = tri_pre[M], total_int = int_pre[M];
    const int ntiles = grid_for(total, 4096);
    // global scratch: table, prefixes, keys x2, codes, values x2, mesh keys x2, histograms, counters
    size_t off[10], bytes = 0;
    const size_t sizes[10] = {sizeof(MeshBuild) * (size_t)M, 8 * (size_t)(M + 1), 8 * (size_t)(M + 1),
                              sizeof(K) * (size_t)total, sizeof(K) * (size_t)total, sizeof(K) * (size_t)total,
                              8 * (size_t)total, 8 * (size_t)total, 4 * 256 * (size_t)ntiles,
                              sizeof(DevCounters) * (size_t)M};
    for (int i = 0; i < 10; ++i) {
        off[i] = bytes;
        bytes += align_up(sizes[i]);
    }
    char* g = nullptr;
    if (pool_alloc(reinterpret_cast<void**>(&g), bytes, s) != RSI_OK) {
        free_all();
        return RSI_ERR_OOM;
    }
    MeshBuild* d_mb = (MeshBuild*)(g + off[0]);
    int64_t* d_tri_pre = (int64_t*)(g + off[1]);
    int64_t* d_int_pre = (int64_t*)(g + off[2]);
    K* ka = (K*)(g + off[3]);
    K* kb = (K*)(g + off[4]);
    K* codes = (K*)(g + off[5]);
    int32_t* va = (int32_t*)(g + off[6]);
    int32_t* vb = va + total;
    uint32_t* mka = (uint32_t*)(g + off[7]);
    uint32_t* mkb = mka + total;
    uint32_t* hist = (uint32_t*)(g + off[8]);
    DevCounters* d_ctr = (DevCounters*)(g + off[9]);
    std::vector<DevCounters> hc(M);
    auto fail_all = [&](int code) {
        cudaStreamSynchronize(s);
        pool_free(g, s);
        free_all();
        return code;
    };
    cudaError_t e = cudaMemcpyAsync(d_mb, mb.data(), sizeof(MeshBuild) * M, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tri_pre, tri_pre.data(), 8 * (size_t)(M + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_int_pre, int_pre.data(), 8 * (size_t)(M + 1), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_all(cuda_fail(e, "lbvh_build_batched: upload"));
    int rc = enqueue_batched_build<K>(d_mb, d_tri_pre, d_int_pre, M, total, total_int, ka, kb, codes, va, vb, mka,
                                      mkb, hist, d_ctr, s, treelet_passes);
    if (rc) return fail_all(rc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), d_ctr, sizeof(DevCounters) * M, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_all(cuda_fail(e, "lbvh_build_batched"));
    for (int m = 0; m < M; ++m) {
        if (hc[m].error) {
            const std::string why = hc[m].error == RSI_ERR_NAN ? "NaN vertex coordinate" : "triangle vertex index out of range";
            return fail_all(fail(hc[m].error, "lbvh_build_batched: mesh " + std::to_string(m) + ": " + why));
        }
    }
    pool_free(g, s);
    for (int m = 0; m < M; ++m) {
        finish_handle(hs[m], hc[m]);
        hs[m]->treelet_passes = treelet_passes;
        out[m] = hs[m];
    }
    return RSI_OK;
}

// ---------------------------------------------------------------- rebuild in place
int rebuild_prepare(const rsi_bvh_t* hs, int M, const float* const* V, const int32_t* const* T, cudaStream_t s,
                    RebuildSpec* out) {
    if (!out || !hs || !V || !T || M < 1) return fail(RSI_ERR_INVALID_ARG, "rebuild: bad arguments");
    RebuildSpec& r = *out;
    r = RebuildSpec{};
    r.M = M;
    r.morton_bits = hs[0] ? hs[0]->morton_bits : 30;
    std::vector<MeshBuild> mb(M);
    std::vector<int64_t> tri_pre(M + 1, 0), int_pre(M + 1, 0);
    for (int m = 0; m < M; ++m) {
        const rsi_bvh_s* h = hs[m];
        if (!h || !V[m] || !T[m])
            return fail(RSI_ERR_INVALID_ARG, "rebuild: mesh " + std::to_string(m) + " lacks a hierarchy or buffer");
        if (h->morton_bits != r.morton_bits)
            return fail(RSI_ERR_INVALID_ARG, "rebuild: the hierarchies differ in morton_bits");
        r.treelet_passes = std::max(r.treelet_passes, h->treelet_passes);
        if (!h->hgt || !h->flags) return fail(RSI_ERR_INVALID_ARG, "rebuild: hierarchy without build scratch");
        mb[m] = MeshBuild{V[m], T[m], h->n_vert, h->n_tri, h->nodes, h->nodes4, h->tris, h->sorted_keys, h->perm,
                          h->left, h->right, h->parent, h->hgt, h->flags, h->box, h->ctr};
        tri_pre[m + 1] = tri_pre[m] + h->n_tri;
        int_pre[m + 1] = int_pre[m] + (h->n_tri > 1 ? h->n_tri - 1 : 0);
    }
    r.total = tri_pre[M];
    r.total_int = int_pre[M];
    r.hs.assign(hs, hs + M);
    for (int m = 0; m < M; ++m) hs[m]->has_q = false;   // the batched build writes no compressed nodes
    const size_t ksz = r.morton_bits == 30 ? 4 : 8;
    const int ntiles = grid_for(r.total, 4096);
    size_t off[10], bytes = 0;
    const size_t sizes[10] = {sizeof(MeshBuild) * (size_t)M, 8 * (size_t)(M + 1), 8 * (size_t)(M + 1),
                              ksz * (size_t)r.total, ksz * (size_t)r.total, ksz * (size_t)r.total,
                              8 * (size_t)r.total, 8 * (size_t)r.total, 4 * 256 * (size_t)ntiles,
                              sizeof(DevCounters) * (size_t)M};
    for (int i = 0; i < 10; ++i) {
        off[i] = bytes;
        bytes += align_up(sizes[i]);
    }
    if (pool_alloc(reinterpret_cast<void**>(&r.mem), bytes, s) != RSI_OK) return RSI_ERR_OOM;
    char* g = r.mem;
    r.d_mb = g + off[0];
    r.d_tri_pre = (int64_t*)(g + off[1]);
    r.d_int_pre = (int64_t*)(g + off[2]);
    r.ka = g + off[3];
    r.kb = g + off[4];
    r.codes = g + off[5];
    r.va = (int32_t*)(g + off[6]);
    r.vb = r.va + r.total;
    r.mka = (uint32_t*)(g + off[7]);
    r.mkb = r.mka + r.total;
    r.hist = (uint32_t*)(g + off[8]);
    r.d_ctr = (DevCounters*)(g + off[9]);
    cudaError_t e = cudaMemcpyAsync(r.d_mb, mb.data(), sizeof(MeshBuild) * M, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.d_tri_pre, tri_pre.data(), 8 * (size_t)(M + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.d_int_pre, int_pre.data(), 8 * (size_t)(M + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host tables above go out of scope
    if (e != cudaSuccess) {
        rebuild_release(r);
        return cuda_fail(e, "rebuild: upload");
    }
    return RSI_OK;
}

int rebuild_enqueue(const RebuildSpec& r, cudaStream_t s) {
    const MeshBuild* d_mb = static_cast<const MeshBuild*>(r.d_mb);
    if (r.morton_bits == 30)
        return enqueue_batched_build<uint32_t>(d_mb, r.d_tri_pre, r.d_int_pre, r.M, r.total, r.total_int,
                                               (uint32_t*)r.ka, (uint32_t*)r.kb, (uint32_t*)r.codes, r.va, r.vb, r.mka,
                                               r.mkb, r.hist, r.d_ctr, s, r.treelet_passes);
    return enqueue_batched_build<uint64_t>(d_mb, r.d_tri_pre, r.d_int_pre, r.M, r.total, r.total_int,
                                           (uint64_t*)r.ka, (uint64_t*)r.kb, (uint64_t*)r.codes, r.va, r.vb, r.mka,
                                           r.mkb, r.hist, r.d_ctr, s, r.treelet_passes);
}

void rebuild_release(RebuildSpec& r) {
    if (r.mem) pool_free(r.mem, 0);
    r.mem = nullptr;
}

int refresh_handles(const RebuildSpec& r, cudaStream_t s) {
    std::vector<DevCounters> hc(r.M);
    RSI_CUDA_TRY(cudaMemcpyAsync(hc.data(), r.d_ctr, sizeof(DevCounters) * r.M, cudaMemcpyDeviceToHost, s));
    RSI_CUDA_TRY(cudaStreamSynchronize(s));
    int rc = RSI_OK;
    for (int m = 0; m < r.M; ++m) {
        if (hc[m].error && rc == RSI_OK) {
            const std::string why = hc[m].error == RSI_ERR_NAN ? "NaN vertex coordinate" : "triangle vertex index out of range";
            rc = fail(hc[m].error, "rebuild: mesh " + std::to_string(m) + ": " + why);
        }
        finish_handle(r.hs[m], hc[m]);
    }
    return rc;
}

}  // namespace rsi

namespace rsi {
namespace {
int build_checked(const char* fn, const float* d_vertices, int64_t n_vertices, const int32_t* d_triangles,
                  int64_t n_triangles, int index_bytes, int morton_bits, int tree_builder, void* stream,
                  rsi_bvh_t* out) {
    const std::string f(fn);
    if (!out) return fail(RSI_ERR_INVALID_ARG, f + ": out is NULL");
    *out = nullptr;
    if (index_bytes != 4)
        return fail(RSI_ERR_DTYPE, f + ": triangle indices must be int32 (index_bytes = 4), got " +
                                       std::to_string(index_bytes) + " bytes");
    if (!d_vertices || !d_triangles) return fail(RSI_ERR_INVALID_ARG, f + ": NULL input pointer");
    if (n_triangles < 1 || n_vertices < 1 || n_triangles > (int64_t)0x3FFFFFFF || n_vertices > ((int64_t)1 << 31))
        return fail(RSI_ERR_INVALID_ARG, f + ": need 1 <= n_triangles < 2^30 and 1 <= n_vertices <= 2^31");
    if (morton_bits != 30 && morton_bits != 63) return fail(RSI_ERR_INVALID_ARG, f + ": morton_bits must be 30 or 63");
    const int builder = tree_builder & 0xFF, passes = tree_builder >> 8;
    if ((builder != RSI_TREE_KARRAS && builder != RSI_TREE_APETREI) || passes < 0 || passes > 3)
        return fail(RSI_ERR_INVALID_ARG, f + ": tree_builder must be RSI_TREE_KARRAS or RSI_TREE_APETREI, "
                                             "optionally | RSI_TREE_TREELETS(1 .. 3)");
    return build_from_device(d_vertices, n_vertices, d_triangles, n_triangles, morton_bits, tree_builder,
                             (cudaStream_t)stream, out);
}
}  // namespace
}  // namespace rsi

extern "C" int lbvh_build(const float* d_vertices, int64_t n_vertices, const int32_t* d_triangles,
                          int64_t n_triangles, int index_bytes, int morton_bits, void* stream, rsi_bvh_t* out) {
    return rsi::build_checked("lbvh_build", d_vertices, n_vertices, d_triangles, n_triangles, index_bytes,
                              morton_bits, RSI_TREE_KARRAS, stream, out);
}

extern "C" int lbvh_build_ex(const float* d_vertices, int64_t n_vertices, const int32_t* d_triangles,
                             int64_t n_triangles, int index_bytes, int morton_bits, int tree_builder, void* stream,
                             rsi_bvh_t* out) {
    return rsi::build_checked("lbvh_build_ex", d_vertices, n_vertices, d_triangles, n_triangles, index_bytes,
                              morton_bits, tree_builder, stream, out);
}

extern "C" int lbvh_build_batched(int n_meshes, const float* const* d_vertices, const int64_t* n_vertices,
                                  const int32_t* const* d_triangles, const int64_t* n_triangles, int index_bytes,
                                  int morton_bits, void* stream, rsi_bvh_t* out) {
    return lbvh_build_batched_ex(n_meshes, d_vertices, n_vertices, d_triangles, n_triangles, index_bytes,
                                 morton_bits, 0, stream, out);
}

extern "C" int lbvh_build_batched_ex(int n_meshes, const float* const* d_vertices, const int64_t* n_vertices,
                                     const int32_t* const* d_triangles, const int64_t* n_triangles, int index_bytes,
                                     int morton_bits, int treelet_passes, void* stream, rsi_bvh_t* out) {
    if (!out || n_meshes < 1 || !d_vertices || !n_vertices || !d_triangles || !n_triangles)
        return rsi::fail(RSI_ERR_INVALID_ARG, "lbvh_build_batched: need n_meshes >= 1 and non-NULL arrays");
    for (int m = 0; m < n_meshes; ++m) out[m] = nullptr;
    if (index_bytes != 4) return rsi::fail(RSI_ERR_DTYPE, "lbvh_build_batched: triangle indices must be int32");
    if (morton_bits != 30 && morton_bits != 63)
        return rsi::fail(RSI_ERR_INVALID_ARG, "lbvh_build_batched: morton_bits must be 30 or 63");
    if (treelet_passes < 0 || treelet_passes > 3)
        return rsi::fail(RSI_ERR_INVALID_ARG, "lbvh_build_batched: treelet_passes must be 0 .. 3");
    int64_t total = 0;
    for (int m = 0; m < n_meshes; ++m) {
        if (!d_vertices[m] || !d_triangles[m] || n_vertices[m] < 1 || n_triangles[m] < 1 ||
            n_vertices[m] > ((int64_t)1 << 31))
            return rsi::fail(RSI_ERR_INVALID_ARG, "lbvh_build_batched: mesh " + std::to_string(m) +
                                                      " has a NULL pointer or a count out of range");
        total += n_triangles[m];
    }
    if (total > 0x3FFFFFFF)
        return rsi::fail(RSI_ERR_INVALID_ARG, "lbvh_build_batched: more than 2^30 triangles in all");
    cudaStream_t s = (cudaStream_t)stream;
    return morton_bits == 30
               ? rsi::build_batched_impl<uint32_t>(n_meshes, d_vertices, n_vertices, d_triangles, n_triangles, 30,
                                                   treelet_passes, s, out)
               : rsi::build_batched_impl<uint64_t>(n_meshes, d_vertices, n_vertices, d_triangles, n_triangles, 63,
                                                   treelet_passes, s, out);
}

extern "C" int lbvh_build_host(const float* h_vertices, int64_t n_vertices, const int32_t* h_triangles,
                               int64_t n_triangles, int index_bytes, int morton_bits, void* stream, rsi_bvh_t* out) {
    return lbvh_build_host_ex(h_vertices, n_vertices, h_triangles, n_triangles, index_bytes, morton_bits,
                              RSI_TREE_KARRAS, stream, out);
}

extern "C" int lbvh_build_host_ex(const float* h_vertices, int64_t n_vertices, const int32_t* h_triangles,
                                  int64_t n_triangles, int index_bytes, int morton_bits, int tree_builder, void* stream,
                                  rsi_bvh_t* out) {
    if (!out) return rsi::fail(RSI_ERR_INVALID_ARG, "lbvh_build_host: out is NULL");
    *out = nullptr;
    if (!h_vertices || !h_triangles || n_vertices < 1 || n_triangles < 1)
        return rsi::fail(RSI_ERR_INVALID_ARG, "lbvh_build_host: bad input");
    const int builder = tree_builder & 0xFF, passes = tree_builder >> 8;
    if ((builder != RSI_TREE_KARRAS && builder != RSI_TREE_APETREI) || passes < 0 || passes > 3)
        return rsi::fail(RSI_ERR_INVALID_ARG, "lbvh_build_host: tree_builder must be RSI_TREE_KARRAS or "
                                              "RSI_TREE_APETREI, optionally | RSI_TREE_TREELETS(1 .. 3)");
    if (index_bytes != 4) return rsi::fail(RSI_ERR_DTYPE, "lbvh_build_host: triangle indices must be int32");
    cudaStream_t s = (cudaStream_t)stream;
    float* dv = nullptr;
    int32_t* dt = nullptr;
    size_t bv = 12 * (size_t)n_vertices, bt = 12 * (size_t)n_triangles;
    if (rsi::pool_alloc(reinterpret_cast<void**>(&dv), bv, s) != RSI_OK ||
        rsi::pool_alloc(reinterpret_cast<void**>(&dt), bt, s) != RSI_OK) {
        rsi::pool_free(dv, s);
        return RSI_ERR_OOM;
    }
    int rc = RSI_OK;
    if (cudaMemcpyAsync(dv, h_vertices, bv, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dt, h_triangles, bt, cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = rsi::cuda_fail(cudaGetLastError(), "lbvh_build_host copy");
    if (rc == RSI_OK) rc = lbvh_build_ex(dv, n_vertices, dt, n_triangles, 4, morton_bits, tree_builder, stream, out);
    rsi::pool_free(dv, s);
    rsi::pool_free(dt, s);
    return rc;
}

extern "C" int lbvh_free(rsi_bvh_t h) {
    if (!h) return RSI_OK;
    cudaDeviceSynchronize();
    rsi::forget_handle(h);         // detach its network, drop the batched plans that name it
    rsi::pool_free(h->nodes, 0);   // base of the single allocation
    rsi::pool_free(h->band_ids, 0);
    rsi::pool_free(h->pair_mem, 0);
    rsi::pool_free(h->order_hist, 0);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    delete h;
    return RSI_OK;
}

extern "C" int lbvh_info(rsi_bvh_t h, rsi_bvh_info* out) {
    if (!h || !out) return rsi::fail(RSI_ERR_INVALID_ARG, "lbvh_info: NULL argument");
    out->n_triangles = h->n_tri;
    out->n_vertices = h->n_vert;
    out->morton_bits = h->morton_bits;
    out->height = h->height;
    out->device_bytes = h->device_bytes + 12 * h->band_cap + h->pair_bytes;
    for (int a = 0; a < 3; ++a) {
        out->extent_lo[a] = h->lo[a];
        out->extent_hi[a] = h->hi[a];
        out->max_tri_extent[a] = h->dmax[a];
    }
    return RSI_OK;
}

extern "C" int lbvh_export(rsi_bvh_t h, void* stream, rsi_bvh_host_view* v) {
    if (!h || !v) return rsi::fail(RSI_ERR_INVALID_ARG, "lbvh_export: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = h->n_tri;
    RSI_CUDA_TRY(cudaStreamSynchronize(s));
    if (v->sorted_keys) {
        if (h->morton_bits == 30) {
            uint32_t* tmp = new uint32_t[n];
            cudaError_t e = cudaMemcpy(tmp, h->sorted_keys, 4 * n, cudaMemcpyDeviceToHost);
            for (int64_t i = 0; i < n; ++i) v->sorted_keys[i] = tmp[i];
            delete[] tmp;
            RSI_CUDA_TRY(e);
        } else {
            RSI_CUDA_TRY(cudaMemcpy(v->sorted_keys, h->sorted_keys, 8 * n, cudaMemcpyDeviceToHost));
        }
    }
    if (v->perm) RSI_CUDA_TRY(cudaMemcpy(v->perm, h->perm, 4 * n, cudaMemcpyDeviceToHost));
    if (n > 1 && v->left) RSI_CUDA_TRY(cudaMemcpy(v->left, h->left, 4 * (n - 1), cudaMemcpyDeviceToHost));
    if (n > 1 && v->right) RSI_CUDA_TRY(cudaMemcpy(v->right, h->right, 4 * (n - 1), cudaMemcpyDeviceToHost));
    if (v->parent) RSI_CUDA_TRY(cudaMemcpy(v->parent, h->parent, 4 * (2 * n - 1), cudaMemcpyDeviceToHost));
    if (v->box) RSI_CUDA_TRY(cudaMemcpy(v->box, h->box, 24 * (2 * n - 1), cudaMemcpyDeviceToHost));
    return RSI_OK;
}

extern "C" size_t lbvh_node_bytes(void) { return sizeof(rsi::Node); }
