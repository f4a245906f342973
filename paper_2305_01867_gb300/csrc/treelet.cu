// treelet.cu -- restructuring of a built hierarchy (an option of lbvh_build_ex).
//
// The paper's hierarchy splits every node at the highest differing bit of the
// triangles' Morton codes (Sec. 3.2, after Karras 2012).  Those midpoint splits
// leave loose boxes in the middle of the tree: on a heightfield of 19,602
// triangles a segment meets ~35 child-pair nodes where a surface-area-guided
// tree of the same triangles needs ~24.  These passes, after the build,
// rewrite small groups of nodes ("treelets") so that the sum of the surface
// areas of the internal nodes -- the usual estimate of the nodes a random
// segment meets -- goes down, in the manner of treelet restructuring (Karras &
// Aila 2013, "Fast parallel construction of high-quality bounding volume
// hierarchies"), with the treelets tiled by depth instead of grown bottom-up:
//
//  * a treelet is an internal node r at depth d with the internal nodes of its
//    subtree down to depth d + 2; its leaves are the children that hang
//    below: subtrees rooted at depth d + 3, or triangles -- at most 7: when 8
//    would hang below, the depth-(d + 2) node of smallest box stays whole
//    (a third of the programme's work for 8 leaves, nearly the same trees);
//  * rewiring a treelet never changes the box of any subtree that hangs below
//    it nor of r itself (a box is the union of the triangles below), so all
//    treelets whose roots share d mod 3 are disjoint and independent: one
//    launch restructures them all, one warp per treelet, and three launches
//    (d mod 3 = 0, 1, 2, depths recomputed in between) make one pass;
//  * the warp finds the binary tree over the treelet's leaves with the
//    smallest sum of internal-node surface areas by dynamic programming over
//    the leaf subsets (every subset's best split, smallest subsets first)
//    and, when it is clearly smaller than the current one, rewires the
//    treelet's own internal nodes into it (same node ids, r keeps its place).
//
// Leaves, their Morton order and the triangles are untouched; only the
// internal nodes' children, parents and boxes change, so every query answers
// exactly as on the plain tree.  The compressed-node layout needs the right
// child at the left one + 1, which the rewired tree no longer has: handles
// built with restructuring have no compressed nodes (node width 3 falls back
// to child-pair nodes).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "rsi_internal.cuh"

namespace rsi {
namespace {

constexpr int kTreeletLevels = 3;          // levels of internal nodes in a treelet
constexpr int kTreeletLeaves = 7;          // a treelet's leaves (of 8 the smallest pair stays joined)
constexpr int kFullSet = (1 << kTreeletLeaves) - 1;
constexpr int kTreeletWarps = 4;           // warps per block of k_treelet
constexpr int kTreeletBlocksPerSm = 12;    // register budget: 12 resident blocks (48 warps) per SM
constexpr unsigned kFull = 0xffffffffu;
constexpr int kClimbMax = 1 << 16;         // climb steps before a pass gives up (RSI_ERR_STACK)

// The non-empty subsets of the 8 treelet leaves ordered by size: the subsets
// of size s are by_size[off[s] .. off[s + 1]).
struct SubsetTable {
    uint8_t by_size[kFullSet];
    uint8_t off[kTreeletLeaves + 2];
};
constexpr int popc_c(int x) { return x ? (x & 1) + popc_c(x >> 1) : 0; }
constexpr SubsetTable make_subset_table() {
    SubsetTable t{};
    int k = 0;
    for (int s = 1; s <= kTreeletLeaves; ++s) {
        t.off[s] = (uint8_t)k;
        for (int m = 1; m <= kFullSet; ++m)
            if (popc_c(m) == s) t.by_size[k++] = (uint8_t)m;
    }
    t.off[kTreeletLeaves + 1] = (uint8_t)k;
    return t;
}
__constant__ SubsetTable c_subsets = make_subset_table();

// One warp's working set for one treelet.
struct TreeletSmem {
    float lbox[kTreeletLeaves][6];   // treelet leaf boxes (min xyz, max xyz)
    int lref[kTreeletLeaves];        // treelet leaf references (tagged as the build tags them)
    int inner[kTreeletLeaves - 1];   // the treelet's internal nodes (inner[0] = its root)
    float lowbox[16][6];             // boxes of the subsets of leaves 0-3 (index: the subset)
    float highbox[8][6];             // boxes of the subsets of leaves 4-6 (index: the subset >> 4)
    int g[4];                        // the third level: child c of r's child s at g[2 * s + c]
    int y[8];                        // the fourth level: child c of g[q] at y[2 * q + c]
    float g_area[4];                 // half areas of the internal g[q]
    float area[kFullSet + 1];        // surface area of the box of each leaf subset
    float cost[kFullSet + 1];        // best summed internal-node area of a tree over the subset
    uint8_t best[kFullSet + 1];      // the part holding the subset's lowest leaf, in that best tree
    int emit_node[kTreeletLeaves - 1], emit_set[kTreeletLeaves - 1];
    int emit_l[kTreeletLeaves - 1], emit_r[kTreeletLeaves - 1];
    int k, ni;                       // leaves, internal nodes
};

__device__ __forceinline__ int64_t slot_of(int32_t ref, int64_t n) {
    return ((uint32_t)ref & kLeafTag) ? (n - 1 + (int64_t)((uint32_t)ref & ~kLeafTag)) : (int64_t)ref;
}

__device__ __forceinline__ float half_area(float dx, float dy, float dz) {
    return fmaxf(dx, 0.0f) * fmaxf(dy, 0.0f) + fmaxf(dy, 0.0f) * fmaxf(dz, 0.0f) + fmaxf(dz, 0.0f) * fmaxf(dx, 0.0f);
}

// Box of node slot i, read through L2 (other warps rewrite boxes during the pass).
__device__ __forceinline__ void load_box(const float* __restrict__ box, int64_t i, float b[6]) {
#pragma unroll
    for (int a = 0; a < 6; ++a) b[a] = __ldcg(box + 6 * i + a);
}


__device__ __forceinline__ bool is_leaf_ref(int32_t ref) { return ((uint32_t)ref & kLeafTag) != 0; }

__device__ __forceinline__ void box_union(float b[6], const float* o) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        b[c] = fminf(b[c], o[c]);
        b[3 + c] = fmaxf(b[3 + c], o[3 + c]);
    }
}

// Box of the leaf subset S (non-empty) from the boxes of its two halves.
__device__ __forceinline__ void subset_box(const TreeletSmem& sm, int S, float b[6]) {
    const int lo = S & 15, hi = S >> 4;
#pragma unroll
    for (int c = 0; c < 6; ++c) b[c] = lo ? sm.lowbox[lo][c] : (c < 3 ? 3.0e38f : -3.0e38f);
    if (hi) box_union(b, sm.highbox[hi]);
}

// Restructure the treelet rooted at internal node r (all 32 lanes call it).
__device__ void restructure(int r, int64_t n, int32_t* __restrict__ left, int32_t* __restrict__ right,
                            int32_t* __restrict__ parent, float* __restrict__ box, TreeletSmem& sm, int lane) {
    // 1. the treelet: r and the internal nodes of the next two levels; their
    //    children below are its leaves.  Three rounds of loads spread over
    //    the lanes -- r's children; their children; the children and boxes
    //    of the level below -- then lane 0 lists leaves and internal nodes
    //    level by level, in child order.
    int32_t v = 0;
    if (lane < 2) v = __ldcg((lane ? right : left) + r);
    const int32_t a = __shfl_sync(kFull, v, 0), b = __shfl_sync(kFull, v, 1);
    v = (int32_t)kLeafTag;   // "no internal node here"
    if (lane < 4) {
        const int32_t p = (lane >> 1) ? b : a;
        if (!is_leaf_ref(p)) v = __ldcg((lane & 1 ? right : left) + p);
        sm.g[lane] = v;
    }
    const int32_t gq = __shfl_sync(kFull, v, (lane >> 1) & 3), gb = __shfl_sync(kFull, v, (lane - 8) & 3);
    if (lane < 8) {
        sm.y[lane] = is_leaf_ref(gq) ? 0 : __ldcg((lane & 1 ? right : left) + gq);
    } else if (lane < 12) {
        float bb[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (!is_leaf_ref(gb)) load_box(box, gb, bb);
        sm.g_area[lane - 8] = half_area(bb[3] - bb[0], bb[4] - bb[1], bb[5] - bb[2]);
    }
    __syncwarp();
    if (lane == 0) {
        int k = 0, ni = 0, n2 = 0;
        int l2q[4];   // the internal nodes of the third level, as indices into g
        sm.inner[ni++] = r;
        if (is_leaf_ref(a)) sm.lref[k++] = a;
        if (is_leaf_ref(b)) sm.lref[k++] = b;
        if (!is_leaf_ref(a)) sm.inner[ni++] = a;
        if (!is_leaf_ref(b)) sm.inner[ni++] = b;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (is_leaf_ref(q < 2 ? a : b)) continue;
            if (is_leaf_ref(sm.g[q])) sm.lref[k++] = sm.g[q];
            else l2q[n2++] = q;
        }
        if (n2 > 0 && k + 2 * n2 > kTreeletLeaves) {
            // eight leaves: the third-level node of smallest box stays whole (a leaf itself)
            int at = 0;
            float amin = 3.0e38f;
            for (int i = 0; i < n2; ++i) {
                const float ai = sm.g_area[l2q[i]];
                if (ai < amin) {
                    amin = ai;
                    at = i;
                }
            }
            sm.lref[k++] = sm.g[l2q[at]];
            l2q[at] = l2q[--n2];
        }
        for (int i = 0; i < n2; ++i) {
            sm.inner[ni++] = sm.g[l2q[i]];
            sm.lref[k++] = sm.y[2 * l2q[i]];
            sm.lref[k++] = sm.y[2 * l2q[i] + 1];
        }
        sm.k = k;
        sm.ni = ni;
    }
    __syncwarp();
    const int k = sm.k, ni = sm.ni;
    if (k < 3) return;   // two leaves: one tree only
    const int full = (1 << k) - 1;
    // 2. leaf boxes; the current cost (summed area of the internal nodes)
    float old = 0.0f;
    if (lane < k) {
        float b[6];
        load_box(box, slot_of(sm.lref[lane], n), b);
#pragma unroll
        for (int a = 0; a < 6; ++a) sm.lbox[lane][a] = b[a];
    }
    if (lane < ni) {
        float b[6];
        load_box(box, sm.inner[lane], b);
        old = half_area(b[3] - b[0], b[4] - b[1], b[5] - b[2]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) old += __shfl_xor_sync(kFull, old, o);
    __syncwarp();
    // 3. the box area of every leaf subset (a single leaf costs nothing):
    //    the boxes of the subsets of leaves 0-3 (lanes 1-15) and of leaves
    //    4-6 (lanes 17-23) first; a subset's box is the union of its halves'
    if (lane >= 1 && lane < 16 && lane <= full) {
        float bb[6] = {3.0e38f, 3.0e38f, 3.0e38f, -3.0e38f, -3.0e38f, -3.0e38f};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if ((lane >> i) & 1) box_union(bb, sm.lbox[i]);
#pragma unroll
        for (int c = 0; c < 6; ++c) sm.lowbox[lane][c] = bb[c];
    } else if (lane >= 17 && lane < 24 && ((lane - 16) << 4) <= full) {
        float bb[6] = {3.0e38f, 3.0e38f, 3.0e38f, -3.0e38f, -3.0e38f, -3.0e38f};
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (((lane - 16) >> i) & 1) box_union(bb, sm.lbox[4 + i]);
#pragma unroll
        for (int c = 0; c < 6; ++c) sm.highbox[lane - 16][c] = bb[c];
    }
    __syncwarp();
    for (int S = lane + 1; S <= full; S += 32) {
        float bb[6];
        subset_box(sm, S, bb);
        sm.area[S] = half_area(bb[3] - bb[0], bb[4] - bb[1], bb[5] - bb[2]);
        sm.cost[S] = 0.0f;
        sm.best[S] = 0;
    }
    __syncwarp();
    // 4. best split of every subset, smallest subsets first.  A split is the
    //    part Q holding the subset's lowest leaf (Q != S): Q = lowest | sub,
    //    sub a proper submask of the rest.  Subsets of up to five leaves take
    //    one lane each; a six-leaf subset takes four lanes and the whole set
    //    of seven all 32: lane g of a group of G = 2^b lanes fixes the top b
    //    bits of the rest at the pattern g and walks the submasks of the
    //    remaining low bits.
    for (int sz = 2; sz <= k; ++sz) {
        const int o0 = c_subsets.off[sz], ns = c_subsets.off[sz + 1] - o0;
        const int lg = sz <= 5 ? 0 : (sz == 6 ? 2 : 5), G = 1 << lg;
        for (int base = 0; base < ns; base += 32 / G) {   // uniform trip count
            const int i = base + (lane >> lg), g = lane & (G - 1);
            float bc = 3.0e38f;
            int bq = 0;
            const int S = i < ns ? (int)c_subsets.by_size[o0 + i] : 0;
            if (S != 0 && S <= full) {
                const int low = S & -S, rest = S ^ low;
                int lowbits = rest, hi = 0;   // rest without its top lg set bits; g spread over those
                for (int t = 0; t < lg; ++t) {
                    const int b = 1 << (31 - __clz(lowbits));
                    lowbits ^= b;
                    if ((g >> (lg - 1 - t)) & 1) hi |= b;
                }
                int sub = lowbits;
                while (true) {   // submasks of lowbits, decreasing, with the fixed top pattern
                    const int m = hi | sub;
                    if (m != rest) {
                        const int Q = low | m;
                        const float c = sm.cost[Q] + sm.cost[S ^ Q];
                        if (c < bc || (c == bc && Q < bq)) {
                            bc = c;
                            bq = Q;
                        }
                    }
                    if (sub == 0) break;
                    sub = (sub - 1) & lowbits;
                }
            }
            if (G > 1) {
                for (int o = G >> 1; o; o >>= 1) {
                    const float oc = __shfl_xor_sync(kFull, bc, o);
                    const int oq = __shfl_xor_sync(kFull, bq, o);
                    if (oc < bc || (oc == bc && oq < bq)) {
                        bc = oc;
                        bq = oq;
                    }
                }
            }
            if (S != 0 && S <= full && g == 0) {
                sm.cost[S] = sm.area[S] + bc;
                sm.best[S] = (uint8_t)bq;
            }
        }
        __syncwarp();
    }
    // 5. rewire only for a clear gain
    if (!(sm.cost[full] < old * 0.99999f)) return;
    if (lane == 0) {   // the new internal nodes, top down: node id, its leaf subset, its children
        int st_set[kTreeletLeaves - 1], st_node[kTreeletLeaves - 1];
        int sp = 0, next_id = 1, m = 0;
        st_set[sp] = full;
        st_node[sp++] = sm.inner[0];
        while (sp > 0) {
            --sp;
            const int S = st_set[sp], id = st_node[sp];
            const int Q = sm.best[S];
            int refs[2];
            const int parts[2] = {Q, S ^ Q};
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int T = parts[c];
                if ((T & (T - 1)) == 0) {
                    refs[c] = sm.lref[__ffs(T) - 1];
                } else {
                    const int nid = sm.inner[next_id++];
                    st_set[sp] = T;
                    st_node[sp++] = nid;
                    refs[c] = nid;
                }
            }
            sm.emit_node[m] = id;
            sm.emit_set[m] = S;
            sm.emit_l[m] = refs[0];
            sm.emit_r[m] = refs[1];
            ++m;
        }
    }
    __syncwarp();
    if (lane < ni) {   // lane i writes new internal node i (the root's box stays as it is)
        const int id = sm.emit_node[lane], S = sm.emit_set[lane];
        const int lr = sm.emit_l[lane], rr = sm.emit_r[lane];
        left[id] = lr;
        right[id] = rr;
        parent[slot_of(lr, n)] = id;
        parent[slot_of(rr, n)] = id;
        if (lane > 0) {
            float bb[6];
            subset_box(sm, S, bb);
            float* bo = box + 6 * (int64_t)id;
#pragma unroll
            for (int c = 0; c < 6; ++c) bo[c] = bb[c];
        }
    }
}

// Depth of every node slot (root 0) by its parent chain; with `height` the
// largest leaf depth is also raised into it (the tree height).  With off >= 0
// the internal nodes at depth = off (mod kTreeletLevels) are appended to
// roots[] (count in *n_roots).
__global__ void k_depth(int64_t n, const int32_t* __restrict__ parent, int32_t* __restrict__ depth,
                        DevCounters* c, int height, int off, int32_t* __restrict__ roots, int* __restrict__ n_roots) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int d = 0;
    if (i < 2 * n - 1) {
        for (int32_t p = parent[i]; p >= 0; p = parent[p]) {
            if (++d == kClimbMax) {   // a parent chain longer than any tree
                atomicCAS(&c->error, 0, RSI_ERR_STACK);
                break;
            }
        }
        depth[i] = d;
        if (height && i >= n - 1) atomicMax(&c->height, d);
    }
    if (off < 0) return;
    const bool root = i < n - 1 && d % kTreeletLevels == off;
    const unsigned m = __ballot_sync(kFull, root);   // one atomic per warp
    if (!m) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(n_roots, __popc(m));
    base = __shfl_sync(kFull, base, __ffs(m) - 1);
    if (root) roots[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
}

// The treelets whose roots k_depth listed: each warp takes roots in turn.
__global__ void __launch_bounds__(32 * kTreeletWarps, kTreeletBlocksPerSm) k_treelet(int64_t n, int32_t* __restrict__ left,
                                                                int32_t* __restrict__ right,
                                                                int32_t* __restrict__ parent,
                                                                float* __restrict__ box,
                                                                const int32_t* __restrict__ roots,
                                                                const int* __restrict__ n_roots) {
    __shared__ TreeletSmem sm[kTreeletWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nr = *n_roots;
    for (int t = blockIdx.x * kTreeletWarps + w; t < nr; t += gridDim.x * kTreeletWarps)
        restructure(roots[t], n, left, right, parent, box, sm[w], lane);
}

// Packed child-pair node i of a tree whose boxes are final.
__device__ __forceinline__ void pack_node(int64_t n, const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                                          const float* __restrict__ box, Node* __restrict__ nodes, int64_t i) {
    const int32_t lc = left[i], rc = right[i];
    const float* bl = box + 6 * slot_of(lc, n);
    const float* br = box + 6 * slot_of(rc, n);
    const int pl = ((uint32_t)lc & kLeafTag) ? ~(int)((uint32_t)lc & ~kLeafTag) : (int)lc;
    const int pr = ((uint32_t)rc & kLeafTag) ? ~(int)((uint32_t)rc & ~kLeafTag) : (int)rc;
    Node nd;
    nd.lmin = make_float4(bl[0], bl[1], bl[2], __int_as_float(pl));
    nd.lmax = make_float4(bl[3], bl[4], bl[5], __int_as_float(pr));
    nd.rmin = make_float4(br[0], br[1], br[2], 0.0f);
    nd.rmax = make_float4(br[3], br[4], br[5], 0.0f);
    nodes[i] = nd;
}

// The packed child-pair nodes of the new tree.
__global__ void k_pack_nodes(int64_t n, const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                             const float* __restrict__ box, Node* __restrict__ nodes) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n - 1) pack_node(n, left, right, box, nodes, i);
}

// ---------------------------------------------------------------- many meshes
// The same passes over all meshes of a batched build: a thread finds its mesh
// by a binary search over the prefix of the per-mesh counts.
__device__ __forceinline__ int mesh_index(const int64_t* __restrict__ pre, int M, int64_t g) {
    int lo = 0, hi = M - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(pre + mid) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int chain_depth(const int32_t* __restrict__ parent, int64_t slot, DevCounters* c) {
    int d = 0;
    for (int32_t p = parent[slot]; p >= 0; p = parent[p]) {
        if (++d == kClimbMax) {
            atomicCAS(&c->error, 0, RSI_ERR_STACK);
            break;
        }
    }
    return d;
}

// The internal nodes at depth = off (mod kTreeletLevels) of every mesh, as
// (node, mesh) pairs.
__global__ void k_roots_seg(const MeshBuild* __restrict__ d, const int64_t* __restrict__ int_pre, int M,
                            int64_t total_int, int off, int32_t* __restrict__ roots_node,
                            int32_t* __restrict__ roots_mesh, int* __restrict__ n_roots) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool root = false;
    int m = 0, i = 0;
    if (g < total_int) {
        m = mesh_index(int_pre, M, g);
        i = (int)(g - __ldg(int_pre + m));
        root = chain_depth(d[m].parent, i, d[m].ctr) % kTreeletLevels == off;
    }
    const unsigned mk = __ballot_sync(kFull, root);   // one atomic per warp
    if (!mk) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == __ffs(mk) - 1) base = atomicAdd(n_roots, __popc(mk));
    base = __shfl_sync(kFull, base, __ffs(mk) - 1);
    if (root) {
        const int at = base + __popc(mk & ((1u << lane) - 1u));
        roots_node[at] = i;
        roots_mesh[at] = m;
    }
}

__global__ void __launch_bounds__(32 * kTreeletWarps, kTreeletBlocksPerSm) k_treelet_seg(const MeshBuild* __restrict__ d,
                                                                    const int32_t* __restrict__ roots_node,
                                                                    const int32_t* __restrict__ roots_mesh,
                                                                    const int* __restrict__ n_roots) {
    __shared__ TreeletSmem sm[kTreeletWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nr = *n_roots;
    for (int t = blockIdx.x * kTreeletWarps + w; t < nr; t += gridDim.x * kTreeletWarps) {
        const MeshBuild& b = d[roots_mesh[t]];
        restructure(roots_node[t], b.nt, b.left, b.right, b.parent, b.box, sm[w], lane);
    }
}

__global__ void k_zero_height_seg(const MeshBuild* __restrict__ d, int M) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) d[m].ctr->height = 0;
}

// Every mesh's height: the largest depth of its leaves.
__global__ void k_height_seg(const MeshBuild* __restrict__ d, const int64_t* __restrict__ tri_pre, int M,
                             int64_t total) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int m = mesh_index(tri_pre, M, g);
    const MeshBuild& b = d[m];
    if (b.nt < 2) return;
    const int64_t j = g - __ldg(tri_pre + m);
    atomicMax(&b.ctr->height, chain_depth(b.parent, b.nt - 1 + j, b.ctr));
}

__global__ void k_pack_seg(const MeshBuild* __restrict__ d, const int64_t* __restrict__ int_pre, int M,
                           int64_t total_int) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total_int) return;
    const int m = mesh_index(int_pre, M, g);
    const MeshBuild& b = d[m];
    pack_node(b.nt, b.left, b.right, b.box, b.nodes, g - __ldg(int_pre + m));
}

// Blocks of a treelet launch: a warp for every internal node that could be a
// root (about a third are), so that no warp takes two treelets in a row;
// blocks past the root count return at once.
int treelet_grid(int64_t n_internal) {
    return (int)std::max<int64_t>(1, (n_internal + kTreeletWarps - 1) / kTreeletWarps);
}

}  // namespace

// Restructuring passes over a finished single build, in stream order without
// host synchronization: each pass restructures the treelets rooted at depths
// 0, 1 and 2 (mod 3) in turn (a depth kernel lists the roots, a persistent
// kernel takes them); then the packed nodes are rewritten and the tree
// height recomputed.  `depth` is build scratch of 2n - 1 ints (the build's
// height array), `list` build scratch of at least n + 16 ints (the sort's).
int enqueue_treelets(rsi_bvh_s* h, int passes, int32_t* depth, int32_t* list, cudaStream_t s) {
    const int64_t n = h->n_tri;
    if (n < 2 || passes <= 0) return RSI_OK;
    passes = passes > 3 ? 3 : passes;
    int* counts = list + n;   // one root count per (pass, offset)
    RSI_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * 3 * kTreeletLevels, s));
    const int nodes_grid = (int)((2 * n - 1 + 255) / 256);
    const int tl_grid = treelet_grid(n - 1);
    int launches = 0;
    for (int p = 0; p < passes; ++p) {
        for (int off = 0; off < kTreeletLevels; ++off) {
            int* cnt = counts + p * kTreeletLevels + off;
            k_depth<<<nodes_grid, 256, 0, s>>>(n, h->parent, depth, h->ctr, 0, off, list, cnt);
            k_treelet<<<tl_grid, 32 * kTreeletWarps, 0, s>>>(n, h->left, h->right, h->parent, h->box, list, cnt);
            launches += 2;
        }
    }
    RSI_CUDA_TRY(cudaMemsetAsync(&h->ctr->height, 0, sizeof(int), s));
    k_depth<<<nodes_grid, 256, 0, s>>>(n, h->parent, depth, h->ctr, 1, -1, nullptr, nullptr);
    k_pack_nodes<<<(int)((n - 1 + 255) / 256), 256, 0, s>>>(n, h->left, h->right, h->box, h->nodes);
    note_launches(launches + 2);
    RSI_CUDA_TRY(cudaGetLastError());
    return RSI_OK;
}

int enqueue_treelets_batched(const MeshBuild* d_mb, const int64_t* d_tri_pre, const int64_t* d_int_pre, int M,
                             int64_t total, int64_t total_int, int passes, int32_t* roots_node, int32_t* roots_mesh,
                             int* counts, cudaStream_t s) {
    if (total_int <= 0 || passes <= 0) return RSI_OK;
    passes = passes > 3 ? 3 : passes;
    RSI_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int) * 3 * kTreeletLevels, s));
    const int int_grid = (int)((total_int + 255) / 256);
    const int tl_grid = treelet_grid(total_int);
    for (int p = 0; p < passes; ++p) {
        for (int off = 0; off < kTreeletLevels; ++off) {
            int* cnt = counts + p * kTreeletLevels + off;
            k_roots_seg<<<int_grid, 256, 0, s>>>(d_mb, d_int_pre, M, total_int, off, roots_node, roots_mesh, cnt);
            k_treelet_seg<<<tl_grid, 32 * kTreeletWarps, 0, s>>>(d_mb, roots_node, roots_mesh, cnt);
        }
    }
    k_zero_height_seg<<<(M + 127) / 128, 128, 0, s>>>(d_mb, M);
    k_height_seg<<<(int)((total + 255) / 256), 256, 0, s>>>(d_mb, d_tri_pre, M, total);
    k_pack_seg<<<int_grid, 256, 0, s>>>(d_mb, d_int_pre, M, total_int);
    note_launches(2 * kTreeletLevels * passes + 3);
    RSI_CUDA_TRY(cudaGetLastError());
    return RSI_OK;
}

}  // namespace rsi
