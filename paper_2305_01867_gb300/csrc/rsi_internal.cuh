// rsi_internal.cuh -- device data layout and host helpers shared by the
// library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "rsi.h"

namespace rsi {

// Packed child-pair node: the boxes of both children next to the two child
// references, so one 64-byte fetch (two 32-byte loads, one L1 sector each)
// lets a segment test both children.  lmin.w holds the left reference, lmax.w the
// right one (as int bits): an internal node index >= 0 or ~leaf for a leaf.
struct __align__(64) Node {
    float4 lmin, lmax, rmin, rmax;
};
static_assert(sizeof(Node) == 64, "node layout");

// Four-wide node of the FP32 traversal: the binary node i at even depth
// together with its children, so that one fetch of 128 bytes (one L1 line)
// tests up to four boxes and the segment's chain of dependent fetches is
// half as long.  Child c's box sits in lane c of the six float4 (structure of
// arrays), ref[c] is its reference (a four-wide node = the binary index of an
// even-depth node, ~leaf for a leaf, kEmpty4 for no child).  Stored at the
// binary index, so slots of odd-depth nodes stay unused.
struct __align__(128) Node4 {
    float4 xlo, xhi, ylo, yhi, zlo, zhi;
    int4 ref;
    int4 pad;
};
static_assert(sizeof(Node4) == 128, "node4 layout");
constexpr int kEmpty4 = 0x7FFFFFFE;   // no child in this lane of a Node4

// Compressed child-pair node (32 bytes, one 32-byte load): the node's own
// box minimum as the frame origin, a power-of-two grid step per axis and the
// children's boxes as 8-bit grid coordinates, rounded outward when built and
// rebuilt with directed-rounding FMAs when read, so a rebuilt box always
// contains the exact one (culling stays conservative).  In Karras numbering
// the right child is the left one + 1, so one index names both children.
//   meta bits 0-7 / 8-15 / 16-23: biased exponents of the x / y / z steps
//   (step = 2^(e - 127)); bit 24: the left child is a leaf; bit 25: the right.
//   q bytes, low byte first: w0 = l.xlo l.ylo l.zlo l.xhi,
//   w1 = l.yhi l.zhi r.xlo r.ylo, w2 = r.zlo r.xhi r.yhi r.zhi.
struct __align__(32) NodeQ {
    float ox, oy, oz;
    uint32_t meta;
    uint32_t w0, w1, w2;
    int32_t split;   // left child index (leaf or internal); right child = split + 1
};
static_assert(sizeof(NodeQ) == 32, "compressed node layout");

// Triangle in leaf (Morton) order: three float4 vertices; v0.w carries the
// caller's triangle id (int bits).  Padded to 64 bytes so that a lane fetches
// it with two 32-byte loads, each reading one whole L1 sector.
struct __align__(64) Tri {
    float4 v0, v1, v2, pad;
};
static_assert(sizeof(Tri) == 64, "triangle layout");

constexpr uint32_t kLeafTag = 0x80000000u;   // leaf tag of the exported tree
constexpr float kTau = 1e-6f;                // relative margin of the band
constexpr double kTauD = 1e-6;
constexpr double kTMerge = 1e-9;             // crossings merged within this t
constexpr int kMaxInclusive = 64;            // inclusive hits kept per FP64 ray

// Per-handle device scratch words.
struct DevCounters {
    int error;          // first RSI_ERR_* raised by a kernel (0 = none)
    int band_count;     // rays queued for the FP64 re-test
    int height;         // tree height (written by the refit)
    int amb_seg_count;  // FP64 pass, count mode: ambiguous segments listed for the crossing count
    unsigned long long node_visits, tri_tests, ambiguous;
    unsigned long long next_ray;   // work counter of the persistent traversal
    unsigned long long ready;      // segments available to the work queue
    int n_fallback;                // learned query: segments left to the tree search
    int n_confirmed;               // learned query: hits confirmed by the proposal
    unsigned int ext_bits[6];   // extent as order-preserving uint (min xyz, max xyz)
    unsigned int dmax_bits[3];  // largest triangle box side per axis (float bits)
    int tpend_count;            // FP64 pass, count mode: certain hits of those whose t is computed
    int pair_count;             // FP64 pass: (segment, triangle) pairs listed
    int fb_count;               // FP64 pass: segments left to the warp-per-segment kernel
    int hard_count;             // FP64 pass: pairs the certain FP64 test left undecided
    int n_finish;               // nearest mode: hitting segments listed for the finish
    int n_finish64;             // nearest mode: of those, left to the FP64 evaluation
    int todo_count;             // FP64 pass: listed pairs the FP32 test left undecided
};

}  // namespace rsi

struct rsi_bvh_s {
    int64_t n_tri = 0, n_vert = 0;
    int morton_bits = 30;
    int height = 0;
    float lo[3], hi[3], dmax[3];
    // packed traversal data
    rsi::Node* nodes = nullptr;   // [max(n_tri - 1, 1)]
    rsi::Node4* nodes4 = nullptr; // [max(n_tri - 1, 1)], even-depth slots used
    rsi::NodeQ* nodesq = nullptr; // [max(n_tri - 1, 1)] compressed child-pair nodes
    bool has_q = false;           // nodesq written (single builds)
    int treelet_passes = 0;       // restructuring passes of its build (a rebuild repeats them)
    rsi::Tri* tris = nullptr;     // [n_tri]
    // exported build arrays
    void* sorted_keys = nullptr;  // uint32 or uint64 [n_tri]
    int32_t* perm = nullptr;      // [n_tri]
    int32_t* left = nullptr;      // [n_tri - 1]
    int32_t* right = nullptr;     // [n_tri - 1]
    int32_t* parent = nullptr;    // [2 n_tri - 1]
    float* box = nullptr;         // [6 (2 n_tri - 1)]
    // scratch
    rsi::DevCounters* ctr = nullptr;
    rsi::DevCounters h_ctr_store{};                // host copy for read-back
    rsi::DevCounters* h_ctr = &h_ctr_store;
    int32_t* band_ids = nullptr;         // [band_cap] rays queued for FP64 (then order,
                                         // proposals and the FP64 fallback list, band_cap each)
    int64_t band_cap = 0;
    char* pair_mem = nullptr;            // pair lists of the FP64 pass (see PairScratch)
    int64_t pair_seg_cap = 0, pair_cap = 0, pair_bytes = 0;
    int64_t device_bytes = 0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};   // traversal / re-test timing
    bool timed = false;
    unsigned int* order_hist = nullptr;   // rsi_segment_order's cell counts (2^15), on first use
    int32_t* hgt = nullptr;               // build scratch in the handle's allocation: node heights,
    int32_t* flags = nullptr;             // arrival flags / range ends (rebuilds reuse them)
    uint64_t gen = 0;                 // process-unique id (plans name hierarchies by it)
    rsi_mlp_s* mlp = nullptr;         // attached proposal network (rsi_mlp_attach)
};

namespace rsi {

// Thread-local last-error message and helpers that turn CUDA failures into
// RSI_ERR_* codes.
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define RSI_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return rsi::cuda_fail(e_, #expr); \
    } while (0)

inline int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : g);
}

int device_sm_count();

// Per-device library context: a private stream-ordered memory pool (freed
// blocks stay cached, frees do not synchronize the device) and the staging
// of host-buffer queries, shared by all handles of the device and serialized
// by `host_mu`.
constexpr int kMaxCtxDevices = 64;
struct DeviceCtx {
    cudaMemPool_t pool = nullptr;
    std::mutex host_mu;
    char* stage = nullptr;                 // two slots of host-query staging
    int64_t stage_chunk = 0;
    cudaStream_t st_in = nullptr, st_out = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_q[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
    DevCounters* h_chunk_ctr = nullptr;    // pinned counters of every chunk of a call
    int64_t h_chunk_cap = 0;
    char* whole = nullptr;                 // whole-batch staging of host-buffer queries
    int64_t whole_cap = 0;                 // segments it holds (30 B each)
    cudaEvent_t ev_chunk[64] = {};         // copy-in events of the whole-batch chunks
    unsigned long long* h_ready = nullptr; // pinned: segments copied in so far, per chunk
    unsigned int* d_done = nullptr;        // device: finished segments per output chunk of a whole-batch query
    unsigned int* h_done = nullptr;        // pinned: the host's copy of them
    cudaStream_t st_poll = nullptr;        // copies of those counters
};
DeviceCtx* device_ctx();   // the current device's context (NULL without a device)
int pool_alloc(void** p, size_t bytes, cudaStream_t s);
void pool_free(void* p, cudaStream_t s);

// Allocation-failure injection (rsi_debug_fail_allocations): true when the
// current allocation is to fail.  Every device and pinned allocation of the
// library asks it first.
bool alloc_injected();
// cudaMalloc / cudaMallocHost that honour the injection and leave *p NULL
// after any failure, so a later release never sees a stale pointer.
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) {
    cudaError_t e = alloc_injected() ? cudaErrorMemoryAllocation : cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e != cudaSuccess) *p = nullptr;
    return e;
}
template <class T>
cudaError_t host_malloc_pinned(T** p, size_t bytes) {
    cudaError_t e =
        alloc_injected() ? cudaErrorMemoryAllocation : cudaMallocHost(reinterpret_cast<void**>(p), bytes);
    if (e != cudaSuccess) *p = nullptr;
    return e;
}

// Count of kernel launches made by the library (rsi_kernel_launches).
void note_launches(int n);
// One mesh of a batched build (build.cu, treelet.cu): its inputs and the
// arrays of its handle.
struct MeshBuild {
    const float* V;
    const int32_t* T;
    int64_t nv, nt;
    Node* nodes;
    Node4* nodes4;
    Tri* tris;
    void* keys;   // the handle's sorted keys (uint32 or uint64)
    int32_t *perm, *left, *right, *parent, *hgt, *ends;
    float* box;
    DevCounters* ctr;
};

// Restructuring passes after a single build (treelet.cu).
int enqueue_treelets(rsi_bvh_s* h, int passes, int32_t* depth, int32_t* list, cudaStream_t s);
// The same over all meshes of a batched build (roots_node / roots_mesh: the
// internal-node count of ints each; counts: 9 ints).
int enqueue_treelets_batched(const MeshBuild* d_mb, const int64_t* d_tri_pre, const int64_t* d_int_pre, int M,
                             int64_t total, int64_t total_int, int passes, int32_t* roots_node, int32_t* roots_mesh,
                             int* counts, cudaStream_t s);

// A batched rebuild prepared for capture: the hierarchies' own arrays are
// rebuilt in place from the meshes' current buffers (the sizes fixed at
// preparation), by kernels that rebuild_enqueue issues without any host
// synchronization.  d_ctr receives every mesh's build counters (errors,
// height, extent, padding); refresh_handles copies them to the handles.
struct RebuildSpec {
    char* mem = nullptr;        // one allocation: table, prefixes, sort buffers, counters
    int M = 0, morton_bits = 30;
    int treelet_passes = 0;     // the most any of the hierarchies was built with
    int64_t total = 0, total_int = 0;
    void* d_mb = nullptr;       // [M] per-mesh build descriptors
    int64_t* d_tri_pre = nullptr;
    int64_t* d_int_pre = nullptr;
    void *ka = nullptr, *kb = nullptr, *codes = nullptr;
    int32_t *va = nullptr, *vb = nullptr;
    uint32_t *mka = nullptr, *mkb = nullptr, *hist = nullptr;
    DevCounters* d_ctr = nullptr;
    std::vector<rsi_bvh_t> hs;
};
int rebuild_prepare(const rsi_bvh_t* hs, int M, const float* const* V, const int32_t* const* T, cudaStream_t s,
                    RebuildSpec* out);
int rebuild_enqueue(const RebuildSpec& r, cudaStream_t s);
void rebuild_release(RebuildSpec& r);
// Host copies of the hierarchies' extent, padding and height after a rebuild
// has run (synchronizes s); the first mesh error found, else RSI_OK.
int refresh_handles(const RebuildSpec& r, cudaStream_t s);

// Process-unique id of a new hierarchy (never 0, never reused).
uint64_t next_handle_gen();
// Attachments of proposal networks to hierarchies (rsi_mlp_attach): every
// change goes through these, so that freeing either side detaches both.
void attach_mlp(rsi_bvh_t h, rsi_mlp_s* m);
void forget_handle(rsi_bvh_t h);   // lbvh_free: detach, drop cached plans naming h
void forget_mlp(rsi_mlp_s* m);     // rsi_mlp_free: detach from every hierarchy
// The batched-query plan cache (query.cu): drop every plan naming `gen`.
void drop_plans_of(uint64_t gen);

namespace mlpk {
// Tensor-core inference of the proposal network (mlp.cu).
int forward_tc(rsi_mlp_s* m, rsi_bvh_t h, const float* from, const float* to, int64_t n, float* logits,
               uint8_t* top4, cudaStream_t s);
// The same kernel with the proposal verified in place: settled segments get
// hit = 1 (amb = 0), the others are listed in `order` (count in
// ctr->n_fallback); ctr must be reset first.
int propose_verify(rsi_mlp_s* m, rsi_bvh_t h, const float* from, const float* to, int64_t n, uint8_t* hit,
                   uint8_t* amb, int32_t* order, DevCounters* ctr, int stats, cudaStream_t s);
}  // namespace mlpk

}  // namespace rsi
