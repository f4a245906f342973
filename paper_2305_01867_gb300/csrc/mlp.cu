// mlp.cu -- the cluster-proposal network of the learned any-hit query:
// segment end points -> 128 -> 128 -> 256 cluster logits (GELU), BF16
// weights and layer inputs, FP32 accumulation.  (Not in the paper: the
// proposal, its training and the proposal-verify-fallback query are added
// on top of the method; the fallback is the paper's full tree search, so
// answers stay exactly those of the plain query.)
//
//  k_mlp_tc<VERIFY>  persistent inference on the 5th-generation tensor
//                    cores: per tile of 128 segments three tcgen05.mma
//                    chains (K = 16, 128, 128; N = 128, 128, 256) with FP32
//                    accumulators in TMEM, operands in shared memory in the
//                    no-swizzle K-major core-matrix layout; two tile groups
//                    alternate so that one group's TMEM->register epilogue
//                    (bias, GELU, BF16 rounding, top-4 cluster selection)
//                    runs while the other group's chains run.  With VERIFY
//                    the top-4 never leave registers: the proposed clusters'
//                    triangles are tested in the same kernel and the
//                    segments they do not settle are listed for the tree
//                    search.
//  training          FP32 SIMT kernels (tiled GEMMs, fused elementwise
//                    steps, Adam) on the same BF16 roundings; the network is
//                    small and training is a one-off set-up cost.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "rsi_internal.cuh"
#include "segtest.cuh"

namespace rsi {
namespace mlpk {

constexpr int kIn = 16, kH = 128, kOut = 256;
constexpr int kW1 = kIn * kH, kW2 = kH * kH, kW3 = kH * kOut;   // element counts
constexpr int kParams = kW1 + kH + kW2 + kH + kW3 + kOut;        // W1 b1 W2 b2 W3 b3
constexpr int kOffW1 = 0, kOffB1 = kW1, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kW2, kOffW3 = kOffB2 + kH,
              kOffB3 = kOffW3 + kW3;
// BF16 images of W^T (N rows x K columns, K-major core matrices) in the order
// the forward kernel copies them to shared memory
constexpr int kImgW1 = 0, kImgW2 = kImgW1 + kH * kIn * 2, kImgW3 = kImgW2 + kH * kH * 2,
              kImgBytes = kImgW3 + kOut * kH * 2;   // 102400 bytes

// Byte offset of element (row, k) of a K-major operand with K columns: core
// matrices of 8 rows x 8 elements (128 B), K-adjacent ones 128 B apart
// (leading byte offset), row-adjacent groups K * 16 B apart (stride offset).
__host__ __device__ constexpr uint32_t cm_offset(int row, int k, int K) {
    return (uint32_t)((row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// GELU in its tanh form (Hendrycks & Gimpel 2016, "Gaussian Error Linear
// Units"): GELU(z) = 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).
// Inference evaluates tanh with the hardware approximation tanh.approx.f32
// (one special-function instruction; its error stays below 2^-10.5 of the
// result, far below the BF16 resolution of the layer outputs except at
// rounding boundaries); training evaluates it with CUDA's tanhf and
// differentiates the same formula.
constexpr float kG0 = 0.7978845608028654f;     // sqrt(2 / pi)
constexpr float kG1 = 0.035677408136300125f;   // 0.044715 sqrt(2 / pi)
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu_fast(float z) {
    const float h = 0.5f * z;
    return fmaf(h, tanh_fast(z * fmaf(kG1, z * z, kG0)), h);
}
__device__ __forceinline__ float gelu(float z) {
    const float h = 0.5f * z;
    return fmaf(h, tanhf(z * fmaf(kG1, z * z, kG0)), h);
}
__device__ __forceinline__ float gelu_grad(float z) {
    const float z2 = z * z;
    const float t = tanhf(z * fmaf(kG1, z2, kG0));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * fmaf(3.0f * kG1, z2, kG0);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Features of segment r: both end points mapped by the extent to [-1, 1],
// clamped to [-4, 4]; inputs 6..15 are zero.
__device__ __forceinline__ void seg_features(const float* __restrict__ from, const float* __restrict__ to, int64_t r,
                                             const float lo[3], const float sc[3], float f[6]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f[a] = fminf(fmaxf((from[3 * r + a] - lo[a]) * sc[a] - 1.0f, -4.0f), 4.0f);
        f[3 + a] = fminf(fmaxf((to[3 * r + a] - lo[a]) * sc[a] - 1.0f, -4.0f), 4.0f);
    }
}

// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared memory matrix descriptor: start >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29), stride byte offset >> 4 (32-45), version 1 (46-47),
// base offset 0, no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B in BF16 (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for an mbarrier phase: the waiting thread is suspended by the
// hardware between checks (suspend-time hint 1 ms) instead of spinning;
// false after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    const unsigned long long t0 = now_ns();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase), "r"(1000000u)
            : "memory");
        if (done) return true;
        if (now_ns() - t0 > 2000000000ull) return false;
    }
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
    uint32_t r[32];
    __syncwarp();   // .sync.aligned: the whole warp issues the load together
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Shared memory map of the tensor-core kernel (bytes from a 1024-aligned
// base): the weight images, then per tile group its layer inputs, the
// biases, the top-4 exchange between the two column halves of a row and
// their verification flags, the mbarriers and the TMEM address.
constexpr int kXBytes = 128 * kIn * 2;          // [128 x 16] BF16 features of one tile
constexpr int kHBytes = 128 * kH * 2;           // [128 x 128] BF16 hidden activations
constexpr int kSmX = kImgBytes;                 // group g: kSmX + g kXBytes
constexpr int kSmH = kSmX + 2 * kXBytes;        // group g: kSmH + g kHBytes
constexpr int kSmBias = kSmH + 2 * kHBytes;     // 512 floats
constexpr int kSmXchg = kSmBias + 512 * 4;      // [group][half][row] 4 keys
// verification, per group: the rows' segments (start, direction, |d|_1),
// proposed clusters, hit flags, the list of rows left after the best
// cluster and its length
constexpr int kVerBytes = 128 * 32 + 128 * 4 + 128 * 4 + 128 * 4 + 16;
constexpr int kSmVer = kSmXchg + 2 * 2 * 128 * 16;
constexpr int kSmBar = kSmVer + 2 * kVerBytes;   // bar_in[2], bar_mma[2], bar_x[2], TMEM address
constexpr int kSmBytes = kSmBar + 64;
constexpr int kTmemCols = 512;
// 16 warps: two tile groups of 8 (4 TMEM lane quarters x 2 column halves);
// lane 0 of each group's first warp issues that group's tensor-core chains.
constexpr int kTcThreads = 16 * 32;

struct TcArgs {
    const uint8_t* img;    // BF16 weight images
    const float* bias;     // b1 | b2 | b3
    const float* from;
    const float* to;
    int n;
    float lo0, lo1, lo2, sc0, sc1, sc2;   // feature map: (p - lo) * sc - 1
    int* err;              // RSI_ERR_TIMEOUT if a wait ran out
    // inference outputs (rsi_mlp_forward)
    float* logits;         // [n][256] or NULL
    uint8_t* top4;         // [n][4] or NULL (cluster ids, best first)
    // verification (the learned query)
    const Tri* tris;
    int n_tri;
    int cluster_max;       // triangles of the largest cluster: ceil(n_tri / 256)
    float dmax0, dmax1, dmax2;
    uint8_t* hit;
    uint8_t* amb;
    int32_t* order;        // segments left to the tree search
    DevCounters* ctr;      // n_fallback, n_confirmed, tri_tests
    int stats;
};

// Top-4 selection keys: the FP32 logit with its low 8 bits replaced by
// 255 - cluster, compared as floats.  Logits are thereby compared to 24
// significant bits, no two keys of a row are equal, and on equal 24-bit
// prefixes the lower cluster ranks first for a positive logit (the higher
// for a negative one).  The insertion keeps t0 >= t1 >= t2 >= t3.
__device__ __forceinline__ float logit_key(float z, int cluster) {
    return __uint_as_float((__float_as_uint(z) & 0xFFFFFF00u) | (uint32_t)(255 - cluster));
}
__device__ __forceinline__ int key_cluster(float k) { return 255 - (int)(__float_as_uint(k) & 255u); }
__device__ __forceinline__ void top4_insert(float k, float t[4]) {
    const float m0 = fminf(t[0], k), m1 = fminf(t[1], k), m2 = fminf(t[2], k);
    t[3] = fmaxf(t[3], m2);
    t[2] = fmaxf(t[2], m1);
    t[1] = fmaxf(t[1], m0);
    t[0] = fmaxf(t[0], k);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Two 32-column TMEM loads of this thread's lane, one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float v[64]) {
    uint32_t r[64];
    __syncwarp();
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
          "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr + 32));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 64; ++j) v[j] = __uint_as_float(r[j]);
}

// Hidden-layer epilogue of this thread's 64 columns c0 .. c0 + 63 of its
// row: + bias -> GELU -> BF16 -> the next layer's K-major A operand.
__device__ __forceinline__ void epilogue_hidden(uint32_t taddr, const float* __restrict__ bias, uint8_t* sH, int row,
                                                int c0) {
    float v[64];
    tmem_ld64(taddr + c0, v);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int k0 = c0 + 8 * q;
        uint4 w;
        w.x = pack_bf16x2(gelu_fast(v[8 * q + 0] + bias[k0 + 0]), gelu_fast(v[8 * q + 1] + bias[k0 + 1]));
        w.y = pack_bf16x2(gelu_fast(v[8 * q + 2] + bias[k0 + 2]), gelu_fast(v[8 * q + 3] + bias[k0 + 3]));
        w.z = pack_bf16x2(gelu_fast(v[8 * q + 4] + bias[k0 + 4]), gelu_fast(v[8 * q + 5] + bias[k0 + 5]));
        w.w = pack_bf16x2(gelu_fast(v[8 * q + 6] + bias[k0 + 6]), gelu_fast(v[8 * q + 7] + bias[k0 + 7]));
        *reinterpret_cast<uint4*>(sH + cm_offset(row, k0, kH)) = w;
    }
}

// Persistent tensor-core kernel of the proposal network, one CTA per SM.
//
// Two tile groups of 8 warps each work on alternate 128-segment tiles so
// that one group's SIMT epilogue (bias, GELU, BF16 packing, top-4, proposal
// verification) overlaps the other group's tensor-core chains.  Group g owns
// TMEM columns 256 g .. 256 g + 255: layer 1 accumulates into the first 128,
// layer 2 into the second 128, layer 3 (N = 256) into all of them once the
// layer-2 epilogue has read its accumulator.  Per layer, the group's warps
// arrive on bar_in[g] when the layer's A operand is in shared memory; the
// group's issuing thread waits for all eight, issues the chain and commits
// it to bar_mma[g], on which the group waits.  The two groups issue
// independently; the tensor cores interleave their chains.  Every wait is
// bounded (about 2 s: RSI_ERR_TIMEOUT, then the kernel leaves its loops,
// waits for its last commit and frees TMEM).
//
// VERIFY = false: logits and top-4 cluster ids are written (rsi_mlp_forward).
// VERIFY = true: the top-4 stay in registers; the row's two column halves
// each test the triangles of two of the proposed clusters in FP32; a
// certain decisive hit settles the segment (hit = 1, not ambiguous), every
// other segment is appended to `order` for the tree search.
template <bool VERIFY>
__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_tc(TcArgs P) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* sBias = reinterpret_cast<float*>(sm + kSmBias);
    const uint32_t bar0 = smem_addr(sm + kSmBar);   // bar_in[0..1], bar_mma[0..1], bar_x[0..1]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kSmBar + 48);

    for (int i = tid; i < kImgBytes / 16; i += kTcThreads)
        reinterpret_cast<uint4*>(sm)[i] = reinterpret_cast<const uint4*>(P.img)[i];
    for (int i = tid; i < 512; i += kTcThreads) sBias[i] = P.bias[i];
    if (tid == 0) {
        mbar_init(bar0, 8);   // bar_in: one arrival per warp of the group
        mbar_init(bar0 + 8, 8);
        mbar_init(bar0 + 16, 1);
        mbar_init(bar0 + 24, 1);
        mbar_init(bar0 + 32, 8);
        mbar_init(bar0 + 40, 8);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *tslot;
    const int64_t n_tiles = ((int64_t)P.n + 127) / 128;
    const int64_t G = gridDim.x;

    const uint32_t aW1 = smem_addr(sm + kImgW1), aW2 = smem_addr(sm + kImgW2), aW3 = smem_addr(sm + kImgW3);
    {
        // ---------------------------------------------------------------- tile groups
        const int g = warp >> 3, q = warp & 3, half = (warp >> 2) & 1;
        const bool issuer = (warp & 7) == 0 && lane == 0;
        const uint32_t aX = smem_addr(sm + kSmX + g * kXBytes), aH = smem_addr(sm + kSmH + g * kHBytes);
        const uint32_t dcol = tbase + 256u * (uint32_t)g;
        uint32_t pin = 0, issued = 0;
        const int row = 32 * q + lane;
        uint8_t* sX = sm + kSmX + g * kXBytes;
        uint8_t* sH = sm + kSmH + g * kHBytes;
        float4* sXchg = reinterpret_cast<float4*>(sm + kSmXchg);
        uint8_t* sVer = sm + kSmVer + g * kVerBytes;
        float4* sSeg = reinterpret_cast<float4*>(sVer);                       // [row][2]: s | dl1, d
        uchar4* sCl = reinterpret_cast<uchar4*>(sVer + 128 * 32);              // [row] proposed clusters
        int* sHit = reinterpret_cast<int*>(sVer + 128 * 32 + 512);             // [row] -1 none, 0 open, 1 hit
        int* sList = reinterpret_cast<int*>(sVer + 128 * 32 + 1024);           // rows left after cluster 0
        int* sLeft = reinterpret_cast<int*>(sVer + 128 * 32 + 1536);           // their number
        const int tg = (warp & 7) * 32 + lane;                                 // thread in the group
        const uint32_t bar_in = bar0 + 8 * g, bar_mma = bar0 + 16 + 8 * g, bar_x = bar0 + 32 + 8 * g;
        const uint32_t tl = tbase + ((uint32_t)(32 * q) << 16) + 256u * (uint32_t)g;
        const float lo[3] = {P.lo0, P.lo1, P.lo2}, sc[3] = {P.sc0, P.sc1, P.sc2};
        uint32_t ph = 0, px = 0;
        int64_t confirmed_n = 0, tests = 0;
        float nxt[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        auto load_seg = [&](int64_t t) {
            const int64_t r = t * 128 + row;
            if (t < n_tiles && r < P.n) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    nxt[a] = __ldg(P.from + 3 * r + a);
                    nxt[3 + a] = __ldg(P.to + 3 * r + a);
                }
            }
        };
        // waits are decided per warp (__all_sync), so that a warp leaves its
        // loop as a whole and its lanes keep meeting the same warp-wide steps
        auto wait_mma = [&]() -> bool {
            const bool ok = __all_sync(0xffffffffu, mbar_wait(bar_mma, ph));
            ph ^= 1u;
            if (!ok) atomicCAS(P.err, 0, RSI_ERR_TIMEOUT);
            fence_after();
            return ok;
        };
        // the layer's A operand is in shared memory: arrive; the issuing
        // thread waits for the group's eight warps and issues the chain
        auto arrive_in = [&](int layer) {
            fence_proxy_async();   // generic-proxy writes of the operand -> visible to the tensor cores
            fence_before();        // this thread's TMEM reads are complete
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_in);
            if (issuer) {
                const bool ok = mbar_wait(bar_in, pin);
                pin ^= 1u;
                if (!ok) {
                    atomicCAS(P.err, 0, RSI_ERR_TIMEOUT);
                    return;   // nothing issued: the group's wait for this chain runs out
                }
                fence_after();
                if (layer == 0) {
                    mma_bf16(dcol, smem_desc(aX, 128, kIn * 16), smem_desc(aW1, 128, kIn * 16), idesc_bf16(128, kH), 0);
                } else if (layer == 1) {
                    for (int ks = 0; ks < kH / 16; ++ks)
                        mma_bf16(dcol + 128, smem_desc(aH + 256 * ks, 128, kH * 16),
                                 smem_desc(aW2 + 256 * ks, 128, kH * 16), idesc_bf16(128, kH), ks > 0);
                } else {
                    for (int ks = 0; ks < kH / 16; ++ks)
                        mma_bf16(dcol, smem_desc(aH + 256 * ks, 128, kH * 16), smem_desc(aW3 + 256 * ks, 128, kH * 16),
                                 idesc_bf16(128, kOut), ks > 0);
                }
                mma_commit(bar_mma);
                ++issued;
            }
        };
        // the two column halves of a row exchange through shared memory
        auto xchg_sync = [&]() -> bool {
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_x);
            const bool ok = __all_sync(0xffffffffu, mbar_wait(bar_x, px));
            px ^= 1u;
            if (!ok) atomicCAS(P.err, 0, RSI_ERR_TIMEOUT);
            return ok;
        };
        int64_t tile = blockIdx.x + G * g;
        load_seg(tile);
        for (; tile < n_tiles; tile += 2 * G) {
            const int64_t r = tile * 128 + row;
            const bool valid = r < P.n;
            float seg[6];
#pragma unroll
            for (int a = 0; a < 6; ++a) seg[a] = nxt[a];
            load_seg(tile + 2 * G);   // the next tile's segment, in flight during this tile
            if (half == 0) {
                float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (valid) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        f[a] = fminf(fmaxf((seg[a] - lo[a]) * sc[a] - 1.0f, -4.0f), 4.0f);
                        f[3 + a] = fminf(fmaxf((seg[3 + a] - lo[a]) * sc[a] - 1.0f, -4.0f), 4.0f);
                    }
                }
                uint4 w0;
                w0.x = pack_bf16x2(f[0], f[1]);
                w0.y = pack_bf16x2(f[2], f[3]);
                w0.z = pack_bf16x2(f[4], f[5]);
                w0.w = 0u;
                *reinterpret_cast<uint4*>(sX + cm_offset(row, 0, kIn)) = w0;
                *reinterpret_cast<uint4*>(sX + cm_offset(row, 8, kIn)) = make_uint4(0u, 0u, 0u, 0u);
            }
            arrive_in(0);
            if (!wait_mma()) break;
            epilogue_hidden(tl, sBias, sH, row, 64 * half);
            arrive_in(1);
            if (!wait_mma()) break;
            epilogue_hidden(tl + 128, sBias + kH, sH, row, 64 * half);
            arrive_in(2);
            if (!wait_mma()) break;
            // logits of this half (128 columns): bias, keys, top-4
            float t4[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
#pragma unroll 1
            for (int cc = 0; cc < 2; ++cc) {
                const int c0 = 128 * half + 64 * cc;
                float v[64];
                tmem_ld64(tl + c0, v);
#pragma unroll
                for (int j = 0; j < 64; ++j) {
                    v[j] += sBias[2 * kH + c0 + j];
                    top4_insert(logit_key(v[j], c0 + j), t4);
                }
                if (!VERIFY && P.logits && valid) {
                    float4* dst = reinterpret_cast<float4*>(P.logits + r * kOut + c0);
#pragma unroll
                    for (int j = 0; j < 16; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
            }
            fence_before();   // TMEM reads of this tile are complete before the group's next arrival
            sXchg[(g * 2 + half) * 128 + row] = make_float4(t4[0], t4[1], t4[2], t4[3]);
            if (!xchg_sync()) break;
            {
                const float4 o = sXchg[(g * 2 + (half ^ 1)) * 128 + row];
                top4_insert(o.x, t4);
                top4_insert(o.y, t4);
                top4_insert(o.z, t4);
                top4_insert(o.w, t4);
            }
            if (!VERIFY) {
                if (half == 0 && P.top4 && valid)
                    *reinterpret_cast<uchar4*>(P.top4 + 4 * r) =
                        make_uchar4((uint8_t)key_cluster(t4[0]), (uint8_t)key_cluster(t4[1]),
                                    (uint8_t)key_cluster(t4[2]), (uint8_t)key_cluster(t4[3]));
            } else {
                // Verification, packed over the group's 256 threads: every
                // open row's best cluster first (one (row, triangle) pair per
                // slot), then clusters 2-4 of the rows that cluster 1 left.
                // A slot tests one triangle; a certain decisive hit settles
                // its row.  No lane waits on another row's longer list.
                if (half == 0) {
                    const float3 s = make_float3(seg[0], seg[1], seg[2]), e = make_float3(seg[3], seg[4], seg[5]);
                    const bool open = valid && !(segtest::bad3(s) || segtest::bad3(e));
                    const float3 d = make_float3(e.x - s.x, e.y - s.y, e.z - s.z);
                    sSeg[2 * row] = make_float4(s.x, s.y, s.z, fabsf(d.x) + fabsf(d.y) + fabsf(d.z));
                    sSeg[2 * row + 1] = make_float4(d.x, d.y, d.z, 0.0f);
                    sCl[row] = make_uchar4((uint8_t)key_cluster(t4[0]), (uint8_t)key_cluster(t4[1]),
                                           (uint8_t)key_cluster(t4[2]), (uint8_t)key_cluster(t4[3]));
                    sHit[row] = open ? 0 : -1;
                }
                if (tg == 0) *sLeft = 0;
                if (!xchg_sync()) break;
                const int W = P.cluster_max;
                auto test_slot = [&](int rw, int c, int k) {
                    const int j = segtest::cluster_begin(c, P.n_tri) + k;
                    if (j >= segtest::cluster_begin(c + 1, P.n_tri)) return;
                    const float4 a = sSeg[2 * rw], b = sSeg[2 * rw + 1];
                    segtest::SegF sg;
                    sg.s = make_float3(a.x, a.y, a.z);
                    sg.d = make_float3(b.x, b.y, b.z);
                    sg.dl1 = a.w;
                    ++tests;
                    if (segtest::tri_certain_hit(sg, segtest::load_tri(P.tris, j))) sHit[rw] = 1;
                };
#pragma unroll 1
                for (int slot = tg; slot < 128 * W; slot += 256) {   // cluster 1 of every open row
                    const int rw = slot / W;
                    if (sHit[rw] == 0) test_slot(rw, sCl[rw].x, slot - rw * W);
                }
                if (!xchg_sync()) break;
                if (half == 0 && sHit[row] == 0) sList[atomicAdd(sLeft, 1)] = row;
                if (!xchg_sync()) break;
                const int left = *sLeft;
#pragma unroll 1
                for (int slot = tg; slot < left * 3 * W; slot += 256) {   // clusters 2-4 of the rows left
                    const int i = slot / (3 * W), rem = slot - i * 3 * W;
                    const int rw = sList[i], ci = rem / W;
                    const uchar4 cl = sCl[rw];
                    test_slot(rw, ci == 0 ? cl.y : (ci == 1 ? cl.z : cl.w), rem - ci * W);
                }
                if (!xchg_sync()) break;
                if (half == 0) {
                    const bool confirmed = sHit[row] == 1;
                    if (valid && confirmed) {
                        P.hit[r] = 1;
                        if (P.amb) P.amb[r] = 0;
                        ++confirmed_n;
                    }
                    const bool left_row = valid && !confirmed;
                    const unsigned m = __ballot_sync(0xffffffffu, left_row);
                    int base = 0;
                    if (lane == 0 && m) base = atomicAdd(&P.ctr->n_fallback, __popc(m));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (left_row) P.order[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)r;
                }
            }
        }
        // after a timeout the group may have left with a chain still running:
        // wait for the issuer's last commit (bounded) before TMEM is freed
        if (issuer && issued) mbar_wait(bar_mma, (issued - 1u) & 1u);
        if (VERIFY) {
            for (int off = 16; off; off >>= 1) {
                confirmed_n += __shfl_xor_sync(0xffffffffu, confirmed_n, off);
                tests += __shfl_xor_sync(0xffffffffu, tests, off);
            }
            if (lane == 0 && confirmed_n) atomicAdd(&P.ctr->n_confirmed, (int)confirmed_n);
            if (lane == 0 && P.stats && tests) atomicAdd(&P.ctr->tri_tests, (unsigned long long)tests);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
    }
}

// The network's activation pieces on a vector (tests): the hardware tanh
// approximation, CUDA's tanhf beside it, and GELU as inference applies it.
__global__ void k_activation(const float* __restrict__ z, int64_t n, float* __restrict__ tanh_a,
                             float* __restrict__ tanh_cuda, float* __restrict__ g) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    tanh_a[i] = tanh_fast(z[i]);
    tanh_cuda[i] = tanhf(z[i]);
    g[i] = gelu_fast(z[i]);
}

// FP32 master parameters -> BF16 images of W1^T, W2^T, W3^T (core-matrix
// layout) and the FP32 biases.
__global__ void k_mlp_pack(const float* __restrict__ p, uint8_t* __restrict__ img, float* __restrict__ bias) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    __nv_bfloat16* im = reinterpret_cast<__nv_bfloat16*>(img);
    if (i < kW1) {   // W1[k][n], k < 16, n < 128
        const int k = i / kH, n = i % kH;
        im[(kImgW1 + cm_offset(n, k, kIn)) / 2] = __float2bfloat16_rn(p[kOffW1 + i]);
    } else if (i < kW1 + kW2) {
        const int j = i - kW1, k = j / kH, n = j % kH;
        im[(kImgW2 + cm_offset(n, k, kH)) / 2] = __float2bfloat16_rn(p[kOffW2 + j]);
    } else if (i < kW1 + kW2 + kW3) {
        const int j = i - kW1 - kW2, k = j / kOut, n = j % kOut;
        im[(kImgW3 + cm_offset(n, k, kH)) / 2] = __float2bfloat16_rn(p[kOffW3 + j]);
    }
    if (i < kH) {
        bias[i] = p[kOffB1 + i];
        bias[kH + i] = p[kOffB2 + i];
    }
    if (i < kOut) bias[2 * kH + i] = p[kOffB3 + i];
}

// ---------------------------------------------------------------- training
// C[M][N] = op(A)[M][K] op(B)[K][N] in FP32; op(A)[m][k] = TA ? A[k][m] :
// A[m][k] (row-major, leading dimension lda), likewise B.  64 x 64 tiles,
// 256 threads, 4 x 4 outputs per thread.
// blockIdx.z splits K into chunks of kchunk; with more than one chunk the
// partial products are added into C (zeroed by the caller).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(const float* __restrict__ A, const float* __restrict__ B,
                                              float* __restrict__ C, int M, int N, int K, int lda, int ldb, int ldc,
                                              int kchunk) {
    __shared__ float As[16][64 + 4], Bs[16][64 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    float acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += 16) {
        for (int i = threadIdx.x; i < 16 * 64; i += 256) {
            const int kk = i / 64, mm = i % 64;
            const int m = m0 + mm, k = k0 + kk, n = n0 + mm;
            As[kk][mm] = (m < M && k < ke) ? (TA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k]) : 0.0f;
            Bs[kk][mm] = (n < N && k < ke) ? (TB ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n]) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                b[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                if (gridDim.z > 1) atomicAdd(C + (int64_t)m * ldc + n, acc[i][j]);
                else C[(int64_t)m * ldc + n] = acc[i][j];
            }
        }
}

// BF16-rounded copies of the weight matrices (the values the forward uses).
__global__ void k_round_weights(const float* __restrict__ p, float* __restrict__ wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kW1) wb[i] = bf16r(p[kOffW1 + i]);
    else if (i < kW1 + kW2) wb[i] = bf16r(p[kOffW2 + i - kW1]);
    else if (i < kW1 + kW2 + kW3) wb[i] = bf16r(p[kOffW3 + i - kW1 - kW2]);
}

__global__ void k_train_features(const float* __restrict__ from, const float* __restrict__ to, int n, float lo0,
                                 float lo1, float lo2, float sc0, float sc1, float sc2, float* __restrict__ x) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float lo[3] = {lo0, lo1, lo2}, sc[3] = {sc0, sc1, sc2};
    float f[6];
    seg_features(from, to, r, lo, sc, f);
#pragma unroll
    for (int k = 0; k < kIn; ++k) x[(int64_t)r * kIn + k] = k < 6 ? bf16r(f[k]) : 0.0f;
}

// z += b (kept for the backward); a = BF16(GELU(z)).
__global__ void k_bias_gelu(float* __restrict__ z, const float* __restrict__ b, float* __restrict__ a, int rows, int cols) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * cols) return;
    const float v = z[i] + b[i % cols];
    z[i] = v;
    a[i] = bf16r(gelu(v));
}

// Mean BCE with logits over n x 256: dz = (sigmoid(z + b3) - y) / (n 256);
// the loss sum goes to *loss.
__global__ void k_bce(float* __restrict__ z, const float* __restrict__ b3, const uint32_t* __restrict__ labels, int n,
                      float* __restrict__ loss) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (i < (int64_t)n * kOut) {
        const int c = (int)(i % kOut);
        const int64_t r = i / kOut;
        const float v = z[i] + b3[c];
        const float y = (float)((labels[r * 8 + (c >> 5)] >> (c & 31)) & 1u);
        l = fmaxf(v, 0.0f) - v * y + log1pf(expf(-fabsf(v)));
        z[i] = (1.0f / (1.0f + expf(-v)) - y) / ((float)n * kOut);
    }
    for (int off = 16; off; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// dz = da * GELU'(z)
__global__ void k_gelu_back(const float* __restrict__ da, const float* __restrict__ z, float* __restrict__ dz, int64_t m) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) dz[i] = da[i] * gelu_grad(z[i]);
}

// g[c] += sum over a chunk of 256 rows of d[r][c] (g zeroed by the caller)
__global__ void k_colsum(const float* __restrict__ d, int rows, int cols, float* __restrict__ g) {
    const int c = threadIdx.x;
    const int r0 = blockIdx.x * 256, r1 = min(rows, r0 + 256);
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = r0; r < r1; ++r) s += d[(int64_t)r * cols + c];
    atomicAdd(g + c, s);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace mlpk
}  // namespace rsi

struct rsi_mlp_s {
    float* params = nullptr;   // FP32 master weights [kParams]
    float* grads = nullptr;    // [kParams]
    float* adam_m = nullptr;   // [kParams]
    float* adam_v = nullptr;   // [kParams]
    uint8_t* img = nullptr;    // BF16 images
    float* bias = nullptr;     // 512
    int* scratch_i = nullptr;  // tile counter, error
    int64_t step = 0;
    bool packed = false;
    // training scratch
    float* act = nullptr;
    int64_t act_cap = 0;
    float* d_loss = nullptr;
};

namespace rsi {
namespace mlpk {

int ensure_packed(rsi_mlp_s* m, cudaStream_t s) {
    if (m->packed) return RSI_OK;
    k_mlp_pack<<<grid_for(kW1 + kW2 + kW3, 256), 256, 0, s>>>(m->params, m->img, m->bias);
    note_launches(1);
    RSI_CUDA_TRY(cudaGetLastError());
    m->packed = true;
    return RSI_OK;
}

void feature_map(rsi_bvh_t h, float lo[3], float sc[3]) {
    for (int a = 0; a < 3; ++a) {
        lo[a] = h->lo[a];
        sc[a] = h->hi[a] > h->lo[a] ? 2.0f / (h->hi[a] - h->lo[a]) : 0.0f;
    }
}

// Launch of the tensor-core kernel: one CTA per SM (or per pair of tiles).
template <bool VERIFY>
int launch_tc(const TcArgs& P, int64_t n, cudaStream_t s) {
    // set on every launch: the attribute belongs to the current device's context
    RSI_CUDA_TRY(cudaFuncSetAttribute(k_mlp_tc<VERIFY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kSmBytes + 1024));
    const int64_t tiles = (n + 127) / 128;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + 1) / 2, (int64_t)device_sm_count()));
    k_mlp_tc<VERIFY><<<grid, kTcThreads, kSmBytes + 1024, s>>>(P);
    note_launches(1);
    RSI_CUDA_TRY(cudaGetLastError());
    return RSI_OK;
}

TcArgs tc_args(rsi_mlp_s* m, rsi_bvh_t h, const float* from, const float* to, int64_t n) {
    TcArgs P{};
    P.img = m->img;
    P.bias = m->bias;
    P.from = from;
    P.to = to;
    P.n = (int)n;
    float lo[3], sc[3];
    feature_map(h, lo, sc);
    P.lo0 = lo[0];
    P.lo1 = lo[1];
    P.lo2 = lo[2];
    P.sc0 = sc[0];
    P.sc1 = sc[1];
    P.sc2 = sc[2];
    return P;
}

int forward_tc(rsi_mlp_s* m, rsi_bvh_t h, const float* from, const float* to, int64_t n, float* logits,
               uint8_t* top4, cudaStream_t s) {
    int rc = ensure_packed(m, s);
    if (rc) return rc;
    RSI_CUDA_TRY(cudaMemsetAsync(m->scratch_i, 0, 2 * sizeof(int), s));
    TcArgs P = tc_args(m, h, from, to, n);
    P.logits = logits;
    P.top4 = top4;
    P.err = m->scratch_i + 1;
    return launch_tc<false>(P, n, s);
}

int propose_verify(rsi_mlp_s* m, rsi_bvh_t h, const float* from, const float* to, int64_t n, uint8_t* hit,
                   uint8_t* amb, int32_t* order, DevCounters* ctr, int stats, cudaStream_t s) {
    int rc = ensure_packed(m, s);
    if (rc) return rc;
    TcArgs P = tc_args(m, h, from, to, n);
    P.err = &ctr->error;
    P.tris = h->tris;
    P.n_tri = (int)h->n_tri;
    P.cluster_max = (int)((h->n_tri + 255) / 256);
    P.dmax0 = h->dmax[0];
    P.dmax1 = h->dmax[1];
    P.dmax2 = h->dmax[2];
    P.hit = hit;
    P.amb = amb;
    P.order = order;
    P.ctr = ctr;
    P.stats = stats;
    return launch_tc<true>(P, n, s);
}

// C = op(A) op(B).  A long reduction (the batch, for weight gradients) is
// split into chunks of 512 accumulated atomically so the grid fills the GPU.
template <bool TA, bool TB>
int gemm(const float* A, const float* B, float* C, int M, int N, int K, int lda, int ldb, int ldc, cudaStream_t s) {
    const int chunks = K >= 2048 ? (K + 511) / 512 : 1;
    if (chunks > 1) RSI_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * ldc, s));
    dim3 grid((N + 63) / 64, (M + 63) / 64, chunks);
    k_gemm<TA, TB><<<grid, 256, 0, s>>>(A, B, C, M, N, K, lda, ldb, ldc, chunks > 1 ? 512 : K);
    note_launches(1);
    return RSI_OK;
}

int colsum(const float* d, int rows, int cols, float* g, cudaStream_t s) {
    RSI_CUDA_TRY(cudaMemsetAsync(g, 0, sizeof(float) * cols, s));
    k_colsum<<<(rows + 255) / 256, cols, 0, s>>>(d, rows, cols, g);
    note_launches(1);
    return RSI_OK;
}

// One training step on a batch of n <= 65536 segments: forward with the
// BF16 roundings of the inference kernel, mean BCE, backward (roundings as
// identity), gradients into m->grads, then Adam when `apply`.
int train_step(rsi_mlp_s* m, rsi_bvh_t h, const float* from, const float* to, const uint32_t* labels, int n, float lr,
               int apply, float* h_loss, cudaStream_t s) {
    const int64_t need = (int64_t)n * (kIn + 4 * kH + kOut + kH) + kW1 + kW2 + kW3 + 1;
    if (m->act_cap < need) {
        if (m->act) {
            RSI_CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(m->act);
            m->act = nullptr;
            m->act_cap = 0;
        }
        if (rsi::dev_malloc(&m->act, sizeof(float) * need) != cudaSuccess) {
            cudaGetLastError();
            return fail(RSI_ERR_OOM, "rsi_mlp_train_step: activation buffers");
        }
        m->act_cap = need;
    }
    float* x = m->act;                     // [n][16]
    float* z1 = x + (int64_t)n * kIn;      // [n][128]
    float* a1 = z1 + (int64_t)n * kH;
    float* z2 = a1 + (int64_t)n * kH;
    float* a2 = z2 + (int64_t)n * kH;
    float* z3 = a2 + (int64_t)n * kH;      // [n][256], then dz3
    float* da = z3 + (int64_t)n * kOut;    // [n][128]
    float* wb = da + (int64_t)n * kH;      // BF16-rounded W1 | W2 | W3
    float* loss = wb + kW1 + kW2 + kW3;
    float *W1b = wb, *W2b = wb + kW1, *W3b = wb + kW1 + kW2;
    float* g = m->grads;
    float lo[3], sc[3];
    feature_map(h, lo, sc);
    k_round_weights<<<grid_for(kW1 + kW2 + kW3, 256), 256, 0, s>>>(m->params, wb);
    k_train_features<<<grid_for(n, 256), 256, 0, s>>>(from, to, n, lo[0], lo[1], lo[2], sc[0], sc[1], sc[2], x);
    note_launches(2);
    gemm<false, false>(x, W1b, z1, n, kH, kIn, kIn, kH, kH, s);
    k_bias_gelu<<<grid_for((int64_t)n * kH, 256), 256, 0, s>>>(z1, m->params + kOffB1, a1, n, kH);
    gemm<false, false>(a1, W2b, z2, n, kH, kH, kH, kH, kH, s);
    k_bias_gelu<<<grid_for((int64_t)n * kH, 256), 256, 0, s>>>(z2, m->params + kOffB2, a2, n, kH);
    gemm<false, false>(a2, W3b, z3, n, kOut, kH, kH, kOut, kOut, s);
    RSI_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), s));
    k_bce<<<grid_for((int64_t)n * kOut, 256), 256, 0, s>>>(z3, m->params + kOffB3, labels, n, loss);
    note_launches(3);
    // backward: z3 now holds dz3
    gemm<true, false>(a2, z3, g + kOffW3, kH, kOut, n, kH, kOut, kOut, s);          // a2^T dz3
    colsum(z3, n, kOut, g + kOffB3, s);
    gemm<false, true>(z3, W3b, da, n, kH, kOut, kOut, kOut, kH, s);                 // dz3 W3^T
    k_gelu_back<<<grid_for((int64_t)n * kH, 256), 256, 0, s>>>(da, z2, z2, (int64_t)n * kH);   // z2 <- dz2
    gemm<true, false>(a1, z2, g + kOffW2, kH, kH, n, kH, kH, kH, s);                // a1^T dz2
    colsum(z2, n, kH, g + kOffB2, s);
    gemm<false, true>(z2, W2b, da, n, kH, kH, kH, kH, kH, s);                       // dz2 W2^T
    k_gelu_back<<<grid_for((int64_t)n * kH, 256), 256, 0, s>>>(da, z1, z1, (int64_t)n * kH);   // z1 <- dz1
    gemm<true, false>(x, z1, g + kOffW1, kIn, kH, n, kIn, kH, kH, s);               // x^T dz1
    colsum(z1, n, kH, g + kOffB1, s);
    note_launches(2);
    if (apply) {
        ++m->step;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.0f - std::pow(b1, (float)m->step), c2 = 1.0f - std::pow(b2, (float)m->step);
        k_adam<<<grid_for(kParams, 256), 256, 0, s>>>(m->params, g, m->adam_m, m->adam_v, kParams, lr, b1, b2, 1e-8f,
                                                       c1, c2);
        note_launches(1);
        m->packed = false;
    }
    RSI_CUDA_TRY(cudaGetLastError());
    if (h_loss) {
        float l = 0.0f;
        RSI_CUDA_TRY(cudaMemcpyAsync(&l, loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        RSI_CUDA_TRY(cudaStreamSynchronize(s));
        *h_loss = l / ((float)n * kOut);
    }
    return RSI_OK;
}

// He-style initial weights from a counter-based generator (splitmix64 +
// Box-Muller), so a seed gives the same network on any host.
uint64_t splitmix(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double gauss(uint64_t& st) {
    double u1 = ((splitmix(st) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    double u2 = (splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace mlpk
}  // namespace rsi

using namespace rsi::mlpk;

extern "C" int rsi_mlp_create(uint64_t seed, rsi_mlp_t* out) {
    if (!out) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_mlp_create: out is NULL");
    *out = nullptr;
    auto* m = new rsi_mlp_s();
    const size_t pb = sizeof(float) * kParams;
    char* base = nullptr;
    if (rsi::dev_malloc(&base, 4 * pb + kImgBytes + 512 * 4 + 256) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return rsi::fail(RSI_ERR_OOM, "rsi_mlp_create: allocation failed");
    }
    m->params = reinterpret_cast<float*>(base);
    m->grads = reinterpret_cast<float*>(base + pb);
    m->adam_m = reinterpret_cast<float*>(base + 2 * pb);
    m->adam_v = reinterpret_cast<float*>(base + 3 * pb);
    m->img = reinterpret_cast<uint8_t*>(base + 4 * pb);
    m->bias = reinterpret_cast<float*>(base + 4 * pb + kImgBytes);
    m->scratch_i = reinterpret_cast<int*>(base + 4 * pb + kImgBytes + 512 * 4);
    std::vector<float> p(kParams, 0.0f);
    uint64_t st = seed * 0x2545F4914F6CDD1Dull + 0x4D4C50ull;
    for (int k = 0; k < 6; ++k)
        for (int n = 0; n < kH; ++n) p[kOffW1 + k * kH + n] = (float)(gauss(st) * std::sqrt(2.0 / 6.0));
    for (int i = 0; i < kW2; ++i) p[kOffW2 + i] = (float)(gauss(st) * std::sqrt(2.0 / kH));
    for (int i = 0; i < kW3; ++i) p[kOffW3 + i] = (float)(gauss(st) * std::sqrt(1.0 / kH));
    cudaError_t e = cudaMemcpy(m->params, p.data(), pb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->adam_m, 0, 2 * pb);
    if (e == cudaSuccess) e = cudaMemset(m->img, 0, kImgBytes);
    if (e != cudaSuccess) {
        cudaFree(base);
        delete m;
        return rsi::cuda_fail(e, "rsi_mlp_create");
    }
    *out = m;
    return RSI_OK;
}

extern "C" int rsi_mlp_free(rsi_mlp_t m) {
    if (!m) return RSI_OK;
    cudaDeviceSynchronize();
    rsi::forget_mlp(m);
    cudaFree(m->params);
    if (m->act) cudaFree(m->act);
    delete m;
    return RSI_OK;
}

extern "C" int rsi_mlp_num_params(void) { return kParams; }

extern "C" int rsi_mlp_attach(rsi_bvh_t h, rsi_mlp_t m) {
    if (!h) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_mlp_attach: NULL hierarchy");
    rsi::attach_mlp(h, m);
    return RSI_OK;
}

extern "C" int rsi_mlp_set_params(rsi_mlp_t m, const float* h_params, void* stream) {
    if (!m || !h_params) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_mlp_set_params: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    RSI_CUDA_TRY(cudaMemcpyAsync(m->params, h_params, sizeof(float) * kParams, cudaMemcpyHostToDevice, s));
    RSI_CUDA_TRY(cudaStreamSynchronize(s));
    m->packed = false;
    return RSI_OK;
}

extern "C" int rsi_mlp_get_params(rsi_mlp_t m, float* h_params, float* h_grads, void* stream) {
    if (!m) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_mlp_get_params: NULL handle");
    cudaStream_t s = (cudaStream_t)stream;
    if (h_params) RSI_CUDA_TRY(cudaMemcpyAsync(h_params, m->params, sizeof(float) * kParams, cudaMemcpyDeviceToHost, s));
    if (h_grads) RSI_CUDA_TRY(cudaMemcpyAsync(h_grads, m->grads, sizeof(float) * kParams, cudaMemcpyDeviceToHost, s));
    RSI_CUDA_TRY(cudaStreamSynchronize(s));
    return RSI_OK;
}

extern "C" int rsi_mlp_forward(rsi_mlp_t m, rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n,
                               float* d_logits, uint8_t* d_top4, void* stream) {
    if (!m || !h || n < 0 || n > 0x7FFFFF00ll || (n > 0 && (!d_from || !d_to)))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_mlp_forward: bad arguments");
    if (n == 0) return RSI_OK;
    return forward_tc(m, h, d_from, d_to, n, d_logits, d_top4, (cudaStream_t)stream);
}

extern "C" int rsi_mlp_status(rsi_mlp_t m, void* stream) {
    if (!m) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_mlp_status: NULL handle");
    int v[2] = {0, 0};
    RSI_CUDA_TRY(cudaMemcpyAsync(v, m->scratch_i, sizeof v, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    RSI_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (v[1]) return rsi::fail(v[1], "rsi_mlp: a tensor-core wait ran out");
    return RSI_OK;
}

extern "C" int rsi_mlp_train_step(rsi_mlp_t m, rsi_bvh_t h, const float* d_from, const float* d_to,
                                  const uint32_t* d_labels, int64_t n, float lr, int apply, float* h_loss,
                                  void* stream) {
    if (!m || !h || !d_from || !d_to || !d_labels || n < 1 || n > 65536)
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_mlp_train_step: need 1 <= n <= 65536 and all buffers");
    return train_step(m, h, d_from, d_to, d_labels, (int)n, lr, apply, h_loss, (cudaStream_t)stream);
}

extern "C" int rsi_mlp_reset_optimizer(rsi_mlp_t m, void* stream) {
    if (!m) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_mlp_reset_optimizer: NULL handle");
    RSI_CUDA_TRY(cudaMemsetAsync(m->adam_m, 0, 2 * sizeof(float) * kParams, (cudaStream_t)stream));
    m->step = 0;
    return RSI_OK;
}

extern "C" int rsi_mlp_activation(const float* d_z, int64_t n, float* d_tanh, float* d_tanh_cuda, float* d_gelu,
                                  void* stream) {
    if (n < 0 || (n > 0 && (!d_z || !d_tanh || !d_tanh_cuda || !d_gelu)))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_mlp_activation: bad arguments");
    if (n == 0) return RSI_OK;
    k_activation<<<rsi::grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(d_z, n, d_tanh, d_tanh_cuda, d_gelu);
    rsi::note_launches(1);
    RSI_CUDA_TRY(cudaGetLastError());
    return RSI_OK;
}
