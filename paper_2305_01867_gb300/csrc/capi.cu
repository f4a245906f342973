// capi.cu -- error reporting and device queries behind the C ABI.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "rsi_internal.cuh"

namespace rsi {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return RSI_ERR_CUDA;
}

static std::atomic<unsigned long long> g_launches{0};

void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

static std::mutex g_ctx_mu;
static DeviceCtx* g_ctx[kMaxCtxDevices] = {};

DeviceCtx* device_ctx() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxCtxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_ctx_mu);
    if (!g_ctx[dev]) {
        auto* c = new DeviceCtx();
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return nullptr;
        }
        uint64_t keep = 4ull << 30;   // up to 4 GiB of freed blocks stay cached for later handles
        cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_ctx[dev] = c;
    }
    return g_ctx[dev];
}

// Allocations left before injected failures start; -1 = no injection.
static std::atomic<long long> g_alloc_left{-1};

bool alloc_injected() {
    long long v = g_alloc_left.load(std::memory_order_relaxed);
    while (v > 0 && !g_alloc_left.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) {
    }
    return v == 0;
}

int pool_alloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (alloc_injected())
        return fail(RSI_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected)");
    DeviceCtx* c = device_ctx();
    if (!c) return fail(RSI_ERR_CUDA, "no CUDA device context");
    if (cudaMallocFromPoolAsync(p, bytes, c->pool, s) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(RSI_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return RSI_OK;
}

void pool_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

static std::atomic<uint64_t> g_gen{0};

uint64_t next_handle_gen() { return ++g_gen; }

static std::mutex g_attach_mu;
static std::vector<std::pair<rsi_bvh_t, rsi_mlp_s*>> g_attach;   // (hierarchy, network)

void attach_mlp(rsi_bvh_t h, rsi_mlp_s* m) {
    std::lock_guard<std::mutex> lock(g_attach_mu);
    for (size_t i = 0; i < g_attach.size(); ++i) {
        if (g_attach[i].first == h) {
            g_attach.erase(g_attach.begin() + (long)i);
            break;
        }
    }
    h->mlp = m;
    if (m) g_attach.emplace_back(h, m);
}

void forget_handle(rsi_bvh_t h) {
    {
        std::lock_guard<std::mutex> lock(g_attach_mu);
        for (size_t i = 0; i < g_attach.size(); ++i) {
            if (g_attach[i].first == h) {
                g_attach.erase(g_attach.begin() + (long)i);
                break;
            }
        }
        h->mlp = nullptr;
    }
    drop_plans_of(h->gen);
}

void forget_mlp(rsi_mlp_s* m) {
    std::lock_guard<std::mutex> lock(g_attach_mu);
    for (size_t i = 0; i < g_attach.size();) {
        if (g_attach[i].second == m) {
            g_attach[i].first->mlp = nullptr;
            g_attach.erase(g_attach.begin() + (long)i);
        } else {
            ++i;
        }
    }
}

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace rsi

extern "C" const char* rsi_last_error(void) { return rsi::g_last_error.c_str(); }

extern "C" uint64_t rsi_kernel_launches(void) { return rsi::g_launches.load(); }

extern "C" int rsi_debug_fail_allocations(int64_t after) {
    rsi::g_alloc_left.store(after < 0 ? -1 : (long long)after);
    return RSI_OK;
}
