// capi.cu -- error reporting and device queries behind the C ABI.
#include <cuda_runtime.h>

#include <atomic>
#include <string>

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

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace rsi

extern "C" const char* rsi_last_error(void) { return rsi::g_last_error.c_str(); }

extern "C" uint64_t rsi_kernel_launches(void) { return rsi::g_launches.load(); }
