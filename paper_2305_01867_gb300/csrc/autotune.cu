// autotune.cu -- picks the launch shape of the traversal (threads per block,
// resident blocks per SM) and the in-tile segment reordering of a query by
// timing candidates on a sample of its own segments with CUDA events, and
// reports the traversal stack the tree needs (the smallest of 32 / 64 / 128
// entries above the tree height).  Choices are cached in a JSON file keyed
// by device, mode and the sizes of the problem (log2 buckets).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "rsi_internal.cuh"

namespace {

struct Choice {
    int block = 256, bps = 4, tile = 0, stack = 32;
    float ms = 0.0f;
};

int log2_bucket(int64_t x) {
    int b = 0;
    while (x > 1) {
        x >>= 1;
        ++b;
    }
    return b;
}

std::string tuning_key(int mode, int64_t n_tri, int64_t n_rays) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    std::string name = "unknown";
    int sms = 0;
    if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) {
        name = p.name;
        sms = p.multiProcessorCount;
    }
    for (char& c : name)
        if (c == '"' || c == '\\') c = '_';
    std::ostringstream k;
    k << name << "|sm" << sms << "|" << (mode == RSI_COUNT ? "count" : "any_hit") << "|t" << log2_bucket(n_tri) << "|r"
      << log2_bucket(n_rays);
    return k.str();
}

// The cache holds one entry per line:  "key": {"block": B, "blocks_per_sm": S,
// "ray_sort_tile": T, "stack": K, "ms": M},
int field(const std::string& line, const char* name, int dflt) {
    std::string pat = std::string("\"") + name + "\":";
    size_t p = line.find(pat);
    if (p == std::string::npos) return dflt;
    return std::atoi(line.c_str() + p + pat.size());
}

std::map<std::string, std::string> read_cache(const char* path) {
    std::map<std::string, std::string> m;
    if (!path || !*path) return m;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        size_t a = line.find('"');
        if (a == std::string::npos) continue;
        size_t b = line.find("\": {", a + 1);
        if (b == std::string::npos) continue;
        m[line.substr(a + 1, b - a - 1)] = line.substr(b + 3);
    }
    return m;
}

bool write_cache(const char* path, const std::map<std::string, std::string>& m) {
    if (!path || !*path) return true;
    std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream f(tmp);
        if (!f) return false;
        f << "{\n";
        size_t i = 0;
        for (const auto& kv : m) {
            std::string v = kv.second;
            while (!v.empty() && (v.back() == ',' || v.back() == ' ' || v.back() == '\r')) v.pop_back();
            f << "  \"" << kv.first << "\": " << v << (++i < m.size() ? ",\n" : "\n");
        }
        f << "}\n";
    }
    return std::rename(tmp.c_str(), path) == 0;
}

std::string encode(const Choice& c) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "{\"block\": %d, \"blocks_per_sm\": %d, \"ray_sort_tile\": %d, \"stack\": %d, \"ms\": %.4f}",
                  c.block, c.bps, c.tile, c.stack, c.ms);
    return buf;
}

}  // namespace

extern "C" int rsi_autotune(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays, int mode,
                            const char* cache_path, rsi_options* inout, rsi_tuning* result, void* stream) {
    if (!h || !inout || !d_from || !d_to || n_rays < 1 || (mode != RSI_ANY_HIT && mode != RSI_COUNT))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_autotune: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    Choice best;
    best.stack = h->height < 32 ? 32 : (h->height < 64 ? 64 : 128);
    const std::string key = tuning_key(mode, h->n_tri, n_rays);
    auto cache = read_cache(cache_path);
    auto it = cache.find(key);
    int candidates = 0, from_cache = 0;
    if (it != cache.end()) {
        best.block = field(it->second, "block", 256);
        best.bps = field(it->second, "blocks_per_sm", 4);
        best.tile = field(it->second, "ray_sort_tile", 0);
        from_cache = 1;
    } else {
        const int64_t n = std::min<int64_t>(n_rays, (int64_t)1 << 21);   // sample: the first 2M segments
        uint8_t* hit = nullptr;
        int32_t* cnt = nullptr;
        if (cudaMallocAsync(&hit, (size_t)n, s) != cudaSuccess ||
            cudaMallocAsync(&cnt, 4 * (size_t)n, s) != cudaSuccess) {
            if (hit) cudaFreeAsync(hit, s);
            cudaGetLastError();
            return rsi::fail(RSI_ERR_OOM, "rsi_autotune: sample buffers");
        }
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const int shapes[][2] = {{256, 4}, {256, 3}, {256, 2}, {128, 8}, {128, 6}, {64, 16}};
        const int tiles[] = {0, 2048, 8192};
        float best_ms = INFINITY;
        int rc = RSI_OK;
        for (const auto& sh : shapes) {
            for (int tile : tiles) {
                rsi_options o = *inout;
                o.block = sh[0];
                o.blocks_per_sm = sh[1];
                o.ray_sort_tile = tile;
                o.time_kernels = 0;
                o.collect_stats = 0;
                float total = 0.0f;
                for (int rep = 0; rep < 4 && rc == RSI_OK; ++rep) {
                    cudaEventRecord(e0, s);
                    rc = rsi_query(h, d_from, d_to, n, mode, &o, hit, mode == RSI_COUNT ? cnt : nullptr, nullptr,
                                   nullptr, stream);
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) total += ms;   // the first run warms up
                }
                if (rc != RSI_OK) break;
                ++candidates;
                const float ms = total / 3.0f;
                if (ms < best_ms) {
                    best_ms = ms;
                    best.block = sh[0];
                    best.bps = sh[1];
                    best.tile = tile;
                    best.ms = ms;
                }
            }
            if (rc != RSI_OK) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFreeAsync(hit, s);
        cudaFreeAsync(cnt, s);
        if (rc != RSI_OK) return rc;
        cache[key] = encode(best);
        if (!write_cache(cache_path, cache)) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_autotune: cannot write cache");
    }
    inout->block = best.block;
    inout->blocks_per_sm = best.bps;
    inout->ray_sort_tile = best.tile;
    if (result) {
        result->block = best.block;
        result->blocks_per_sm = best.bps;
        result->ray_sort_tile = best.tile;
        result->stack = best.stack;
        result->ms = best.ms;
        result->from_cache = from_cache;
        result->candidates = candidates;
    }
    return RSI_OK;
}
