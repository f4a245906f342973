// autotune.cu -- picks the launch shape of the traversal (threads per block,
// resident blocks per SM), the node width it fetches (child-pair,
// compressed child-pair or four-wide) and the in-tile segment reordering of
// a query by timing candidates on a sample of its own segments with CUDA
// events, and reports the traversal stack the tree needs (the smallest of
// 32 / 64 / 128 entries that holds the chosen walk's worst case).  For
// batched plans it also times the stack size (that bucket or the next).
// Choices are cached in a JSON file keyed by device, mode and the sizes of
// the problem (log2 buckets).
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
    int block = 256, bps = 4, tile = 0, stack = 32, width = 2;
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
// "ray_sort_tile": T, "stack": K, "node_width": W, "ms": M},
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
    char buf[200];
    std::snprintf(buf, sizeof buf,
                  "{\"block\": %d, \"blocks_per_sm\": %d, \"ray_sort_tile\": %d, \"stack\": %d, \"node_width\": %d, "
                  "\"ms\": %.4f}",
                  c.block, c.bps, c.tile, c.stack, c.width, c.ms);
    return buf;
}

}  // namespace

extern "C" int rsi_autotune(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays, int mode,
                            const char* cache_path, rsi_options* inout, rsi_tuning* result, void* stream) {
    if (!h || !inout || !d_from || !d_to || n_rays < 1 || (mode != RSI_ANY_HIT && mode != RSI_COUNT))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_autotune: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    Choice best;
    // stack entries of the walk: one per level (child-pair), three per
    // four-wide level; the four-wide walk needs <= 128 (tree height <= 82)
    auto stack_for = [&](int width) {
        const int need = width == 4 ? 3 * ((h->height + 2) / 2) : h->height + 1;
        return need <= 32 ? 32 : (need <= 64 ? 64 : 128);
    };
    const bool wide_ok = 3 * ((h->height + 2) / 2) <= 128;
    const std::string key = tuning_key(mode, h->n_tri, n_rays);
    auto cache = read_cache(cache_path);
    auto it = cache.find(key);
    int candidates = 0, from_cache = 0;
    if (it != cache.end()) {
        best.block = field(it->second, "block", 256);
        best.bps = field(it->second, "blocks_per_sm", 4);
        best.tile = field(it->second, "ray_sort_tile", 0);
        best.width = field(it->second, "node_width", 2);
        if (best.width == 4 && !wide_ok) best.width = 2;
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
        const int widths[] = {2, 3, 4};
        float best_ms = INFINITY;
        int rc = RSI_OK;
        for (const auto& sh : shapes) {
            for (int c = 0; c < 9; ++c) {
                const int tile = tiles[c % 3], width = widths[c / 3];
                if (width == 4 && !wide_ok) continue;
                rsi_options o = *inout;
                o.block = sh[0];
                o.blocks_per_sm = sh[1];
                o.ray_sort_tile = tile;
                o.node_width = width;
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
                    best.width = width;
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
        best.stack = stack_for(best.width);
        cache[key] = encode(best);
        if (!write_cache(cache_path, cache)) return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_autotune: cannot write cache");
    }
    inout->block = best.block;
    inout->blocks_per_sm = best.bps;
    inout->ray_sort_tile = best.tile;
    inout->node_width = best.width;
    best.stack = stack_for(best.width);
    inout->stack = best.stack;
    if (result) {
        result->block = best.block;
        result->blocks_per_sm = best.bps;
        result->ray_sort_tile = best.tile;
        result->stack = best.stack;
        result->ms = best.ms;
        result->from_cache = from_cache;
        result->candidates = candidates;
        result->node_width = best.width;
    }
    return RSI_OK;
}

// ---------------------------------------------------------------- batched plans
extern "C" int rsi_batch_autotune(const rsi_ray_batch* batches, int n_batches, int mode, const char* cache_path,
                                  rsi_options* inout, rsi_tuning* result, void* stream) {
    if (!batches || n_batches < 1 || !inout || (mode != RSI_ANY_HIT && mode != RSI_COUNT))
        return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_autotune: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t tri = 0, rays = 0;
    int height = 0;
    for (int i = 0; i < n_batches; ++i) {
        if (!batches[i].bvh || batches[i].n_rays < 0)
            return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_autotune: batch " + std::to_string(i) + " is malformed");
        tri += batches[i].bvh->n_tri;
        rays += batches[i].n_rays;
        height = std::max(height, batches[i].bvh->height);
    }
    auto stack_need = [&](int width) { return width == 4 ? 3 * ((height + 2) / 2) : height + 1; };
    auto bucket = [](int need) { return need <= 32 ? 32 : (need <= 64 ? 64 : 128); };
    const bool wide_ok = 3 * ((height + 2) / 2) <= 128;
    std::ostringstream kk;
    kk << tuning_key(mode, tri, rays) << "|batched" << n_batches;
    const std::string key = kk.str();
    auto cache = read_cache(cache_path);
    auto it = cache.find(key);
    Choice best;
    best.bps = 3;
    int candidates = 0, from_cache = 0;
    if (it != cache.end()) {
        best.block = field(it->second, "block", 256);
        best.bps = field(it->second, "blocks_per_sm", 3);
        best.tile = field(it->second, "ray_sort_tile", 0);
        best.width = field(it->second, "node_width", 2);
        best.stack = field(it->second, "stack", 0);
        if (best.width == 4 && !wide_ok) best.width = 2;
        if (best.stack < bucket(stack_need(best.width))) best.stack = bucket(stack_need(best.width));
        from_cache = 1;
    } else {
        // a sample plan: every batch cut to its first 2^17 segments, outputs in scratch
        const int64_t cut = (int64_t)1 << 17;
        std::vector<rsi_ray_batch> sample(batches, batches + n_batches);
        int64_t total = 0;
        for (auto& b : sample) {
            b.n_rays = std::min<int64_t>(b.n_rays, cut);
            total += b.n_rays;
        }
        // outputs: hit bytes, ambiguity bytes, then the int32 counts from a
        // 256-byte boundary (2 * total bytes need not be a multiple of 4)
        char* out = nullptr;
        const size_t count_off = ((size_t)2 * (size_t)total + 255) & ~(size_t)255;
        if (rsi::dev_malloc(&out, count_off + 4 * (size_t)std::max<int64_t>(total, 1)) != cudaSuccess) {
            cudaGetLastError();
            return rsi::fail(RSI_ERR_OOM, "rsi_batch_autotune: sample outputs");
        }
        int64_t off = 0;
        for (auto& b : sample) {
            b.d_hit = reinterpret_cast<uint8_t*>(out) + off;
            b.d_ambiguous = reinterpret_cast<uint8_t*>(out) + total + off;
            b.d_count = reinterpret_cast<int32_t*>(out + count_off) + off;
            off += b.n_rays;
        }
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const int shapes[][2] = {{256, 3}, {256, 2}, {256, 4}, {128, 6}, {128, 8}};
        const int widths[] = {2, 4};
        const int tiles[] = {0, 8192};
        float best_ms = INFINITY;
        int rc = RSI_OK;
        for (const auto& sh : shapes) {
            for (int width : widths) {
                if (width == 4 && !wide_ok) continue;
                const int st0 = bucket(stack_need(width));
                for (int stack : {st0, std::min(2 * st0, 128)}) {
                    if (stack != st0 && st0 == 128) continue;
                    for (int tile : tiles) {
                        rsi_options o = *inout;
                        o.block = sh[0];
                        o.blocks_per_sm = sh[1];
                        o.node_width = width;
                        o.ray_sort_tile = tile;
                        o.stack = stack;
                        o.timeout_ns = 0;
                        o.collect_stats = 0;
                        rsi_batch_t plan = nullptr;
                        rc = rsi_batch_create(sample.data(), n_batches, mode, &o, stream, &plan);
                        if (rc != RSI_OK) break;
                        float total_ms = 0.0f;
                        for (int rep = 0; rep < 4 && rc == RSI_OK; ++rep) {
                            cudaEventRecord(e0, s);
                            rc = rsi_batch_launch(plan, stream);
                            cudaEventRecord(e1, s);
                            cudaEventSynchronize(e1);
                            float ms = 0.0f;
                            cudaEventElapsedTime(&ms, e0, e1);
                            if (rep > 0) total_ms += ms;   // the first launch warms up
                        }
                        rsi_batch_free(plan);
                        if (rc != RSI_OK) break;
                        ++candidates;
                        const float ms = total_ms / 3.0f;
                        if (ms < best_ms) {
                            best_ms = ms;
                            best.block = sh[0];
                            best.bps = sh[1];
                            best.width = width;
                            best.tile = tile;
                            best.stack = stack;
                            best.ms = ms;
                        }
                    }
                    if (rc != RSI_OK) break;
                }
                if (rc != RSI_OK) break;
            }
            if (rc != RSI_OK) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(out);
        if (rc != RSI_OK) return rc;
        cache[key] = encode(best);
        if (!write_cache(cache_path, cache))
            return rsi::fail(RSI_ERR_INVALID_ARG, "rsi_batch_autotune: cannot write cache");
    }
    inout->block = best.block;
    inout->blocks_per_sm = best.bps;
    inout->ray_sort_tile = best.tile;
    inout->node_width = best.width;
    inout->stack = best.stack;
    if (result) {
        result->block = best.block;
        result->blocks_per_sm = best.bps;
        result->ray_sort_tile = best.tile;
        result->stack = best.stack;
        result->ms = best.ms;
        result->from_cache = from_cache;
        result->candidates = candidates;
        result->node_width = best.width;
    }
    return RSI_OK;
}
