// grbk_alloc.cu -- device blocks for contexts.
//
// A context holds a few GB of device buffers (A, B, C, R, A A^T, the split
// planes).  cudaMalloc and cudaFree of GB-sized blocks cost milliseconds and
// cudaFree synchronises the device, which dominates a create / solve / destroy
// cycle on the host's data.  Blocks freed here are kept, per device and rounded
// size, and handed to the next request of the same size; a cudaMalloc that
// fails releases every kept block and retries.  At most kCacheCap bytes are
// kept; beyond that a freed block goes back to the driver.
#include <cuda_runtime.h>
#include <stddef.h>
#include <map>
#include <mutex>
#include <unordered_map>
#include <utility>

#include "grbk_internal.cuh"

namespace grbk {

namespace {  // the cache's state

struct Block {
    size_t bytes;
    int dev;
};

std::mutex g_mu;
std::unordered_map<void*, Block> g_live;             // handed out
std::multimap<std::pair<int, size_t>, void*> g_kept;  // (device, bytes) -> block
size_t g_kept_bytes = 0;
constexpr size_t kCacheCap = size_t(64) << 30;

size_t rounded(size_t b)
{
    const size_t g = b > (size_t(1) << 20) ? (size_t(2) << 20) : 256;
    return (b + g - 1) / g * g;
}

void free_on(int dev, void* p)
{
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    cudaFree(p);
    if (cur != dev) cudaSetDevice(cur);
}

void release_kept_locked()
{
    for (auto& kv : g_kept) free_on(kv.first.first, kv.second);
    g_kept.clear();
    g_kept_bytes = 0;
}

}  // namespace

cudaError_t dev_alloc(void** p, size_t bytes)
{
    *p = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t r = rounded(bytes > 0 ? bytes : 1);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_kept.find({dev, r});
        if (it != g_kept.end()) {
            *p = it->second;
            g_kept.erase(it);
            g_kept_bytes -= r;
            g_live[*p] = {r, dev};
            return cudaSuccess;
        }
    }
    e = cudaMalloc(p, r);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        {
            std::lock_guard<std::mutex> lk(g_mu);
            release_kept_locked();
        }
        e = cudaMalloc(p, r);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_live[*p] = {r, dev};
    return cudaSuccess;
}

void dev_free(void* p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_live.find(p);
    if (it == g_live.end()) {  // not from dev_alloc
        cudaFree(p);
        return;
    }
    const Block b = it->second;
    g_live.erase(it);
    if (g_kept_bytes + b.bytes > kCacheCap) {
        free_on(b.dev, p);
        return;
    }
    g_kept.insert({{b.dev, b.bytes}, p});
    g_kept_bytes += b.bytes;
}

}  // namespace grbk

extern "C" void grbk_trim_cache(void)
{
    std::lock_guard<std::mutex> lk(grbk::g_mu);
    grbk::release_kept_locked();
}
