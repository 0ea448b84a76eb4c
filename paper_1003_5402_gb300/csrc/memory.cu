// Process-wide memory caches behind every plan context.
//
// Device memory: one stream-ordered pool per device (cudaMemPoolCreate) whose
// release threshold keeps the memory of destroyed contexts mapped for the next
// one, so that creating and destroying plans in a long-lived process (a
// server, a batch of re-plans) costs sub-allocations instead of cudaMalloc /
// cudaFree, which map and unmap pages and synchronise the device.
//
// Pinned host memory: a small free list of page-locked blocks.  A context
// needs well under a megabyte of it (read-back staging), but cudaMallocHost
// and cudaFreeHost each take a few hundred microseconds.
#include <algorithm>
#include <mutex>
#include <vector>

#include "dao_internal.h"

namespace dao {

namespace {

std::mutex g_mu;
std::vector<cudaMemPool_t> g_pools;          // per device, created on first use

struct PinnedBlock {
    void* p;
    size_t bytes;
};
std::vector<PinnedBlock> g_pinned_free;      // cached page-locked blocks
size_t g_pinned_cached = 0;
constexpr size_t PINNED_CACHE_MAX = 64u << 20;

cudaError_t pool_for(int device, cudaMemPool_t* out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_pools.size() <= device) g_pools.resize(device + 1, nullptr);
    if (g_pools[device] == nullptr) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool = nullptr;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        size_t free_b = 0, total_b = 0;
        e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        cuuint64_t keep = std::min<cuuint64_t>(POOL_KEEP_MAX, total_b / 16);
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pools[device] = pool;
    }
    *out = g_pools[device];
    return cudaSuccess;
}

}  // namespace

cudaError_t pool_alloc(void** p, size_t bytes, int device, cudaStream_t s) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = pool_for(device, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), pool, s);
}

cudaError_t pool_free(void* p, cudaStream_t s) { return p ? cudaFreeAsync(p, s) : cudaSuccess; }

cudaError_t pinned_alloc(void** p, size_t* bytes_io) {
    const size_t bytes = *bytes_io;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        // smallest cached block that is large enough
        int best = -1;
        for (int i = 0; i < (int)g_pinned_free.size(); ++i)
            if (g_pinned_free[i].bytes >= bytes && (best < 0 || g_pinned_free[i].bytes < g_pinned_free[best].bytes))
                best = i;
        if (best >= 0) {
            *p = g_pinned_free[best].p;
            *bytes_io = g_pinned_free[best].bytes;
            g_pinned_cached -= g_pinned_free[best].bytes;
            g_pinned_free.erase(g_pinned_free.begin() + best);
            return cudaSuccess;
        }
    }
    return cudaMallocHost(p, bytes);
}

void pinned_release(void* p, size_t bytes) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_pinned_cached + bytes <= PINNED_CACHE_MAX) {
            g_pinned_free.push_back({p, bytes});
            g_pinned_cached += bytes;
            return;
        }
    }
    cudaFreeHost(p);
}

cudaError_t release_cached_memory(int device) {
    std::vector<PinnedBlock> blocks;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        blocks.swap(g_pinned_free);
        g_pinned_cached = 0;
        if (device >= 0 && device < (int)g_pools.size()) pool = g_pools[device];
    }
    for (const PinnedBlock& b : blocks) cudaFreeHost(b.p);
    return pool ? cudaMemPoolTrimTo(pool, 0) : cudaSuccess;
}

}  // namespace dao
