// Device-memory cache of the single-problem API: buffers released by
// acs_problem_destroy (and the scratch of the device build) are kept per
// device, up to a cap, and handed to later allocations of a size they fit,
// so that a create/solve/destroy loop does not pay cudaMalloc and cudaFree
// (each of which synchronises the device) for every buffer.  A block is
// reused for a request of 80-100 % of its size; a cudaMalloc that fails
// releases the cache and retries once.  The cap is ACS_DEVICE_CACHE_MB
// (default 4096); acs_device_cache_trim releases everything.
#include <stdint.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <vector>

#include "acs_internal.cuh"

namespace acs {
namespace {

struct DeviceCache {
    std::multimap<size_t, void*> free;        // size -> block
    size_t cached = 0;
    long long hits = 0, misses = 0;
};

std::mutex g_mu;
std::vector<DeviceCache> g_cache;             // by device ordinal

size_t cache_cap() {
    static const size_t cap = [] {
        const char* e = getenv("ACS_DEVICE_CACHE_MB");
        const long long mb = e ? atoll(e) : 4096;
        return (size_t)(mb > 0 ? mb : 0) << 20;
    }();
    return cap;
}

DeviceCache& cache_of(int device) {
    if ((int)g_cache.size() <= device) g_cache.resize(device + 1);
    return g_cache[device];
}

// every cached block of the device back to the driver (lock held)
void trim_locked(int device) {
    DeviceCache& C = cache_of(device);
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != device) cudaSetDevice(device);
    for (auto& kv : C.free) cudaFree(kv.second);
    C.free.clear();
    C.cached = 0;
    if (cur >= 0 && cur != device) cudaSetDevice(cur);
}

}  // namespace

void* dev_alloc(int device, size_t bytes, size_t* got) {
    const size_t want = ((bytes > 0 ? bytes : 1) + 511) & ~(size_t)511;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        DeviceCache& C = cache_of(device);
        auto it = C.free.lower_bound(want);
        if (it != C.free.end() && it->first - want <= it->first / 5) {
            void* p = it->second;
            *got = it->first;
            C.cached -= it->first;
            C.free.erase(it);
            ++C.hits;
            return p;
        }
        ++C.misses;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        {
            std::lock_guard<std::mutex> lk(g_mu);
            trim_locked(device);
        }
        p = nullptr;
        if (cudaMalloc(&p, want) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
    }
    *got = want;
    return p;
}

void dev_release(int device, void* p, size_t bytes) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceCache& C = cache_of(device);
    if (C.cached + bytes <= cache_cap()) {
        C.free.emplace(bytes, p);
        C.cached += bytes;
    } else {
        cudaFree(p);
    }
}

}  // namespace acs

extern "C" {

int acs_device_cache_trim(int32_t device) {
    std::lock_guard<std::mutex> lk(acs::g_mu);
    if (device >= 0) {
        acs::trim_locked(device);
    } else {
        for (int d = 0; d < (int)acs::g_cache.size(); ++d) acs::trim_locked(d);
    }
    return ACS_SOLVED;
}

int acs_device_cache_stats(int32_t device, int64_t* out3) {
    if (!out3 || device < 0) return ACS_ERR_ARG;
    std::lock_guard<std::mutex> lk(acs::g_mu);
    acs::DeviceCache& C = acs::cache_of(device);
    out3[0] = (int64_t)C.cached;
    out3[1] = C.hits;
    out3[2] = C.misses;
    return ACS_SOLVED;
}

}  // extern "C"
