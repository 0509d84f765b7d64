// Device and pinned-host allocations of the library, through one registry:
// every live allocation is counted (lbm_debug_alloc_stats), and the
// LBM_DEBUG_FAIL_ALLOC environment variable makes allocations fail on the
// host, without touching the GPU, so that the tests can check every error
// path of lbm_create, lbm_batch_create and the tape for leaks.
//
// LBM_DEBUG_FAIL_ALLOC=n: once n allocations have succeeded since the
// variable took its current value, every further allocation fails with
// cudaErrorMemoryAllocation (n = 0: all of them).  Unset: no effect.
#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>
#include <string>
#include <unordered_map>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {
namespace {

std::mutex g_mu;
std::unordered_map<void *, bool> g_live;   // pointer -> pinned host (true) or device (false)
long long g_live_dev = 0, g_live_host = 0;
std::string g_fail_value;                  // LBM_DEBUG_FAIL_ALLOC as last seen
long long g_since = 0;                     // allocations since it took that value

// True when the injection says this allocation must fail (g_mu held).
bool inject_failure() {
    const char *v = std::getenv("LBM_DEBUG_FAIL_ALLOC");
    const std::string cur = v ? v : "";
    if (cur != g_fail_value) {
        g_fail_value = cur;
        g_since = 0;
    }
    if (cur.empty()) return false;
    char *end = nullptr;
    const long long n = std::strtoll(cur.c_str(), &end, 10);
    if (end == cur.c_str() || n < 0) return false;
    if (g_since >= n) return true;
    ++g_since;
    return false;
}

}  // namespace

cudaError_t dev_alloc_raw(void **p, size_t bytes) {
    *p = nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    if (inject_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess && *p) {
        g_live[*p] = false;
        ++g_live_dev;
    }
    return e;
}

cudaError_t host_alloc_raw(void **p, size_t bytes) {
    *p = nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    if (inject_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaHostAlloc(p, bytes, cudaHostAllocDefault);
    if (e == cudaSuccess && *p) {
        g_live[*p] = true;
        ++g_live_host;
    }
    return e;
}

void dev_free(void *p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_live.find(p);
        if (it != g_live.end() && !it->second) {
            g_live.erase(it);
            --g_live_dev;
        }
    }
    cudaFree(p);
}

void host_free(void *p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_live.find(p);
        if (it != g_live.end() && it->second) {
            g_live.erase(it);
            --g_live_host;
        }
    }
    cudaFreeHost(p);
}

}  // namespace lbm

extern "C" lbm_status lbm_debug_alloc_stats(long long *live_device, long long *live_host) {
    if (!live_device || !live_host) return LBM_E_INVALID;
    std::lock_guard<std::mutex> lock(lbm::g_mu);
    *live_device = lbm::g_live_dev;
    *live_host = lbm::g_live_host;
    return LBM_OK;
}
