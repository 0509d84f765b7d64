// Device and pinned-host allocations of the library, through one registry:
// every live allocation is counted (lbm_debug_alloc_stats), and the
// LBM_DEBUG_FAIL_ALLOC environment variable makes allocations fail on the
// host, without touching the GPU, so that the tests can check every error
// path of lbm_create, lbm_batch_create and the tape for leaks.
//
// In the bounds-checked build (-DLBM_CHECKED) each device allocation also
// carries a canary past its end (lbm_debug_check_canaries).
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
// LBM_CHECKED builds: every device allocation carries kCanary bytes of a
// known pattern past its end; lbm_debug_check_canaries reads them back
#ifdef LBM_CHECKED
constexpr size_t kCanary = 256;
constexpr unsigned char kCanaryByte = 0xA5;
std::unordered_map<void *, size_t> g_size;   // device pointer -> requested bytes
#endif
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
#ifdef LBM_CHECKED
    cudaError_t e = cudaMalloc(p, bytes + kCanary);
    if (e == cudaSuccess && *p) {
        e = cudaMemset((unsigned char *)*p + bytes, kCanaryByte, kCanary);
        if (e != cudaSuccess) {
            cudaFree(*p);
            *p = nullptr;
            return e;
        }
        g_size[*p] = bytes;
    }
#else
    cudaError_t e = cudaMalloc(p, bytes);
#endif
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
#ifdef LBM_CHECKED
        g_size.erase(p);
#endif
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

extern "C" lbm_status lbm_debug_check_canaries(long long *damaged) {
    if (!damaged) return LBM_E_INVALID;
#ifdef LBM_CHECKED
    std::lock_guard<std::mutex> lock(lbm::g_mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return LBM_E_CUDA;
    long long bad = 0;
    unsigned char buf[lbm::kCanary];
    for (const auto &kv : lbm::g_size) {
        if (cudaMemcpy(buf, (unsigned char *)kv.first + kv.second, lbm::kCanary, cudaMemcpyDeviceToHost) != cudaSuccess)
            return LBM_E_CUDA;
        for (size_t i = 0; i < lbm::kCanary; ++i)
            if (buf[i] != lbm::kCanaryByte) {
                ++bad;
                break;
            }
    }
    *damaged = bad;
#else
    *damaged = -1;   // no canaries in this build
#endif
    return LBM_OK;
}

extern "C" lbm_status lbm_debug_alloc_stats(long long *live_device, long long *live_host) {
    if (!live_device || !live_host) return LBM_E_INVALID;
    std::lock_guard<std::mutex> lock(lbm::g_mu);
    *live_device = lbm::g_live_dev;
    *live_host = lbm::g_live_host;
    return LBM_OK;
}
