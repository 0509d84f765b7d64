// lbm_step_noalloc: one time step that allocates nothing.
//
// Some callers cannot call cudaMalloc: a host framework that owns every
// device allocation (a fixed pool it hands out itself), or a latency-critical
// loop where cudaMalloc's implicit device-wide synchronisation is not
// allowed.  This entry point lets them run the two-pass step on buffers they
// already own.  The only device memory it needs beyond the caller's f_in and
// f_out -- the potential field of the step and the error word -- lives in a
// fixed file-scope array of LBM_STATIC_SCRATCH_BYTES that every GPU loading
// the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[LBM_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr size_t kErrBytes = 256;  // error word, padded so the field stays 256-byte aligned

std::mutex g_scratch_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The array's
// name is a host-side stand-in in host code, so its address is looked up
// once per device with that device current.
lbm_status scratch_on_current_device(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_E_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return LBM_E_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LBM_OK;
}

// The step of lbm_step's two-pass form: T is the arithmetic type, TS the
// storage type of f (FP32 lattices: FP32 distributions, FP64 arithmetic and an
// FP64 potential field, as lbm_step computes them).
template <typename TS, typename T>
lbm_status run_step(const lbm_params &p, const lbm::ModelScalars &ms, const void *f_in, void *f_out, void *scratch) {
    using namespace lbm;
    Model<T> m{};
    m.nx = p.nx;
    m.ny = p.ny;
    m.eos = p.eos;
    m.RT = (T)ms.RT;
    m.a = (T)ms.a;
    m.b = (T)ms.b;
    m.aal = (T)ms.aal;
    m.k = (T)ms.k;
    m.omega = (T)(1.0 / p.tau);
    const int radius = p.hdm_radius ? p.hdm_radius : (p.prec == LBM_F64 ? 40 : 26);
    double wx[kMaxRadius + 1] = {}, wy[kMaxRadius + 1] = {};
    m.walls = (p.flags & LBM_FLAG_WALLS_Y) ? 1 : 0;
    const int ny_line = m.walls ? 2 * p.ny : p.ny;   // walls: the mirrored column's period
    if (lbm_hdm_weights(p.nx, radius, wx, &m.kx) != LBM_OK || lbm_hdm_weights(ny_line, radius, wy, &m.ky) != LBM_OK)
        return LBM_E_INVALID;
    for (int j = 0; j <= kMaxRadius; ++j) {
        m.wx[j] = (T)wx[j];
        m.wy[j] = (T)wy[j];
    }
    cudaStream_t s = (cudaStream_t)p.stream;
    int *err = (int *)scratch;
    m.chk = err;
    T *q = (T *)((unsigned char *)scratch + kErrBytes);
    const bool sc = p.force == LBM_FORCE_SC, cdm = p.grad == LBM_GRAD_CDM;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return LBM_E_CUDA;
    cudaError_t e;
    if constexpr (sizeof(TS) == sizeof(T)) {
        e = launch_potential<T>(m, sc, (const T *)f_in, q, err, s);
        if (e == cudaSuccess) e = launch_collide<T>(m, sc, cdm, (const T *)f_in, q, (T *)f_out, s);
    } else {
        e = launch_potential_mixed(m, sc, (const float *)f_in, q, err, s);
        if (e == cudaSuccess) e = launch_collide_mixed(m, sc, cdm, (const float *)f_in, q, (float *)f_out, s);
    }
    if (e != cudaSuccess) return LBM_E_CUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LBM_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_E_CUDA;
    return (h & kErrUnstable) ? LBM_E_UNSTABLE : LBM_OK;
}

}  // namespace

namespace {
// the potential field is FP64 for both precisions
long long max_cells() { return (long long)((LBM_STATIC_SCRATCH_BYTES - kErrBytes) / sizeof(double)); }
}  // namespace

extern "C" lbm_status lbm_step_noalloc(const lbm_params *p, const void *f_in, void *f_out) {
    if (!p || !f_in || !f_out || f_in == f_out) return LBM_E_INVALID;
    const char *why = "";
    if (lbm::check_params(*p, &why) != LBM_OK) return LBM_E_INVALID;
    if ((long long)p->nx * p->ny > max_cells()) return LBM_E_INVALID;
    lbm::ModelScalars ms;
    if (lbm::model_scalars(*p, &ms) != LBM_OK) return LBM_E_INVALID;
    void *scratch = nullptr;
    lbm_status st = scratch_on_current_device(&scratch);
    if (st != LBM_OK) return st;
    return p->prec == LBM_F64 ? run_step<double, double>(*p, ms, f_in, f_out, scratch)
                              : run_step<float, double>(*p, ms, f_in, f_out, scratch);
}
