// C ABI of the library (include/lbm.h): context life cycle, parameter
// validation, host<->device marshalling and the launch sequence of a step.
#include <sys/mman.h>
#include <unistd.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <algorithm>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace lbm {

lbm_status check_params(const lbm_params &p, const char **why) {
    auto bad = [&](const char *w) {
        *why = w;
        return LBM_E_INVALID;
    };
    if (p.nx < 1 || p.ny < 1) return bad("nx, ny must be >= 1");
    if ((long long)p.nx * p.ny > (1LL << 31)) return bad("lattice larger than 2^31 cells");
    if (p.prec != LBM_F32 && p.prec != LBM_F64) return bad("prec must be LBM_F32 or LBM_F64");
    if (p.eos < LBM_EOS_VDW || p.eos > LBM_EOS_PSI_EXP) return bad("unknown eos");
    if (p.force != LBM_FORCE_SC && p.force != LBM_FORCE_ZC) return bad("unknown force form");
    if (p.grad != LBM_GRAD_HDM && p.grad != LBM_GRAD_CDM) return bad("unknown gradient");
    if (p.hdm_radius < 0 || p.hdm_radius > kMaxRadius) return bad("hdm_radius must be in [0, 48]");
    if (p.flags & ~(LBM_FLAG_TWO_PASS | LBM_FLAG_WALLS_Y | LBM_FLAG_F32_ARITH | LBM_FLAG_STAGED_HOST))
        return bad("unknown flags");
    if (!(p.tau > 0.5) || !std::isfinite(p.tau)) return bad("tau must be > 0.5");
    if (p.eos == LBM_EOS_PSI_EXP) {
        if (!std::isfinite(p.G) || p.G == 0.0) return bad("G must be finite and non-zero");
        if (!(p.rho0 > 0) || !std::isfinite(p.rho0)) return bad("rho0 must be > 0");
        return LBM_OK;
    }
    if (!(p.a >= 0) || !(p.b > 0) || !(p.R > 0)) return bad("need a >= 0, b > 0, R > 0");
    if (!(p.Tr > 0) || !std::isfinite(p.Tr)) return bad("Tr must be > 0");
    if (!std::isfinite(p.k) || !std::isfinite(p.omega)) return bad("k, omega must be finite");
    return LBM_OK;
}

lbm_status model_scalars(const lbm_params &p, ModelScalars *s) {
    *s = ModelScalars{};
    if (p.eos == LBM_EOS_PSI_EXP) {  // Eq. 4-5
        s->a = 0.5 * p.G;
        s->b = 1.0 / p.rho0;
        s->k = 1.0;
        return LBM_OK;
    }
    double Tc = p.Tc, rc = 0;
    if (!(Tc > 0) && (p.a <= 0 || lbm_critical_point(p.eos, p.a, p.b, p.R, &Tc, &rc) != LBM_OK))
        return LBM_E_INVALID;
    const double T = p.Tr * Tc;
    double alpha = 1.0, dalpha = 0.0, m, q;
    switch (p.eos) {
    case LBM_EOS_PR:   // alpha = (1 + m (1 - sqrt(T/Tc)))^2, Eq. 28
    case LBM_EOS_RKS:  // the Soave form after Eq. 27
        m = p.eos == LBM_EOS_PR ? 0.37464 + 1.54226 * p.omega - 0.26992 * p.omega * p.omega
                                : 0.480 + 1.574 * p.omega - 0.176 * p.omega * p.omega;
        q = 1.0 + m * (1.0 - std::sqrt(T / Tc));
        alpha = q * q;
        dalpha = -q * m / std::sqrt(T * Tc);
        break;
    case LBM_EOS_RK:  // alpha = T^-1/2, Eq. 27
        alpha = 1.0 / std::sqrt(T);
        dalpha = -0.5 / (T * std::sqrt(T));
        break;
    default:
        break;
    }
    s->T = T;
    s->Tc = Tc;
    s->a = p.a;
    s->b = p.b;
    s->aal = p.a * alpha;
    s->aalp = p.a * dalpha;
    s->k = p.k;
    s->RT = p.R * T;
    return LBM_OK;
}

}  // namespace lbm

// Reverse sweep: segment k's recomputed states (or records) and stencil fields
// live in slot k % kTapeSlots, so the recompute on its own stream may run up
// to kTapeSlots - 1 segments ahead of the adjoint steps.  Two: a third slot
// (the recompute two segments ahead) measured no faster at 512^2, 5000 steps,
// and either stream at the higher priority starved the other (11 % slower).
constexpr int kTapeSlots = 2;
static_assert(kTapeSlots >= 2, "the recompute runs at least one segment ahead");

struct lbm_ctx {
    lbm_params p{};
    ModelScalars ms{};              // host scalars of p (temperature, EOS constants)
    int kx = 0, ky = 0;
    double wx[kMaxRadius + 1] = {}, wy[kMaxRadius + 1] = {};
    size_t esz = 4;               // bytes per value (float or double)
    long long n = 0;              // cells
    void *f[2] = {nullptr, nullptr};
    int cur = 0;                  // f[cur] holds the current state
    void *q = nullptr;            // potential field of the current pass
    bool fused = false;           // FP32 single-pass step in use
    void *qpad[2] = {nullptr, nullptr};  // padded potential of f[0] / f[1] (fused path)
    bool qpad_valid = false;      // qpad[cur] holds the potential of f[cur]
    int seg_rows = 0;             // rows per CTA segment of the fused path (0: automatic)
    int num_sms = 0;              // SMs of the context's device
    bool direct_host = false;     // the device reads the caller's pageable host arrays in place
    void *mom = nullptr;          // rho, vx, vy scratch (3 n values), lazily allocated
    double *partial = nullptr;    // reduction partials
    lbm_obs *obs_dev = nullptr;
    int *err = nullptr;           // device error word
    cudaStream_t stream = nullptr;
    bool initialized = false;
    bool unstable = false;
    std::string msg;
    // pinned host staging for precision conversion of host fields
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // event accounting of lbm_step (lbm_set_timing)
    bool timing = false;
    lbm_timing tm{};
    struct Pending { cudaEvent_t a, b; int slot; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    // reverse-mode tape (lbm_adjoint_forward / lbm_adjoint_backward)
    std::vector<void *> ckpt;       // states at t = 0, C, 2C, ... (9 n values each)
    // single-pass contexts: the padded stencil field of each checkpointed state
    // as the forward formed it (the single-pass kernel finishes the field of
    // t+1 from its partial densities, a different rounding from the potential
    // kernel), so that a recompute from a checkpoint repeats the forward bit for bit
    std::vector<void *> ckptq;
    void *tmp[2] = {nullptr, nullptr};
    void *qpad_tape[2] = {nullptr, nullptr};
    int tape_steps = -1, tape_C = 0;
    bool fused_rev = false;         // the single-pass kernel's CTA order of the next step (alternates)
    bool tape_last_ready = false;   // the last two segments' states are in their sweep slots (set by the forward)
    // reverse sweep buffers, allocated with the tape: the states recomputed
    // inside a segment (single-pass contexts: the forward kernel's record of
    // every state of a segment), the stencil field of every state of a
    // segment, the adjoint ping-pong, kernel scratch and the FP64 dL/dT slots
    // (kTapeSlots sets: the recompute of the next earlier segments runs on
    // rstream while the adjoint steps of a segment run on astream)
    std::vector<void *> seg, segq;
    cudaStream_t rstream = nullptr;
    cudaStream_t astream = nullptr;   // the adjoint steps
    cudaEvent_t rec_done[kTapeSlots] = {}, adj_done[kTapeSlots] = {}, bw_start = nullptr;
    void *lam[2] = {nullptr, nullptr};
    void *aux = nullptr;
    double *slots = nullptr;
};

namespace {

std::string g_create_error = "no error";

lbm_status fail(lbm_ctx *c, lbm_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->msg = buf; else g_create_error = buf;
    return st;
}

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *what) {
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_E_NOMEM : LBM_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(c, expr, what)                                   \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

template <typename T>
Model<T> model_of(const lbm_ctx *c) {
    Model<T> m{};
    m.chk = c->err;
    m.nx = c->p.nx;
    m.ny = c->p.ny;
    m.eos = c->p.eos;
    m.kx = c->kx;
    m.ky = c->ky;
    m.walls = (c->p.flags & LBM_FLAG_WALLS_Y) ? 1 : 0;
    m.RT = (T)c->ms.RT;
    m.a = (T)c->ms.a;
    m.b = (T)c->ms.b;
    m.aal = (T)c->ms.aal;
    m.k = (T)c->ms.k;
    m.omega = (T)(1.0 / c->p.tau);
    for (int j = 0; j <= kMaxRadius; ++j) {
        m.wx[j] = (T)c->wx[j];
        m.wy[j] = (T)c->wy[j];
    }
    return m;
}

bool is_f64(const lbm_ctx *c) { return c->p.prec == LBM_F64; }
bool is_sc(const lbm_ctx *c) { return c->p.force == LBM_FORCE_SC; }
bool is_cdm(const lbm_ctx *c) { return c->p.grad == LBM_GRAD_CDM; }
// The reverse mode takes the single-pass kernel (its recording variant and
// the padded layout) for HDM lattices only; CDM lattices tape with the
// two-pass kernels.
bool tape_fused(const lbm_ctx *c) { return c->fused && !is_cdm(c); }

cudaError_t take_event(lbm_ctx *c, cudaEvent_t *ev) {
    if (!c->event_pool.empty()) {
        *ev = c->event_pool.back();
        c->event_pool.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(ev);
}

// Resolve recorded event pairs into the per-slot sums (synchronises on them).
cudaError_t resolve_timing(lbm_ctx *c) {
    for (auto &p : c->pending) {
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e != cudaSuccess) return e;
        float ms = 0;
        e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess) return e;
        c->tm.ms_kernel[p.slot] += ms;
        c->tm.count_kernel[p.slot] += 1;
        c->event_pool.push_back(p.a);
        c->event_pool.push_back(p.b);
    }
    c->pending.clear();
    return cudaSuccess;
}

// Launch one kernel of a step through `fn`, bracketed by an event pair when
// timing is enabled.
template <typename Fn>
cudaError_t timed_launch(lbm_ctx *c, int slot, Fn fn, int kernels = 1) {
    if (!c->timing) return fn();
    if (c->pending.size() >= 8192) {
        cudaError_t e = resolve_timing(c);
        if (e != cudaSuccess) return e;
    }
    cudaEvent_t a, b;
    cudaError_t e = take_event(c, &a);
    if (e == cudaSuccess) e = take_event(c, &b);
    if (e == cudaSuccess) e = cudaEventRecord(a, c->stream);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
    if (e != cudaSuccess) return e;
    c->pending.push_back({a, b, slot});
    c->tm.launches += kernels;
    return cudaSuccess;
}

// One time step: potential of f[cur] into q, then force/collide/stream into f[1-cur].
template <typename T>
cudaError_t step_once(lbm_ctx *c, const Model<T> &m) {
    const T *f = (const T *)c->f[c->cur];
    T *g = (T *)c->f[1 - c->cur];
    cudaError_t e = timed_launch(c, 0, [&] { return launch_potential<T>(m, is_sc(c), f, (T *)c->q, c->err, c->stream); });
    if (e != cudaSuccess) return e;
    e = timed_launch(c, 1, [&] { return launch_collide<T>(m, is_sc(c), is_cdm(c), f, (const T *)c->q, g, c->stream); });
    if (e != cudaSuccess) return e;
    if (c->timing) c->tm.steps += 1;
    c->cur = 1 - c->cur;
    return cudaSuccess;
}

// One time step of an FP32 lattice in the two-pass form: FP32 distributions,
// FP64 arithmetic and an FP64 potential field (see lbm_kernels.cu).
cudaError_t step_once_mixed(lbm_ctx *c, const Model<double> &m) {
    const float *f = (const float *)c->f[c->cur];
    float *g = (float *)c->f[1 - c->cur];
    cudaError_t e = timed_launch(c, 0, [&] { return launch_potential_mixed(m, is_sc(c), f, (double *)c->q, c->err, c->stream); });
    if (e != cudaSuccess) return e;
    e = timed_launch(c, 1, [&] { return launch_collide_mixed(m, is_sc(c), is_cdm(c), f, (const double *)c->q, g, c->stream); });
    if (e != cudaSuccess) return e;
    if (c->timing) c->tm.steps += 1;
    c->cur = 1 - c->cur;
    return cudaSuccess;
}

int seg_rows_of(const lbm_ctx *c) {
    return c->seg_rows > 0 ? c->seg_rows : fused_auto_seg_rows(c->p.nx, c->p.ny, c->num_sms);
}

// One time step by the single-pass FP32 kernel.
cudaError_t step_fused(lbm_ctx *c, const Model<float> &m) {
    const float *f = (const float *)c->f[c->cur];
    cudaError_t e;
    if (!c->qpad_valid) {
        e = timed_launch(c, 0, [&] {
            return launch_potential_padded(m, is_sc(c), f, (float *)c->qpad[c->cur], c->err, c->stream);
        });
        if (e != cudaSuccess) return e;
        c->qpad_valid = true;
    }
    e = timed_launch(c, 2, [&] {
        return launch_fused_step(m, is_sc(c), is_cdm(c), f, (const float *)c->qpad[c->cur], (float *)c->f[1 - c->cur],
                                 (float *)c->qpad[1 - c->cur], c->err, seg_rows_of(c), c->stream, true, nullptr,
                                 c->fused_rev);
    });
    if (e != cudaSuccess) return e;
    c->fused_rev = !c->fused_rev;   // the CTA order alternates step by step
    if (c->timing) c->tm.steps += 1;
    c->cur = 1 - c->cur;
    return cudaSuccess;
}

// Density and Eq. 11 velocity of the current state, in the arithmetic of the
// lattice's step: FP32 for FP32 lattices on the single-pass kernel (or with
// LBM_FLAG_F32_ARITH), FP64 for the other FP32 lattices (the mixed kernels).
template <typename T>
cudaError_t moments_into(lbm_ctx *c, T *r, T *vx, T *vy) {
    Model<T> m = model_of<T>(c);
    const T *f = (const T *)c->f[c->cur];
    cudaError_t e = launch_potential<T>(m, is_sc(c), f, (T *)c->q, c->err, c->stream);
    if (e != cudaSuccess) return e;
    return launch_moments<T>(m, is_sc(c), is_cdm(c), f, (const T *)c->q, r, vx, vy, c->stream);
}
template <>
cudaError_t moments_into<float>(lbm_ctx *c, float *r, float *vx, float *vy) {
    if (c->fused || (c->p.flags & LBM_FLAG_F32_ARITH)) {
        Model<float> mf = model_of<float>(c);
        const float *f = (const float *)c->f[c->cur];
        cudaError_t e = launch_potential<float>(mf, is_sc(c), f, (float *)c->q, c->err, c->stream);
        if (e != cudaSuccess) return e;
        return launch_moments<float>(mf, is_sc(c), is_cdm(c), f, (const float *)c->q, r, vx, vy, c->stream);
    }
    Model<double> m = model_of<double>(c);
    const float *f = (const float *)c->f[c->cur];
    cudaError_t e = launch_potential_mixed(m, is_sc(c), f, (double *)c->q, c->err, c->stream);
    if (e != cudaSuccess) return e;
    return launch_moments_mixed(m, is_sc(c), is_cdm(c), f, (const double *)c->q, r, vx, vy, c->stream);
}

// Three fields of scratch and, past them, the 8-byte word of the host-array
// check (mom_bad).
size_t mom_fields_bytes(const lbm_ctx *c) { return (3 * c->n * c->esz + 255) / 256 * 256; }

lbm_status ensure_mom(lbm_ctx *c) {
    if (c->mom) return LBM_OK;
    CK(c, dev_alloc(&c->mom, mom_fields_bytes(c) + 256), "cudaMalloc(moments)");
    return LBM_OK;
}

unsigned long long *mom_bad(lbm_ctx *c) {
    return (unsigned long long *)((char *)c->mom + mom_fields_bytes(c));
}

// True if every page of [p, p + bytes) is resident in host memory (mincore):
// device writes then meet no page that has to be populated first.
bool pages_resident(const void *p, size_t bytes) {
    static const long ps = sysconf(_SC_PAGESIZE);
    if (ps <= 0 || bytes == 0) return false;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p) / ps * ps;
    const uintptr_t end = reinterpret_cast<uintptr_t>(p) + bytes;
    const size_t pages = (end - a + ps - 1) / ps;
    std::vector<unsigned char> vec(pages);
    if (mincore(reinterpret_cast<void *>(a), end - a, vec.data()) != 0) return false;
    for (unsigned char v : vec)
        if (!(v & 1)) return false;
    return true;
}

lbm_status read_error_word(lbm_ctx *c) {
    int h = 0;
    CK(c, cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read error word");
    CK(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (h & kErrUnstable) {
        c->unstable = true;
        return fail(c, LBM_E_UNSTABLE, "unstable: NaN or non-positive density on the lattice");
    }
    if (h & kErrTimeout) return fail(c, LBM_E_TIMEOUT, "a device-side wait timed out");
    if (h & kErrBounds) return fail(c, LBM_E_CUDA, "a device-side bounds check failed");
    return LBM_OK;
}

lbm_status check_ready(lbm_ctx *c) {
    if (!c) return LBM_E_INVALID;
    if (!c->initialized) return fail(c, LBM_E_STATE, "lattice not initialised (call lbm_init_density or lbm_set_f)");
    if (c->unstable) return fail(c, LBM_E_UNSTABLE, "lattice is in the error state; re-initialise it");
    return LBM_OK;
}

lbm_status mark_initialized(lbm_ctx *c) {
    CK(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), "clear error word");
    c->initialized = true;
    c->unstable = false;
    c->qpad_valid = false;
    return LBM_OK;
}

lbm_status ensure_stage(lbm_ctx *c, size_t bytes) {
    if (c->stage_bytes >= bytes) return LBM_OK;
    CK(c, cudaStreamSynchronize(c->stream), "sync before staging realloc");
    if (c->stage) host_free(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    CK(c, host_alloc(&c->stage, bytes), "cudaHostAlloc(stage)");
    c->stage_bytes = bytes;
    return LBM_OK;
}

void free_tape(lbm_ctx *c) {
    for (void *p : c->ckpt) dev_free(p);
    c->ckpt.clear();
    for (void *p : c->ckptq) dev_free(p);
    c->ckptq.clear();
    for (void *p : c->seg) dev_free(p);
    for (void *p : c->segq) dev_free(p);
    c->seg.clear();
    c->segq.clear();
    for (int k = 0; k < 2; ++k) {
        dev_free(c->lam[k]);
        c->lam[k] = nullptr;
    }
    for (int k = 0; k < kTapeSlots; ++k) {
        if (c->rec_done[k]) cudaEventDestroy(c->rec_done[k]);
        if (c->adj_done[k]) cudaEventDestroy(c->adj_done[k]);
        c->rec_done[k] = c->adj_done[k] = nullptr;
    }
    if (c->rstream) cudaStreamDestroy(c->rstream);
    if (c->astream) cudaStreamDestroy(c->astream);
    if (c->bw_start) cudaEventDestroy(c->bw_start);
    c->rstream = c->astream = nullptr;
    c->bw_start = nullptr;
    dev_free(c->aux);
    dev_free(c->slots);
    c->aux = nullptr;
    c->slots = nullptr;
    for (int k = 0; k < 2; ++k) {
        dev_free(c->tmp[k]);
        dev_free(c->qpad_tape[k]);
        c->tmp[k] = c->qpad_tape[k] = nullptr;
    }
    c->tape_steps = -1;
}

// One forward step from state `src` to `dst` (explicit buffers).  Single-pass
// path: qsrc holds the padded stencil field of src (valid on entry) and qdst
// receives that of dst.  Two-pass path: the potential of src is formed into
// qsrc first (qdst unused).  rec (single-pass): where the record of src goes,
// or nullptr.
template <typename T>
cudaError_t tape_step(lbm_ctx *c, const Model<T> &m, const void *src, void *dst, void *qsrc, void *qdst,
                      float *rec, bool rev) {
    if constexpr (std::is_same_v<T, float>) {   // (FP64 contexts never take the single-pass kernel)
        if (tape_fused(c))
            return launch_fused_step(m, is_sc(c), is_cdm(c), (const float *)src, (const float *)qsrc, (float *)dst,
                                     (float *)qdst, c->err, seg_rows_of(c), c->stream, true, rec, rev);
    }
    cudaError_t e = launch_potential<T>(m, is_sc(c), (const T *)src, (T *)qsrc, c->err, c->stream);
    if (e != cudaSuccess) return e;
    return launch_collide<T>(m, is_sc(c), is_cdm(c), (const T *)src, (const T *)qsrc, (T *)dst, c->stream);
}

template <typename T>
lbm_status tape_forward(lbm_ctx *c, const T *rho0, int nsteps, int C, T *rhoT) {
    const size_t fbytes = (size_t)kQ * c->n * sizeof(T);
    const int nck = nsteps / C + 1;
    c->tape_steps = -1;
    // a tape of the same shape (checkpoint count and interval) is reused
    const bool reuse = c->slots && c->tape_C == C && c->ckpt.size() == (size_t)nck;
    if (!reuse) {
        free_tape(c);
        for (int k = 0; k < nck; ++k) {
            void *p = nullptr;
            if (dev_alloc(&p, fbytes) != cudaSuccess) {
                free_tape(c);
                return fail(c, LBM_E_NOMEM, "not enough device memory for %d checkpoints", nck);
            }
            c->ckpt.push_back(p);
        }
        if (dev_alloc(&c->tmp[0], fbytes) != cudaSuccess || dev_alloc(&c->tmp[1], fbytes) != cudaSuccess) {
            free_tape(c);
            return fail(c, LBM_E_NOMEM, "tape scratch");
        }
        if (tape_fused(c)) {
            size_t qb = sizeof(float) * (size_t)fused_q_pitch(c->p.nx) * c->p.ny;
            if (dev_alloc(&c->qpad_tape[0], qb) != cudaSuccess || dev_alloc(&c->qpad_tape[1], qb) != cudaSuccess) {
                free_tape(c);
                return fail(c, LBM_E_NOMEM, "tape potential fields");
            }
            for (int k = 0; k < nck; ++k) {
                void *p = nullptr;
                if (dev_alloc(&p, qb) != cudaSuccess) {
                    free_tape(c);
                    return fail(c, LBM_E_NOMEM, "checkpoint potential fields");
                }
                c->ckptq.push_back(p);
            }
        }
        {   // buffers of the reverse sweep
            const bool tau1 = model_of<T>(c).omega == T(1);
            const int qpitch = tape_fused(c) ? fused_q_pitch(c->p.nx) : c->p.nx;
            const size_t qbytes = sizeof(T) * (size_t)qpitch * c->p.ny;
            const AdjLayout lay = adjoint_layout(c->p.nx, c->p.ny, tape_fused(c), tau1);
            const size_t lbytes = (size_t)lay.nlam * lay.lstride * sizeof(T);
            bool ok = true;
            // single-pass contexts keep the forward kernel's record of every state
            // of a segment (five planes); the others keep the states after the first
            const size_t sbytes = tape_fused(c) ? (size_t)5 * c->n * sizeof(float) : fbytes;
            c->seg.assign(tape_fused(c) ? kTapeSlots * C : kTapeSlots * (C > 1 ? C - 1 : 0), nullptr);
            c->segq.assign(kTapeSlots * C, nullptr);
            for (auto &p : c->seg) ok = ok && dev_alloc(&p, sbytes) == cudaSuccess;
            for (auto &p : c->segq) ok = ok && dev_alloc(&p, qbytes) == cudaSuccess;
            // equal priorities (either stream favoured starves the other)
            ok = ok && cudaStreamCreateWithFlags(&c->rstream, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaStreamCreateWithFlags(&c->astream, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->bw_start, cudaEventDisableTiming) == cudaSuccess;
            for (int k = 0; k < kTapeSlots; ++k)
                ok = ok && cudaEventCreateWithFlags(&c->rec_done[k], cudaEventDisableTiming) == cudaSuccess &&
                     cudaEventCreateWithFlags(&c->adj_done[k], cudaEventDisableTiming) == cudaSuccess;
            ok = ok && dev_alloc(&c->lam[0], lbytes) == cudaSuccess && dev_alloc(&c->lam[1], lbytes) == cudaSuccess &&
                 dev_alloc(&c->aux, (size_t)lay.naux * lay.dstride * sizeof(T)) == cudaSuccess &&
                 dev_alloc((void **)&c->slots, sizeof(double) * (adjoint_slots<T>(c->p.nx, c->p.ny) + 1)) == cudaSuccess;
            if (!ok) {
                free_tape(c);
                return fail(c, LBM_E_NOMEM, "not enough device memory for the reverse sweep buffers");
            }
        }
        c->tape_C = C;
    }
    Model<T> m = model_of<T>(c);
    CK(c, cudaMemsetAsync(c->err, 0, sizeof(int), c->stream), "clear error word");
    CK(c, launch_init<T>(m, rho0, nullptr, nullptr, (T *)c->ckpt[0], c->stream), "init kernel");
    // What the reverse sweep needs of the last two segments goes straight
    // into their slots, so the sweep starts with no recompute: segment k's
    // stencil fields of states k C .. in slot k % kTapeSlots, and its states
    // k C + 1 .. (single-pass contexts: the records of states k C .., the
    // states themselves staying in the scratch pair).
    const int K = (nsteps - 1) / C, t0 = K * C, sl = K % kTapeSlots, nseg = C > 1 ? C - 1 : 0;
    const int slp = (K + kTapeSlots - 1) % kTapeSlots;   // the slot of segment K - 1
    const int tp = K >= 1 ? t0 - C : t0;   // the first step of the taped segments
    auto fbuf = [&](int t) -> void * {   // where state t (>= 1) goes
        if (t % C == 0) return c->ckpt[t / C];
        if (!tape_fused(c) && t > t0 && t < nsteps) return c->seg[sl * nseg + (t - t0 - 1)];
        if (!tape_fused(c) && t > tp && t < t0) return c->seg[slp * nseg + (t - tp - 1)];
        return c->tmp[t & 1];
    };
    auto rbuf = [&](int t) -> float * {   // where the record of state t goes (single-pass)
        if (!tape_fused(c) || t < tp) return nullptr;
        return (float *)c->seg[((t / C) % kTapeSlots) * C + t % C];
    };
    auto qbuf = [&](int t) -> void * {   // the stencil field of state t
        if (t >= t0 && t < nsteps) return c->segq[sl * C + (t - t0)];
        if (t >= tp && t < t0) return c->segq[slp * C + (t - tp)];
        if (tape_fused(c) && t % C == 0) return c->ckptq[t / C];
        return tape_fused(c) ? c->qpad_tape[t & 1] : c->q;
    };
    if constexpr (std::is_same_v<T, float>) {
        if (tape_fused(c))
            CK(c, launch_potential_padded(m, is_sc(c), (const float *)c->ckpt[0], (float *)qbuf(0), c->err, c->stream),
               "potential");
    }
    const void *cur = c->ckpt[0];
    for (int t = 0; t < nsteps; ++t) {
        void *dst = fbuf(t + 1);
        CK(c, tape_step<T>(c, m, cur, dst, qbuf(t), qbuf(t + 1), rbuf(t), (t & 1) != 0), "tape forward step");
        cur = dst;
    }
    if (tape_fused(c)) {   // the checkpointed fields of the taped segments, for a later recompute
        const size_t qb = sizeof(float) * (size_t)fused_q_pitch(c->p.nx) * c->p.ny;
        for (int t = tp; t <= t0; t += C)
            CK(c, cudaMemcpyAsync(c->ckptq[t / C], qbuf(t), qb, cudaMemcpyDeviceToDevice, c->stream),
               "checkpoint field");
    }
    c->tape_last_ready = true;
    CK(c, launch_density<T>(c->n, (const T *)cur, rhoT, c->stream), "density");
    // leave the context on the final state too
    CK(c, cudaMemcpyAsync(c->f[0], cur, fbytes, cudaMemcpyDeviceToDevice, c->stream), "copy final state");
    c->cur = 0;
    c->initialized = true;
    c->unstable = false;
    c->qpad_valid = false;
    c->tape_steps = nsteps;
    c->tape_C = C;
    return LBM_OK;
}

template <typename T>
lbm_status tape_backward(lbm_ctx *c, const T *grad_rhoT, T *grad_rho0, double *gT) {
    const int N = c->tape_steps, C = c->tape_C;
    const int nx = c->p.nx, ny = c->p.ny;
    Model<T> m = model_of<T>(c);
    const T R = (T)c->p.R, aalp = (T)c->ms.aalp;
    const bool tau1 = m.omega == T(1);
    const AdjLayout lay = adjoint_layout(nx, ny, tape_fused(c), tau1);
    // stencil fields: the single-pass layout (padded rows) or the plain one
    const int qpitch = tape_fused(c) ? fused_q_pitch(nx) : nx;
    const int qoff = (qpitch - nx) / 2;
    const int nslots = adjoint_slots<T>(nx, ny);
    void **lam = c->lam, *aux = c->aux;
    double *slots = c->slots;
    const int rows = tape_fused(c) ? seg_rows_of(c) : 0;
    const int nseg = C > 1 ? C - 1 : 0;
    // slot sl: states (single-pass: records) seg[sl * nseg + j] (seg[sl * C + j]),
    // stencil fields segq[sl * C + j]
    auto segf = [&](int sl, int j) { return c->seg[sl * nseg + j]; };
    auto segrec = [&](int sl, int j) { return c->seg[sl * C + j]; };
    auto segqf = [&](int sl, int j) { return c->segq[sl * C + j]; };
    // Recompute segment k from its checkpoint with the forward kernels on
    // stream s into slot sl: the stencil field of every state t0 .. t1-1, and
    // the states t0+1 .. t1-1 (single-pass: the records of states t0 .. t1-1,
    // which takes the segment's last step too; the states pass through the
    // scratch pair).
    auto recompute = [&](int k, int sl, cudaStream_t s) {
        const int t0 = k * C, t1 = std::min(N, t0 + C);
        cudaError_t r = cudaSuccess;
        if constexpr (std::is_same_v<T, float>) {   // (FP64 contexts never take the single-pass kernel)
            if (tape_fused(c)) {
                r = cudaMemcpyAsync(segqf(sl, 0), c->ckptq[k], sizeof(float) * (size_t)fused_q_pitch(nx) * ny,
                                    cudaMemcpyDeviceToDevice, s);
                const void *cur = c->ckpt[k];
                for (int t = t0; t < t1 && r == cudaSuccess; ++t) {
                    // (programmatic launches here too: plain ones, which hold no SM
                    // resources while they wait, made the sweep 4 % slower)
                    void *dst = c->tmp[(t + 1) & 1];
                    void *qn = t + 1 < t1 ? segqf(sl, t + 1 - t0) : c->qpad_tape[0];
                    r = launch_fused_step(m, is_sc(c), is_cdm(c), (const float *)cur, (const float *)segqf(sl, t - t0),
                                          (float *)dst, (float *)qn, c->err, rows, s, true, (float *)segrec(sl, t - t0),
                                          (t & 1) != 0);
                    cur = dst;
                }
                return r;
            }
        }
        const void *cur = c->ckpt[k];
        for (int t = t0; t < t1 && r == cudaSuccess; ++t) {
            r = launch_potential<T>(m, is_sc(c), (const T *)cur, (T *)segqf(sl, t - t0), c->err, s);
            if (r == cudaSuccess && t < t1 - 1) {
                r = launch_collide<T>(m, is_sc(c), is_cdm(c), (const T *)cur, (const T *)segqf(sl, t - t0),
                                      (T *)segf(sl, t - t0), s);
                cur = segf(sl, t - t0);
            }
        }
        return r;
    };
    // the sweep runs on the tape's own streams, ordered after the context's
    // stream at the start and before it at the end
    cudaStream_t as = c->astream;
    cudaError_t e = cudaEventRecord(c->bw_start, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(as, c->bw_start, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(slots, 0, sizeof(double) * (nslots + 1), as);
    if (e == cudaSuccess) e = launch_adjoint_seed<T>(nx, ny, tape_fused(c), lay, grad_rhoT, (T *)lam[0], c->err, as);
    // The recompute of segment j (into slot j % kTapeSlots) runs on rstream
    // once the adjoint steps of segment j + kTapeSlots, the slot's previous
    // user, are done; the adjoint steps of segment k (on astream) wait for
    // its recompute.  So the recompute runs up to kTapeSlots - 1 segments
    // ahead of the adjoint steps.
    const int K = (N - 1) / C;
    for (int j = 0; j < kTapeSlots && e == cudaSuccess; ++j)   // orders rstream after the seed
        e = cudaEventRecord(c->adj_done[j], as);
    // segments K and K - 1 are left in their slots by the forward
    const bool taped = c->tape_last_ready;
    c->tape_last_ready = false;   // the sweep reuses the slots
    auto rec = [&](int j) {
        cudaError_t r = cudaStreamWaitEvent(c->rstream, c->adj_done[j % kTapeSlots], 0);
        if (r == cudaSuccess && !(taped && j >= K - 1)) r = recompute(j, j % kTapeSlots, c->rstream);
        if (r == cudaSuccess) r = cudaEventRecord(c->rec_done[j % kTapeSlots], c->rstream);
        return r;
    };
    for (int j = K; j >= std::max(0, K - kTapeSlots + 2) && e == cudaSuccess; --j) e = rec(j);
    int li = 0;
    for (int k = K; k >= 0 && e == cudaSuccess; --k) {
        const int sl = k % kTapeSlots;
        if (k - kTapeSlots + 1 >= 0) e = rec(k - kTapeSlots + 1);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(as, c->rec_done[sl], 0);
        const int t0 = k * C, t1 = std::min(N, t0 + C);
        for (int t = t1 - 1; t >= t0 && e == cudaSuccess; --t) {
            const T *ft = (const T *)(tape_fused(c) ? segrec(sl, t - t0) : (t == t0 ? c->ckpt[k] : segf(sl, t - t0 - 1)));
            e = launch_adjoint_step<T>(m, R, aalp, is_sc(c), is_cdm(c), tau1, tape_fused(c), lay, ft,
                                       (const T *)segqf(sl, t - t0), qpitch, qoff, (const T *)lam[li], (T *)aux,
                                       (T *)lam[1 - li], slots, c->err, /*overlap_prev=*/t != t1 - 1, as);
            li = 1 - li;
        }
        if (e == cudaSuccess) e = cudaEventRecord(c->adj_done[sl], as);
    }
    if (e == cudaSuccess) e = launch_adjoint_initial<T>(nx, ny, lay, (const T *)lam[li], grad_rho0, c->err, as);
    if (e == cudaSuccess) e = launch_sum_slots(slots, nslots, slots + nslots, as);
    if (e == cudaSuccess) e = cudaEventRecord(c->bw_start, as);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->bw_start, 0);
    double h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, slots + nslots, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint");
    *gT = h;
    return read_error_word(c);
}

}  // namespace

namespace {

// fn(lo, hi) over [0, n) split across the host's threads (the precision
// conversions between the caller's FP64 arrays and the pinned FP32 staging run
// at memory speed only when many cores share them); one thread below 1M items.
template <typename F>
void parallel_for(long long n, F fn) {
    const long long kMinPerThread = 1 << 20;
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    nt = (unsigned)std::max<long long>(1, std::min<long long>(nt, n / kMinPerThread));
    if (nt == 1) {
        fn(0LL, n);
        return;
    }
    std::vector<std::thread> pool;
    const long long chunk = (n + nt - 1) / nt;
    for (unsigned t = 1; t < nt; ++t) {
        const long long lo = t * chunk, hi = std::min(n, lo + chunk);
        if (lo < hi) pool.emplace_back([=] { fn(lo, hi); });
    }
    fn(0LL, std::min(n, chunk));
    for (auto &th : pool) th.join();
}

template <typename D, typename S>
void convert(D *dst, const S *src, long long n) {
    parallel_for(n, [=](long long lo, long long hi) {
        for (long long i = lo; i < hi; ++i) dst[i] = (D)src[i];
    });
}

}  // namespace

extern "C" {

lbm_status lbm_adjoint_forward(lbm_ctx *c, const void *rho0, int nsteps, int checkpoint_interval, void *rho_T) {
    NvtxRange nvtx("lbm_adjoint_forward");
    if (!c) return LBM_E_INVALID;
    if (!rho0 || !rho_T) return fail(c, LBM_E_INVALID, "rho0 and rho_T must be device arrays");
    if (nsteps < 1 || checkpoint_interval < 1) return fail(c, LBM_E_INVALID, "need nsteps >= 1, checkpoint_interval >= 1");
    if (c->p.flags & LBM_FLAG_WALLS_Y) return fail(c, LBM_E_INVALID, "the reverse mode covers periodic lattices only");
    return is_f64(c) ? tape_forward<double>(c, (const double *)rho0, nsteps, checkpoint_interval, (double *)rho_T)
                     : tape_forward<float>(c, (const float *)rho0, nsteps, checkpoint_interval, (float *)rho_T);
}

lbm_status lbm_adjoint_backward(lbm_ctx *c, const void *grad_rho_T, void *grad_rho0, double *grad_T, double *grad_Tr,
                                double *grad_G) {
    NvtxRange nvtx("lbm_adjoint_backward");
    if (!c) return LBM_E_INVALID;
    if (c->tape_steps < 1) return fail(c, LBM_E_STATE, "no tape: call lbm_adjoint_forward first");
    if (!grad_rho_T || !grad_rho0) return fail(c, LBM_E_INVALID, "grad arrays must be device arrays");
    double gT = 0;
    lbm_status st = is_f64(c) ? tape_backward<double>(c, (const double *)grad_rho_T, (double *)grad_rho0, &gT)
                              : tape_backward<float>(c, (const float *)grad_rho_T, (float *)grad_rho0, &gT);
    if (st != LBM_OK) return st;
    // the accumulated scalar is dL/dG for the effective mass of Eq. 4, else dL/dT
    const bool psi = c->p.eos == LBM_EOS_PSI_EXP;
    if (grad_T) *grad_T = psi ? 0.0 : gT;
    if (grad_Tr) *grad_Tr = psi ? 0.0 : gT * c->ms.Tc;  // T = Tr Tc
    if (grad_G) *grad_G = psi ? gT : 0.0;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_params *p, lbm_ctx **out) {
    if (!out) return fail(nullptr, LBM_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, LBM_E_INVALID, "params is NULL");
    const char *why = "";
    if (check_params(*p, &why) != LBM_OK) return fail(nullptr, LBM_E_INVALID, "%s", why);
    ModelScalars ms;
    if (model_scalars(*p, &ms) != LBM_OK)
        return fail(nullptr, LBM_E_INVALID, "no critical point for these EOS constants; pass Tc explicitly");

    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_E_NOMEM, "host allocation failed");
    c->p = *p;
    c->stream = (cudaStream_t)p->stream;
    c->esz = p->prec == LBM_F64 ? sizeof(double) : sizeof(float);
    c->n = (long long)p->nx * p->ny;
    c->ms = ms;
    int radius = p->hdm_radius ? p->hdm_radius : (p->prec == LBM_F64 ? 40 : 26);
    lbm_hdm_weights(p->nx, radius, c->wx, &c->kx);
    // with walls the column operator is the periodic one of the mirrored column
    lbm_hdm_weights((p->flags & LBM_FLAG_WALLS_Y) ? 2 * p->ny : p->ny, radius, c->wy, &c->ky);

    auto bail = [&](cudaError_t e, const char *what) {
        lbm_status st = (e == cudaErrorMemoryAllocation) ? LBM_E_NOMEM : LBM_E_CUDA;
        fail(nullptr, st, "%s: %s", what, cudaGetErrorString(e));
        lbm_destroy(c);
        return st;
    };
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return bail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return bail(e, "cudaDeviceGetAttribute");
    {   // coherent access to pageable host memory through the host's page tables
        int pageable = 0, host_tables = 0;
        if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev) != cudaSuccess) {
            cudaGetLastError();
            pageable = host_tables = 0;
        }
        c->direct_host = pageable == 1 && host_tables == 1 && !(p->flags & LBM_FLAG_STAGED_HOST);
    }
    size_t fbytes = (size_t)kQ * c->n * c->esz;
    if ((e = dev_alloc(&c->f[0], fbytes)) != cudaSuccess) return bail(e, "cudaMalloc(f0)");
    if ((e = dev_alloc(&c->f[1], fbytes)) != cudaSuccess) return bail(e, "cudaMalloc(f1)");
    // the potential field of the two-pass kernels is FP64 for both precisions
    if ((e = dev_alloc(&c->q, (size_t)c->n * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc(q)");
    c->fused = p->prec == LBM_F32 && !(p->flags & LBM_FLAG_TWO_PASS) &&
               fused_step_supported(model_of<float>(c), p->grad == LBM_GRAD_CDM, radius);
    if (c->fused) {
        size_t qb = sizeof(float) * (size_t)fused_q_pitch(p->nx) * p->ny;
        if ((e = dev_alloc(&c->qpad[0], qb)) != cudaSuccess) return bail(e, "cudaMalloc(qpad0)");
        if ((e = dev_alloc(&c->qpad[1], qb)) != cudaSuccess) return bail(e, "cudaMalloc(qpad1)");
    }
    if ((e = dev_alloc(&c->partial, sizeof(double) * 6 * observables_partial_count())) != cudaSuccess)
        return bail(e, "cudaMalloc(partial)");
    if ((e = dev_alloc(&c->obs_dev, sizeof(lbm_obs))) != cudaSuccess) return bail(e, "cudaMalloc(obs)");
    if ((e = dev_alloc(&c->err, sizeof(int))) != cudaSuccess) return bail(e, "cudaMalloc(err)");
    if ((e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream)) != cudaSuccess) return bail(e, "cudaMemset(err)");
    *out = c;
    return LBM_OK;
}

lbm_status lbm_set_segment_rows(lbm_ctx *c, int rows) {
    if (!c) return LBM_E_INVALID;
    if (rows < 0 || rows > c->p.ny) return fail(c, LBM_E_INVALID, "segment rows must be in [0, ny = %d]", c->p.ny);
    c->seg_rows = rows;
    return LBM_OK;
}

lbm_status lbm_get_segment_rows(lbm_ctx *c, int *rows) {
    if (!c || !rows) return LBM_E_INVALID;
    *rows = c->fused ? seg_rows_of(c) : 0;
    return LBM_OK;
}

lbm_status lbm_tune_segment_rows(lbm_ctx *c, int trials, int *rows) {
    NvtxRange nvtx("lbm_tune_segment_rows");
    lbm_status st = check_ready(c);
    if (st != LBM_OK) return st;
    if (!rows) return fail(c, LBM_E_INVALID, "rows must be non-NULL");
    if (trials < 1 || trials > 1000) return fail(c, LBM_E_INVALID, "trials must be in [1, 1000]");
    if (!c->fused) {
        *rows = 0;
        return LBM_OK;
    }
    // Every trial launch reads the current state (f and its padded potential)
    // and writes the buffers the next step overwrites, so the state is kept.
    const Model<float> m = model_of<float>(c);
    const float *f = (const float *)c->f[c->cur];
    if (!c->qpad_valid) {
        CK(c, launch_potential_padded(m, is_sc(c), f, (float *)c->qpad[c->cur], c->err, c->stream), "potential");
        c->qpad_valid = true;
    }
    auto launch = [&](int h) {
        return launch_fused_step(m, is_sc(c), is_cdm(c), f, (const float *)c->qpad[c->cur], (float *)c->f[1 - c->cur],
                                 (float *)c->qpad[1 - c->cur], c->err, h, c->stream);
    };
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    // time n launches at height h (after one warm-up launch)
    auto time_height = [&](int h, int n, float *ms) {
        e = launch(h);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], c->stream);
        for (int t = 0; t < n && e == cudaSuccess; ++t) e = launch(h);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, ev[0], ev[1]);
        return e == cudaSuccess;
    };
    // Coarse scan: heights 8k - 2 (whole slabs, no wasted collided rows) up to
    // the lattice or 1022 rows, `trials` launches each; the kFinal fastest go on.
    constexpr int kFinal = 6, kRounds = 3;
    int cand[kFinal];
    float cand_ms[kFinal];
    int ncand = 0;
    const int hmax = std::min(c->p.ny, 1022);
    for (int h = 6; h <= hmax; h += 8) {
        if ((c->p.ny + h - 1) / h > 65535) continue;
        float ms = 0.f;
        if (!time_height(h, trials, &ms)) break;
        int at = ncand < kFinal ? ncand++ : kFinal;   // insertion into the sorted list
        while (at > 0 && cand_ms[at - 1] > ms) {
            if (at < kFinal) {
                cand[at] = cand[at - 1];
                cand_ms[at] = cand_ms[at - 1];
            }
            --at;
        }
        if (at < kFinal) {
            cand[at] = h;
            cand_ms[at] = ms;
        }
    }
    // Final: kRounds interleaved rounds of 8 x trials launches per candidate (a
    // short scan's pick varies by a few tenths of a percent from one run to the
    // next); the smallest total wins.
    float total[kFinal] = {};
    for (int r = 0; r < kRounds && e == cudaSuccess; ++r)
        for (int i = 0; i < ncand && e == cudaSuccess; ++i) {
            float ms = 0.f;
            if (time_height(cand[i], 8 * trials, &ms)) total[i] += ms;
        }
    int bi = -1;
    for (int i = 0; i < ncand; ++i)
        if (bi < 0 || total[i] < total[bi]) bi = i;
    const int best = bi < 0 ? 0 : cand[bi];
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    CK(c, e, "segment-height trials");
    st = read_error_word(c);
    if (st != LBM_OK) return st;
    c->seg_rows = best;
    *rows = best;
    return LBM_OK;
}

lbm_status lbm_init_density_device(lbm_ctx *c, const void *rho, const void *ux, const void *uy) {
    if (!c) return LBM_E_INVALID;
    if (!rho) return fail(c, LBM_E_INVALID, "rho is NULL");
    c->cur = 0;
    cudaError_t e;
    if (is_f64(c))
        e = launch_init<double>(model_of<double>(c), (const double *)rho, (const double *)ux, (const double *)uy,
                                (double *)c->f[0], c->stream);
    else
        e = launch_init<float>(model_of<float>(c), (const float *)rho, (const float *)ux, (const float *)uy,
                               (float *)c->f[0], c->stream);
    CK(c, e, "init kernel");
    return mark_initialized(c);
}

lbm_status lbm_init_density(lbm_ctx *c, const double *rho, const double *ux, const double *uy) {
    if (!c) return LBM_E_INVALID;
    if (!rho) return fail(c, LBM_E_INVALID, "rho is NULL");
    if (c->direct_host) {   // the device reads the caller's arrays in place, checking rho
        lbm_status st = ensure_mom(c);
        if (st != LBM_OK) return st;
        char *dev = (char *)c->mom;
        const size_t fb = c->n * c->esz;
        unsigned long long *badw = mom_bad(c), bad = 0;
        const double *src[3] = {rho, ux, uy};
        CK(c, cudaMemsetAsync(badw, 0xff, sizeof(*badw), c->stream), "clear check word");
        for (int k = 0; k < 3; ++k) {
            if (!src[k]) continue;
            cudaError_t e = is_f64(c) ? launch_from_host<double>(src[k], (double *)(dev + k * fb), c->n,
                                                                  k == 0 ? badw : nullptr, c->stream)
                                      : launch_from_host<float>(src[k], (float *)(dev + k * fb), c->n,
                                                                 k == 0 ? badw : nullptr, c->stream);
            CK(c, e, "read host field");
        }
        CK(c, cudaMemcpyAsync(&bad, badw, sizeof(bad), cudaMemcpyDeviceToHost, c->stream), "read check word");
        CK(c, cudaStreamSynchronize(c->stream), "sync host fields");
        if (bad != ~0ull) return fail(c, LBM_E_INVALID, "rho[%lld] is not a positive finite number", (long long)bad);
        return lbm_init_density_device(c, dev, ux ? dev + fb : nullptr, uy ? dev + 2 * fb : nullptr);
    }
    std::vector<long long> bad(33, -1);   // first bad index per chunk, the lowest reported
    {
        const long long n = c->n;
        const long long chunk = (n + 31) / 32;
        parallel_for(32, [&](long long lo, long long hi) {
            for (long long t = lo; t < hi; ++t)
                for (long long i = t * chunk; i < std::min(n, (t + 1) * chunk); ++i)
                    if (!(rho[i] > 0) || !std::isfinite(rho[i])) {
                        bad[t] = i;
                        break;
                    }
        });
    }
    for (long long i : bad)
        if (i >= 0) return fail(c, LBM_E_INVALID, "rho[%lld] is not a positive finite number", i);
    lbm_status st = ensure_mom(c);
    if (st != LBM_OK) return st;
    char *dev = (char *)c->mom;
    size_t fb = c->n * c->esz;
    const double *src[3] = {rho, ux, uy};
    if (!is_f64(c) && (st = ensure_stage(c, 3 * fb)) != LBM_OK) return st;
    CK(c, cudaStreamSynchronize(c->stream), "sync before staging");  // stage may still feed an earlier copy
    for (int k = 0; k < 3; ++k) {
        if (!src[k]) continue;
        if (is_f64(c)) {
            CK(c, cudaMemcpyAsync(dev + k * fb, src[k], fb, cudaMemcpyHostToDevice, c->stream), "copy init field");
        } else {
            float *h = (float *)c->stage + k * c->n;
            convert(h, src[k], c->n);
            CK(c, cudaMemcpyAsync(dev + k * fb, h, fb, cudaMemcpyHostToDevice, c->stream), "copy init field");
        }
    }
    return lbm_init_density_device(c, dev, ux ? dev + fb : nullptr, uy ? dev + 2 * fb : nullptr);
}

lbm_status lbm_set_f(lbm_ctx *c, const double *f) {
    if (!c) return LBM_E_INVALID;
    if (!f) return fail(c, LBM_E_INVALID, "f is NULL");
    size_t cnt = (size_t)kQ * c->n;
    c->cur = 0;
    if (is_f64(c)) {
        CK(c, cudaMemcpyAsync(c->f[0], f, cnt * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy f");
        CK(c, cudaStreamSynchronize(c->stream), "sync f copy");
    } else {
        lbm_status st = ensure_stage(c, cnt * sizeof(float));
        if (st != LBM_OK) return st;
        CK(c, cudaStreamSynchronize(c->stream), "sync before staging");
        float *h = (float *)c->stage;
        convert(h, f, (long long)cnt);
        CK(c, cudaMemcpyAsync(c->f[0], h, cnt * sizeof(float), cudaMemcpyHostToDevice, c->stream), "copy f");
        CK(c, cudaStreamSynchronize(c->stream), "sync f copy");
    }
    return mark_initialized(c);
}

lbm_status lbm_get_f(lbm_ctx *c, double *f) {
    lbm_status st = check_ready(c);
    if (st != LBM_OK) return st;
    if (!f) return fail(c, LBM_E_INVALID, "f is NULL");
    size_t cnt = (size_t)kQ * c->n;
    if (is_f64(c)) {
        CK(c, cudaMemcpyAsync(f, c->f[c->cur], cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy f");
        CK(c, cudaStreamSynchronize(c->stream), "sync f copy");
    } else {
        lbm_status st2 = ensure_stage(c, cnt * sizeof(float));
        if (st2 != LBM_OK) return st2;
        float *h = (float *)c->stage;
        CK(c, cudaMemcpyAsync(h, c->f[c->cur], cnt * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "copy f");
        CK(c, cudaStreamSynchronize(c->stream), "sync f copy");
        convert(f, h, (long long)cnt);
    }
    return read_error_word(c);
}

}  // extern "C"

namespace {

// ---- saved states (lbm_save / lbm_load) ----
// File: a fixed header, the current distributions in the storage precision
// (nine planes of nx ny), for single-pass contexts the padded stencil field
// the next step reads, and a checksum of those bytes.
struct StateHeader {
    char magic[8];            // "LBMSTAT1"
    int32_t nx, ny, prec, eos, force, grad, hdm_radius, flags;
    double a, b, R, omega, Tr, Tc, k, tau, G, rho0;
    int64_t f_bytes, q_bytes;   // q_bytes 0: no stencil field saved
};
static_assert(sizeof(StateHeader) == 8 + 8 * 4 + 10 * 8 + 2 * 8, "fixed layout");
const char kStateMagic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', '1'};

// FNV-1a over 64 chunks (hashed in parallel), then over the chunk hashes.
uint64_t state_checksum(const unsigned char *p, size_t n) {
    constexpr int kChunks = 64;
    uint64_t h[kChunks];
    parallel_for(kChunks * (1LL << 20), [&](long long lo, long long hi) {
        for (long long k = lo >> 20; k < ((hi + (1LL << 20) - 1) >> 20) && k < kChunks; ++k) {
            const size_t a = n * k / kChunks, b = n * (k + 1) / kChunks;
            uint64_t x = 1469598103934665603ull;
            for (size_t i = a; i < b; ++i) x = (x ^ p[i]) * 1099511628211ull;
            h[k] = x;
        }
    });
    uint64_t x = 1469598103934665603ull;
    for (int k = 0; k < kChunks; ++k)
        for (int byte = 0; byte < 8; ++byte) x = (x ^ ((h[k] >> (8 * byte)) & 0xff)) * 1099511628211ull;
    return x;
}

// The parameters the saved stencil field depends on match the context's.
bool same_physics(const StateHeader &h, const lbm_params &p) {
    return h.eos == p.eos && h.force == p.force && h.grad == p.grad && h.hdm_radius == p.hdm_radius &&
           (h.flags & LBM_FLAG_WALLS_Y) == (p.flags & LBM_FLAG_WALLS_Y) && h.a == p.a && h.b == p.b && h.R == p.R &&
           h.omega == p.omega && h.Tr == p.Tr && h.Tc == p.Tc && h.k == p.k && h.G == p.G && h.rho0 == p.rho0;
}

}  // namespace

extern "C" {

lbm_status lbm_save(lbm_ctx *c, const char *path) {
    lbm_status st = check_ready(c);
    if (st != LBM_OK) return st;
    if (!path) return fail(c, LBM_E_INVALID, "path is NULL");
    if ((st = read_error_word(c)) != LBM_OK) return st;   // no state of a lattice in the error state
    StateHeader h{};
    std::memcpy(h.magic, kStateMagic, sizeof(h.magic));
    const lbm_params &p = c->p;
    h.nx = p.nx; h.ny = p.ny; h.prec = p.prec; h.eos = p.eos; h.force = p.force; h.grad = p.grad;
    h.hdm_radius = p.hdm_radius; h.flags = p.flags;
    h.a = p.a; h.b = p.b; h.R = p.R; h.omega = p.omega; h.Tr = p.Tr; h.Tc = p.Tc; h.k = p.k; h.tau = p.tau;
    h.G = p.G; h.rho0 = p.rho0;
    h.f_bytes = (int64_t)kQ * c->n * c->esz;
    h.q_bytes = c->fused && c->qpad_valid ? (int64_t)sizeof(float) * fused_q_pitch(p.nx) * p.ny : 0;
    if ((st = ensure_stage(c, h.f_bytes + h.q_bytes)) != LBM_OK) return st;
    unsigned char *buf = (unsigned char *)c->stage;
    CK(c, cudaMemcpyAsync(buf, c->f[c->cur], h.f_bytes, cudaMemcpyDeviceToHost, c->stream), "copy f");
    if (h.q_bytes)
        CK(c, cudaMemcpyAsync(buf + h.f_bytes, c->qpad[c->cur], h.q_bytes, cudaMemcpyDeviceToHost, c->stream),
           "copy stencil field");
    CK(c, cudaStreamSynchronize(c->stream), "sync state copy");
    const uint64_t sum = state_checksum(buf, h.f_bytes + h.q_bytes);
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(c, LBM_E_IO, "cannot open %s for writing", path);
    const bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 &&
                    std::fwrite(buf, 1, h.f_bytes + h.q_bytes, fp) == (size_t)(h.f_bytes + h.q_bytes) &&
                    std::fwrite(&sum, sizeof(sum), 1, fp) == 1;
    if (std::fclose(fp) != 0 || !ok) return fail(c, LBM_E_IO, "writing %s failed", path);
    return LBM_OK;
}

lbm_status lbm_load(lbm_ctx *c, const char *path) {
    if (!c) return LBM_E_INVALID;
    if (!path) return fail(c, LBM_E_INVALID, "path is NULL");
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(c, LBM_E_IO, "cannot open %s", path);
    StateHeader h{};
    auto close_fail = [&](lbm_status s2, const char *why) {
        std::fclose(fp);
        return fail(c, s2, "%s: %s", path, why);
    };
    if (std::fread(&h, sizeof(h), 1, fp) != 1 || std::memcmp(h.magic, kStateMagic, sizeof(h.magic)) != 0)
        return close_fail(LBM_E_IO, "not a saved lattice state");
    if (h.nx != c->p.nx || h.ny != c->p.ny || h.prec != c->p.prec)
        return close_fail(LBM_E_INVALID, "lattice size or precision differs from the context's");
    const int64_t fb = (int64_t)kQ * c->n * c->esz;
    const int64_t qb_expected = (int64_t)sizeof(float) * fused_q_pitch(c->p.nx) * c->p.ny;
    if (h.f_bytes != fb || (h.q_bytes != 0 && (h.prec != LBM_F32 || h.q_bytes != qb_expected)))
        return close_fail(LBM_E_IO, "inconsistent header");
    lbm_status st = ensure_stage(c, h.f_bytes + h.q_bytes);
    if (st != LBM_OK) {
        std::fclose(fp);
        return st;
    }
    CK(c, cudaStreamSynchronize(c->stream), "sync before staging");
    unsigned char *buf = (unsigned char *)c->stage;
    uint64_t sum = 0;
    if (std::fread(buf, 1, h.f_bytes + h.q_bytes, fp) != (size_t)(h.f_bytes + h.q_bytes) ||
        std::fread(&sum, sizeof(sum), 1, fp) != 1)
        return close_fail(LBM_E_IO, "truncated");
    std::fclose(fp);
    if (sum != state_checksum(buf, h.f_bytes + h.q_bytes)) return fail(c, LBM_E_IO, "%s: checksum mismatch", path);
    c->cur = 0;
    CK(c, cudaMemcpyAsync(c->f[0], buf, h.f_bytes, cudaMemcpyHostToDevice, c->stream), "copy f");
    // the saved stencil field where this context reads one and the physics
    // matches (a resumed run then repeats the uninterrupted one bit for bit);
    // else the next step forms it from f
    const bool use_q = h.q_bytes != 0 && c->fused && same_physics(h, c->p);
    if (use_q)
        CK(c, cudaMemcpyAsync(c->qpad[0], buf + h.f_bytes, h.q_bytes, cudaMemcpyHostToDevice, c->stream),
           "copy stencil field");
    CK(c, cudaStreamSynchronize(c->stream), "sync state copy");
    st = mark_initialized(c);
    c->qpad_valid = use_q;
    return st;
}

lbm_status lbm_step(lbm_ctx *c, int nsteps) {
    NvtxRange nvtx("lbm_step");
    lbm_status st = check_ready(c);
    if (st != LBM_OK) return st;
    if (nsteps < 0) return fail(c, LBM_E_INVALID, "nsteps must be >= 0");
    if (is_f64(c)) {
        Model<double> m = model_of<double>(c);
        for (int s = 0; s < nsteps; ++s) CK(c, step_once<double>(c, m), "step");
    } else if (c->fused) {
        Model<float> m = model_of<float>(c);
        for (int s = 0; s < nsteps; ++s) CK(c, step_fused(c, m), "fused step");
    } else if (c->p.flags & LBM_FLAG_F32_ARITH) {
        Model<float> m = model_of<float>(c);
        for (int s = 0; s < nsteps; ++s) CK(c, step_once<float>(c, m), "step");
    } else {
        Model<double> m = model_of<double>(c);
        for (int s = 0; s < nsteps; ++s) CK(c, step_once_mixed(c, m), "step");
    }
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx *c) {
    if (!c) return LBM_E_INVALID;
    return read_error_word(c);
}

lbm_status lbm_moments_device(lbm_ctx *c, void *rho, void *vx, void *vy) {
    lbm_status st = check_ready(c);
    if (st != LBM_OK) return st;
    if (!rho || !vx || !vy) return fail(c, LBM_E_INVALID, "rho, vx, vy must be non-NULL device arrays");
    cudaError_t e = is_f64(c) ? moments_into<double>(c, (double *)rho, (double *)vx, (double *)vy)
                              : moments_into<float>(c, (float *)rho, (float *)vx, (float *)vy);
    CK(c, e, "moments kernel");
    return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx *c, double *rho, double *vx, double *vy) {
    lbm_status st = check_ready(c);
    if (st != LBM_OK) return st;
    if (!rho) return fail(c, LBM_E_INVALID, "rho is NULL");
    if ((st = ensure_mom(c)) != LBM_OK) return st;
    char *dev = (char *)c->mom;
    size_t fb = c->n * c->esz;
    double *dst[3] = {rho, vx, vy};
    bool in_place = c->direct_host;   // every page of the caller's arrays resident: the device writes them
    for (int k = 0; k < 3 && in_place; ++k)
        if (dst[k]) in_place = pages_resident(dst[k], c->n * sizeof(double));
    if ((st = lbm_moments_device(c, dev, dev + fb, dev + 2 * fb)) != LBM_OK) return st;
    if (in_place) {
        for (int k = 0; k < 3; ++k) {
            if (!dst[k]) continue;
            cudaError_t e = is_f64(c) ? launch_to_host<double>((const double *)(dev + k * fb), dst[k], c->n, c->stream)
                                      : launch_to_host<float>((const float *)(dev + k * fb), dst[k], c->n, c->stream);
            CK(c, e, "write host field");
        }
        CK(c, cudaStreamSynchronize(c->stream), "sync moments");
        return read_error_word(c);
    }
    if (is_f64(c)) {
        for (int k = 0; k < 3; ++k)
            if (dst[k]) CK(c, cudaMemcpyAsync(dst[k], dev + k * fb, fb, cudaMemcpyDeviceToHost, c->stream), "copy moments");
        CK(c, cudaStreamSynchronize(c->stream), "sync moments");
    } else {
        if ((st = ensure_stage(c, 3 * fb)) != LBM_OK) return st;
        float *h = (float *)c->stage;
        // field k is converted on the host while field k + 1 is still copied
        cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            if (!dst[k]) continue;
            e = cudaMemcpyAsync(h + k * c->n, dev + k * fb, fb, cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = take_event(c, &ev[k]);
            if (e == cudaSuccess) e = cudaEventRecord(ev[k], c->stream);
        }
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            if (!dst[k]) continue;
            e = cudaEventSynchronize(ev[k]);
            if (e == cudaSuccess) convert(dst[k], h + k * c->n, c->n);
        }
        for (cudaEvent_t x : ev)
            if (x) c->event_pool.push_back(x);
        CK(c, e, "copy moments");
    }
    return read_error_word(c);
}

lbm_status lbm_gradient(lbm_ctx *c, const double *q, double h, double *gx, double *gy) {
    if (!c) return LBM_E_INVALID;
    if (!q || !gx || !gy) return fail(c, LBM_E_INVALID, "q, gx and gy must be non-NULL host arrays");
    if (!(h > 0) || !std::isfinite(h)) return fail(c, LBM_E_INVALID, "grid spacing h must be positive and finite");
    lbm_status st = ensure_mom(c);
    if (st != LBM_OK) return st;
    char *dev = (char *)c->mom;
    const size_t fb = c->n * c->esz;
    if (is_f64(c)) {
        CK(c, cudaMemcpyAsync(dev, q, fb, cudaMemcpyHostToDevice, c->stream), "copy field");
        CK(c, launch_gradient<double>(model_of<double>(c), is_cdm(c), (const double *)dev, h, (double *)(dev + fb),
                                      (double *)(dev + 2 * fb), c->stream), "gradient kernel");
        CK(c, cudaMemcpyAsync(gx, dev + fb, fb, cudaMemcpyDeviceToHost, c->stream), "copy gradient");
        CK(c, cudaMemcpyAsync(gy, dev + 2 * fb, fb, cudaMemcpyDeviceToHost, c->stream), "copy gradient");
        CK(c, cudaStreamSynchronize(c->stream), "sync gradient");
    } else {
        if ((st = ensure_stage(c, 3 * fb)) != LBM_OK) return st;
        CK(c, cudaStreamSynchronize(c->stream), "sync before staging");
        float *hs = (float *)c->stage;
        convert(hs, q, c->n);
        CK(c, cudaMemcpyAsync(dev, hs, fb, cudaMemcpyHostToDevice, c->stream), "copy field");
        CK(c, launch_gradient<float>(model_of<float>(c), is_cdm(c), (const float *)dev, (float)h, (float *)(dev + fb),
                                     (float *)(dev + 2 * fb), c->stream), "gradient kernel");
        CK(c, cudaMemcpyAsync(hs + c->n, dev + fb, 2 * fb, cudaMemcpyDeviceToHost, c->stream), "copy gradient");
        CK(c, cudaStreamSynchronize(c->stream), "sync gradient");
        convert(gx, hs + c->n, c->n);
        convert(gy, hs + 2 * c->n, c->n);
    }
    return LBM_OK;
}

lbm_status lbm_observables(lbm_ctx *c, lbm_obs *out) {
    lbm_status st = check_ready(c);
    if (st != LBM_OK) return st;
    if (!out) return fail(c, LBM_E_INVALID, "out is NULL");
    if ((st = ensure_mom(c)) != LBM_OK) return st;
    char *dev = (char *)c->mom;
    size_t fb = c->n * c->esz;
    if ((st = lbm_moments_device(c, dev, dev + fb, dev + 2 * fb)) != LBM_OK) return st;
    cudaError_t e = is_f64(c) ? launch_observables<double>(c->n, (double *)dev, (double *)(dev + fb),
                                                           (double *)(dev + 2 * fb), c->partial, c->obs_dev, c->stream)
                              : launch_observables<float>(c->n, (float *)dev, (float *)(dev + fb),
                                                          (float *)(dev + 2 * fb), c->partial, c->obs_dev, c->stream);
    CK(c, e, "observables kernel");
    CK(c, cudaMemcpyAsync(out, c->obs_dev, sizeof(lbm_obs), cudaMemcpyDeviceToHost, c->stream), "copy observables");
    return read_error_word(c);
}

lbm_status lbm_set_timing(lbm_ctx *c, int enable) {
    if (!c) return LBM_E_INVALID;
    if (enable) {
        CK(c, resolve_timing(c), "resolve timing events");
        c->tm = lbm_timing{};
    }
    c->timing = enable != 0;
    return LBM_OK;
}

lbm_status lbm_get_timing(lbm_ctx *c, lbm_timing *out) {
    if (!c) return LBM_E_INVALID;
    if (!out) return fail(c, LBM_E_INVALID, "out is NULL");
    CK(c, resolve_timing(c), "resolve timing events");
    *out = c->tm;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    dev_free(c->f[0]);
    dev_free(c->f[1]);
    dev_free(c->q);
    dev_free(c->qpad[0]);
    dev_free(c->qpad[1]);
    dev_free(c->mom);
    dev_free(c->partial);
    dev_free(c->obs_dev);
    dev_free(c->err);
    free_tape(c);
    if (c->stage) host_free(c->stage);
    for (auto &p : c->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto ev : c->event_pool) cudaEventDestroy(ev);
    delete c;
}

const char *lbm_last_error(const lbm_ctx *c) {
    return c ? c->msg.c_str() : g_create_error.c_str();
}

int lbm_host_in_place(const lbm_ctx *c) { return c ? (c->direct_host ? 1 : 0) : -1; }

}  // extern "C"
