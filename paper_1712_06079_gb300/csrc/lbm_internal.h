// Internal (C++) launch interface between the C ABI and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "nvtx3/nvToolsExt.h"

namespace lbm {

// An NVTX range over a scope (named in a profiler's timeline; no cost when no
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Host-side scalars of a parameter set.  With an equation of state: T = Tr Tc
// (Tc = p.Tc, or from lbm_critical_point), a, b, a alpha(T) and its
// T-derivative (Eq. 27, 28), k, R T.  With the effective mass of Eq. 4
// (LBM_EOS_PSI_EXP): a = G/2, b = 1/rho0, k = 1, the rest 0 -- the device
// potential is then U = a (1 - exp(-b rho))^2 (Eq. 5 minus rho c_s^2).
struct ModelScalars {
    double T, Tc, a, b, aal, aalp, k, RT;
};
// Range checks of a parameter set shared by every entry point; returns
// LBM_E_INVALID with a reason in *why.
lbm_status check_params(const lbm_params &p, const char **why);
lbm_status model_scalars(const lbm_params &p, ModelScalars *s);

// Every device and pinned-host allocation of the library goes through these
// (alloc.cpp): a registry of live allocations and the allocation-failure
// injection of LBM_DEBUG_FAIL_ALLOC.
cudaError_t dev_alloc_raw(void **p, size_t bytes);
cudaError_t host_alloc_raw(void **p, size_t bytes);
template <typename P>
cudaError_t dev_alloc(P **p, size_t bytes) {
    return dev_alloc_raw((void **)p, bytes);
}
template <typename P>
cudaError_t host_alloc(P **p, size_t bytes) {
    return host_alloc_raw((void **)p, bytes);
}
void dev_free(void *p);
void host_free(void *p);

// f = f^eq(rho, u) (Eq. 2); ux/uy may be null (zero velocity).
template <typename T>
cudaError_t launch_init(const Model<T> &m, const T *rho, const T *ux, const T *uy, T *f, cudaStream_t s);
// n FP64 values of a pageable host array read by the device in place and
// converted to T; only on devices that access pageable memory through the
// host's page tables.  bad (optional): receives the lowest index of a value
// that is not a positive finite number (atomicMin, preset all ones).
template <typename T>
cudaError_t launch_from_host(const double *src, T *dst, long long n, unsigned long long *bad, cudaStream_t s);
// n values of T written as FP64 into a resident pageable host array in place
// (same devices).
template <typename T>
cudaError_t launch_to_host(const T *src, double *dst, long long n, cudaStream_t s);

// Pass 1 of a step: rho = sum_i f_i (Eq. 3) and the potential field
// (Eq. 8 / Eq. 21) into q; flags NaN or rho <= 0 in *err.
template <typename T>
cudaError_t launch_potential(const Model<T> &m, bool sc, const T *f, T *q, int *err, cudaStream_t s);

// Pass 2 of a step: HDM (Eq. 20) or CDM (Eq. 15) gradient of q, force
// (Eq. 22 / Eq. 7), exact-difference forcing + BGK (Eq. 1, 10) and periodic
// push streaming from f into fout.
template <typename T>
cudaError_t launch_collide(const Model<T> &m, bool sc, bool cdm, const T *f, const T *q, T *fout, cudaStream_t s);

// rho (Eq. 3) and the half-step velocity v (Eq. 11) of state f with its q.
template <typename T>
cudaError_t launch_moments(const Model<T> &m, bool sc, bool cdm, const T *f, const T *q, T *rho, T *vx, T *vy,
                           cudaStream_t s);

// The same three launches for FP32-stored distributions with FP64 arithmetic
// and an FP64 potential field q (the two-pass form of FP32 lattices); rho, vx,
// vy are rounded to FP32 on output.
cudaError_t launch_potential_mixed(const Model<double> &m, bool sc, const float *f, double *q, int *err,
                                   cudaStream_t s);
cudaError_t launch_collide_mixed(const Model<double> &m, bool sc, bool cdm, const float *f, const double *q,
                                 float *fout, cudaStream_t s);
cudaError_t launch_moments_mixed(const Model<double> &m, bool sc, bool cdm, const float *f, const double *q,
                                 float *rho, float *vx, float *vy, cudaStream_t s);

// HDM (Eq. 20) or CDM (Eq. 15 times 1/c_s^2) gradient of the periodic field
// q (nx * ny, row-major) on a grid of spacing h into gx, gy.
template <typename T>
cudaError_t launch_gradient(const Model<T> &m, bool cdm, const T *q, T h, T *gx, T *gy, cudaStream_t s);

// FP64 reductions of (rho, vx, vy) over n cells into *out (device memory).
// partial must hold observables_partial_count() * 6 doubles.
int observables_partial_count();
template <typename T>
cudaError_t launch_observables(long long n, const T *rho, const T *vx, const T *vy, double *partial, lbm_obs *out,
                               cudaStream_t s);

// Single-pass FP32 step (fused_step.cu): reads f(t) and the padded potential
// q(t), writes f(t+1) and the padded potential of f(t+1).  The padded
// potential has fused_q_pitch(nx) floats per row, column x stored at x + 32,
// with periodic images in the 32 ghost columns on each side.  A CTA sweeps a
// segment of seg_rows rows of a 120-column strip; fused_auto_seg_rows picks
// the segment height for a lattice on a GPU with num_sms SMs.
bool fused_step_supported(const Model<float> &m, bool cdm, int radius);
int fused_q_pitch(int nx);
int fused_auto_seg_rows(int nx, int ny, int num_sms);
cudaError_t launch_potential_padded(const Model<float> &m, bool sc, const float *f, float *qpad, int *err,
                                    cudaStream_t s);
// pdl: launch with programmatic serialization (the grid may be scheduled while
// the previous one drains; it waits for it before any access).  rec (periodic
// HDM lattices only): also write the reverse mode's record of f(t), five planes of
// nx ny floats: rho, jx, jy and the HDM derivatives Dx, Dy of the stencil field.
// rev: the CTAs take the strips and segments in reverse order (results are the
// same either way; alternated step by step, the first CTAs of a step read the
// rows the last CTAs of the previous step wrote, while they are still in L2).
cudaError_t launch_fused_step(const Model<float> &m, bool sc, bool cdm, const float *f, const float *qin,
                              float *fout, float *qout, int *err, int seg_rows, cudaStream_t s, bool pdl = true,
                              float *rec = nullptr, bool rev = false);

// Adjoint (reverse-time) step (adjoint.cu): from lambda = dL/df at t+1 and the
// state f at t with its stencil field q (row y, column x at
// q[y * qpitch + qoff + x]; |q| = Phi for the Shan-Chen form, U for
// Zhang-Chen), writes lambda at t into lam_out and adds the step's dL/dT to
// the FP64 slots Tpart[0 .. adjoint_slots).  In the padded layout f is not
// the state but the single-pass kernel's record of it (rho, jx, jy, Dx, Dy:
// five planes of nx ny).  lambda has nine fields, or three
// (rho_bar, jx_bar, jy_bar with lambda_i = rho_bar + e_i . j_bar) when tau1;
// aux holds naux scratch fields.  Field k, row y, column x of lambda / aux
// sits at [k * stride + y * pitch + off + x] as adjoint_layout gives: padded
// rows with 32 periodic ghost columns on each side for the FP32 single-pass
// layout (padded = true: q in that layout, nx % 4 == 0, nx >= 64, HDM radius
// 26), plain rows otherwise.  R is the gas constant, aalp = a dalpha/dT; err
// receives kErrTimeout if a bounded wait on a copy gives up.  overlap_prev:
// the preceding launch on the stream is the previous reverse step's kernel B
// (not a kernel that wrote f or q), so in the padded layout this step's first
// kernel may start while it finishes.
struct AdjLayout {
    int dpitch, doff, naux;
    long long dstride;
    int lpitch, loff, nlam;
    long long lstride;
};
AdjLayout adjoint_layout(int nx, int ny, bool padded, bool tau1);
template <typename T>
int adjoint_slots(int nx, int ny);
template <typename T>
cudaError_t launch_adjoint_step(const Model<T> &m, T R, T aalp, bool sc, bool cdm, bool tau1, bool padded,
                                const AdjLayout &l, const T *f, const T *q, int qpitch, int qoff, const T *lam_next,
                                T *aux, T *lam_out, double *Tpart, int *err, bool overlap_prev, cudaStream_t s);
// lambda at the final step from dL/drho_T (rho_T = sum_i f_i).
template <typename T>
cudaError_t launch_adjoint_seed(int nx, int ny, bool padded, const AdjLayout &l, const T *grad_rho, T *lam,
                                int *err, cudaStream_t s);
// dL/drho0 = sum_i w_i lambda_i at t = 0 (f = f^eq(rho0, 0)).
template <typename T>
cudaError_t launch_adjoint_initial(int nx, int ny, const AdjLayout &l, const T *lam, T *grad_rho0, int *err,
                                  cudaStream_t s);
// *out = sum of nslots doubles in index order (one thread).
cudaError_t launch_sum_slots(const double *slots, int nslots, double *out, cudaStream_t s);
template <typename T>
cudaError_t launch_density(long long n, const T *f, T *rho, cudaStream_t s);

}  // namespace lbm
