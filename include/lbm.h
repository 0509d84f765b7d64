/*
 * lbm.h -- C ABI of the GB300 (sm_103a) D2Q9 pseudopotential lattice
 * Boltzmann step with the high-order-difference (HDM) interaction force of
 * Qin, Zhao, Chen, Zhang & Wen, "A pseudopotential multiphase lattice
 * Boltzmann model based on high-order difference" (arXiv:1712.06079).
 *
 * One time step (Sec. 2 and Sec. 4 of the paper) is
 *   rho = sum_i f_i, rho u = sum_i e_i f_i                        (Eq. 3)
 *   p = k p_EOS(rho, T)  (Hu scaling, Sec. 5; EOS Eq. 24, 27-29)
 *   U = p - rho c_s^2 (Eq. 8),  Phi = sqrt|U| (Eq. 21)
 *   grad by the HDM compact scheme of Eq. 20 (or the CDM of Eq. 15)
 *   F = -2 s Phi grad Phi (Shan-Chen form, Eq. 22; s = sign U at the cell)
 *     or F = -grad U      (Zhang-Chen form, Eq. 7)
 *   f_i* = f_i - (f_i - f_i^eq(rho,u))/tau
 *          + f_i^eq(rho, u + F/rho) - f_i^eq(rho, u)           (Eq. 1, 2, 10)
 *   f_i(x + e_i, t+1) = f_i*(x)  on a lattice periodic in x and y  (Eq. 1),
 *     or periodic in x with half-way bounce-back walls in y (LBM_FLAG_WALLS_Y)
 *
 * Conventions shared by every entry point:
 *  - Fields are row-major, x fastest: index = y * nx + x, nx * ny entries.
 *  - Distributions are SoA: f[i * nx*ny + y*nx + x], i = 0..8 in the order
 *    rest, +x, +y, -x, -y, (+1,+1), (-1,+1), (-1,-1), (+1,-1).
 *  - "host" arrays are caller-owned CPU memory, copied in or out before the
 *    call returns; "device" arrays are caller-owned CUDA device memory of the
 *    context's precision (float for LBM_F32, double for LBM_F64), used on the
 *    context's stream without synchronisation.
 *  - The context owns all device memory it allocates; lbm_destroy frees it.
 *  - Errors are status codes, never exceptions or aborts.  A failed call
 *    leaves a message retrievable by lbm_last_error.  A context whose device
 *    error word reports instability (NaN or rho <= 0) answers
 *    LBM_E_UNSTABLE to lbm_step until it is re-initialised.
 *  - Work is queued on params.stream (a cudaStream_t; NULL = the legacy
 *    default stream).  lbm_step is asynchronous; lbm_sync, lbm_moments,
 *    lbm_get_f and lbm_observables synchronise the stream and check the
 *    device error word.
 */
#ifndef LBM_H
#define LBM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;
typedef struct lbm_batch lbm_batch;

typedef enum {
    LBM_OK = 0,
    LBM_E_INVALID = 1,  /* bad argument (null pointer, size, parameter range) */
    LBM_E_NOMEM = 2,    /* device or host allocation failed */
    LBM_E_CUDA = 3,     /* a CUDA runtime call failed */
    LBM_E_UNSTABLE = 4, /* the device error word saw a NaN or rho <= 0 */
    LBM_E_TIMEOUT = 5,  /* a bounded device-side wait gave up */
    LBM_E_STATE = 6,    /* call out of order (e.g. step before init) */
    LBM_E_IO = 7        /* a saved-state file could not be written or read, or is not one */
} lbm_status;

/* Equations of state (Sec. 5.2): van der Waals (Eq. 24), Carnahan-Starling
 * (Eq. 29, with the standard (1 - b rho/4)^3 denominator), Peng-Robinson
 * (Eq. 28), Redlich-Kwong with alpha = 1/sqrt(T) (Eq. 27) and its Soave form
 * (alpha(T) given after Eq. 27).  LBM_EOS_PSI_EXP is the original Shan-Chen
 * model instead (Eq. 4-5): effective mass psi = 1 - exp(-rho/rho0), force
 * F = -G psi grad psi, pressure p = rho/3 + (G/2) psi^2; it has no
 * temperature, critical point or Hu factor (Tr, Tc, a, b, R, omega, k unused). */
typedef enum {
    LBM_EOS_VDW = 0,
    LBM_EOS_CS = 1,
    LBM_EOS_PR = 2,
    LBM_EOS_RK = 3,
    LBM_EOS_RKS = 4,
    LBM_EOS_PSI_EXP = 5
} lbm_eos;
/* Interaction form: Shan-Chen effective mass (Eq. 4 rewritten as Eq. 22) or
 * Zhang-Chen potential (Eq. 7 with U of Eq. 8). */
typedef enum { LBM_FORCE_SC = 0, LBM_FORCE_ZC = 1 } lbm_force;
/* Gradient operator: HDM compact scheme (Eq. 20) or weighted CDM (Eq. 15). */
typedef enum { LBM_GRAD_HDM = 0, LBM_GRAD_CDM = 1 } lbm_grad;
typedef enum { LBM_F32 = 0, LBM_F64 = 1 } lbm_prec;
/* LBM_FLAG_TWO_PASS: never use the single-pass FP32 step kernel (keep the
 * potential pass + collide pass form even where the fused kernel applies).
 * The single-pass kernel takes LBM_F32 lattices with nx a multiple of 4,
 * nx >= 64 and ny >= 54, with the HDM at radius 26 or with the CDM, periodic
 * or walled.
 * LBM_FLAG_WALLS_Y: no-slip walls half a lattice spacing below row 0 and above
 * row ny-1 instead of periodicity in y (the splash case of Sec. 5.5; x stays
 * periodic).  The paper gives no wall closures; the library takes half-way
 * bounce-back (a population that would cross a wall returns to its node,
 * reversed) and continues the interaction field across each wall by its mirror
 * image (zero normal gradient), so Eq. 20 along a column is the periodic
 * operator of the mirrored column of period 2 ny and Eq. 15 reads mirrored
 * neighbours.  Walled FP32 lattices that the single-pass kernel takes run it
 * (mirrored rows in its staging, bounce-back at the wall rows); the others,
 * FP64 and lbm_step_noalloc run the two-pass kernels; the batch and the
 * reverse mode reject walls (LBM_E_INVALID). */
/* LBM_FLAG_F32_ARITH: an LBM_F32 lattice that runs the two-pass kernels
 * computes in FP32 there too instead of FP64 (faster where FP64 is slow, as
 * on GB300; the FP32 1000-step field bar is met only with FP64 arithmetic
 * there).  No effect on the single-pass kernel, which computes in FP32. */
/* LBM_FLAG_STAGED_HOST: the host arrays of lbm_init_density and lbm_moments
 * pass through the library's pinned staging buffer (checked and converted by
 * host threads, one DMA copy each way) even on a device that accesses pageable
 * host memory through the host's page tables (Grace with NVLink-C2C).  There,
 * by default, the device reads lbm_init_density's FP64 arrays in place,
 * checking and converting them itself, and writes lbm_moments' FP64 arrays in
 * place when every page of them is resident (an array written before, as a
 * reused buffer is; fresh pages are populated faster by the host threads of
 * the staging path).  All give the same values and errors. */
enum { LBM_FLAG_TWO_PASS = 1, LBM_FLAG_WALLS_Y = 2, LBM_FLAG_F32_ARITH = 4, LBM_FLAG_STAGED_HOST = 8 };

typedef struct {
    int nx, ny;      /* lattice size, >= 1 each, periodic in both axes (Sec. 5.2)
                        unless flags has LBM_FLAG_WALLS_Y */
    int prec;        /* lbm_prec: storage precision of f.  LBM_F64 computes
                        in FP64; LBM_F32 computes in FP32 in the single-pass
                        kernel and in FP64 in the two-pass kernels (every
                        lattice the single-pass kernel does not take) unless
                        flags has LBM_FLAG_F32_ARITH */
    int eos;         /* lbm_eos */
    int force;       /* lbm_force */
    int grad;        /* lbm_grad */
    int hdm_radius;  /* truncation radius K of the explicit form of Eq. 20;
                        0 = automatic (26 for F32, 40 for F64); max 48 */
    int flags;       /* bit set of LBM_FLAG_* (0 = defaults) */
    double a, b, R;  /* EOS constants (Sec. 5.2: a = 9/49, b = 2/21 VdW; a = 1,
                        b = 4 CS; R = 1) */
    double omega;    /* acentric factor for PR and RKS (0.344 water) */
    double Tr;       /* reduced temperature T/Tc, > 0 */
    double Tc;       /* critical temperature; 0 = computed by lbm_critical_point */
    double k;        /* Hu scaling p = k p_EOS (Sec. 5; 0.01 VdW, 0.02 RK,
                        0.04 PR and CS in Sec. 5.2) */
    double tau;      /* BGK relaxation time (Eq. 1), > 0.5 */
    double G;        /* LBM_EOS_PSI_EXP: interaction strength of Eq. 4, < 0
                        (phase separation below G = -4 rho0 / 3) */
    double rho0;     /* LBM_EOS_PSI_EXP: reference density of psi, > 0 */
    void *stream;    /* cudaStream_t for all work of this context, or NULL */
} lbm_params;

/* FP64 reductions over the lattice (Sec. 5.2 coexistence, Sec. 5.4 spurious
 * currents).  v is the half-step velocity of Eq. 11. */
typedef struct {
    double mass;       /* sum_x rho */
    double mom_x;      /* sum_x rho v_x */
    double mom_y;      /* sum_x rho v_y */
    double max_speed;  /* max_x |v| */
    double rho_min, rho_max;
} lbm_obs;

/* Device-time accounting of lbm_step, for roofline measurements.  When
 * enabled, lbm_step records a CUDA event pair on the context's stream around
 * every kernel it launches; lbm_get_timing synchronises and sums them.  The
 * kernel slots are: 0 potential pass, 1 force/collide/stream pass, 2 fused
 * single-pass step, 3 unused. */
typedef struct {
    long long steps;            /* steps issued while timing was enabled */
    long long launches;         /* kernels launched by lbm_step while enabled */
    double ms_kernel[4];        /* summed device time per kernel slot */
    long long count_kernel[4];  /* launches per kernel slot */
} lbm_timing;

/* Critical point (Tc, rho_c) of an EOS with alpha = 1 (PR, RKS) or
 * alpha = 1/sqrt(T) (RK), i.e. dp/drho = d2p/drho2 = 0 (Sec. 5.2).  Host-only
 * FP64 computation.  Returns LBM_E_INVALID for an unknown EOS or
 * non-positive constants. */
lbm_status lbm_critical_point(int eos, double a, double b, double R, double *Tc, double *rho_c);

/* Coexistence densities of the Maxwell equal-area construction (Sec. 5.2) of
 * the unscaled EOS at T = p->Tr * Tc (Tc = p->Tc, or computed when 0), using
 * p->eos, a, b, R, omega; p_EOS(rho_g) = p_EOS(rho_l) and the p-v areas are
 * equal.  For LBM_EOS_PSI_EXP the same construction on the pressure of Eq. 5
 * (p->G, p->rho0).  Host-only FP64.  LBM_E_INVALID when Tr >= 1 or there is
 * no loop. */
lbm_status lbm_maxwell(const lbm_params *p, double *rho_g, double *rho_l);

/* Weights of the explicit form of the periodic HDM operator (Eq. 20): on a
 * periodic line of n points the solution of the tridiagonal system is
 *   d_i = sum_{j=1..K} w[j] (u_{i+j} - u_{i-j}),
 * with w folded over the period.  Writes w[0..radius] (w[0] = 0) and the
 * effective radius min(radius, (n-1)/2) to *k_eff.  Host-only, FP64. */
lbm_status lbm_hdm_weights(int n, int radius, double *w, int *k_eff);

/* Create a context for one lattice (validates p, resolves Tc, allocates the
 * two distribution buffers, the potential field and reduction scratch on the
 * current CUDA device).  *out is set to NULL on failure. */
lbm_status lbm_create(const lbm_params *p, lbm_ctx **out);

/* f = f^eq(rho, u) (Eq. 2) from host FP64 fields rho (> 0), ux, uy
 * (NULL = zero velocity).  Clears the error state.  Blocks until the copy
 * has been issued and the init kernels are queued. */
lbm_status lbm_init_density(lbm_ctx *c, const double *rho, const double *ux, const double *uy);

/* Same from device arrays of the context precision (ux/uy may be NULL). */
lbm_status lbm_init_density_device(lbm_ctx *c, const void *rho, const void *ux, const void *uy);

/* Set or read the full distribution state f (host FP64, 9*nx*ny entries,
 * SoA as above).  lbm_set_f clears the error state. */
lbm_status lbm_set_f(lbm_ctx *c, const double *f);
lbm_status lbm_get_f(lbm_ctx *c, double *f);

/* Advance nsteps >= 0 time steps (Eq. 1).  Asynchronous on the context's
 * stream.  Returns LBM_E_STATE before any init, LBM_E_UNSTABLE if a previous
 * synchronising call saw the device error word set. */
lbm_status lbm_step(lbm_ctx *c, int nsteps);

/* Wait for the context's stream and check the device error word. */
lbm_status lbm_sync(lbm_ctx *c);

/* Density (Eq. 3) and half-step velocity v (Eq. 11) of the current state into
 * host FP64 arrays (vx, vy may be NULL).  Synchronising. */
lbm_status lbm_moments(lbm_ctx *c, double *rho, double *vx, double *vy);

/* Same into device arrays of the context precision; asynchronous. */
lbm_status lbm_moments_device(lbm_ctx *c, void *rho, void *vx, void *vy);

/* FP64 lattice reductions of the current state.  Synchronising. */
lbm_status lbm_observables(lbm_ctx *c, lbm_obs *out);

/* The context's gradient operator applied to a caller field, with the same
 * device code as the step's interaction (the two-pass kernels' tile stencil):
 * HDM, the periodic solution of Eq. 20 along every row (d/dx) and column
 * (d/dy) as the folded explicit stencil of the context's radius, or CDM, Eq. 15
 * times 1/c_s^2 = 3; both divided by the grid spacing h (the step uses h = 1).
 * With LBM_FLAG_WALLS_Y the columns are closed by the mirror image, as in the
 * step (d/dy of a line of ny points is the periodic operator on 2 ny points).
 * q, gx, gy: host FP64 arrays of nx*ny values, row-major (x fastest), q taken
 * as given (no magnitude, unlike the Shan-Chen field); computed in the
 * context precision (q rounded to FP32 for FP32 contexts).  The lattice state
 * is not touched and need not be initialised.  LBM_E_INVALID for NULL arrays
 * or h <= 0.  Synchronising. */
lbm_status lbm_gradient(lbm_ctx *c, const double *q, double h, double *gx, double *gy);

/* Reverse mode through nsteps steps, for gradients of a function of the final
 * density (e.g. the L2 distance to a target droplet) with respect to the
 * initial density and the model's scalar parameter: the temperature, or the
 * interaction strength G of LBM_EOS_PSI_EXP.  Not a passage of the paper: the
 * adjoint of its step (Eq. 1-3, 7/8, 10, 20-22).
 * lbm_adjoint_forward: f = f^eq(rho0, 0) (Eq. 2) from the device array rho0,
 *   nsteps steps (Eq. 1), density of the final state into the device array
 *   rho_T; the state every checkpoint_interval steps is kept on the device
 *   (checkpoint_interval = ceil(sqrt(nsteps)) gives sqrt(N) checkpointing, 1
 *   keeps every state).  The context is left on the final state.
 * lbm_adjoint_backward: from dL/drho_T (device array) writes dL/drho0 (device
 *   array) and dL/dT, dL/d(T/Tc), dL/dG (host doubles, each may be NULL),
 *   recomputing the states between checkpoints with the same kernels and
 *   running the adjoint step backwards; the scalar gradient is accumulated in
 *   FP64.  Synchronising.
 * All device arrays hold nx*ny values of the context precision.  With an
 * equation of state the interaction strength G of Eq. 4/6 cancels from
 * Eq. 22, so dL/dG = 0; with LBM_EOS_PSI_EXP there is no temperature, so
 * dL/dT = dL/d(T/Tc) = 0 and dL/dG is live. */
lbm_status lbm_adjoint_forward(lbm_ctx *c, const void *rho0, int nsteps, int checkpoint_interval, void *rho_T);
lbm_status lbm_adjoint_backward(lbm_ctx *c, const void *grad_rho_T, void *grad_rho0, double *grad_T, double *grad_Tr,
                                double *grad_G);

/* Launch shape of the single-pass FP32 step (not a passage of the paper): a
 * CTA sweeps `rows` rows of a 120-column strip.  0 (the default) picks the
 * height from the lattice and the device's SM count; 1..ny fixes it.  Results
 * depend on it only through FP32 rounding (the d/dy sums restart at every
 * segment; the same height gives bit-identical results).  LBM_E_INVALID
 * outside [0, ny].  lbm_get_segment_rows reports the height in use, 0 when
 * the context runs the two-pass step. */
lbm_status lbm_set_segment_rows(lbm_ctx *c, int rows);
lbm_status lbm_get_segment_rows(lbm_ctx *c, int *rows);

/* Autotuner for the segment height (not a passage of the paper): times
 * `trials` (1..1000) launches of the single-pass step for every height
 * 8k - 2 <= min(ny, 1022), on the current state, re-times the six fastest in
 * three interleaved rounds of 8 x `trials` launches each, keeps the one with
 * the least total time for the context and returns it in *rows.  The state is kept: each trial reads f
 * and writes only the buffers that the next step overwrites.  *rows = 0 and
 * nothing timed when the context runs the two-pass step.  LBM_E_STATE before
 * initialisation, LBM_E_INVALID for a bad argument, LBM_E_UNSTABLE if the
 * trial steps flag a non-positive density.  Synchronising. */
lbm_status lbm_tune_segment_rows(lbm_ctx *c, int trials, int *rows);

/* Enable (1) or disable (0) the event accounting of lbm_step; enabling
 * resets the counters.  Not synchronising. */
lbm_status lbm_set_timing(lbm_ctx *c, int enable);

/* Read the accounting (synchronising).  Kernels launched while timing was
 * disabled are not counted. */
lbm_status lbm_get_timing(lbm_ctx *c, lbm_timing *out);

/* ---------------------------------------------------------------------------
 * Batched sweep: n independent periodic lattices of uneven size, each with its
 * own EOS, constants, T/Tc, tau, k, force form and gradient (the temperature
 * and EOS sweeps behind the coexistence curves of Sec. 5.2, Fig. 5), advanced
 * together by one persistent launch per lbm_batch_step call (a cooperative
 * grid over all cells, or one thread-block cluster per instance, see
 * lbm_batch_set_cluster), replayed from a CUDA graph.  All instances share p[0].prec and p[0].stream.
 * Host fields are concatenated instance after instance: a density field has
 * nx_i*ny_i entries per instance, a distribution array 9*nx_i*ny_i (SoA within
 * the instance).  Grid-wide waits inside the launch are bounded (2 s); a wait
 * that gives up makes the launch return early and the next synchronising call
 * answer LBM_E_TIMEOUT.
 * ------------------------------------------------------------------------- */

/* Validate p[0..n-1] and allocate the batch on the current device.  Each
 * instance holds at most 2^30 cells and the instances together, each padded to
 * a multiple of 512 cells, fewer than 2^31; otherwise LBM_E_INVALID before any
 * allocation. */
lbm_status lbm_batch_create(const lbm_params *p, int n, lbm_batch **out);

/* f = f^eq(rho, 0) (Eq. 2) for every instance from concatenated host FP64 rho. */
lbm_status lbm_batch_init_density(lbm_batch *b, const double *rho);

/* Set / read the full state (concatenated host FP64, 9*nx_i*ny_i per instance).
 * lbm_batch_get_f synchronises. */
lbm_status lbm_batch_set_f(lbm_batch *b, const double *f);
lbm_status lbm_batch_get_f(lbm_batch *b, double *f);

/* Advance every instance nsteps steps (Eq. 1): one persistent launch,
 * asynchronous on the batch's stream. */
lbm_status lbm_batch_step(lbm_batch *b, int nsteps);

/* Wait for the batch's stream and check its error word. */
lbm_status lbm_batch_sync(lbm_batch *b);

/* Density (Eq. 3) of every instance into concatenated host FP64 rho.  Synchronising. */
lbm_status lbm_batch_density(lbm_batch *b, double *rho);

/* Density (Eq. 3) and half-step velocity v = (sum_i e_i f_i + F/2) / rho
 * (Eq. 11, F the step's interaction force) of every instance, in the batch's
 * precision, into concatenated host FP64 arrays (nx_i*ny_i entries per
 * instance, instance after instance; vx, vy may be NULL).  The conventions of
 * lbm_moments, per instance.  LBM_E_STATE before initialisation, LBM_E_NOMEM
 * if its buffers (three fields of the batch, allocated on the first call)
 * cannot be had.  Synchronising. */
lbm_status lbm_batch_moments(lbm_batch *b, double *rho, double *vx, double *vy);

/* Launch shape of the persistent kernel: threads per block (128, 256 or 512)
 * and co-resident blocks per SM (1 .. the occupancy limit).  Selects the grid
 * form (a cluster form set earlier, by lbm_batch_set_cluster or the tuner, is
 * dropped). */
lbm_status lbm_batch_set_launch(lbm_batch *b, int block_threads, int blocks_per_sm);
lbm_status lbm_batch_get_launch(lbm_batch *b, int *block_threads, int *grid_blocks);

/* Cluster form of the batch: one thread-block cluster of `cluster` CTAs
 * (2, 4 or 8: portable cluster sizes) per instance, block_threads (128, 256, 512 or 1024)
 * threads each, the clusters taking the instances largest first, the instance's distributions and potential field held in shared
 * memory for the whole launch and the stencil halos and boundary populations
 * exchanged through distributed shared memory; hardware cluster barriers
 * replace the grid barriers.  The per-cell arithmetic is the grid form's, so
 * both forms give the same results.  CTA k of an instance's cluster owns the
 * columns [k nx / cluster, (k + 1) nx / cluster).  Every instance must split:
 * its narrowest slice at least as wide as its x halo (the HDM radius, 1 for
 * CDM), and both distribution buffers plus the haloed field of the widest
 * slice within a block's shared memory; otherwise LBM_E_INVALID and the batch
 * keeps its form.  cluster = 0 returns to the grid
 * form.  lbm_batch_get_launch then reports block_threads and cluster * n. */
lbm_status lbm_batch_set_cluster(lbm_batch *b, int cluster, int block_threads);
/* The batch's form: 0 grid, 2/4/8 the cluster form's cluster size, -1 grouped. */
lbm_status lbm_batch_get_cluster(lbm_batch *b, int *cluster);

/* Grouped cluster form: each instance takes the smallest cluster size of 2, 4
 * and 8 whose slices split it (as for lbm_batch_set_cluster) within
 * max_smem_bytes of shared memory per CTA (0: the device's opt-in maximum;
 * LBM_GROUPS_BALANCED: the shared memory of the widest slice any instance has
 * on 8 CTAs, so that no CTA holds more than the largest lattice's 8-CTA
 * slice), else the smallest within the opt-in maximum; the instances of one cluster
 * size form a group, run as one cluster launch with that group's own shared
 * memory size and block_threads (256, 512 or 1024) threads per CTA, each group
 * on its own stream forked from the batch's stream and joined back before the
 * step call's work ends (captured into the same CUDA graph).  Small instances
 * thus hold fewer SMs, and a small cap lets several CTAs share an SM.  The
 * per-cell arithmetic is the other forms', so the results are the same.
 * LBM_E_INVALID (the batch keeps its form) if an instance does not split over
 * 8 CTAs or a group's cluster cannot be placed; LBM_E_NOMEM if its order table
 * cannot be had.  lbm_batch_get_launch then reports block_threads and the
 * total CTA count; lbm_batch_set_launch or lbm_batch_set_cluster leave it. */
enum { LBM_GROUPS_BALANCED = -1 };
lbm_status lbm_batch_set_groups(lbm_batch *b, int max_smem_bytes, int block_threads);
/* Groups of the grouped form (ngroups = 0 otherwise): cluster size, instance
 * count and shared memory per CTA of each, largest cluster first; cluster,
 * count and smem_bytes may be NULL, else hold at least 3 entries. */
lbm_status lbm_batch_get_groups(lbm_batch *b, int *ngroups, int *cluster, int *count, int *smem_bytes);

/* Autotuner: time trial_steps steps for every candidate launch shape (grid
 * form: block size x blocks per SM; cluster form: cluster size x block size,
 * where the instances split; grouped form: shared-memory cap (balanced, the
 * opt-in maximum, 72 KB) x block size) on a copy of the current state, keep the fastest
 * (its block size and grid, as lbm_batch_get_launch reports them, written to
 * the out pointers, which may be NULL) and restore the state.  Synchronising. */
lbm_status lbm_batch_tune(lbm_batch *b, int trial_steps, int *block_threads, int *grid_blocks);

/* Test hook for the bounded grid barrier: block `block` (or none when -1)
 * skips its first arrival, so the other blocks give up after limit_seconds
 * (at most 60) and the next synchronising call answers LBM_E_TIMEOUT.  While
 * armed, steps take the grid form. */
lbm_status lbm_batch_debug_skip_barrier(lbm_batch *b, int block, double limit_seconds);

const char *lbm_batch_last_error(const lbm_batch *b);
void lbm_batch_destroy(lbm_batch *b);

/* Size of the fixed device scratch array used by lbm_step_noalloc. */
#define LBM_STATIC_SCRATCH_BYTES (4u << 20)

/* One time step that allocates nothing (the paper has no counterpart: this is
 * a deployment variant of lbm_step).  For callers that cannot call cudaMalloc
 * -- a host framework that owns every device allocation, or a latency-
 * critical loop that must not take cudaMalloc's implicit synchronisation.
 *   p      lattice and model parameters, as for lbm_create (p->stream is used;
 *          p->flags is accepted but the step always takes the two-pass form,
 *          with FP64 arithmetic for LBM_F32: LBM_FLAG_F32_ARITH is ignored);
 *   f_in   device array, 9*nx*ny values of the precision p->prec, SoA as
 *          above: the state at t (read only);
 *   f_out  device array of the same size, distinct from f_in: receives the
 *          state at t+1.  Both stay owned by the caller.
 * The step is lbm_step's two-pass form (for LBM_F32: FP32 distributions,
 * FP64 arithmetic).  Its potential field (FP64 in both precisions) and the
 * error word live in one file-scope device array of LBM_STATIC_SCRATCH_BYTES
 * (4 MiB) that every GPU loading the library holds until the process exits,
 * so nx*ny may be at most (4 MiB - 256 B) / 8 = 524,256 cells; larger
 * lattices are rejected with LBM_E_INVALID before any device work.  The first call on a
 * device looks the array's device address up (with that device current), so
 * make the first call before any stream capture.  Every call, on any stream,
 * shares the one array and leaves its contents behind; the error word is
 * cleared at the start of each call.  Calls whose work overlaps on the GPU
 * therefore race and must be serialised by the caller.  Synchronising:
 * returns LBM_E_UNSTABLE if the step saw a NaN or rho <= 0, LBM_E_CUDA on a
 * CUDA error, LBM_E_INVALID on bad arguments.  Calls no cudaMalloc, cudaFree
 * or other allocating routine. */
lbm_status lbm_step_noalloc(const lbm_params *p, const void *f_in, void *f_out);

/* Test hook (not a passage of the paper): the number of device and of pinned
 * host allocations the library holds right now, over all contexts and
 * batches.  With the environment variable LBM_DEBUG_FAIL_ALLOC=n set, once n
 * allocations have succeeded since it took its current value, every further
 * allocation of the library fails as if the memory were exhausted (n = 0: all
 * of them); the failing call answers LBM_E_NOMEM and frees what it took, so a
 * test can walk every allocation of an entry point and check for leaks.  The
 * failure is made on the host; no GPU call fails. */
lbm_status lbm_debug_alloc_stats(long long *live_device, long long *live_host);

/* Test hook (not a passage of the paper) of the bounds-checked build, a
 * library compiled with -DLBM_CHECKED: its kernels check the indices of their
 * global and distributed-shared-memory accesses, skip an access that would
 * fall outside its buffer and set a bit in the error word instead (the next
 * synchronising call answers LBM_E_CUDA, "a device-side bounds check
 * failed"), and every device allocation carries 256 bytes of a known pattern
 * past its end.  *damaged receives the number of live allocations whose
 * pattern changed (synchronises the device), or -1 in the normal build,
 * which has neither checks nor canaries. */
lbm_status lbm_debug_check_canaries(long long *damaged);

/* Saved lattice states (not a passage of the paper: checkpoint and resume).
 * lbm_save writes the current distributions in the storage precision to the
 * file `path` (created or truncated), with a header of the lattice's
 * parameters, for a context on the single-pass kernel the stencil field its
 * next step reads, and a checksum.  LBM_E_STATE before initialisation,
 * LBM_E_UNSTABLE for a lattice in the error state, LBM_E_IO if the file cannot
 * be written.  Synchronising.
 * lbm_load reads such a file into a context of the same nx, ny and precision
 * (else LBM_E_INVALID; other parameters may differ: a restart at another
 * temperature, say) and leaves it initialised on that state.  The saved
 * stencil field is used where the context runs the single-pass kernel and
 * every parameter the field depends on matches, so that a resumed run repeats
 * an uninterrupted one bit for bit; otherwise the next step forms the field
 * from the distributions.  LBM_E_IO for a file that cannot be read, is not a
 * saved state, is truncated or fails its checksum; the context then keeps its
 * state.  Synchronising. */
lbm_status lbm_save(lbm_ctx *c, const char *path);
lbm_status lbm_load(lbm_ctx *c, const char *path);

/* Free everything the context owns.  NULL is a no-op. */
void lbm_destroy(lbm_ctx *c);

/* Message of the last failed call on c (or of the last failed lbm_create
 * when c is NULL).  Never NULL. */
const char *lbm_last_error(const lbm_ctx *c);

/* 1 if the device accesses this context's host arrays in place where it can
 * (see LBM_FLAG_STAGED_HOST), 0 if they always pass through the pinned
 * staging buffer, -1 for NULL. */
int lbm_host_in_place(const lbm_ctx *c);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
