// Batched sweep: many independent periodic lattices of uneven size, each with
// its own equation of state, temperature and relaxation time, advanced by one
// persistent cooperative launch (captured in a CUDA graph) instead of two
// launches per instance per step.
//
// Layout.  The instances' cells are concatenated; instance i owns cells
// [off_i, off_i + nx_i ny_i) of every array, with off_i a multiple of 512 so
// that any chunk of 128..512 consecutive cells belongs to one instance.  f is
// SoA over the whole batch: f[q * ntot + cell].
//
// One step = phase A (rho = sum f, potential field of Eq. 8/21 for every cell)
// + grid barrier + phase B (HDM/CDM gradient of the potential, force Eq. 22 /
// Eq. 7, exact-difference forcing + BGK of Eq. 1, 2, 10, periodic push
// streaming within the instance) + grid barrier.  Blocks take 'chunks' of
// blockDim cells of one instance (its parameters are uniform in the block).
// The grid barrier is a counter/generation pair in global memory; every wait
// is bounded by %globaltimer and sets LBM_E_TIMEOUT and an abort flag that
// all blocks check, so no block can spin forever.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kAlign = 512;       // instance offsets are multiples of this many cells
constexpr int kTableGrain = 128;  // cells per entry of the chunk -> instance table

template <typename T>
struct Inst {
    Model<T> m;
    int off;  // first cell of the instance in the concatenated arrays
    int sc;   // Shan-Chen (Eq. 22) or Zhang-Chen (Eq. 7) form
    int cdm;  // CDM (Eq. 15) instead of HDM (Eq. 20)
};

struct BarrierState {
    unsigned int count;
    unsigned int gen;
    int abort;
};

template <typename T>
struct BatchArgs {
    const Inst<T> *inst;
    const int *table;      // instance of each kTableGrain-cell group (-1 = padding)
    T *f[2];               // the two distribution buffers (ping-pong by step parity)
    T *q;                  // potential field
    long long ntot;        // cells in the concatenated arrays (padded)
    int nsteps;
    int parity0;           // buffer holding the state at the first step
    int *err;
    BarrierState *bar;
    unsigned long long limit_ns;
    int skip_block;        // test hook: this block never arrives at the first barrier (-1: none)
};

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a wall-time bound.  Returns false if the batch was
// aborted (by a timeout here or elsewhere).
__device__ bool grid_sync(BarrierState *b, unsigned int nblocks, int *err, unsigned long long limit_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &b->gen;
        volatile int *vabort = &b->abort;
        const unsigned int g = *vgen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == nblocks - 1) {
            b->count = 0;
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const unsigned long long t0 = gtimer();
            unsigned int it = 0;
            while (*vgen == g && !*vabort) {
                if ((++it & 255) == 0 && gtimer() - t0 > limit_ns) {
                    atomicOr(err, kErrTimeout);
                    atomicExch(&b->abort, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        ok = !*vabort;
    }
    __syncthreads();
    return ok;
}

template <typename T>
__device__ __forceinline__ T qabs(T v, bool sc) {
    return sc ? fabs(v) : v;
}

// Moments (Eq. 3), exact-difference forcing (Eq. 10) and BGK (Eq. 1) of one
// cell with interaction force (Fx, Fy): the post-collision populations
// post[i]; the rest population takes rho minus the other eight.
template <typename T>
__device__ __forceinline__ void collide_cell(const Model<T> &m, const T (&fi)[kQ], T Fx, T Fy, T (&post)[kQ]) {
    T r = T(0), jx = T(0), jy = T(0);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        r += fi[i];
        jx += T(ex(i)) * fi[i];
        jy += T(ey(i)) * fi[i];
    }
    const T inv = T(1) / r;
    const T ux = jx * inv, uy = jy * inv;
    const T vx = ux + Fx * inv, vy = uy + Fy * inv;
    const T uu = ux * ux + uy * uy, vv = vx * vx + vy * vy;
    T moved = T(0);
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        const T eu = T(ex(i)) * ux + T(ey(i)) * uy;
        const T ev = T(ex(i)) * vx + T(ey(i)) * vy;
        const T feq = r * wq<T>(i) * (T(1) + T(3) * eu + T(4.5) * eu * eu - T(1.5) * uu);
        const T fsh = r * wq<T>(i) * (T(1) + T(3) * ev + T(4.5) * ev * ev - T(1.5) * vv);
        post[i] = fi[i] - (fi[i] - feq) * m.omega + (fsh - feq);
        moved += post[i];
    }
    post[0] = r - moved;
}

// Interaction force at cell `cell` = (x, y) of instance I from the potential
// field q (concatenated layout): the HDM gradient (explicit periodic form of
// Eq. 20, folded weights for short lines) or the CDM of Eq. 15, then Eq. 22
// (Shan-Chen, q = s Phi) or Eq. 7 (Zhang-Chen).
template <typename T>
__device__ __forceinline__ void inst_force(const Inst<T> &I, const T *__restrict__ q, long long cell, int x, int y,
                                           T &Fx, T &Fy) {
    const Model<T> &m = I.m;
    const bool sc = I.sc != 0;
    const T *qi = q + I.off;
    const T *qrow = qi + (long long)y * m.nx;
    T dx = T(0), dy = T(0);
    if (I.cdm) {
        // Eq. 15 times 1/c_s^2 on the instance's periodic lattice
        const int xp = x + 1 == m.nx ? 0 : x + 1, xm = x == 0 ? m.nx - 1 : x - 1;
        const int yp = y + 1 == m.ny ? 0 : y + 1, ym = y == 0 ? m.ny - 1 : y - 1;
        auto at = [&](int yy, int xx) { return qabs(__ldg(qi + (long long)yy * m.nx + xx), sc); };
        const T e = at(y, xp), w = at(y, xm), nn = at(yp, x), s = at(ym, x);
        const T ne = at(yp, xp), nw = at(yp, xm), se = at(ym, xp), sw = at(ym, xm);
        dx = T(1.0 / 3.0) * (e - w) + T(1.0 / 12.0) * ((ne + se) - (nw + sw));
        dy = T(1.0 / 3.0) * (nn - s) + T(1.0 / 12.0) * ((ne + nw) - (se + sw));
    } else {
        // explicit periodic form of Eq. 20 (folded weights for short lines)
        for (int j = 1; j <= m.kx; ++j) {
            int xp = x + j, xm = x - j;
            if (xp >= m.nx) xp -= m.nx;
            if (xm < 0) xm += m.nx;
            dx += m.wx[j] * (qabs(__ldg(qrow + xp), sc) - qabs(__ldg(qrow + xm), sc));
        }
        for (int j = 1; j <= m.ky; ++j) {
            int yp = y + j, ym = y - j;
            if (yp >= m.ny) yp -= m.ny;
            if (ym < 0) ym += m.ny;
            dy += m.wy[j] * (qabs(__ldg(qi + (long long)yp * m.nx + x), sc) -
                             qabs(__ldg(qi + (long long)ym * m.nx + x), sc));
        }
    }
    const T qc = q[cell];
    if (sc) {  // Eq. 22: F = -2 s Phi grad Phi, q = s Phi
        Fx = T(-2) * qc * dx;
        Fy = T(-2) * qc * dy;
    } else {   // Eq. 7
        Fx = -dx;
        Fy = -dy;
    }
}

template <typename T>
__global__ void batch_kernel(const BatchArgs<T> a) {
    const unsigned int nblocks = gridDim.x;
    const int B = blockDim.x;
    const long long nchunks = a.ntot / B;
    for (int step = 0; step < a.nsteps; ++step) {
        const bool odd = ((a.parity0 + step) & 1) != 0;  // (a select, not a dynamic index into the parameters)
        const T *__restrict__ f = odd ? a.f[1] : a.f[0];
        T *__restrict__ fo = odd ? a.f[0] : a.f[1];
        // ---- phase A: density and potential field ----
        for (long long ch = blockIdx.x; ch < nchunks; ch += nblocks) {
            const long long cell = ch * B + threadIdx.x;
            const int ii = a.table[(ch * B) / kTableGrain];
            if (ii < 0) continue;
            const Inst<T> &I = a.inst[ii];
            const long long local = cell - I.off;
            if (local >= (long long)I.m.nx * I.m.ny) continue;
            T r = T(0);
#pragma unroll
            for (int i = 0; i < kQ; ++i) r += f[i * a.ntot + cell];
            if (!(r > T(0)) || !isfinite(r)) atomicOr(a.err, kErrUnstable);
            a.q[cell] = potential_field(I.m, r, I.sc != 0);
        }
        if (step == 0 && (int)blockIdx.x == a.skip_block) return;  // test hook: never arrive
        if (!grid_sync(a.bar, nblocks, a.err, a.limit_ns)) return;
        // ---- phase B: gradient, force, forcing + BGK, periodic push streaming ----
        for (long long ch = blockIdx.x; ch < nchunks; ch += nblocks) {
            const long long cell = ch * B + threadIdx.x;
            const int ii = a.table[(ch * B) / kTableGrain];
            if (ii < 0) continue;
            const Inst<T> &I = a.inst[ii];
            const Model<T> &m = I.m;
            const int local = (int)(cell - I.off);
            if (local >= m.nx * m.ny) continue;
            const int y = local / m.nx, x = local - y * m.nx;
            T Fx, Fy;
            inst_force(I, a.q, cell, x, y, Fx, Fy);
            T fi[kQ], post[kQ];
#pragma unroll
            for (int i = 0; i < kQ; ++i) fi[i] = f[i * a.ntot + cell];
            collide_cell(m, fi, Fx, Fy, post);
            const int xp = x + 1 == m.nx ? 0 : x + 1, xm = x == 0 ? m.nx - 1 : x - 1;
            const int yp = y + 1 == m.ny ? 0 : y + 1, ym = y == 0 ? m.ny - 1 : y - 1;
#pragma unroll
            for (int i = 1; i < kQ; ++i) {
                const int dxs = ex(i) == 1 ? xp : (ex(i) == -1 ? xm : x);
                const int dys = ey(i) == 1 ? yp : (ey(i) == -1 ? ym : y);
                const long long k = i * a.ntot + I.off + (long long)dys * m.nx + dxs;
                if (in_bounds(k, kQ * a.ntot, m.chk)) fo[k] = post[i];
            }
            fo[cell] = post[0];
        }
        if (!grid_sync(a.bar, nblocks, a.err, a.limit_ns)) return;
    }
}

// Cluster form: one thread-block cluster of C CTAs per instance, with the
// instance's state on chip for the whole launch.  CTA rank k owns the columns
// [k nx / C, (k + 1) nx / C) of every row (widths differ by one at most); its two distribution buffers and
// its potential field (with hx halo columns on each side) live in shared
// memory.  One step: phase A (rho and the potential field of the owned cells),
// a cluster barrier, the halo columns copied from the neighbouring ranks'
// shared memory (ranks k - 1 and k + 1 modulo C: x is periodic), phase B
// (gradient, force, forcing + BGK, push streaming: a population that leaves
// the owned columns is stored into the neighbour's buffer), a cluster barrier.
// Global f is read before the first step and written after the last.  The
// only waits are the cluster barriers, reached the same number of times by
// every thread, and no CTA exits before the last barrier, so no access reaches
// the shared memory of a CTA that has left.  The per-cell arithmetic is the
// grid form's, term for term.
template <typename T>
struct ClusterArgs {
    const Inst<T> *inst;
    const int *order;  // instance of each cluster: largest first, so no large one starts last
    const T *fin;    // state at the first step (concatenated layout)
    T *fout;         // receives the state after nsteps (may be fin)
    long long ntot;
    int nsteps;
    int *err;
};

template <typename T>
__global__ void cluster_batch_kernel(const ClusterArgs<T> a) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const Inst<T> &I = a.inst[a.order[blockIdx.x / C]];   // clusters lie along x, one per instance
    const Model<T> &m = I.m;
    const bool sc = I.sc != 0, cdm = I.cdm != 0;
    const int nx = m.nx, ny = m.ny;
    // rank k owns columns [k nx / C, (k + 1) nx / C): widths differ by one at
    // most; every rank lays its slice out with the pitch of the widest, so a
    // neighbour's element sits at the same offset in every CTA
    const int x0 = (int)((long long)rank * nx / C), w = (int)((long long)(rank + 1) * nx / C) - x0;
    const int wmax = (nx + C - 1) / C;
    const int hx = cdm ? 1 : m.kx;
    const int W = wmax + 2 * hx;                // potential row pitch
    const int ncell = w * ny;                   // owned cells
    const int plane = wmax * ny;                // distribution plane stride
    T *fa = reinterpret_cast<T *>(smem_raw);   // [kQ][ny][wmax]
    T *fb = fa + (size_t)kQ * plane;
    T *ph = fb + (size_t)kQ * plane;           // [ny][W], owned column xl at hx + xl
    const int left = rank == 0 ? C - 1 : rank - 1, right = rank == C - 1 ? 0 : rank + 1;
    const int wl = (int)((long long)(left + 1) * nx / C) - (int)((long long)left * nx / C);   // the left rank's width

    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const int y = c / w, xl = c - y * w;
        const long long g = I.off + (long long)y * nx + x0 + xl;
#pragma unroll
        for (int i = 0; i < kQ; ++i)
            if (in_bounds(i * a.ntot + g, kQ * a.ntot, m.chk)) fa[i * plane + y * wmax + xl] = a.fin[i * a.ntot + g];
    }
    __syncthreads();
    for (int step = 0; step < a.nsteps; ++step) {
        // ---- phase A: density and potential field of the owned cells ----
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int y = c / w, xl = c - y * w;
            T r = T(0);
#pragma unroll
            for (int i = 0; i < kQ; ++i) r += fa[i * plane + y * wmax + xl];
            if (!(r > T(0)) || !isfinite(r)) atomicOr(a.err, kErrUnstable);
            ph[y * W + hx + xl] = potential_field(m, r, sc);
        }
        cluster.sync();
        // ---- halo: the left neighbour's columns wl - hx .. wl - 1, the right one's 0 .. hx - 1 ----
        {
            const T *pl = cluster.map_shared_rank(ph, left);
            const T *pr = cluster.map_shared_rank(ph, right);
            const int nh = hx * ny;
            for (int c = threadIdx.x; c < 2 * nh; c += blockDim.x) {
                const int side = c < nh ? 0 : 1, k = c - side * nh;
                const int y = k / hx, j = k - y * hx;
                if (side == 0) ph[y * W + j] = pl[y * W + wl + j];
                else ph[y * W + hx + w + j] = pr[y * W + hx + j];
            }
        }
        __syncthreads();
        // ---- phase B: gradient, force, forcing + BGK, push streaming ----
        T *fbl = cluster.map_shared_rank(fb, left);
        T *fbr = cluster.map_shared_rank(fb, right);
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int y = c / w, xl = c - y * w;
            const T *row = ph + y * W + hx + xl;   // row[j]: the field at column xl + j
            T dx = T(0), dy = T(0);
            if (cdm) {
                // Eq. 15 times 1/c_s^2
                const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
                auto at = [&](int yy, int dxo) { return qabs(ph[yy * W + hx + xl + dxo], sc); };
                const T e = at(y, 1), wv = at(y, -1), nn = at(yp, 0), so = at(ym, 0);
                const T ne = at(yp, 1), nw = at(yp, -1), se = at(ym, 1), sw = at(ym, -1);
                dx = T(1.0 / 3.0) * (e - wv) + T(1.0 / 12.0) * ((ne + se) - (nw + sw));
                dy = T(1.0 / 3.0) * (nn - so) + T(1.0 / 12.0) * ((ne + nw) - (se + sw));
            } else {
                // explicit periodic form of Eq. 20 (folded weights for short lines)
                for (int j = 1; j <= m.kx; ++j) dx += m.wx[j] * (qabs(row[j], sc) - qabs(row[-j], sc));
                for (int j = 1; j <= m.ky; ++j) {
                    int yp = y + j, ym = y - j;
                    if (yp >= ny) yp -= ny;
                    if (ym < 0) ym += ny;
                    dy += m.wy[j] * (qabs(ph[yp * W + hx + xl], sc) - qabs(ph[ym * W + hx + xl], sc));
                }
            }
            const T qc = row[0];
            T Fx, Fy;
            if (sc) {  // Eq. 22: F = -2 s Phi grad Phi, q = s Phi
                Fx = T(-2) * qc * dx;
                Fy = T(-2) * qc * dy;
            } else {   // Eq. 7
                Fx = -dx;
                Fy = -dy;
            }
            T fi[kQ], post[kQ];
#pragma unroll
            for (int i = 0; i < kQ; ++i) fi[i] = fa[i * plane + y * wmax + xl];
            collide_cell(m, fi, Fx, Fy, post);
            const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
#pragma unroll
            for (int i = 1; i < kQ; ++i) {
                const int dys = ey(i) == 1 ? yp : (ey(i) == -1 ? ym : y);
                const int xd = xl + ex(i);
                T *dst = xd < 0 ? fbl : (xd >= w ? fbr : fb);
                const int xc = xd < 0 ? wl - 1 : (xd >= w ? 0 : xd);
                if (in_bounds(i * plane + dys * wmax + xc, (long long)kQ * plane, m.chk))
                    dst[i * plane + dys * wmax + xc] = post[i];   // own buffer or a neighbour's (same layout)
            }
            fb[y * wmax + xl] = post[0];
        }
        cluster.sync();
        T *t = fa;
        fa = fb;
        fb = t;
    }
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const int y = c / w, xl = c - y * w;
        const long long g = I.off + (long long)y * nx + x0 + xl;
#pragma unroll
        for (int i = 0; i < kQ; ++i)
            if (in_bounds(i * a.ntot + g, kQ * a.ntot, m.chk)) a.fout[i * a.ntot + g] = fa[i * plane + y * wmax + xl];
    }
}

template <typename T>
__global__ void batch_init_kernel(const Inst<T> *inst, const int *table, const T *rho, T *f, long long ntot) {
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < ntot;
         cell += (long long)gridDim.x * blockDim.x) {
        const int ii = table[cell / kTableGrain];
        const bool valid = ii >= 0 && cell - inst[ii].off < (long long)inst[ii].m.nx * inst[ii].m.ny;
        const T r = valid ? rho[cell] : T(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) f[i * ntot + cell] = r * wq<T>(i);  // f^eq(rho, 0), Eq. 2
    }
}

template <typename T>
__global__ void batch_density_kernel(const Inst<T> *inst, const int *table, const T *f, T *rho, long long ntot) {
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < ntot;
         cell += (long long)gridDim.x * blockDim.x) {
        T r = T(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) r += f[i * ntot + cell];
        rho[cell] = r;
    }
}

// Density (Eq. 3) and the potential field (Eq. 8 / 21) of every cell: phase A
// of the step as a launch of its own (for lbm_batch_moments).
template <typename T>
__global__ void batch_potential_kernel(const Inst<T> *inst, const int *table, const T *f, T *q, long long ntot,
                                       int *err) {
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < ntot;
         cell += (long long)gridDim.x * blockDim.x) {
        const int ii = table[cell / kTableGrain];
        if (ii < 0) continue;
        const Inst<T> &I = inst[ii];
        if (cell - I.off >= (long long)I.m.nx * I.m.ny) continue;
        T r = T(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) r += f[i * ntot + cell];
        if (!(r > T(0)) || !isfinite(r)) atomicOr(err, kErrUnstable);
        q[cell] = potential_field(I.m, r, I.sc != 0);
    }
}

// rho (Eq. 3) and the half-step velocity v = (sum_i e_i f_i + F/2) / rho of
// Eq. 11, with F the step's interaction force from the potential field q.
template <typename T>
__global__ void batch_moments_kernel(const Inst<T> *inst, const int *table, const T *f, const T *q, T *rho, T *vx,
                                     T *vy, long long ntot) {
    for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < ntot;
         cell += (long long)gridDim.x * blockDim.x) {
        const int ii = table[cell / kTableGrain];
        if (ii < 0) continue;
        const Inst<T> &I = inst[ii];
        const int local = (int)(cell - I.off);
        if (local >= I.m.nx * I.m.ny) continue;
        const int y = local / I.m.nx, x = local - y * I.m.nx;
        T Fx, Fy;
        inst_force(I, q, cell, x, y, Fx, Fy);
        T r = T(0), jx = T(0), jy = T(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const T v = f[i * ntot + cell];
            r += v;
            jx += T(ex(i)) * v;
            jy += T(ey(i)) * v;
        }
        rho[cell] = r;
        vx[cell] = (jx + T(0.5) * Fx) / r;
        vy[cell] = (jy + T(0.5) * Fy) / r;
    }
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_batch {
    int n = 0;
    int prec = LBM_F32;
    size_t esz = 4;
    long long ntot = 0;
    std::vector<lbm_params> params;
    std::vector<long long> off;
    void *inst_dev = nullptr;
    int *table_dev = nullptr;
    int *order_dev = nullptr;      // instances by decreasing cell count (cluster form)
    void *f[2] = {nullptr, nullptr};
    void *q = nullptr;
    void *stage_dev = nullptr;   // rho staging (ntot values of the precision)
    void *stage_host = nullptr;  // pinned host staging
    void *mom_dev = nullptr;     // rho, vx, vy of lbm_batch_moments (3 ntot values, allocated on first use)
    void *mom_host = nullptr;    // their pinned host copy
    int *err = nullptr;
    BarrierState *bar = nullptr;
    int cur = 0;
    cudaStream_t stream = nullptr;
    int block_threads = 256;
    int grid_blocks = 0;
    int cluster = 0;               // CTAs per instance in the cluster form (0: grid form, -1: grouped)
    int cluster_threads = 256;
    size_t cluster_smem = 0;       // dynamic shared memory per CTA of the cluster form
    // grouped cluster form: one cluster launch per cluster size, each on its own
    // stream (forked from and joined to the batch's stream), instances of group
    // g at gorder_dev[first .. first + count) by decreasing cell count
    struct Group {
        int cluster, first, count;
        size_t smem;
    };
    std::vector<Group> groups;
    int *gorder_dev = nullptr;
    cudaStream_t gstream[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t gfork = nullptr, gjoin[3] = {nullptr, nullptr, nullptr};
    int groups_gen = 0;            // changes with every grouping (graph cache key)
    std::vector<int> halo;         // x halo of each instance (kx for HDM, 1 for CDM)
    unsigned long long limit_ns = 2000000000ull;  // 2 s per barrier wait
    int skip_block = -1;
    bool initialized = false;
    bool unstable = false;
    // graphs of the last step count, one per starting buffer parity
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
    int graph_steps[2] = {-1, -1}, graph_block[2] = {-1, -1}, graph_grid[2] = {-1, -1};
    int graph_cluster[2] = {-1, -1}, graph_gen[2] = {-1, -1};
    bool use_graph = true;
    int graph_launches = 0;  // persistent launches issued through a graph
    std::string msg;
};

namespace {

lbm_status bfail(lbm_batch *b, lbm_status st, const std::string &m) {
    if (b) b->msg = m;
    return st;
}

#define BCK(b, expr, what)                                                                         \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? LBM_E_NOMEM : LBM_E_CUDA,            \
                         std::string(what) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

template <typename T>
lbm_status build_instances(lbm_batch *b, std::vector<Inst<T>> &out) {
    out.resize(b->n);
    b->halo.assign(b->n, 0);
    for (int i = 0; i < b->n; ++i) {
        const lbm_params &p = b->params[i];
        Inst<T> &I = out[i];
        I = Inst<T>{};
        ModelScalars ms;
        if (model_scalars(p, &ms) != LBM_OK)
            return bfail(b, LBM_E_INVALID, "no critical point for instance " + std::to_string(i));
        I.m.nx = p.nx;
        I.m.ny = p.ny;
        I.m.eos = p.eos;
        I.m.RT = (T)ms.RT;
        I.m.a = (T)ms.a;
        I.m.b = (T)ms.b;
        I.m.aal = (T)ms.aal;
        I.m.k = (T)ms.k;
        I.m.omega = (T)(1.0 / p.tau);
        const int radius = p.hdm_radius ? p.hdm_radius : (b->prec == LBM_F64 ? 40 : 26);
        double wx[kMaxRadius + 1] = {}, wy[kMaxRadius + 1] = {};
        lbm_hdm_weights(p.nx, radius, wx, &I.m.kx);
        lbm_hdm_weights(p.ny, radius, wy, &I.m.ky);
        for (int j = 0; j <= kMaxRadius; ++j) {
            I.m.wx[j] = (T)wx[j];
            I.m.wy[j] = (T)wy[j];
        }
        I.off = (int)b->off[i];
        I.sc = p.force == LBM_FORCE_SC;
        I.cdm = p.grad == LBM_GRAD_CDM;
        b->halo[i] = I.cdm ? 1 : I.m.kx;
    }
    return LBM_OK;
}

template <typename T>
BatchArgs<T> make_args(lbm_batch *b, int nsteps) {
    BatchArgs<T> a{};
    a.inst = (const Inst<T> *)b->inst_dev;
    a.table = b->table_dev;
    a.f[0] = (T *)b->f[0];
    a.f[1] = (T *)b->f[1];
    a.q = (T *)b->q;
    a.ntot = b->ntot;
    a.nsteps = nsteps;
    a.parity0 = b->cur;
    a.err = b->err;
    a.bar = b->bar;
    a.limit_ns = b->limit_ns;
    a.skip_block = b->skip_block;
    return a;
}

template <typename T>
int max_blocks_per_sm(int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<T>, threads, 0) != cudaSuccess) return 0;
    return nb;
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

// Shared memory per CTA of the cluster form with `cluster` CTAs per instance
// (both distribution buffers and the haloed potential field of the widest
// slice), or 0 when some instance does not split: a slice narrower than the
// instance's x halo, or more than the opt-in shared memory of a block.
size_t cluster_smem_bytes(const lbm_batch *b, int cluster) {
    size_t need = 0;
    for (int i = 0; i < b->n; ++i) {
        const int nx = b->params[i].nx, ny = b->params[i].ny;
        const int wmin = nx / cluster, wmax = (nx + cluster - 1) / cluster;   // slice widths
        if (b->halo[i] > wmin) return 0;
        const size_t bytes = ((size_t)2 * kQ * wmax * ny + (size_t)ny * (wmax + 2 * b->halo[i])) * b->esz;
        need = std::max(need, bytes);
    }
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return need <= (size_t)optin ? need : 0;
}

template <typename T>
cudaLaunchConfig_t cluster_config(const lbm_batch *b, int cluster, int threads, size_t smem,
                                  cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(cluster * b->n));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = b->stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Prepare the cluster kernel for this shape and check that at least one
// cluster of it can be resident.  Returns 0 or an error message.
template <typename T>
const char *configure_cluster(const lbm_batch *b, int cluster, int threads, size_t smem) {
    if (cudaFuncSetAttribute(cluster_batch_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return "shared memory of the cluster form not available";
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config<T>(b, cluster, threads, smem, attr);
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, cluster_batch_kernel<T>, &cfg) != cudaSuccess || nc < 1) {
        cudaGetLastError();
        return "no cluster of this shape fits on the device";
    }
    return nullptr;
}

// Queue one launch running nsteps steps: the cluster form when one is set
// (and no barrier test hook is armed), else the persistent cooperative grid form.
template <typename T>
cudaError_t enqueue(lbm_batch *b, int nsteps) {
    if (b->cluster < 0 && b->skip_block < 0) {   // grouped: fork, one launch per group, join
        cudaError_t e = cudaEventRecord(b->gfork, b->stream);
        for (size_t g = 0; g < b->groups.size() && e == cudaSuccess; ++g) {
            const lbm_batch::Group &G = b->groups[g];
            ClusterArgs<T> ca{};
            ca.inst = (const Inst<T> *)b->inst_dev;
            ca.order = b->gorder_dev + G.first;
            ca.fin = (const T *)b->f[b->cur];
            ca.fout = (T *)b->f[(b->cur + nsteps) & 1];
            ca.ntot = b->ntot;
            ca.nsteps = nsteps;
            ca.err = b->err;
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t cfg = cluster_config<T>(b, G.cluster, b->cluster_threads, G.smem, attr);
            cfg.gridDim = dim3((unsigned)(G.cluster * G.count));
            cfg.stream = b->gstream[g];
            e = cudaStreamWaitEvent(b->gstream[g], b->gfork, 0);
            if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, cluster_batch_kernel<T>, ca);
            if (e == cudaSuccess) e = cudaEventRecord(b->gjoin[g], b->gstream[g]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->gjoin[g], 0);
        }
        return e;
    }
    if (b->cluster > 0 && b->skip_block < 0) {
        ClusterArgs<T> ca{};
        ca.inst = (const Inst<T> *)b->inst_dev;
        ca.order = b->order_dev;
        ca.fin = (const T *)b->f[b->cur];
        ca.fout = (T *)b->f[(b->cur + nsteps) & 1];
        ca.ntot = b->ntot;
        ca.nsteps = nsteps;
        ca.err = b->err;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_config<T>(b, b->cluster, b->cluster_threads, b->cluster_smem, attr);
        return cudaLaunchKernelEx(&cfg, cluster_batch_kernel<T>, ca);
    }
    cudaError_t e = cudaMemsetAsync(b->bar, 0, sizeof(BarrierState), b->stream);
    if (e != cudaSuccess) return e;
    BatchArgs<T> a = make_args<T>(b, nsteps);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(b->grid_blocks);
    cfg.blockDim = dim3(b->block_threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_kernel<T>, a);
}

void drop_graph(lbm_batch *b, int k) {
    if (b->graph_exec[k]) cudaGraphExecDestroy(b->graph_exec[k]);
    if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
    b->graph_exec[k] = nullptr;
    b->graph[k] = nullptr;
    b->graph_steps[k] = -1;
}

// nsteps steps as one persistent launch, replayed from a CUDA graph captured
// for this (step count, starting buffer, launch shape).
template <typename T>
lbm_status run_steps(lbm_batch *b, int nsteps) {
    if (nsteps == 0) return LBM_OK;
    const int k = b->cur;
    if (b->use_graph && b->skip_block < 0) {
        const int shape_block = b->cluster != 0 ? b->cluster_threads : b->block_threads;
        if (!b->graph_exec[k] || b->graph_steps[k] != nsteps || b->graph_block[k] != shape_block ||
            b->graph_grid[k] != b->grid_blocks || b->graph_cluster[k] != b->cluster ||
            b->graph_gen[k] != b->groups_gen) {
            drop_graph(b, k);
            bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                cudaError_t e1 = enqueue<T>(b, nsteps);
                cudaError_t e2 = cudaStreamEndCapture(b->stream, &b->graph[k]);
                ok = e1 == cudaSuccess && e2 == cudaSuccess &&
                     cudaGraphInstantiate(&b->graph_exec[k], b->graph[k], 0) == cudaSuccess;
            }
            if (!ok) {  // graphs unavailable for this launch: plain launches from now on
                cudaGetLastError();
                drop_graph(b, k);
                b->use_graph = false;
            } else {
                b->graph_steps[k] = nsteps;
                b->graph_block[k] = shape_block;
                b->graph_grid[k] = b->grid_blocks;
                b->graph_cluster[k] = b->cluster;
                b->graph_gen[k] = b->groups_gen;
            }
        }
        if (b->graph_exec[k]) {
            BCK(b, cudaGraphLaunch(b->graph_exec[k], b->stream), "cudaGraphLaunch");
            b->graph_launches += 1;
            b->cur = (b->cur + nsteps) & 1;
            return LBM_OK;
        }
    }
    BCK(b, enqueue<T>(b, nsteps), "batch launch");
    b->cur = (b->cur + nsteps) & 1;
    return LBM_OK;
}

lbm_status batch_sync(lbm_batch *b) {
    int h = 0;
    BCK(b, cudaMemcpyAsync(&h, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "read error word");
    BCK(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (h & kErrTimeout) return bfail(b, LBM_E_TIMEOUT, "a grid barrier wait timed out");
    if (h & kErrUnstable) {
        b->unstable = true;
        return bfail(b, LBM_E_UNSTABLE, "unstable: NaN or non-positive density");
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(const lbm_params *p, int n, lbm_batch **out) {
    if (!out) return LBM_E_INVALID;
    *out = nullptr;
    if (!p || n < 1) return LBM_E_INVALID;
    const int prec = p[0].prec;
    if (prec != LBM_F32 && prec != LBM_F64) return LBM_E_INVALID;
    long long padded = 0;
    for (int i = 0; i < n; ++i) {
        const lbm_params &q = p[i];
        const char *why = "";
        if (q.prec != prec || check_params(q, &why) != LBM_OK || (long long)q.nx * q.ny > (1LL << 30) ||
            (q.flags & LBM_FLAG_WALLS_Y))   // the batch steps periodic lattices only
            return LBM_E_INVALID;
        padded += ((long long)q.nx * q.ny + kAlign - 1) / kAlign * kAlign;
    }
    // instance offsets are int cell indices on the device: the padded total
    // must stay below 2^31 cells
    if (padded >= (1LL << 31)) return LBM_E_INVALID;
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_E_NOMEM;
    b->n = n;
    b->prec = prec;
    b->esz = prec == LBM_F64 ? sizeof(double) : sizeof(float);
    b->params.assign(p, p + n);
    b->stream = (cudaStream_t)p[0].stream;
    long long o = 0;
    for (int i = 0; i < n; ++i) {
        b->off.push_back(o);
        long long cells = (long long)p[i].nx * p[i].ny;
        o += (cells + kAlign - 1) / kAlign * kAlign;
    }
    b->ntot = o;
    auto bail = [&](lbm_status st) {
        lbm_batch_destroy(b);
        return st;
    };

    std::vector<int> table(b->ntot / kTableGrain, -1);
    for (int i = 0; i < n; ++i) {
        long long cells = (long long)p[i].nx * p[i].ny;
        for (long long g = b->off[i] / kTableGrain; g < (b->off[i] + cells + kTableGrain - 1) / kTableGrain; ++g)
            table[g] = i;
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) {
        return (long long)p[u].nx * p[u].ny > (long long)p[v].nx * p[v].ny;
    });
    size_t inst_bytes;
    std::vector<unsigned char> inst_host;
    if (prec == LBM_F64) {
        std::vector<Inst<double>> v;
        if (build_instances<double>(b, v) != LBM_OK) return bail(LBM_E_INVALID);
        inst_bytes = v.size() * sizeof(Inst<double>);
        inst_host.assign((unsigned char *)v.data(), (unsigned char *)v.data() + inst_bytes);
    } else {
        std::vector<Inst<float>> v;
        if (build_instances<float>(b, v) != LBM_OK) return bail(LBM_E_INVALID);
        inst_bytes = v.size() * sizeof(Inst<float>);
        inst_host.assign((unsigned char *)v.data(), (unsigned char *)v.data() + inst_bytes);
    }
    const size_t fbytes = (size_t)kQ * b->ntot * b->esz;
    if (dev_alloc(&b->inst_dev, inst_bytes) != cudaSuccess || dev_alloc((void **)&b->table_dev, table.size() * sizeof(int)) != cudaSuccess ||
        dev_alloc(&b->f[0], fbytes) != cudaSuccess || dev_alloc(&b->f[1], fbytes) != cudaSuccess ||
        dev_alloc(&b->q, b->ntot * b->esz) != cudaSuccess || dev_alloc(&b->stage_dev, b->ntot * b->esz) != cudaSuccess ||
        dev_alloc((void **)&b->err, sizeof(int)) != cudaSuccess || dev_alloc((void **)&b->bar, sizeof(BarrierState)) != cudaSuccess ||
        dev_alloc((void **)&b->order_dev, n * sizeof(int)) != cudaSuccess ||
        host_alloc(&b->stage_host, b->ntot * sizeof(double)) != cudaSuccess)
        return bail(LBM_E_NOMEM);
    // the instances' bounds-check error word (LBM_CHECKED builds) is the batch's
    for (int i = 0; i < n; ++i) {
        if (prec == LBM_F64) reinterpret_cast<Inst<double> *>(inst_host.data())[i].m.chk = b->err;
        else reinterpret_cast<Inst<float> *>(inst_host.data())[i].m.chk = b->err;
    }
    if (cudaMemcpy(b->inst_dev, inst_host.data(), inst_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->table_dev, table.data(), table.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->order_dev, order.data(), n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->f[0], 0, fbytes) != cudaSuccess || cudaMemset(b->f[1], 0, fbytes) != cudaSuccess ||
        cudaMemset(b->err, 0, sizeof(int)) != cudaSuccess)
        return bail(LBM_E_CUDA);
    // default launch shape: 256 threads, as many co-resident blocks as occupancy allows
    const int per_sm = prec == LBM_F64 ? max_blocks_per_sm<double>(256) : max_blocks_per_sm<float>(256);
    if (per_sm < 1) return bail(LBM_E_CUDA);
    b->block_threads = 256;
    b->grid_blocks = per_sm * sm_count();
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_set_launch(lbm_batch *b, int block_threads, int blocks_per_sm) {
    if (!b) return LBM_E_INVALID;
    if (block_threads != 128 && block_threads != 256 && block_threads != 512)
        return bfail(b, LBM_E_INVALID, "block_threads must be 128, 256 or 512");
    const int maxb = b->prec == LBM_F64 ? max_blocks_per_sm<double>(block_threads) : max_blocks_per_sm<float>(block_threads);
    if (blocks_per_sm < 1 || blocks_per_sm > maxb)
        return bfail(b, LBM_E_INVALID, "blocks_per_sm must be in [1, " + std::to_string(maxb) + "]");
    b->block_threads = block_threads;
    b->grid_blocks = blocks_per_sm * sm_count();
    b->cluster = 0;   // an explicit grid shape selects the grid form
    return LBM_OK;
}

lbm_status lbm_batch_get_launch(lbm_batch *b, int *block_threads, int *grid_blocks) {
    if (!b || !block_threads || !grid_blocks) return LBM_E_INVALID;
    *block_threads = b->cluster != 0 ? b->cluster_threads : b->block_threads;
    int blocks = b->grid_blocks;
    if (b->cluster > 0) blocks = b->cluster * b->n;
    if (b->cluster < 0) {
        blocks = 0;
        for (const auto &G : b->groups) blocks += G.cluster * G.count;
    }
    *grid_blocks = blocks;
    return LBM_OK;
}

lbm_status lbm_batch_set_cluster(lbm_batch *b, int cluster, int block_threads) {
    if (!b) return LBM_E_INVALID;
    if (cluster == 0) {
        b->cluster = 0;
        return LBM_OK;
    }
    if (cluster != 2 && cluster != 4 && cluster != 8)
        return bfail(b, LBM_E_INVALID, "cluster must be 0, 2, 4 or 8");
    if (block_threads != 128 && block_threads != 256 && block_threads != 512 && block_threads != 1024)
        return bfail(b, LBM_E_INVALID, "block_threads must be 128, 256, 512 or 1024");
    const size_t smem = cluster_smem_bytes(b, cluster);
    if (smem == 0) return bfail(b, LBM_E_INVALID, "an instance does not split over a cluster of this size");
    const char *why = b->prec == LBM_F64 ? configure_cluster<double>(b, cluster, block_threads, smem)
                                         : configure_cluster<float>(b, cluster, block_threads, smem);
    if (why) return bfail(b, LBM_E_INVALID, why);
    b->cluster = cluster;
    b->cluster_threads = block_threads;
    b->cluster_smem = smem;
    return LBM_OK;
}

lbm_status lbm_batch_set_groups(lbm_batch *b, int max_smem_bytes, int block_threads) {
    if (!b) return LBM_E_INVALID;
    if (block_threads != 256 && block_threads != 512 && block_threads != 1024)
        return bfail(b, LBM_E_INVALID, "block_threads must be 256, 512 or 1024");
    if (max_smem_bytes < LBM_GROUPS_BALANCED) return bfail(b, LBM_E_INVALID, "max_smem_bytes must be >= -1");
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return bfail(b, LBM_E_CUDA, "device attributes");
    auto slice_bytes = [&](int i, int C) {   // both buffers and the haloed field of instance i's widest slice
        const int nx = b->params[i].nx, ny = b->params[i].ny, wmax = (nx + C - 1) / C;
        return ((size_t)2 * kQ * wmax * ny + (size_t)ny * (wmax + 2 * b->halo[i])) * b->esz;
    };
    size_t cap = max_smem_bytes > 0 ? std::min<size_t>(max_smem_bytes, optin) : (size_t)optin;
    if (max_smem_bytes == LBM_GROUPS_BALANCED) {   // no CTA holds more than the largest 8-CTA slice
        cap = 0;
        for (int i = 0; i < b->n; ++i) cap = std::max(cap, slice_bytes(i, 8));
        cap = std::min(cap, (size_t)optin);
    }
    // each instance: the smallest cluster whose slices split it (no slice
    // narrower than the x halo) within `cap`, else within the opt-in maximum
    const int sizes[3] = {2, 4, 8};
    std::vector<int> pick(b->n, -1);
    std::vector<size_t> need(b->n, 0);
    for (int i = 0; i < b->n; ++i) {
        const int nx = b->params[i].nx;
        for (size_t limit : {cap, (size_t)optin}) {
            for (int g = 0; g < 3 && pick[i] < 0; ++g) {
                const int C = sizes[g], wmin = nx / C;
                const size_t bytes = slice_bytes(i, C);
                if (b->halo[i] <= wmin && bytes <= limit) {
                    pick[i] = g;
                    need[i] = bytes;
                }
            }
            if (pick[i] >= 0) break;
        }
        if (pick[i] < 0)
            return bfail(b, LBM_E_INVALID, "instance " + std::to_string(i) + " does not split over a cluster of 8");
    }
    std::vector<int> order(b->n);
    for (int i = 0; i < b->n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) {   // by group, then largest first
        if (pick[u] != pick[v]) return pick[u] > pick[v];
        return (long long)b->params[u].nx * b->params[u].ny > (long long)b->params[v].nx * b->params[v].ny;
    });
    std::vector<lbm_batch::Group> groups;
    size_t smax = 0;
    for (int k = 0; k < b->n; ++k) {
        const int i = order[k];
        if (groups.empty() || groups.back().cluster != sizes[pick[i]])
            groups.push_back({sizes[pick[i]], k, 0, 0});
        groups.back().count += 1;
        groups.back().smem = std::max(groups.back().smem, need[i]);
        smax = std::max(smax, need[i]);
    }
    // every group must place at least one cluster (the kernel attribute then
    // covers the largest group's shared memory)
    const bool f64 = b->prec == LBM_F64;
    for (const auto &G : groups) {
        const char *why = f64 ? configure_cluster<double>(b, G.cluster, block_threads, G.smem)
                              : configure_cluster<float>(b, G.cluster, block_threads, G.smem);
        if (why) return bfail(b, LBM_E_INVALID, why);
    }
    cudaError_t e = f64 ? cudaFuncSetAttribute(cluster_batch_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smax)
                        : cudaFuncSetAttribute(cluster_batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smax);
    BCK(b, e, "cudaFuncSetAttribute(grouped cluster form)");
    if (!b->gorder_dev) BCK(b, dev_alloc((void **)&b->gorder_dev, b->n * sizeof(int)), "cudaMalloc(group order)");
    for (int g = 0; g < 3; ++g) {
        if (!b->gstream[g]) BCK(b, cudaStreamCreateWithFlags(&b->gstream[g], cudaStreamNonBlocking), "stream");
        if (!b->gjoin[g]) BCK(b, cudaEventCreateWithFlags(&b->gjoin[g], cudaEventDisableTiming), "event");
    }
    if (!b->gfork) BCK(b, cudaEventCreateWithFlags(&b->gfork, cudaEventDisableTiming), "event");
    BCK(b, cudaMemcpyAsync(b->gorder_dev, order.data(), b->n * sizeof(int), cudaMemcpyHostToDevice, b->stream),
        "group order upload");
    BCK(b, cudaStreamSynchronize(b->stream), "group order upload");
    b->groups = groups;
    b->cluster = -1;
    b->cluster_threads = block_threads;
    b->groups_gen += 1;
    return LBM_OK;
}

lbm_status lbm_batch_get_groups(lbm_batch *b, int *ngroups, int *cluster, int *count, int *smem_bytes) {
    if (!b || !ngroups) return LBM_E_INVALID;
    *ngroups = b->cluster < 0 ? (int)b->groups.size() : 0;
    for (int g = 0; g < *ngroups; ++g) {
        if (cluster) cluster[g] = b->groups[g].cluster;
        if (count) count[g] = b->groups[g].count;
        if (smem_bytes) smem_bytes[g] = (int)b->groups[g].smem;
    }
    return LBM_OK;
}

lbm_status lbm_batch_get_cluster(lbm_batch *b, int *cluster) {
    if (!b || !cluster) return LBM_E_INVALID;
    *cluster = b->cluster;
    return LBM_OK;
}

lbm_status lbm_batch_init_density(lbm_batch *b, const double *rho) {
    if (!b || !rho) return LBM_E_INVALID;
    // scatter the concatenated fields (instance after instance, nx*ny each) to the padded layout
    std::vector<unsigned char> tmp;
    const size_t esz = b->esz;
    unsigned char *h = (unsigned char *)b->stage_host;
    BCK(b, cudaStreamSynchronize(b->stream), "sync before staging");
    std::fill(h, h + b->ntot * esz, 0);
    long long src = 0;
    for (int i = 0; i < b->n; ++i) {
        long long cells = (long long)b->params[i].nx * b->params[i].ny;
        for (long long c = 0; c < cells; ++c) {
            double v = rho[src + c];
            if (!(v > 0) || !std::isfinite(v)) return bfail(b, LBM_E_INVALID, "rho must be positive and finite");
            if (esz == sizeof(double)) ((double *)h)[b->off[i] + c] = v;
            else ((float *)h)[b->off[i] + c] = (float)v;
        }
        src += cells;
    }
    BCK(b, cudaMemcpyAsync(b->stage_dev, h, b->ntot * esz, cudaMemcpyHostToDevice, b->stream), "copy rho");
    b->cur = 0;
    const int blocks = (int)std::min<long long>((b->ntot + 255) / 256, 152 * 16);
    if (b->prec == LBM_F64)
        batch_init_kernel<double><<<blocks, 256, 0, b->stream>>>((const Inst<double> *)b->inst_dev, b->table_dev,
                                                                 (const double *)b->stage_dev, (double *)b->f[0], b->ntot);
    else
        batch_init_kernel<float><<<blocks, 256, 0, b->stream>>>((const Inst<float> *)b->inst_dev, b->table_dev,
                                                                (const float *)b->stage_dev, (float *)b->f[0], b->ntot);
    BCK(b, cudaGetLastError(), "init kernel");
    BCK(b, cudaMemsetAsync(b->err, 0, sizeof(int), b->stream), "clear error word");
    b->initialized = true;
    b->unstable = false;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, int nsteps) {
    NvtxRange nvtx("lbm_batch_step");
    if (!b) return LBM_E_INVALID;
    if (!b->initialized) return bfail(b, LBM_E_STATE, "batch not initialised");
    if (b->unstable) return bfail(b, LBM_E_UNSTABLE, "batch is in the error state");
    if (nsteps < 0) return bfail(b, LBM_E_INVALID, "nsteps must be >= 0");
    return b->prec == LBM_F64 ? run_steps<double>(b, nsteps) : run_steps<float>(b, nsteps);
}

lbm_status lbm_batch_sync(lbm_batch *b) {
    if (!b) return LBM_E_INVALID;
    return batch_sync(b);
}

lbm_status lbm_batch_density(lbm_batch *b, double *rho) {
    if (!b || !rho) return LBM_E_INVALID;
    if (!b->initialized) return bfail(b, LBM_E_STATE, "batch not initialised");
    const int blocks = (int)std::min<long long>((b->ntot + 255) / 256, 152 * 16);
    if (b->prec == LBM_F64)
        batch_density_kernel<double><<<blocks, 256, 0, b->stream>>>((const Inst<double> *)b->inst_dev, b->table_dev,
                                                                    (const double *)b->f[b->cur], (double *)b->stage_dev, b->ntot);
    else
        batch_density_kernel<float><<<blocks, 256, 0, b->stream>>>((const Inst<float> *)b->inst_dev, b->table_dev,
                                                                   (const float *)b->f[b->cur], (float *)b->stage_dev, b->ntot);
    BCK(b, cudaGetLastError(), "density kernel");
    BCK(b, cudaMemcpyAsync(b->stage_host, b->stage_dev, b->ntot * b->esz, cudaMemcpyDeviceToHost, b->stream), "copy rho");
    lbm_status st = batch_sync(b);
    if (st != LBM_OK && st != LBM_E_UNSTABLE) return st;
    long long dst = 0;
    for (int i = 0; i < b->n; ++i) {
        long long cells = (long long)b->params[i].nx * b->params[i].ny;
        for (long long c = 0; c < cells; ++c)
            rho[dst + c] = b->esz == sizeof(double) ? ((double *)b->stage_host)[b->off[i] + c]
                                                    : (double)((float *)b->stage_host)[b->off[i] + c];
        dst += cells;
    }
    return st;
}

lbm_status lbm_batch_moments(lbm_batch *b, double *rho, double *vx, double *vy) {
    if (!b || !rho) return LBM_E_INVALID;
    if (!b->initialized) return bfail(b, LBM_E_STATE, "batch not initialised");
    const size_t fb = b->ntot * b->esz;
    if (!b->mom_dev && dev_alloc(&b->mom_dev, 3 * fb) != cudaSuccess)
        return bfail(b, LBM_E_NOMEM, "moment buffers");
    if (!b->mom_host && host_alloc(&b->mom_host, 3 * fb) != cudaSuccess)
        return bfail(b, LBM_E_NOMEM, "pinned moment staging");
    const int blocks = (int)std::min<long long>((b->ntot + 255) / 256, 152 * 16);
    unsigned char *md = (unsigned char *)b->mom_dev;
    if (b->prec == LBM_F64) {
        const Inst<double> *inst = (const Inst<double> *)b->inst_dev;
        const double *f = (const double *)b->f[b->cur];
        batch_potential_kernel<double><<<blocks, 256, 0, b->stream>>>(inst, b->table_dev, f, (double *)b->q, b->ntot,
                                                                     b->err);
        batch_moments_kernel<double><<<blocks, 256, 0, b->stream>>>(inst, b->table_dev, f, (const double *)b->q,
                                                                    (double *)md, (double *)(md + fb),
                                                                    (double *)(md + 2 * fb), b->ntot);
    } else {
        const Inst<float> *inst = (const Inst<float> *)b->inst_dev;
        const float *f = (const float *)b->f[b->cur];
        batch_potential_kernel<float><<<blocks, 256, 0, b->stream>>>(inst, b->table_dev, f, (float *)b->q, b->ntot,
                                                                    b->err);
        batch_moments_kernel<float><<<blocks, 256, 0, b->stream>>>(inst, b->table_dev, f, (const float *)b->q,
                                                                   (float *)md, (float *)(md + fb),
                                                                   (float *)(md + 2 * fb), b->ntot);
    }
    BCK(b, cudaGetLastError(), "moments kernels");
    BCK(b, cudaMemcpyAsync(b->mom_host, b->mom_dev, 3 * fb, cudaMemcpyDeviceToHost, b->stream), "copy moments");
    lbm_status st = batch_sync(b);
    if (st != LBM_OK && st != LBM_E_UNSTABLE) return st;
    double *out[3] = {rho, vx, vy};
    for (int k = 0; k < 3; ++k) {
        if (!out[k]) continue;
        const unsigned char *h = (const unsigned char *)b->mom_host + k * fb;
        long long dst = 0;
        for (int i = 0; i < b->n; ++i) {
            const long long cells = (long long)b->params[i].nx * b->params[i].ny;
            for (long long c = 0; c < cells; ++c)
                out[k][dst + c] = b->esz == sizeof(double) ? ((const double *)h)[b->off[i] + c]
                                                           : (double)((const float *)h)[b->off[i] + c];
            dst += cells;
        }
    }
    return st;
}

lbm_status lbm_batch_get_f(lbm_batch *b, double *f) {
    if (!b || !f) return LBM_E_INVALID;
    if (!b->initialized) return bfail(b, LBM_E_STATE, "batch not initialised");
    long long total = 0;
    for (int i = 0; i < b->n; ++i) total += (long long)b->params[i].nx * b->params[i].ny;
    std::vector<unsigned char> all((size_t)kQ * b->ntot * b->esz);
    BCK(b, cudaMemcpyAsync(all.data(), b->f[b->cur], all.size(), cudaMemcpyDeviceToHost, b->stream), "copy f");
    lbm_status st = batch_sync(b);
    if (st != LBM_OK && st != LBM_E_UNSTABLE) return st;
    // output: instance after instance, each 9 x ny x nx (SoA within the instance)
    long long dst = 0;
    for (int i = 0; i < b->n; ++i) {
        long long cells = (long long)b->params[i].nx * b->params[i].ny;
        for (int k = 0; k < kQ; ++k)
            for (long long c = 0; c < cells; ++c) {
                size_t idx = (size_t)k * b->ntot + b->off[i] + c;
                f[dst + k * cells + c] = b->esz == sizeof(double) ? ((double *)all.data())[idx]
                                                                  : (double)((float *)all.data())[idx];
            }
        dst += kQ * cells;
    }
    return st;
}

lbm_status lbm_batch_set_f(lbm_batch *b, const double *f) {
    if (!b || !f) return LBM_E_INVALID;
    std::vector<unsigned char> all((size_t)kQ * b->ntot * b->esz, 0);
    long long src = 0;
    for (int i = 0; i < b->n; ++i) {
        long long cells = (long long)b->params[i].nx * b->params[i].ny;
        for (int k = 0; k < kQ; ++k)
            for (long long c = 0; c < cells; ++c) {
                size_t idx = (size_t)k * b->ntot + b->off[i] + c;
                double v = f[src + k * cells + c];
                if (b->esz == sizeof(double)) ((double *)all.data())[idx] = v;
                else ((float *)all.data())[idx] = (float)v;
            }
        src += kQ * cells;
    }
    BCK(b, cudaMemcpyAsync(b->f[0], all.data(), all.size(), cudaMemcpyHostToDevice, b->stream), "copy f");
    BCK(b, cudaStreamSynchronize(b->stream), "sync f copy");
    BCK(b, cudaMemsetAsync(b->err, 0, sizeof(int), b->stream), "clear error word");
    b->cur = 0;
    b->initialized = true;
    b->unstable = false;
    return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch *b, int trial_steps, int *block_threads, int *grid_blocks) {
    NvtxRange nvtx("lbm_batch_tune");
    if (!b || trial_steps < 2) return LBM_E_INVALID;
    if (!b->initialized) return bfail(b, LBM_E_STATE, "batch not initialised");
    // work on a copy of the state: the trials advance it
    const size_t fbytes = (size_t)kQ * b->ntot * b->esz;
    void *save = nullptr;
    BCK(b, dev_alloc(&save, fbytes), "cudaMalloc(tune state)");
    const int cur0 = b->cur;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_t = b->block_threads, best_g = b->grid_blocks;
    int best_c = b->cluster, best_ct = b->cluster_threads;
    const int threads[3] = {128, 256, 512};
    lbm_status st = LBM_OK;
    if (cudaMemcpyAsync(save, b->f[cur0], fbytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess) st = LBM_E_CUDA;
    // a warm-up launch, then a timed one (plain launches: no graph per trial)
    auto trial = [&](float *ms) -> bool {
        const bool g = b->use_graph;
        b->use_graph = false;
        lbm_status s1 = b->prec == LBM_F64 ? run_steps<double>(b, 2) : run_steps<float>(b, 2);
        cudaEventRecord(e0, b->stream);
        lbm_status s2 = b->prec == LBM_F64 ? run_steps<double>(b, trial_steps) : run_steps<float>(b, trial_steps);
        cudaEventRecord(e1, b->stream);
        b->use_graph = g;
        if (s1 != LBM_OK || s2 != LBM_OK || cudaEventSynchronize(e1) != cudaSuccess) return false;
        return cudaEventElapsedTime(ms, e0, e1) == cudaSuccess;
    };
    // grid form: block sizes x co-resident blocks per SM
    b->cluster = 0;
    for (int ti = 0; ti < 3 && st == LBM_OK; ++ti) {
        const int maxb = b->prec == LBM_F64 ? max_blocks_per_sm<double>(threads[ti]) : max_blocks_per_sm<float>(threads[ti]);
        for (int per = 1; per <= maxb && st == LBM_OK; per = per < maxb && per * 2 > maxb ? maxb : per * 2) {
            b->block_threads = threads[ti];
            b->grid_blocks = per * sm_count();
            float ms = 0;
            if (!trial(&ms)) { st = LBM_E_CUDA; break; }
            if (ms < best) { best = ms; best_t = b->block_threads; best_g = b->grid_blocks; best_c = 0; }
            if (per == maxb) break;
        }
    }
    // cluster form: CTAs per instance x threads per CTA, where the instances split
    const int grid_t = best_t, grid_g = best_g;
    const int cthreads[3] = {256, 512, 1024};
    for (int c = 2; c <= 8 && st == LBM_OK; c *= 2) {
        for (int ti = 0; ti < 3 && st == LBM_OK; ++ti) {
            if (lbm_batch_set_cluster(b, c, cthreads[ti]) != LBM_OK) continue;
            float ms = 0;
            if (!trial(&ms)) { st = LBM_E_CUDA; break; }
            if (ms < best) {
                best = ms;
                best_c = c;
                best_ct = cthreads[ti];
            }
        }
    }
    // grouped cluster form: each instance on the smallest cluster whose slices
    // fit a shared-memory cap (balanced against the largest 8-CTA slice, the
    // whole opt-in size, or 72 KB), one launch per cluster size
    const int caps[3] = {LBM_GROUPS_BALANCED, 0, 72 * 1024};
    int best_cap = -1;
    for (int ci = 0; ci < 3 && st == LBM_OK; ++ci) {
        for (int ti = 0; ti < 3 && st == LBM_OK; ++ti) {
            if (lbm_batch_set_groups(b, caps[ci], cthreads[ti]) != LBM_OK) continue;
            float ms = 0;
            if (!trial(&ms)) { st = LBM_E_CUDA; break; }
            if (ms < best) {
                best = ms;
                best_c = -1;
                best_ct = cthreads[ti];
                best_cap = caps[ci];
            }
        }
    }
    b->block_threads = grid_t;
    b->grid_blocks = grid_g;
    b->cluster = 0;
    if (best_c > 0 && st == LBM_OK && lbm_batch_set_cluster(b, best_c, best_ct) != LBM_OK)
        st = LBM_E_CUDA;   // re-applies the kernel attributes of the winning shape
    if (best_c < 0 && st == LBM_OK && lbm_batch_set_groups(b, best_cap, best_ct) != LBM_OK) st = LBM_E_CUDA;
    // restore the state and the error word
    if (cudaMemcpyAsync(b->f[cur0], save, fbytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess) st = LBM_E_CUDA;
    b->cur = cur0;
    cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);
    cudaStreamSynchronize(b->stream);
    dev_free(save);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int t_out = 0, g_out = 0;
    lbm_batch_get_launch(b, &t_out, &g_out);
    if (block_threads) *block_threads = t_out;
    if (grid_blocks) *grid_blocks = g_out;
    return st == LBM_OK ? LBM_OK : bfail(b, st, "autotuning failed");
}

lbm_status lbm_batch_debug_skip_barrier(lbm_batch *b, int block, double limit_seconds) {
    if (!b || !(limit_seconds > 0) || limit_seconds > 60) return LBM_E_INVALID;
    b->skip_block = block;
    b->limit_ns = (unsigned long long)(limit_seconds * 1e9);
    return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->msg.c_str() : "null batch"; }

void lbm_batch_destroy(lbm_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    drop_graph(b, 0);
    drop_graph(b, 1);
    dev_free(b->inst_dev);
    dev_free(b->table_dev);
    dev_free(b->order_dev);
    dev_free(b->gorder_dev);
    for (int g = 0; g < 3; ++g) {
        if (b->gstream[g]) cudaStreamDestroy(b->gstream[g]);
        if (b->gjoin[g]) cudaEventDestroy(b->gjoin[g]);
    }
    if (b->gfork) cudaEventDestroy(b->gfork);
    dev_free(b->f[0]);
    dev_free(b->f[1]);
    dev_free(b->q);
    dev_free(b->stage_dev);
    dev_free(b->mom_dev);
    if (b->mom_host) host_free(b->mom_host);
    dev_free(b->err);
    dev_free(b->bar);
    if (b->stage_host) host_free(b->stage_host);
    delete b;
}

}  // extern "C"
