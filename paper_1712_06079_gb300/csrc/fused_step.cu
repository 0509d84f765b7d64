// Single-pass FP32 D2Q9 HDM pseudopotential step for sm_103a.
//
// One launch per time step reads f(t) and the potential field q(t) and
// writes f(t+1) and q(t+1) = potential of f(t+1), so a step moves 9 floats
// in + 9 floats out + 1 float in + 1 float out per cell (80 B) instead of
// the 116 B of the two-pass form.  The field is Phi = sqrt|U| (Eq. 21) for
// the Shan-Chen form, whose sign s at the cell itself is re-derived from the
// cell's own density, and U (Eq. 8) for the Zhang-Chen form.
//
// Decomposition.  A CTA of 8 warps owns a strip of TXI = 120 columns and a
// segment of up to SEG_H = 128 rows.  It sweeps the segment in slabs of 8
// rows, one warp per row and one lane per 4 consecutive cells (float4 SoA
// loads, 16 B per lane, 512 B per warp).  Lanes 1..30 hold the strip's
// columns; lanes 0 and 31 hold the 4-column groups just outside it, whose
// collision is recomputed so that rho(t+1) of every strip cell can be formed
// on chip (post-collision values of all eight neighbours are needed).
//
// Per slab:
//  1. the potential rows the HDM stencil needs (radius FK = 26 rows above and
//     below, FK columns left and right) are staged in an 80-row shared ring,
//     8 rows per chunk, by the bulk-copy engine (cp.async.bulk, one mbarrier
//     per chunk, issued one slab ahead).  The potential field is stored with
//     32 ghost columns on each side (periodic images), so every staged row is
//     one contiguous 16-byte-aligned copy; rows wrap periodically;
//  2. each lane loads f(t) of its 4 cells (9 float4), evaluates the explicit
//     periodic HDM stencil (the exact solution of the tridiagonal system of
//     Eq. 20, truncated at radius 26 where the neglected tail of the weights
//     changes the derivative of a smooth field by < 3e-9) along x
//     and y, the force (Eq. 22 Shan-Chen or Eq. 7 Zhang-Chen), the moments
//     (Eq. 3) and the exact-difference forcing with BGK (Eq. 1, 2, 10), and
//     stores the nine post-collision float4 into a 10-row shared ring.  The
//     rest population is formed as rho minus the other eight, so the FP32
//     collision conserves mass up to unbiased rounding (the FP32 D2Q9 weights
//     themselves do not sum to one);
//  3. after a barrier each warp gathers row y-1 of the slab (streaming: pull
//     from the ring, x shifts by warp shuffles), sums rho(t+1), evaluates the
//     EOS potential (Eq. 8, 21) and writes f(t+1) and q(t+1) (with ghosts).
// The segment's first slab is shifted one row up so that the rows above the
// segment are recomputed too; the collision work overhead is 8/120 in x and
// about 8/128 in y.
#include <cuda_runtime.h>

#include <algorithm>

#include "lbm_internal.h"
#include "ptx.cuh"

namespace lbm {
namespace {

constexpr int FK = 26;              // HDM radius of this path
constexpr int TXI = 120;            // interior columns per strip
constexpr int QG = 32;              // ghost columns on each side of a padded potential row
constexpr int QW = TXI + 2 * QG;    // floats per staged potential row
constexpr int SLAB = 8;             // rows per slab (one warp each)
constexpr int QCH = 10;             // chunks in the potential ring
constexpr int QRING = QCH * SLAB;   // staged potential rows
constexpr int QBASE = 33;           // chunk 0 starts at row ys - QBASE
constexpr int FROWS = 10;           // post-collision rows kept
constexpr int SEG_H = 128;          // rows per CTA segment
constexpr int NTHR = 32 * SLAB;
constexpr uint64_t kWaitLimitNs = 200ull * 1000 * 1000;  // 0.2 s per chunk wait

constexpr size_t kQsBytes = sizeof(float) * QRING * QW;
constexpr size_t kFsBytes = sizeof(float4) * 9 * FROWS * 32;
constexpr size_t kSmemBytes = kQsBytes + kFsBytes + sizeof(uint64_t) * QCH;

struct FusedArgs {
    Model<float> m;
    const float *f;
    float *fout;
    const float *qin;   // padded field of f(t): row pitch qpitch, column x at x + QG
    float *qout;        // padded field of f(t+1)
    int *err;
    int qpitch;         // nx + 2 * QG
};

__device__ __forceinline__ int wrapi(int i, int n) {
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}

// Field staged for the stencil: Phi = sqrt|U| (SC, Eq. 21) or U (ZC, Eq. 8).
__device__ __forceinline__ float stencil_field(const Model<float> &m, float rho, bool sc) {
    float U = potential_u(m, rho);
    return sc ? sqrtf(fabsf(U)) : U;
}

// Post-collision populations of one cell (Eq. 1 with the exact-difference
// forcing of Eq. 10): f_i* = (1 - omega)(f_i - feq_i(u)) + feq_i(u + F/rho)
// for i = 1..8 and f_0* = rho - sum_{i>0} f_i*.
__device__ __forceinline__ void collide_cell(float (&f)[9], float r, float Fx, float Fy, float omega) {
    float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    float jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
    float inv = 1.0f / r;
    float ux = jx * inv, uy = jy * inv;
    float vx = ux + Fx * inv, vy = uy + Fy * inv;
    const float om1 = 1.0f - omega;
    float uu = ux * ux + uy * uy, vv = vx * vx + vy * vy;
    float r9 = r * (1.0f / 9.0f), r36 = r * (1.0f / 36.0f);
    float au = 1.0f - 1.5f * uu, av = 1.0f - 1.5f * vv;
    float eq_u[9], eq_v[9];
    {   // axis pairs (1,3) along x, (2,4) along y
        float su = au + 4.5f * ux * ux, sv = av + 4.5f * vx * vx;
        eq_u[1] = r9 * (su + 3.0f * ux); eq_u[3] = r9 * (su - 3.0f * ux);
        eq_v[1] = r9 * (sv + 3.0f * vx); eq_v[3] = r9 * (sv - 3.0f * vx);
        su = au + 4.5f * uy * uy; sv = av + 4.5f * vy * vy;
        eq_u[2] = r9 * (su + 3.0f * uy); eq_u[4] = r9 * (su - 3.0f * uy);
        eq_v[2] = r9 * (sv + 3.0f * vy); eq_v[4] = r9 * (sv - 3.0f * vy);
    }
    {   // diagonal pairs (5,7) along (1,1), (6,8) along (-1,1)
        float p = ux + uy, q = vx + vy;
        float su = au + 4.5f * p * p, sv = av + 4.5f * q * q;
        eq_u[5] = r36 * (su + 3.0f * p); eq_u[7] = r36 * (su - 3.0f * p);
        eq_v[5] = r36 * (sv + 3.0f * q); eq_v[7] = r36 * (sv - 3.0f * q);
        p = uy - ux; q = vy - vx;
        su = au + 4.5f * p * p; sv = av + 4.5f * q * q;
        eq_u[6] = r36 * (su + 3.0f * p); eq_u[8] = r36 * (su - 3.0f * p);
        eq_v[6] = r36 * (sv + 3.0f * q); eq_v[8] = r36 * (sv - 3.0f * q);
    }
    float moved = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        f[i] = fmaf(om1, f[i] - eq_u[i], eq_v[i]);
        moved += f[i];
    }
    f[0] = r - moved;
}

template <bool SC>
__global__ void __launch_bounds__(NTHR, 2) fused_step_kernel(const __grid_constant__ FusedArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    float *qs = reinterpret_cast<float *>(smem);                        // [QRING][QW]
    float4 *fs = reinterpret_cast<float4 *>(smem + kQsBytes);           // [9][FROWS][32]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kQsBytes + kFsBytes);

    const Model<float> &m = A.m;
    const int nx = m.nx, ny = m.ny;
    const long long N = (long long)nx * ny;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * TXI;
    const int nint = min(TXI, nx - x0);             // interior columns (multiple of 4)
    const int ys = blockIdx.y * SEG_H;
    const int hseg = min(SEG_H, ny - ys);
    const int nslab = hseg > 6 ? (hseg - 6 + SLAB - 1) / SLAB + 1 : 1;
    const int nchunks = nslab + 8;
    const uint32_t row_bytes = (uint32_t)(nint + 2 * QG) * sizeof(float);
    const int glast = nint / 4 + 1;                 // right ring lane
    const bool active = lane <= glast;
    const bool interior = lane >= 1 && lane < glast;

    if (threadIdx.x == 0) {
        for (int i = 0; i < QCH; ++i) ptx::mbar_init(&bars[i], 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();

    // chunk c holds relative rows 8c .. 8c+7, i.e. global rows ys - QBASE + 8c + k,
    // in ring rows (8c + k) mod QRING
    auto issue_chunk = [&](int c) {
        uint64_t *bar = &bars[c % QCH];
        ptx::mbar_arrive_expect_tx(bar, SLAB * row_bytes);
        for (int k = 0; k < SLAB; ++k) {
            int ry = SLAB * c + k;
            int y = wrapi(ys - QBASE + ry, ny);
            ptx::bulk_g2s(qs + (ry % QRING) * QW, A.qin + (long long)y * A.qpitch + x0, row_bytes, bar);
        }
    };
    int issued = 0;  // chunks issued so far (meaningful in thread 0)
    if (threadIdx.x == 0)
        for (; issued < min(QCH, nchunks); ++issued) issue_chunk(issued);

    const int xg = x0 - 4 + 4 * lane;               // first of this lane's 4 columns
    const int xgw = wrapi(xg, nx);
    bool timed_out = false;

    for (int s = 0; s < nslab; ++s) {
        if (threadIdx.x == 0 && s >= 1 && s + QCH - 1 < nchunks) {
            ptx::fence_proxy_async_smem();
            issue_chunk(s + QCH - 1);
            issued = s + QCH;
        }
        // ---- collision of row yc = ys - 1 + 8s + warp ----
        const int yc = ys - 1 + SLAB * s + warp;
        const int ryc = SLAB * s + warp + QBASE - 1;     // relative row of yc
        float fv[4][9];
        if (active) {
            const float *src = A.f + (long long)wrapi(yc, ny) * nx + xgw;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                float4 v = __ldg(reinterpret_cast<const float4 *>(src + i * N));
                fv[0][i] = v.x; fv[1][i] = v.y; fv[2][i] = v.z; fv[3][i] = v.w;
            }
        }
        {
            const int cfirst = s == 0 ? 0 : s + 8, clast = min(s + 8, nchunks - 1);
            for (int c = cfirst; c <= clast; ++c)
                if (!ptx::mbar_wait_bounded(&bars[c % QCH], (c / QCH) & 1, kWaitLimitNs)) timed_out = true;
        }
        if (active && !timed_out) {
            float dx[4] = {0.f, 0.f, 0.f, 0.f}, dy[4] = {0.f, 0.f, 0.f, 0.f}, qc[4];
            // d/dx: window of staged columns 4 lane .. 4 lane + 59 of row yc; the
            // lane's cells sit at window positions 28..31
            {
                const float *qrow = qs + (ryc % QRING) * QW + 4 * lane;
#pragma unroll
                for (int k = 0; k < 15; ++k) {
                    float4 v4 = *reinterpret_cast<const float4 *>(qrow + 4 * k);
                    const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int pos = 4 * k + e;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int j = pos - 28 - c;
                            if (j >= 1 && j <= FK) dx[c] = fmaf(m.wx[j], v[e], dx[c]);
                            if (j <= -1 && j >= -FK) dx[c] = fmaf(-m.wx[-j], v[e], dx[c]);
                            if (j == 0) qc[c] = v[e];
                        }
                    }
                }
            }
            // d/dy: rows yc - FK .. yc + FK at the lane's 4 columns (ring wraps once at most)
            {
                const float *qcol = qs + 28 + 4 * lane;
                const int base = ryc % QRING;
#pragma unroll
                for (int j = -FK; j <= FK; ++j) {
                    if (j == 0) continue;
                    int row = base + j;
                    if (j > 0) row = row >= QRING ? row - QRING : row;
                    else row = row < 0 ? row + QRING : row;
                    float4 v = *reinterpret_cast<const float4 *>(qcol + row * QW);
                    const float w = j > 0 ? m.wy[j] : -m.wy[-j];
                    dy[0] = fmaf(w, v.x, dy[0]);
                    dy[1] = fmaf(w, v.y, dy[1]);
                    dy[2] = fmaf(w, v.z, dy[2]);
                    dy[3] = fmaf(w, v.w, dy[3]);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float r = ((fv[c][0] + fv[c][1]) + (fv[c][2] + fv[c][3])) +
                          ((fv[c][4] + fv[c][5]) + (fv[c][6] + fv[c][7])) + fv[c][8];
                if (!(r > 0.f) || !isfinite(r)) atomicOr(A.err, kErrUnstable);
                float Fx, Fy;
                if (SC) {   // Eq. 22: F = -2 s Phi grad Phi, s the sign of U at the cell
                    float sphi = potential_u(m, r) >= 0.f ? qc[c] : -qc[c];
                    Fx = -2.0f * sphi * dx[c];
                    Fy = -2.0f * sphi * dy[c];
                } else {    // Eq. 7: F = -grad U
                    Fx = -dx[c];
                    Fy = -dy[c];
                }
                collide_cell(fv[c], r, Fx, Fy, m.omega);
            }
            const int slot = (SLAB * s + warp + 2) % FROWS;
#pragma unroll
            for (int i = 0; i < 9; ++i)
                fs[(i * FROWS + slot) * 32 + lane] = make_float4(fv[0][i], fv[1][i], fv[2][i], fv[3][i]);
        }
        if (__syncthreads_or(timed_out)) break;

        // ---- streaming gather and outputs for row yo = ys + 8s - 2 + warp ----
        const int yo = ys + SLAB * s - 2 + warp;
        if (yo >= ys && yo < ys + hseg) {           // warp-uniform
            const int ro = SLAB * s + warp + 1;     // relative row of yo in the f* ring
            float4 nf[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int slot = (ro - ey(i) + FROWS) % FROWS;
                float4 a = fs[(i * FROWS + slot) * 32 + lane];
                if (ex(i) == 1) {          // f_i(x) = f_i*(x - 1)
                    float left = __shfl_up_sync(0xffffffffu, a.w, 1);
                    a = make_float4(left, a.x, a.y, a.z);
                } else if (ex(i) == -1) {  // f_i(x) = f_i*(x + 1)
                    float right = __shfl_down_sync(0xffffffffu, a.x, 1);
                    a = make_float4(a.y, a.z, a.w, right);
                }
                nf[i] = a;
            }
            if (interior) {
                float4 rho;
                rho.x = ((nf[0].x + nf[1].x) + (nf[2].x + nf[3].x)) + ((nf[4].x + nf[5].x) + (nf[6].x + nf[7].x)) + nf[8].x;
                rho.y = ((nf[0].y + nf[1].y) + (nf[2].y + nf[3].y)) + ((nf[4].y + nf[5].y) + (nf[6].y + nf[7].y)) + nf[8].y;
                rho.z = ((nf[0].z + nf[1].z) + (nf[2].z + nf[3].z)) + ((nf[4].z + nf[5].z) + (nf[6].z + nf[7].z)) + nf[8].z;
                rho.w = ((nf[0].w + nf[1].w) + (nf[2].w + nf[3].w)) + ((nf[4].w + nf[5].w) + (nf[6].w + nf[7].w)) + nf[8].w;
                float4 q;
                q.x = stencil_field(m, rho.x, SC);
                q.y = stencil_field(m, rho.y, SC);
                q.z = stencil_field(m, rho.z, SC);
                q.w = stencil_field(m, rho.w, SC);
                float *dst = A.fout + (long long)yo * nx + xg;
#pragma unroll
                for (int i = 0; i < 9; ++i) __stcs(reinterpret_cast<float4 *>(dst + i * N), nf[i]);
                float *qrow = A.qout + (long long)yo * A.qpitch + QG;
                *reinterpret_cast<float4 *>(qrow + xg) = q;
                if (xg < QG) *reinterpret_cast<float4 *>(qrow + xg + nx) = q;        // right ghost image
                if (xg >= nx - QG) *reinterpret_cast<float4 *>(qrow + xg - nx) = q;  // left ghost image
            }
        }
        __syncthreads();
    }

    if (timed_out) {
        if (threadIdx.x == 0) {
            atomicOr(A.err, kErrTimeout);
            // let copies still in flight land before the CTA's shared memory is released
            for (int c = max(0, issued - QCH); c < issued; ++c)
                (void)ptx::mbar_wait_bounded(&bars[c % QCH], (c / QCH) & 1, kWaitLimitNs);
        }
        __syncthreads();
    }
}

// Padded stencil field: qpad[y][QG + x] for x in [-QG, nx + QG), periodic.
__global__ void potential_pad_kernel(Model<float> m, bool sc, const float *__restrict__ f, float *__restrict__ qpad,
                                     int qpitch, int *__restrict__ err) {
    const long long n = (long long)m.nx * m.ny;
    const long long total = (long long)qpitch * m.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total; c += (long long)gridDim.x * blockDim.x) {
        int y = (int)(c / qpitch), px = (int)(c - (long long)y * qpitch);
        int x = wrapi(px - QG, m.nx);
        long long cell = (long long)y * m.nx + x;
        float r = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) r += f[i * n + cell];
        if (!(r > 0.f) || !isfinite(r)) atomicOr(err, kErrUnstable);
        qpad[c] = stencil_field(m, r, sc);
    }
}

}  // namespace

bool fused_step_supported(const Model<float> &m, bool cdm, int radius) {
    return !cdm && radius == FK && m.kx == FK && m.ky == FK && m.nx % 4 == 0 && m.nx >= 2 * QG &&
           m.ny >= 2 * FK + 2;
}

int fused_q_pitch(int nx) { return nx + 2 * QG; }

cudaError_t launch_potential_padded(const Model<float> &m, bool sc, const float *f, float *qpad, int *err,
                                    cudaStream_t s) {
    const int pitch = fused_q_pitch(m.nx);
    long long total = (long long)pitch * m.ny;
    int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
    potential_pad_kernel<<<blocks, 256, 0, s>>>(m, sc, f, qpad, pitch, err);
    return cudaGetLastError();
}

cudaError_t launch_fused_step(const Model<float> &m, bool sc, const float *f, const float *qin, float *fout,
                              float *qout, int *err, cudaStream_t s) {
    FusedArgs a;
    a.m = m;
    a.f = f;
    a.fout = fout;
    a.qin = qin;
    a.qout = qout;
    a.err = err;
    a.qpitch = fused_q_pitch(m.nx);
    dim3 grid((m.nx + TXI - 1) / TXI, (m.ny + SEG_H - 1) / SEG_H);
    auto kern = sc ? fused_step_kernel<true> : fused_step_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    kern<<<grid, NTHR, kSmemBytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbm
