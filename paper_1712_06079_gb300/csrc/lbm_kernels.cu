// Two-pass D2Q9 HDM pseudopotential step for sm_103a (FP32 and FP64).
//
// Pass 1 (potential_kernel): one thread per cell reads the nine SoA
// distributions (coalesced along x), forms rho (Eq. 3) and writes the
// potential field q: the signed root s*sqrt|U| for the Shan-Chen form
// (Eq. 21/22) or U itself for the Zhang-Chen form (Eq. 7/8).
//
// Pass 2 (collide_kernel): a CTA owns a TX x TY tile.  It stages q over the
// tile plus the cross-shaped halo the gradient needs (K cells left/right on
// the tile's rows for d/dx, K rows above/below on its columns for d/dy, with
// the periodic wrap, or across no-slip walls in y the mirror image of the
// field) in shared memory, then each thread takes TY/TYT cells of one column:
// the explicit HDM stencil (the exact periodic solve of Eq. 20, truncated at
// radius K where the weights fall below the working precision; with walls the
// periodic operator of the mirrored column) or the CDM of Eq. 15, the force
// (Eq. 22 or Eq. 7), the exact-difference forcing with BGK (Eq. 1, 2, 10),
// and a push store of f_i* to x + e_i (with walls, a population that would
// cross one returns to its cell reversed: half-way bounce-back).
//
// FP32 lattices run these kernels in the mixed form: the distributions stay
// FP32 in memory, every operation is FP64, and the potential field between the
// passes is FP64.  A plain FP32 evaluation of the step drifts the interfaces of
// a flat PR slab by ~1e-4 of a cell in 1000 steps through rounding that is
// identical in neighbouring cells (so it does not average out), while FP32
// storage alone stays within 1e-5 of the FP64 result; the single-pass FP32
// kernel keeps FP32 arithmetic.
//
// gradient_kernel applies the same staging and operator to a caller's field.
// The bytes per cell are f read twice (pass 1 and 2), f written once and q
// written once and read once (halo re-reads hit L2).
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {
namespace {

template <typename T>
struct Tile;
template <>
struct Tile<float> {
    static constexpr int TX = 64, TY = 32, TYT = 4;
};
template <>
struct Tile<double> {
    static constexpr int TX = 32, TY = 16, TYT = 4;
};

template <typename T>
__global__ void init_kernel(Model<T> m, const T *__restrict__ rho, const T *__restrict__ ux,
                            const T *__restrict__ uy, T *__restrict__ f) {
    const long long n = (long long)m.nx * m.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        T r = rho[c];
        T u = ux ? ux[c] : T(0), v = uy ? uy[c] : T(0);
        T uu = u * u + v * v;
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            T eu = T(ex(i)) * u + T(ey(i)) * v;
            f[i * n + c] = r * wq<T>(i) * (T(1) + T(3) * eu + T(4.5) * eu * eu - T(1.5) * uu);
        }
    }
}

// TS: storage type of f; T: arithmetic type (and the type of q).
template <typename TS, typename T>
__global__ void potential_kernel(Model<T> m, bool sc, const TS *__restrict__ f, T *__restrict__ q,
                                 int *__restrict__ err) {
    const long long n = (long long)m.nx * m.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        T r = T(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) r += T(f[i * n + c]);
        if (!(r > T(0)) || !isfinite(r)) atomicOr(err, kErrUnstable);
        q[c] = potential_field(m, r, sc);
    }
}

// One cell's gradient from the staged tile.  `row` points at the cell in
// shared memory; W is the row pitch.
template <typename T, bool SC, bool CDM>
__device__ __forceinline__ void gradient(const Model<T> &m, const T *row, int W, T &dx, T &dy) {
    if (CDM) {
        // Eq. 15 times 1/c_s^2: (1/3)(q_E - q_W) + (1/12)(q_NE + q_SE - q_NW - q_SW)
        auto g = [&](int o) { return SC ? fabs(row[o]) : row[o]; };
        T e = g(1), w = g(-1), nn = g(W), s = g(-W);
        T ne = g(W + 1), nw = g(W - 1), se = g(-W + 1), sw = g(-W - 1);
        dx = T(1.0 / 3.0) * (e - w) + T(1.0 / 12.0) * ((ne + se) - (nw + sw));
        dy = T(1.0 / 3.0) * (nn - s) + T(1.0 / 12.0) * ((ne + nw) - (se + sw));
    } else {
        T ax = T(0), ay = T(0);
        for (int j = 1; j <= m.kx; ++j) {
            T d = SC ? fabs(row[j]) - fabs(row[-j]) : row[j] - row[-j];
            ax += m.wx[j] * d;
        }
        for (int j = 1; j <= m.ky; ++j) {
            T d = SC ? fabs(row[j * W]) - fabs(row[-j * W]) : row[j * W] - row[-j * W];
            ay += m.wy[j] * d;
        }
        dx = ax;
        dy = ay;
    }
}

// Stage q over the tile and its halo (rows y0-hy .. y0+TY+hy-1, columns
// x0-hx .. x0+TX+hx-1; the four corners only for CDM).
template <typename T, int TX, int TY, bool CDM>
__device__ __forceinline__ void stage_tile(const Model<T> &m, const T *__restrict__ q, T *S, int hx, int hy, int x0,
                                           int y0) {
    const int W = TX + 2 * hx, H = TY + 2 * hy;
    const int nthr = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int idx = tid; idx < W * H; idx += nthr) {
        int r = idx / W, c = idx - r * W;
        bool inx = c >= hx && c < hx + TX, iny = r >= hy && r < hy + TY;
        if (!CDM && !inx && !iny) continue;
        int gx = wrap_index(x0 - hx + c, m.nx);
        int gy = m.walls ? mirror_index(y0 - hy + r, m.ny) : wrap_index(y0 - hy + r, m.ny);
        const long long k = (long long)gy * m.nx + gx;
        S[idx] = in_bounds(k, (long long)m.nx * m.ny, m.chk) ? q[k] : T(0);
    }
}

// TS: storage type of f and of the outputs; T: arithmetic type (and the type
// of q and of the staged tile).
template <typename TS, typename T, int TX, int TY, int TYT, bool SC, bool CDM, bool MOMENTS>
__global__ void __launch_bounds__(TX *TYT) collide_kernel(Model<T> m, const TS *__restrict__ f, const T *__restrict__ q,
                                                          TS *__restrict__ fout, TS *__restrict__ rho_out,
                                                          TS *__restrict__ vx_out, TS *__restrict__ vy_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    const int hx = CDM ? 1 : m.kx, hy = CDM ? 1 : m.ky;
    const int W = TX + 2 * hx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    stage_tile<T, TX, TY, CDM>(m, q, S, hx, hy, x0, y0);
    __syncthreads();

    const long long n = (long long)m.nx * m.ny;
    const int lx = threadIdx.x, x = x0 + lx;
    if (x >= m.nx) return;
    const int xp = x + 1 == m.nx ? 0 : x + 1, xm = x == 0 ? m.nx - 1 : x - 1;
#pragma unroll 2
    for (int k = 0; k < TY / TYT; ++k) {
        const int ly = threadIdx.y + k * TYT, y = y0 + ly;
        if (y >= m.ny) break;
        const T *row = S + (ly + hy) * W + (lx + hx);
        T dx, dy;
        gradient<T, SC, CDM>(m, row, W, dx, dy);
        T Fx, Fy;
        if (SC) {  // Eq. 22: F = -2 s Phi grad Phi, row[0] = s Phi
            Fx = T(-2) * row[0] * dx;
            Fy = T(-2) * row[0] * dy;
        } else {  // Eq. 7: F = -grad U
            Fx = -dx;
            Fy = -dy;
        }
        const long long c = (long long)y * m.nx + x;
        T fi[kQ];
#pragma unroll
        for (int i = 0; i < kQ; ++i) fi[i] = in_bounds(i * n + c, kQ * n, m.chk) ? T(f[i * n + c]) : T(0);
        T r = T(0), jx = T(0), jy = T(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            r += fi[i];
            jx += T(ex(i)) * fi[i];
            jy += T(ey(i)) * fi[i];
        }
        if (MOMENTS) {  // Eq. 3 and Eq. 11
            rho_out[c] = TS(r);
            vx_out[c] = TS((jx + T(0.5) * Fx) / r);
            vy_out[c] = TS((jy + T(0.5) * Fy) / r);
            continue;
        }
        const T inv = T(1) / r;
        const T ux = jx * inv, uy = jy * inv;
        const T vx = ux + Fx * inv, vy = uy + Fy * inv;  // u + du, du = F/rho (Eq. 10)
        const T uu = ux * ux + uy * uy, vv = vx * vx + vy * vy;
        const int yp = y + 1 == m.ny ? 0 : y + 1, ym = y == 0 ? m.ny - 1 : y - 1;
        // f_i* for the eight moving populations; the rest population takes the
        // remainder so that the collision conserves mass up to rounding
        T moved = T(0);
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            const T eu = T(ex(i)) * ux + T(ey(i)) * uy;
            const T ev = T(ex(i)) * vx + T(ey(i)) * vy;
            const T feq = r * wq<T>(i) * (T(1) + T(3) * eu + T(4.5) * eu * eu - T(1.5) * uu);
            const T fsh = r * wq<T>(i) * (T(1) + T(3) * ev + T(4.5) * ev * ev - T(1.5) * vv);
            const T post = fi[i] - (fi[i] - feq) * m.omega + (fsh - feq);
            moved += post;
            const int dxs = ex(i) == 1 ? xp : (ex(i) == -1 ? xm : x);
            const int dys = ey(i) == 1 ? yp : (ey(i) == -1 ? ym : y);
            const long long k = m.walls && ((ey(i) == 1 && y == m.ny - 1) || (ey(i) == -1 && y == 0))
                                    ? opp(i) * n + c                             // half-way bounce-back off the wall
                                    : i * n + (long long)dys * m.nx + dxs;
            if (in_bounds(k, kQ * n, m.chk)) fout[k] = TS(post);
        }
        if (in_bounds(c, kQ * n, m.chk)) fout[c] = TS(r - moved);
    }
}

// Gradient of a plain field (no magnitude taken), divided by the grid spacing:
// the same tile staging and operator as the collision pass.
template <typename T, int TX, int TY, int TYT, bool CDM>
__global__ void __launch_bounds__(TX *TYT) gradient_kernel(Model<T> m, const T *__restrict__ q, T inv_h,
                                                           T *__restrict__ gx, T *__restrict__ gy) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    const int hx = CDM ? 1 : m.kx, hy = CDM ? 1 : m.ky;
    const int W = TX + 2 * hx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    stage_tile<T, TX, TY, CDM>(m, q, S, hx, hy, x0, y0);
    __syncthreads();
    const int lx = threadIdx.x, x = x0 + lx;
    if (x >= m.nx) return;
    for (int k = 0; k < TY / TYT; ++k) {
        const int ly = threadIdx.y + k * TYT, y = y0 + ly;
        if (y >= m.ny) break;
        T dx, dy;
        gradient<T, false, CDM>(m, S + (ly + hy) * W + (lx + hx), W, dx, dy);
        const long long c = (long long)y * m.nx + x;
        gx[c] = dx * inv_h;
        gy[c] = dy * inv_h;
    }
}

template <typename T>
dim3 grid_for(const Model<T> &m) {
    using Tl = Tile<T>;
    return dim3((m.nx + Tl::TX - 1) / Tl::TX, (m.ny + Tl::TY - 1) / Tl::TY);
}

template <typename T>
size_t smem_for(const Model<T> &m, bool cdm) {
    using Tl = Tile<T>;
    int hx = cdm ? 1 : m.kx, hy = cdm ? 1 : m.ky;
    return sizeof(T) * (size_t)(Tl::TX + 2 * hx) * (Tl::TY + 2 * hy);
}

template <typename TS, typename T, bool SC, bool CDM, bool MOM>
cudaError_t launch_collide_t(const Model<T> &m, const TS *f, const T *q, TS *fout, TS *r, TS *vx, TS *vy,
                             cudaStream_t s) {
    using Tl = Tile<T>;
    auto kern = collide_kernel<TS, T, Tl::TX, Tl::TY, Tl::TYT, SC, CDM, MOM>;
    size_t smem = smem_for(m, CDM);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid_for(m), dim3(Tl::TX, Tl::TYT), smem, s>>>(m, f, q, fout, r, vx, vy);
    return cudaGetLastError();
}

template <typename TS, typename T, bool MOM>
cudaError_t dispatch_collide(const Model<T> &m, bool sc, bool cdm, const TS *f, const T *q, TS *fout, TS *r, TS *vx,
                             TS *vy, cudaStream_t s) {
    if (sc) return cdm ? launch_collide_t<TS, T, true, true, MOM>(m, f, q, fout, r, vx, vy, s)
                       : launch_collide_t<TS, T, true, false, MOM>(m, f, q, fout, r, vx, vy, s);
    return cdm ? launch_collide_t<TS, T, false, true, MOM>(m, f, q, fout, r, vx, vy, s)
               : launch_collide_t<TS, T, false, false, MOM>(m, f, q, fout, r, vx, vy, s);
}

int flat_blocks(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

constexpr int kObsThreads = 256;
constexpr int kObsBlocks = 152 * 2;

template <typename T>
__global__ void obs_partial_kernel(long long n, const T *__restrict__ rho, const T *__restrict__ vx,
                                   const T *__restrict__ vy, double *__restrict__ partial) {
    double s_m = 0, s_x = 0, s_y = 0, v_max = 0, r_min = INFINITY, r_max = -INFINITY;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        double r = rho[c], u = vx[c], v = vy[c];
        s_m += r;
        s_x += r * u;
        s_y += r * v;
        v_max = fmax(v_max, sqrt(u * u + v * v));
        r_min = fmin(r_min, r);
        r_max = fmax(r_max, r);
    }
    __shared__ double sh[6][kObsThreads];
    sh[0][threadIdx.x] = s_m; sh[1][threadIdx.x] = s_x; sh[2][threadIdx.x] = s_y;
    sh[3][threadIdx.x] = v_max; sh[4][threadIdx.x] = r_min; sh[5][threadIdx.x] = r_max;
    __syncthreads();
    for (int st = kObsThreads / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            int o = threadIdx.x + st;
            sh[0][threadIdx.x] += sh[0][o]; sh[1][threadIdx.x] += sh[1][o]; sh[2][threadIdx.x] += sh[2][o];
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][o]);
            sh[4][threadIdx.x] = fmin(sh[4][threadIdx.x], sh[4][o]);
            sh[5][threadIdx.x] = fmax(sh[5][threadIdx.x], sh[5][o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) partial[k * gridDim.x + blockIdx.x] = sh[k][0];
}

__global__ void obs_final_kernel(int nb, const double *__restrict__ partial, lbm_obs *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[6] = {0, 0, 0, 0, INFINITY, -INFINITY};
    for (int b = 0; b < nb; ++b) {
        s[0] += partial[b]; s[1] += partial[nb + b]; s[2] += partial[2 * nb + b];
        s[3] = fmax(s[3], partial[3 * nb + b]);
        s[4] = fmin(s[4], partial[4 * nb + b]);
        s[5] = fmax(s[5], partial[5 * nb + b]);
    }
    out->mass = s[0]; out->mom_x = s[1]; out->mom_y = s[2];
    out->max_speed = s[3]; out->rho_min = s[4]; out->rho_max = s[5];
}

}  // namespace

// Host arrays read by the GPU in place: on a device that reads pageable host
// memory through the host's page tables (coherent NVLink-C2C), n FP64 values
// of a caller's array are converted to T on the device.  With `bad`, the
// lowest index of a value that is not a positive finite number is kept there
// (atomicMin; all ones if none).
template <typename T>
__global__ void from_host_kernel(const double *__restrict__ src, T *__restrict__ dst, long long n,
                                 unsigned long long *bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = src[i];
        if (bad && !(v > 0.0 && v <= 1.7976931348623157e308)) atomicMin(bad, (unsigned long long)i);
        dst[i] = (T)v;
    }
}

template <typename T>
cudaError_t launch_from_host(const double *src, T *dst, long long n, unsigned long long *bad, cudaStream_t s) {
    from_host_kernel<T><<<flat_blocks(n, 256), 256, 0, s>>>(src, dst, n, bad);
    return cudaGetLastError();
}

// ... and written back: n values of T converted to FP64 into a caller's
// resident pageable array, two per thread and step (16-byte stores where the
// array is 16-byte aligned).
template <typename T>
__global__ void to_host_kernel(const T *__restrict__ src, double *__restrict__ dst, long long n) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        const long long n2 = n / 2;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += stride)
            reinterpret_cast<double2 *>(dst)[i] = make_double2((double)src[2 * i], (double)src[2 * i + 1]);
        if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) dst[n - 1] = (double)src[n - 1];
    } else {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
            dst[i] = (double)src[i];
    }
}

template <typename T>
cudaError_t launch_to_host(const T *src, double *dst, long long n, cudaStream_t s) {
    to_host_kernel<T><<<flat_blocks(n / 2 + 1, 256), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init(const Model<T> &m, const T *rho, const T *ux, const T *uy, T *f, cudaStream_t s) {
    long long n = (long long)m.nx * m.ny;
    init_kernel<T><<<flat_blocks(n, 256), 256, 0, s>>>(m, rho, ux, uy, f);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_potential(const Model<T> &m, bool sc, const T *f, T *q, int *err, cudaStream_t s) {
    long long n = (long long)m.nx * m.ny;
    potential_kernel<T, T><<<flat_blocks(n, 256), 256, 0, s>>>(m, sc, f, q, err);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_collide(const Model<T> &m, bool sc, bool cdm, const T *f, const T *q, T *fout, cudaStream_t s) {
    return dispatch_collide<T, T, false>(m, sc, cdm, f, q, fout, nullptr, nullptr, nullptr, s);
}

template <typename T>
cudaError_t launch_moments(const Model<T> &m, bool sc, bool cdm, const T *f, const T *q, T *rho, T *vx, T *vy,
                           cudaStream_t s) {
    return dispatch_collide<T, T, true>(m, sc, cdm, f, q, nullptr, rho, vx, vy, s);
}

cudaError_t launch_potential_mixed(const Model<double> &m, bool sc, const float *f, double *q, int *err,
                                   cudaStream_t s) {
    long long n = (long long)m.nx * m.ny;
    potential_kernel<float, double><<<flat_blocks(n, 256), 256, 0, s>>>(m, sc, f, q, err);
    return cudaGetLastError();
}

cudaError_t launch_collide_mixed(const Model<double> &m, bool sc, bool cdm, const float *f, const double *q,
                                 float *fout, cudaStream_t s) {
    return dispatch_collide<float, double, false>(m, sc, cdm, f, q, fout, nullptr, nullptr, nullptr, s);
}

cudaError_t launch_moments_mixed(const Model<double> &m, bool sc, bool cdm, const float *f, const double *q,
                                 float *rho, float *vx, float *vy, cudaStream_t s) {
    return dispatch_collide<float, double, true>(m, sc, cdm, f, q, nullptr, rho, vx, vy, s);
}

template <typename T>
cudaError_t launch_gradient(const Model<T> &m, bool cdm, const T *q, T h, T *gx, T *gy, cudaStream_t s) {
    using Tl = Tile<T>;
    auto kern = cdm ? gradient_kernel<T, Tl::TX, Tl::TY, Tl::TYT, true> : gradient_kernel<T, Tl::TX, Tl::TY, Tl::TYT, false>;
    const size_t smem = smem_for(m, cdm);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid_for(m), dim3(Tl::TX, Tl::TYT), smem, s>>>(m, q, T(1) / h, gx, gy);
    return cudaGetLastError();
}

int observables_partial_count() { return kObsBlocks; }

template <typename T>
cudaError_t launch_observables(long long n, const T *rho, const T *vx, const T *vy, double *partial, lbm_obs *out,
                               cudaStream_t s) {
    obs_partial_kernel<T><<<kObsBlocks, kObsThreads, 0, s>>>(n, rho, vx, vy, partial);
    obs_final_kernel<<<1, 32, 0, s>>>(kObsBlocks, partial, out);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE(T)                                                                                      \
    template cudaError_t launch_init<T>(const Model<T> &, const T *, const T *, const T *, T *, cudaStream_t);  \
    template cudaError_t launch_from_host<T>(const double *, T *, long long, unsigned long long *, cudaStream_t); \
    template cudaError_t launch_to_host<T>(const T *, double *, long long, cudaStream_t);                       \
    template cudaError_t launch_potential<T>(const Model<T> &, bool, const T *, T *, int *, cudaStream_t);      \
    template cudaError_t launch_collide<T>(const Model<T> &, bool, bool, const T *, const T *, T *, cudaStream_t); \
    template cudaError_t launch_moments<T>(const Model<T> &, bool, bool, const T *, const T *, T *, T *, T *,   \
                                           cudaStream_t);                                                        \
    template cudaError_t launch_observables<T>(long long, const T *, const T *, const T *, double *, lbm_obs *,  \
                                               cudaStream_t);                                                    \
    template cudaError_t launch_gradient<T>(const Model<T> &, bool, const T *, T, T *, T *, cudaStream_t);
LBM_INSTANTIATE(float)
LBM_INSTANTIATE(double)

}  // namespace lbm
