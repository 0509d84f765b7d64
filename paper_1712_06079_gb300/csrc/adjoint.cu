// Reverse-time (adjoint) step of the D2Q9 HDM pseudopotential update, for
// gradients of a function of the final density with respect to the initial
// density field and the temperature.
//
// Forward step at a cell (Eq. 1-3, 7/8, 10, 20-22): rho = sum f, j = sum e f,
// U = k p_EOS(rho, T) - rho/3, stencil field Phi = sqrt|U| (SC) or U (ZC),
// D = (Dx, Dy) = the periodic HDM (or CDM) derivative of Phi, F = -2 s Phi D
// (SC, s = sign U) or -D (ZC), u = j/rho, v = u + F/rho,
// f_i* = (1 - omega)(f_i - feq_i(rho, u)) + feq_i(rho, v), streamed to x + e_i.
//
// Given lambda = dL/df at t+1, the adjoint at t is, per cell, with
// g_i = lambda_i(x + e_i) (the transpose of the streaming):
//   a_i = -(1 - omega) g_i, b_i = g_i                (weights of feq(u), feq(v))
//   rho_bar = sum_i (a_i feq_i(u) + b_i feq_i(v)) / rho
//   u_bar = sum_i a_i rho w_i (3 e_i + 9 (e_i.u) e_i - 3 u)
//   v_bar = sum_i b_i rho w_i (3 e_i + 9 (e_i.v) e_i - 3 v)
//   u_bar += v_bar, F_bar = v_bar / rho, rho_bar -= v_bar.F / rho^2
//   j_bar = u_bar / rho, rho_bar -= u_bar.u / rho
//   SC: D_bar = -2 s Phi F_bar, Phi_bar_centre = -2 s (F_bar.D);  ZC: D_bar = -F_bar
// and, because the periodic derivative is an antisymmetric circulant (its
// transpose is its negative),
//   Phi_bar = Phi_bar_centre - Dx[Dx_bar] - Dy[Dy_bar]
//   U_bar = Phi_bar s / (2 Phi) (SC) or Phi_bar (ZC)
//   rho_bar += U_bar dU/drho,  T_bar += U_bar dU/dtheta
// with theta = T for an equation of state (dU/dT = k dp/dT) and theta = G for
// the effective mass of Eq. 4 (dU/dG = psi^2 / 2).
//   lambda_i(t) = (1 - omega) g_i + rho_bar + e_i . j_bar.
//
// Two tiled kernels per step.  Kernel A does everything up to D_bar, with
// the centre term already folded into rho_bar and T_bar; it writes D_bar, the
// partial rho_bar and rho.  Kernel B stages D_bar with its halo and finishes
// rho_bar, T_bar and lambda(t).  For tau = 1 (omega = 1) every lambda_i(t) is
// rho_bar + e_i . j_bar, so lambda is kept as the three fields (rho_bar,
// jx_bar, jy_bar) instead of nine, staged in shared memory with a one-cell
// halo for the pull g_i = lambda_i(x + e_i).  On plain rows kernel A stages
// the stencil field of its tile with the halo and differentiates it; in the
// padded FP32 layout of the single-pass kernel it reads instead that kernel's
// record of the state (rho, j and the derivatives D the forward step used,
// written by the taped and the recomputed forward steps), so the reverse step
// differentiates only D_bar.  The HDM stencils run at a compile-time radius
// (26 in FP32, 40 in FP64) over weights that are zero past the folded radius
// of the lattice; in the padded layout kernel B forms the tile's derivatives
// once, in recurrence form on packed pairs, before its per-cell work.  The
// padded FP32 kernels are launched with programmatic serialization: A reads
// the record and forms the forward quantities while the previous step's B
// finishes, and every read of a predecessor's output and every write waits
// for it (griddepcontrol.wait).  T_bar
// terms are summed over each warp in the working precision (32 terms), then
// added in FP64 to one slot per warp of each CTA (one writer per slot and
// launch, and the launches are ordered, so the sum is reproducible), over the
// steps in the same slots, and over the slots in a fixed order at the end.
#include <cuda_runtime.h>

#include <cmath>

#include "lbm_internal.h"
#include "ptx.cuh"

namespace lbm {
namespace {

template <typename T>
struct AdjTile;
template <>
struct AdjTile<float> {   // two cells per thread, 512 threads (the padded tile phase needs ~50 registers)
    static constexpr int TX = 64, TY = 16, TYT = 8;
};
template <>
struct AdjTile<double> {  // two cells per thread (register budget)
    static constexpr int TX = 32, TY = 16, TYT = 8;
};

__device__ __forceinline__ float rcp_fast(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_fast(double x) { return 1.0 / x; }
__device__ __forceinline__ float rsqrt_fast(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_fast(double x) { return 1.0 / sqrt(x); }

// Two cells' values as one packed FP32 pair (Blackwell's paired add, multiply
// and fma; each component rounds as the scalar operation), so that the local
// adjoint of a thread's two cells runs as one pass.
struct F2 {
    float2 v;
    F2() = default;
    __device__ explicit F2(double c) : v(make_float2((float)c, (float)c)) {}
    __device__ F2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ F2 f2_of(float2 x) {
    F2 r;
    r.v = x;
    return r;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return f2_of(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return f2_of(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return f2_of(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return f2_of(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2 &operator-=(F2 &a, F2 b) { return a = a - b; }

// a b + c: one fma (scalar types: the contraction the compiler forms anyway)
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ F2 fmadd(F2 a, F2 b, F2 c) { return f2_of(__ffma2_rn(a.v, b.v, c.v)); }

// e_i . (vx, vy) from the signs of e_i (no multiplications by 0 or 1)
template <typename T>
__device__ __forceinline__ T dot_e(int i, T vx, T vy) {
    switch (i) {
        case 1: return vx;
        case 2: return vy;
        case 3: return -vx;
        case 4: return -vy;
        case 5: return vx + vy;
        case 6: return vy - vx;
        case 7: return -(vx + vy);
        case 8: return vx - vy;
        default: return T(0);
    }
}

// U (Eq. 8) with its derivatives in rho and in the model's scalar parameter
// theta: with an equation of state U = k p_EOS - rho/3 and theta = T (Eq. 24,
// 27-29; m.RT = R T, m.aal = a alpha(T), aalp = a dalpha/dT, R the gas
// constant); with the effective mass of Eq. 4 U = (G/2) psi^2 (Eq. 5, m.a =
// G/2, m.b = 1/rho0) and theta = G.  Reciprocals by the fast FP32 form (the
// denominators are positive and well scaled).
template <typename T>
__device__ __forceinline__ void eos_derivs(const Model<T> &m, T R, T aalp, T rho, T &U, T &dUdr, T &dUdth) {
    if (m.eos == LBM_EOS_PSI_EXP) {
        const T e = exp(-rho * m.b), psi = T(1) - e;
        U = m.a * psi * psi;
        dUdr = T(2) * m.a * psi * e * m.b;
        dUdth = T(0.5) * psi * psi;
        return;
    }
    T p, dpdr, dpdT;
    if (m.eos == LBM_EOS_CS) {
        const T e = m.b * rho * T(0.25);
        const T om = T(1) - e;
        const T inv = rcp_fast(om);
        const T inv3 = inv * inv * inv;
        const T num = T(1) + e + e * e - e * e * e;
        const T Z = num * inv3;
        const T dZ = ((T(1) + T(2) * e - T(3) * e * e) * om + T(3) * num) * inv3 * inv;
        p = rho * m.RT * Z - m.a * rho * rho;
        dpdr = m.RT * (Z + e * dZ) - T(2) * m.a * rho;
        dpdT = R * rho * Z;
    } else {
        const T inv = rcp_fast(T(1) - m.b * rho);
        const T rep = rho * m.RT * inv;
        const T drep_dr = m.RT * inv * inv, drep_dT = R * rho * inv;
        if (m.eos == LBM_EOS_VDW) {
            p = rep - m.a * rho * rho;
            dpdr = drep_dr - T(2) * m.a * rho;
            dpdT = drep_dT;
        } else if (m.eos == LBM_EOS_PR) {
            const T id = rcp_fast(T(1) + T(2) * m.b * rho - m.b * m.b * rho * rho);
            p = rep - m.aal * rho * rho * id;
            dpdr = drep_dr - m.aal * T(2) * rho * (T(1) + m.b * rho) * id * id;
            dpdT = drep_dT - aalp * rho * rho * id;
        } else {  // RK, RKS
            const T id = rcp_fast(T(1) + m.b * rho);
            p = rep - m.aal * rho * rho * id;
            dpdr = drep_dr - m.aal * rho * (T(2) + m.b * rho) * id * id;
            dpdT = drep_dT - aalp * rho * rho * id;
        }
    }
    U = m.k * p - rho * T(1.0 / 3.0);
    dUdr = m.k * dpdr - T(1.0 / 3.0);
    dUdth = m.k * dpdT;
}

// kappa = dPhi/dU dU/drho and theta = dPhi/dU dU/dtheta at density rho, with
// dPhi/dU = s / (2 Phi) for the Shan-Chen field and 1 for Zhang-Chen;
// sgn = s.
template <typename T, bool SC>
__device__ __forceinline__ void eos_coeffs(const Model<T> &m, T R, T aalp, T rho, T &kappa, T &theta, T &sgn) {
    T U, dUdr, dUdth;
    eos_derivs(m, R, aalp, rho, U, dUdr, dUdth);
    T d = T(1);
    sgn = U >= T(0) ? T(1) : T(-1);
    if (SC) {
        const T aU = fabs(U);
        d = aU > T(0) ? T(0.5) * sgn * rsqrt_fast(aU) : T(0);
    }
    kappa = d * dUdr;
    theta = d * dUdth;
}

template <typename T>
struct AdjArgs {
    Model<T> m;
    T R;            // gas constant
    T aalp;         // a dalpha/dT
    const T *f;     // state at t (nine unpadded fields); padded layout: its record (five)
    // Every other field is addressed as base[k * stride + y * pitch + off + x].
    const T *q;     // stencil field of f; |q| = Phi (SC) or U (ZC)
    int qpitch, qoff;
    const T *lam;   // adjoint at t+1 (nine fields, or three for tau = 1)
    T *lam_out;     // adjoint at t
    long long lstride;
    int lpitch, loff;
    T *aux;         // D_bar_x, D_bar_y, partial rho_bar, rho[, j_bar_x, j_bar_y]
    long long dstride;
    int dpitch, doff;
    double *Tpart;  // one FP64 slot per warp of each CTA of A, then of B
    int *err;       // error word (a bounded wait that gave up)
    long long nf, nq, nl, nd;   // elements of f (or the record), q, each lambda buffer, aux (checked build)
    T r, r5, r25;   // r = (sqrt 5 - 3)/2 of Eq. 20's operator and its powers (padded FP32 tiles)
};

// FP64 dL/dT slots of a tile kernel's CTAs: one per warp.
template <typename T>
constexpr int adj_warps() { return AdjTile<T>::TX * AdjTile<T>::TYT / 32; }

// Sum of v over each warp (in T), added in FP64 to the warp's own slot
// cta_slots[w].  Each slot has one writer per launch and the launches are
// ordered, so the sums are reproducible; the addition is issued without
// waiting for its result, and no warp waits for the others.
template <typename T>
__device__ __forceinline__ void warp_sum_into(T v, double *cta_slots) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if ((tid & 31) == 0) atomicAdd(cta_slots + (tid >> 5), (double)v);
}

// Copies the rectangle [lx0, lx1) x [ly0, ly1) of a shared array of pitch P
// from the periodic field src (row pitch spitch, column offset soff), whose
// element (gx0 + lx, gy0 + ly) lands at dst[ly * P + lx].  Asynchronous,
// element by element (cp.async).
template <typename T, int TX, int TYT>
__device__ __forceinline__ void stage_rect(T *dst, int P, const T *src, long long nsrc, int spitch, int soff, int nx,
                                           int ny, int gx0, int gy0, int lx0, int lx1, int ly0, int ly1, int *err) {
    for (int lx = lx0 + (int)threadIdx.x; lx < lx1; lx += TX) {
        const int gx = wrap_index(gx0 + lx, nx) + soff;
        for (int ly = ly0 + (int)threadIdx.y; ly < ly1; ly += TYT) {
            const long long g = (long long)wrap_index(gy0 + ly, ny) * spitch + gx;
            if (in_bounds(g, nsrc, err)) ptx::cp_async<sizeof(T)>(dst + ly * P + lx, src + g);
        }
    }
}

// Checked global accesses (the LBM_CHECKED build skips one outside its buffer
// of n elements and flags it; otherwise plain accesses).
template <typename T>
__device__ __forceinline__ T ld_chk(const T *base, long long i, long long n, int *err) {
    return in_bounds(i, n, err) ? base[i] : T(0);
}
template <typename T>
__device__ __forceinline__ void st_chk(T *base, long long i, long long n, T v, int *err) {
    if (in_bounds(i, n, err)) base[i] = v;
}
// Bulk copy of `bytes` from src element off into shared memory, if that range
// lies in the buffer of n elements (else skipped: the barrier's wait then
// gives up and reports it).
template <typename T>
__device__ __forceinline__ void bulk_chk(T *dst, const T *src, long long off, uint32_t bytes, long long n, uint64_t *bar,
                                         int *err) {
    if (in_bounds(off, n, err) && in_bounds(off + bytes / sizeof(T) - 1, n, err)) ptx::bulk_g2s(dst, src + off, bytes, bar);
}

// Antisymmetric stencil sum_j w_j (v[j s] - v[-j s]) with the x (YAX false)
// or y weights of the model, at compile-time radius KC (weights zero past the
// folded radius) or at the runtime radius (KC = 0).
template <typename T, int KC, bool ABS, bool YAX>
__device__ __forceinline__ T stencil(const T *v, int s, const Model<T> &m) {
    auto val = [&](int o) { return ABS ? fabs(v[o]) : v[o]; };
    T acc = T(0);
    if (KC > 0) {
#pragma unroll
        for (int j = 1; j <= KC; ++j) acc += (YAX ? m.wy[j] : m.wx[j]) * (val(j * s) - val(-j * s));
    } else {
        const int k = YAX ? m.ky : m.kx;
        for (int j = 1; j <= k; ++j) acc += (YAX ? m.wy[j] : m.wx[j]) * (val(j * s) - val(-j * s));
    }
    return acc;
}

// Store of a padded field value at column x of row `row`, with its periodic
// image in the ghost columns (PAD) when x lies within kGhost of an edge.
constexpr int kGhost = 32;
__device__ __forceinline__ int yp_of(int y, int ny) { return y + 1 == ny ? 0 : y + 1; }
__device__ __forceinline__ int ym_of(int y, int ny) { return y == 0 ? ny - 1 : y - 1; }
template <typename T, bool PAD>
__device__ __forceinline__ void store_field(T *base, long long n, long long row, int x, int nx, T v, int *err) {
    st_chk(base, row + x, n, v, err);
    if (PAD) {
        if (x < kGhost) st_chk(base, row + x + nx, n, v, err);
        if (x >= nx - kGhost) st_chk(base, row + x - nx, n, v, err);
    }
}

// Padded staging geometry (FP32 single-pass layout, HDM radius KC <= 28):
// a staged row keeps the tile's column 0 at XO, so a row with the x halo is
// one 16-byte-aligned copy of TX + 2 XO values starting at tile column -XO.
constexpr int XO = 28;   // x halo columns staged (>= radius, XO * 4 bytes a multiple of 16)
constexpr int LO = 4;    // lambda halo columns staged (>= 1)

// HDM derivatives of a padded FP32 tile (64 x 16 cells) of a staged field,
// written to D[ly * 64 + lx] (along x) and D[1024 + ly * 64 + lx] (along y),
// both radius-26 operators in recurrence form on packed pairs (hdm_window4_paired).
// Along x, tile row ly is staged at X + ly * XP with tile column c at X + ly *
// XP + 28 + c; work items 0..255 take four cells of a row each from one
// 60-value window of 16-byte loads.  Along y, tile cell (lx, ly) is staged at
// Y + (26 + ly) * YP + yc0 + lx (26 halo rows on each side); items 256..511
// take four cells of a column each from one 56-row window.  Thread k of the
// CTA (at least 512 threads) takes item k; the caller synchronises the CTA
// before and after.  ABS: the field enters as its magnitude.
template <bool ABS>
__device__ __forceinline__ void tile_hdm(const float *X, int XP, const float *Y, int YP, int yc0, float *D,
                                         const Model<float> &m, float r, float r5, float r25) {
    auto mag = [](float v) { return ABS ? fabsf(v) : v; };
    const int item = threadIdx.x + blockDim.x * threadIdx.y;
    if (item >= 512) return;
    float t[60], d[4];
    float2 tp[28];   // deviations paired about the window's centre (hdm_window4_paired)
#pragma unroll
    for (int p = 0; p < 60; ++p) t[p] = 0.f;
    if (item < 256) {
        const int ly = item >> 4, g = item & 15;
        const float *w = X + ly * XP + 4 * g;    // window position p = tile column 4g - 28 + p
#pragma unroll
        for (int k = 0; k < 15; ++k) {
            const float4 v4 = *reinterpret_cast<const float4 *>(w + 4 * k);
            t[4 * k] = v4.x; t[4 * k + 1] = v4.y; t[4 * k + 2] = v4.z; t[4 * k + 3] = v4.w;
        }
        const float ref = mag(t[29]);
#pragma unroll
        for (int j = 0; j < 28; ++j) tp[j] = make_float2(mag(t[2 + j]) - ref, mag(t[57 - j]) - ref);
        hdm_window4_paired(tp, m.wx[1], m.wx[2], r, r5, r25, d);
        *reinterpret_cast<float4 *>(D + ly * 64 + 4 * g) = make_float4(d[0], d[1], d[2], d[3]);
    } else {
        const int i = item - 256, cx = i & 63, h = i >> 6;
        const float *col = Y + 4 * h * YP + yc0 + cx;   // window position p = staged row 4h - 2 + p
#pragma unroll
        for (int p = 2; p <= 57; ++p) t[p] = col[(p - 2) * YP];
        const float ref = mag(t[29]);
#pragma unroll
        for (int j = 0; j < 28; ++j) tp[j] = make_float2(mag(t[2 + j]) - ref, mag(t[57 - j]) - ref);
        hdm_window4_paired(tp, m.wy[1], m.wy[2], r, r5, r25, d);
#pragma unroll
        for (int c = 0; c < 4; ++c) D[1024 + (4 * h + c) * 64 + cx] = d[c];
    }
}

// Bounded wait of the whole CTA for the bulk copies on bars[k]; on timeout
// flags the error word, lets the copies in flight on all nbar barriers land
// and returns false.
__device__ __forceinline__ bool cta_wait_copies(uint64_t *bars, int nbar, int k, int *err) {
    constexpr uint64_t kLimitNs = 200ull * 1000 * 1000;
    const bool ok = ptx::mbar_wait_bounded(&bars[k], 0, kLimitNs);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            atomicOr(err, kErrTimeout);
            for (int b = 0; b < nbar; ++b) (void)ptx::mbar_wait_bounded(&bars[b], 0, kLimitNs);
        }
        __syncthreads();
        return false;
    }
    return true;
}

// The local adjoint of one cell's forcing and collision.  From g_i =
// lambda_i(x + e_i) and the cell's forward quantities (rho, 1/rho, u, v, F,
// D, Phi or U, s) it forms rho_bar without the transposed-derivative and EOS
// terms, j_bar, D_bar and the centre part pc of Phi_bar (Shan-Chen).  With
// feq_i(rho, v) = w_i rho (a + e_i.v (3 + 4.5 e_i.v)), a = 1 - 1.5 |v|^2,
//   sum_i b_i dfeq_i/drho = sum_i b_i w_i (a + e_i.v (3 + 4.5 e_i.v)),
//   sum_i b_i dfeq_i/dv = rho (sum_i b_i w_i e_i (3 + 9 e_i.v) - 3 v sum_i b_i w_i),
// so one pass over the directions forms the weighted sums (e_i.v by its signs).
template <typename T, bool SC, bool TAU1>
__device__ __forceinline__ void adj_local(const T (&g)[kQ], T om1, T r, T inv, T ux, T uy, T vx, T vy, T Fx, T Fy,
                                          T Dx, T Dy, T phi, T sgn, T &rb, T &jbx, T &jby, T &Dbx, T &Dby, T &pc) {
    T G0 = T(0), Gx = T(0), Gy = T(0), Rv = T(0), Hx = T(0), Hy = T(0), Ru = T(0);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const T gw = g[i] * T(wq<double>(i));
        G0 += gw;
        if (i == 0) continue;
        const T ev = dot_e(i, vx, vy);
        const T gt = gw * fmadd(T(9), ev, T(3));
        if (ex(i) == 1) Gx += gt;
        if (ex(i) == -1) Gx -= gt;
        if (ey(i) == 1) Gy += gt;
        if (ey(i) == -1) Gy -= gt;
        Rv = fmadd(gw * ev, fmadd(T(4.5), ev, T(3)), Rv);
        if (!TAU1) {
            const T eu = dot_e(i, ux, uy);
            const T gu = gw * fmadd(T(9), eu, T(3));
            if (ex(i) == 1) Hx += gu;
            if (ex(i) == -1) Hx -= gu;
            if (ey(i) == 1) Hy += gu;
            if (ey(i) == -1) Hy -= gu;
            Ru = fmadd(gw * eu, fmadd(T(4.5), eu, T(3)), Ru);
        }
    }
    const T vv = fmadd(vx, vx, vy * vy);
    rb = fmadd(fmadd(T(-1.5), vv, T(1)), G0, Rv);
    const T vbx = r * fmadd(T(-3) * vx, G0, Gx), vby = r * fmadd(T(-3) * vy, G0, Gy);
    T ubx = vbx, uby = vby;
    if (!TAU1) {   // the f^eq(u) terms enter with the weights -(1 - omega) g_i
        const T uu = fmadd(ux, ux, uy * uy);
        rb -= om1 * fmadd(fmadd(T(-1.5), uu, T(1)), G0, Ru);
        ubx -= om1 * r * fmadd(T(-3) * ux, G0, Hx);
        uby -= om1 * r * fmadd(T(-3) * uy, G0, Hy);
    }
    const T Fbx = vbx * inv, Fby = vby * inv;
    rb -= fmadd(vbx, Fx, vby * Fy) * inv * inv;
    jbx = ubx * inv;
    jby = uby * inv;
    rb -= fmadd(ubx, ux, uby * uy) * inv;
    if (SC) {
        const T m2s = T(-2) * sgn;
        Dbx = m2s * phi * Fbx;
        Dby = m2s * phi * Fby;
        pc = m2s * fmadd(Fbx, Dx, Fby * Dy);
    } else {
        Dbx = -Fbx;
        Dby = -Fby;
        pc = T(0);
    }
}

// Kernel A on plain rows (FP64, and FP32 off the single-pass layout): the
// stencil field is staged with its halo (element-wise asynchronous copies)
// and differentiated here.
template <typename T, bool SC, bool CDM, bool TAU1, int KC>
__global__ void __launch_bounds__(AdjTile<T>::TX *AdjTile<T>::TYT) adj_a_kernel(const AdjArgs<T> a) {
    constexpr int TX = AdjTile<T>::TX, TY = AdjTile<T>::TY, TYT = AdjTile<T>::TYT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Model<T> &m = a.m;
    const int nx = m.nx, ny = m.ny;
    const long long n = (long long)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int hx = CDM ? 1 : (KC ? KC : m.kx), hy = CDM ? 1 : (KC ? KC : m.ky);
    // staged field: S[ly * W + hx + lx] = q(x0 + lx, y0 - hy + ly); lambda tile
    // L[(k * LH + ly) * LW + 1 + lx] = lambda_k(x0 + lx, y0 - 1 + ly)
    const int W = TX + 2 * hx, H = TY + 2 * hy;
    constexpr int LW = TX + 2, LH = TY + 2;
    T *S = reinterpret_cast<T *>(smem_raw);
    T *L = S + W * H;
    // element-wise: a cross for the separable HDM, the full box for the CDM
    if (CDM) {
        stage_rect<T, TX, TYT>(S, W, a.q, a.nq, a.qpitch, a.qoff, nx, ny, x0 - hx, y0 - hy, 0, W, 0, H, a.m.chk);
    } else {
        stage_rect<T, TX, TYT>(S, W, a.q, a.nq, a.qpitch, a.qoff, nx, ny, x0 - hx, y0 - hy, 0, W, hy, hy + TY, a.m.chk);
        stage_rect<T, TX, TYT>(S, W, a.q, a.nq, a.qpitch, a.qoff, nx, ny, x0 - hx, y0 - hy, hx, hx + TX, 0, hy, a.m.chk);
        stage_rect<T, TX, TYT>(S, W, a.q, a.nq, a.qpitch, a.qoff, nx, ny, x0 - hx, y0 - hy, hx, hx + TX, hy + TY, H,
                               a.m.chk);
    }
    if (TAU1)
        for (int k = 0; k < 3; ++k)
            stage_rect<T, TX, TYT>(L + k * LW * LH, LW, a.lam + k * a.lstride, a.nl - k * a.lstride, a.lpitch, a.loff,
                                   nx, ny, x0 - 1, y0 - 1, 0, LW, 0, LH, a.m.chk);
    ptx::cp_async_wait_all();
    __syncthreads();

    // Every thread runs the cell loop; cells outside the lattice compute on a
    // clamped index and store nothing.
    T tacc = T(0);
    const int lx = threadIdx.x, x = x0 + lx;
    const int xc = min(x, nx - 1);
    const int xp = xc + 1 == nx ? 0 : xc + 1, xm = xc == 0 ? nx - 1 : xc - 1;
#pragma unroll
    for (int k = 0; k < TY / TYT; ++k) {
        const int ly = threadIdx.y + k * TYT, y = y0 + ly;
        const bool valid = x < nx && y < ny;
        const int yc = min(y, ny - 1);
        const int yp = yc + 1 == ny ? 0 : yc + 1, ym = yc == 0 ? ny - 1 : yc - 1;
        const long long c = (long long)yc * nx + xc;
        T r = T(0), jx = T(0), jy = T(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const T fi = ld_chk(a.f, i * n + c, a.nf, a.m.chk);
            r += fi;
            if (ex(i) == 1) jx += fi;
            if (ex(i) == -1) jx -= fi;
            if (ey(i) == 1) jy += fi;
            if (ey(i) == -1) jy -= fi;
        }
        T kappa, theta, sgn;
        eos_coeffs<T, SC>(m, a.R, a.aalp, r, kappa, theta, sgn);
        const T inv = rcp_fast(r);
        const T ux = jx * inv, uy = jy * inv;
        // D of the field at the cell (Eq. 15 / 20) from the staged tile
        const T *row = S + (ly + hy) * W + (hx + lx);
        auto fld = [&](int o) { return SC ? fabs(row[o]) : row[o]; };
        T Dx, Dy;
        if (CDM) {
            const T e = fld(1), w = fld(-1), nn = fld(W), s = fld(-W);
            const T ne = fld(W + 1), nw = fld(W - 1), se = fld(-W + 1), sw = fld(-W - 1);
            Dx = T(1.0 / 3.0) * (e - w) + T(1.0 / 12.0) * ((ne + se) - (nw + sw));
            Dy = T(1.0 / 3.0) * (nn - s) + T(1.0 / 12.0) * ((ne + nw) - (se + sw));
        } else {
            Dx = stencil<T, KC, SC, false>(row, 1, m);
            Dy = stencil<T, KC, SC, true>(row, W, m);
        }
        const T phi = fld(0);  // Phi (SC) or U (ZC)
        T Fx, Fy;
        if (SC) { Fx = T(-2) * sgn * phi * Dx; Fy = T(-2) * sgn * phi * Dy; }
        else { Fx = -Dx; Fy = -Dy; }
        const T vx = ux + Fx * inv, vy = uy + Fy * inv;
        T g[kQ];
#pragma unroll
        for (int i = 0; i < kQ; ++i) {  // g_i = lambda_i(x + e_i)
            if (TAU1) {   // lambda_i = rho_bar + e_i . j_bar, by the signs of e_i
                const int o = (ly + 1 + ey(i)) * LW + (1 + lx + ex(i));
                T gi = L[o];
                if (ex(i) == 1) gi += L[LW * LH + o];
                if (ex(i) == -1) gi -= L[LW * LH + o];
                if (ey(i) == 1) gi += L[2 * LW * LH + o];
                if (ey(i) == -1) gi -= L[2 * LW * LH + o];
                g[i] = gi;
            } else {
                const int dxs = ex(i) == 1 ? xp : (ex(i) == -1 ? xm : xc);
                const int dys = ey(i) == 1 ? yp : (ey(i) == -1 ? ym : yc);
                g[i] = ld_chk(a.lam, i * a.lstride + (long long)dys * a.lpitch + a.loff + dxs, a.nl, a.m.chk);
            }
        }
        T rb, jbx, jby, Dbx, Dby, pc;
        adj_local<T, SC, TAU1>(g, T(1) - m.omega, r, inv, ux, uy, vx, vy, Fx, Fy, Dx, Dy, phi, sgn, rb, jbx, jby,
                               Dbx, Dby, pc);
        if (SC) {
            rb += pc * kappa;
            if (valid) tacc += pc * theta;
        }
        if (valid) {
            const long long d0 = (long long)y * a.dpitch + a.doff + x;
            st_chk(a.aux, d0, a.nd, Dbx, a.m.chk);
            st_chk(a.aux, a.dstride + d0, a.nd, Dby, a.m.chk);
            st_chk(a.aux, 2 * a.dstride + d0, a.nd, rb, a.m.chk);
            st_chk(a.aux, 3 * a.dstride + d0, a.nd, r, a.m.chk);
            if (TAU1) {
                const long long l0 = (long long)y * a.lpitch + a.loff + x;
                st_chk(a.lam_out, a.lstride + l0, a.nl, jbx, a.m.chk);
                st_chk(a.lam_out, 2 * a.lstride + l0, a.nl, jby, a.m.chk);
            } else {
                st_chk(a.aux, 4 * a.dstride + d0, a.nd, jbx, a.m.chk);
                st_chk(a.aux, 5 * a.dstride + d0, a.nd, jby, a.m.chk);
            }
        }
    }
    if (SC) warp_sum_into(tacc, a.Tpart + (size_t)(blockIdx.x + gridDim.x * blockIdx.y) * adj_warps<T>());
}

// Kernel A in the padded FP32 layout of the single-pass kernel.  The forward
// quantities come from that kernel's record of the state (rho, j and the HDM
// derivatives D it used), so nothing is differentiated here: the kernel reads
// the record and the field at each of its cells, and for tau = 1 stages the
// lambda tile (three fields, one-cell halo) by per-row bulk copies.  Launched
// with programmatic serialization: everything before griddep_wait reads only
// the record and the field, written at least one launch back on another
// stream (ordered by an event); lambda and every write wait for the previous
// reverse step's kernel B.
template <bool SC, bool TAU1>
__global__ void __launch_bounds__(AdjTile<float>::TX *AdjTile<float>::TYT) adj_a_rec_kernel(const AdjArgs<float> a) {
    constexpr int TX = AdjTile<float>::TX, TY = AdjTile<float>::TY, TYT = AdjTile<float>::TYT, NC = TY / TYT;
    constexpr int LW = TX + 2 * LO, LH = TY + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // lambda tile L[(k * LH + ly) * LW + LO + lx] = lambda_k(x0 + lx, y0 - 1 + ly)
    float *L = reinterpret_cast<float *>(smem_raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(L + (TAU1 ? 3 * LW * LH : 0));
    const Model<float> &m = a.m;
    const int nx = m.nx, ny = m.ny;
    const long long n = (long long)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.x + TX * threadIdx.y;
    const int ncore = min(TX, nx - x0);   // a multiple of 4
    const uint32_t lrow = (ncore + 2 * LO) * sizeof(float);
    if (TAU1) {
        if (tid == 0) {
            ptx::mbar_init(bar, 1);
            ptx::fence_mbar_init();
            ptx::mbar_arrive_expect_tx(bar, 3 * LH * lrow);
        }
        __syncthreads();
    }
    // the next kernel (B of this step) may begin launching
    ptx::griddep_launch_dependents();

    const int lx = threadIdx.x, x = x0 + lx;
    const int xc = min(x, nx - 1);
    float r_k[NC], jx_k[NC], jy_k[NC], Dx_k[NC], Dy_k[NC], q_k[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int yc = min(y0 + (int)threadIdx.y + k * TYT, ny - 1);
        const long long c = (long long)yc * nx + xc;
        r_k[k] = ld_chk(a.f, c, a.nf, a.m.chk);
        jx_k[k] = ld_chk(a.f, n + c, a.nf, a.m.chk);
        jy_k[k] = ld_chk(a.f, 2 * n + c, a.nf, a.m.chk);
        Dx_k[k] = ld_chk(a.f, 3 * n + c, a.nf, a.m.chk);
        Dy_k[k] = ld_chk(a.f, 4 * n + c, a.nf, a.m.chk);
        q_k[k] = ld_chk(a.q, (long long)yc * a.qpitch + a.qoff + xc, a.nq, a.m.chk);
    }
    float inv_k[NC], ux_k[NC], uy_k[NC], vx_k[NC], vy_k[NC], Fx_k[NC], Fy_k[NC], phi_k[NC], sgn_k[NC];
    float kap_k[NC], th_k[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        eos_coeffs<float, SC>(m, a.R, a.aalp, r_k[k], kap_k[k], th_k[k], sgn_k[k]);
        const float inv = rcp_fast(r_k[k]);
        const float phi = SC ? fabsf(q_k[k]) : q_k[k];   // Phi (SC) or U (ZC)
        float Fx, Fy;
        if (SC) { Fx = -2.0f * sgn_k[k] * phi * Dx_k[k]; Fy = -2.0f * sgn_k[k] * phi * Dy_k[k]; }
        else { Fx = -Dx_k[k]; Fy = -Dy_k[k]; }
        inv_k[k] = inv;
        ux_k[k] = jx_k[k] * inv;
        uy_k[k] = jy_k[k] * inv;
        vx_k[k] = ux_k[k] + Fx * inv;
        vy_k[k] = uy_k[k] + Fy * inv;
        Fx_k[k] = Fx;
        Fy_k[k] = Fy;
        phi_k[k] = phi;
    }
    ptx::griddep_wait();
    if (TAU1) {
        if (tid < 32) {  // warp 0 issues one bulk copy per lambda row
            for (int rr = tid; rr < 3 * LH; rr += 32) {
                const int kk = rr / LH, ry = rr - kk * LH;
                const long long off = kk * a.lstride + (long long)wrap_index(y0 - 1 + ry, ny) * a.lpitch + a.loff + x0;
                bulk_chk(L + rr * LW, a.lam, off - LO, lrow, a.nl, bar, a.m.chk);
            }
        }
        if (!cta_wait_copies(bar, 1, 0, a.err)) return;
    }
    static_assert(NC == 2, "the local adjoint runs on the thread's two cells as packed pairs");
    float tacc = 0.0f;
    const int xp = xc + 1 == nx ? 0 : xc + 1, xm = xc == 0 ? nx - 1 : xc - 1;
    float gk[NC][kQ];   // g_i = lambda_i(x + e_i) of both cells
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int ly = threadIdx.y + k * TYT;
        const int yc = min(y0 + ly, ny - 1);
        const int yp = yc + 1 == ny ? 0 : yc + 1, ym = yc == 0 ? ny - 1 : yc - 1;
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            if (TAU1) {   // lambda_i = rho_bar + e_i . j_bar, by the signs of e_i
                const int o = (ly + 1 + ey(i)) * LW + (LO + lx + ex(i));
                float gi = L[o];
                if (ex(i) == 1) gi += L[LW * LH + o];
                if (ex(i) == -1) gi -= L[LW * LH + o];
                if (ey(i) == 1) gi += L[2 * LW * LH + o];
                if (ey(i) == -1) gi -= L[2 * LW * LH + o];
                gk[k][i] = gi;
            } else {
                const int dxs = ex(i) == 1 ? xp : (ex(i) == -1 ? xm : xc);
                const int dys = ey(i) == 1 ? yp : (ey(i) == -1 ? ym : yc);
                gk[k][i] = ld_chk(a.lam, i * a.lstride + (long long)dys * a.lpitch + a.loff + dxs, a.nl, a.m.chk);
            }
        }
    }
    F2 g2[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) g2[i] = F2(gk[0][i], gk[1][i]);
    auto pair = [](const float (&v)[NC]) { return F2(v[0], v[1]); };
    const float om1 = 1.0f - m.omega;
    F2 rb2, jbx2, jby2, Dbx2, Dby2, pc2;
    adj_local<F2, SC, TAU1>(g2, F2(om1, om1), pair(r_k), pair(inv_k), pair(ux_k), pair(uy_k), pair(vx_k),
                            pair(vy_k), pair(Fx_k), pair(Fy_k), pair(Dx_k), pair(Dy_k), pair(phi_k), pair(sgn_k), rb2,
                            jbx2, jby2, Dbx2, Dby2, pc2);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int y = y0 + threadIdx.y + k * TYT;
        const bool valid = x < nx && y < ny;
        float rb = k ? rb2.v.y : rb2.v.x;
        const float jbx = k ? jbx2.v.y : jbx2.v.x, jby = k ? jby2.v.y : jby2.v.x;
        const float Dbx = k ? Dbx2.v.y : Dbx2.v.x, Dby = k ? Dby2.v.y : Dby2.v.x, pc = k ? pc2.v.y : pc2.v.x;
        if (SC) {
            rb += pc * kap_k[k];
            if (valid) tacc += pc * th_k[k];
        }
        if (valid) {
            const long long d0 = (long long)y * a.dpitch + a.doff;
            store_field<float, true>(a.aux, a.nd, d0, x, nx, Dbx, a.m.chk);
            store_field<float, true>(a.aux, a.nd, a.dstride + d0, x, nx, Dby, a.m.chk);
            st_chk(a.aux, 2 * a.dstride + d0 + x, a.nd, rb, a.m.chk);
            st_chk(a.aux, 3 * a.dstride + d0 + x, a.nd, r_k[k], a.m.chk);
            if (TAU1) {
                const long long l0 = (long long)y * a.lpitch + a.loff;
                store_field<float, true>(a.lam_out, a.nl, a.lstride + l0, x, nx, jbx, a.m.chk);
                store_field<float, true>(a.lam_out, a.nl, 2 * a.lstride + l0, x, nx, jby, a.m.chk);
            } else {
                st_chk(a.aux, 4 * a.dstride + d0 + x, a.nd, jbx, a.m.chk);
                st_chk(a.aux, 5 * a.dstride + d0 + x, a.nd, jby, a.m.chk);
            }
        }
    }
    if (SC) warp_sum_into(tacc, a.Tpart + (size_t)(blockIdx.x + gridDim.x * blockIdx.y) * adj_warps<float>());
}

template <typename T, bool SC, bool CDM, bool TAU1, int KC, bool PAD>
__global__ void __launch_bounds__(AdjTile<T>::TX *AdjTile<T>::TYT) adj_b_kernel(const AdjArgs<T> a) {
    constexpr int TX = AdjTile<T>::TX, TY = AdjTile<T>::TY, TYT = AdjTile<T>::TYT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Model<T> &m = a.m;
    const int nx = m.nx, ny = m.ny;
    const int hx = CDM ? 1 : (KC ? KC : m.kx), hy = CDM ? 1 : (KC ? KC : m.ky);
    // D_bar_x over the tile's rows with the x halo, D_bar_y over its columns
    // with the y halo; the CDM takes the full box of halo 1 for both
    const int XS = PAD ? XO : hx;
    const int WX = TX + 2 * XS, HX = CDM ? TY + 2 : TY;
    const int WY = CDM ? TX + 2 : TX, HY = TY + 2 * hy;
    const int ox = CDM ? 1 : 0;  // column offset of the tile in the D_bar_y array
    const int oy = CDM ? 1 : 0;  // row offset of the tile in the D_bar_x array
    T *SX = reinterpret_cast<T *>(smem_raw);
    T *SY = SX + WX * HX;
    uint64_t *bars = reinterpret_cast<uint64_t *>(SY + WY * HY);
    constexpr bool RECUR = PAD && KC == 26 && !CDM;
    static_assert(!RECUR || TX * TYT >= 512, "the tile phase takes one work item per thread");
    T *DT = reinterpret_cast<T *>(bars + 2);   // padded FP32 tiles: D_bar's derivatives over the tile
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    if constexpr (PAD) {
        const int tid = threadIdx.x + TX * threadIdx.y;
        if (tid == 0) {
            ptx::mbar_init(&bars[0], 1);
            ptx::fence_mbar_init();
        }
        __syncthreads();
        // the next reverse step's A may begin its state-only work; this kernel
        // reads A's output, so it waits for A first
        ptx::griddep_launch_dependents();
        ptx::griddep_wait();
        if (tid < 32) {
            const int ncore = min(TX, nx - x0);
            const uint32_t wide = (ncore + 2 * XO) * sizeof(T), core = ncore * sizeof(T);
            if (tid == 0) ptx::mbar_arrive_expect_tx(&bars[0], HX * wide + HY * core);
            __syncwarp();
            for (int ly = tid; ly < HX; ly += 32) {
                const long long off = (long long)wrap_index(y0 + ly, ny) * a.dpitch + a.doff + x0;
                bulk_chk(SX + ly * WX, a.aux, off - XO, wide, a.nd, &bars[0], a.m.chk);
            }
            for (int ly = tid; ly < HY; ly += 32) {
                const long long off = a.dstride + (long long)wrap_index(y0 - hy + ly, ny) * a.dpitch + a.doff + x0;
                bulk_chk(SY + ly * WY, a.aux, off, core, a.nd, &bars[0], a.m.chk);
            }
        }
    } else {
        stage_rect<T, TX, TYT>(SX, WX, a.aux, a.nd, a.dpitch, a.doff, nx, ny, x0 - hx, y0 - oy, 0, WX, 0, HX, a.m.chk);
        stage_rect<T, TX, TYT>(SY, WY, a.aux + a.dstride, a.nd - a.dstride, a.dpitch, a.doff, nx, ny, x0 - ox, y0 - hy,
                               0, WY, 0, HY, a.m.chk);
        ptx::cp_async_wait_all();
        __syncthreads();
    }

    // the density and partial rho_bar of all of the thread's cells first (their
    // loads in flight together), with the EOS terms, while the copies land
    constexpr int NC = TY / TYT;
    T tacc = T(0);
    const int lx = threadIdx.x, x = x0 + lx;
    const int xc = min(x, nx - 1);
    const int xp = xc + 1 == nx ? 0 : xc + 1, xm = xc == 0 ? nx - 1 : xc - 1;
    T rk[NC], rb0k[NC], kap_k[NC], th_k[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const long long d0 = (long long)min(y0 + (int)threadIdx.y + k * TYT, ny - 1) * a.dpitch + a.doff + xc;
        rk[k] = ld_chk(a.aux, 3 * a.dstride + d0, a.nd, a.m.chk);
        rb0k[k] = ld_chk(a.aux, 2 * a.dstride + d0, a.nd, a.m.chk);
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        T sgn;
        eos_coeffs<T, SC>(m, a.R, a.aalp, rk[k], kap_k[k], th_k[k], sgn);
    }
    if (PAD && !cta_wait_copies(bars, 1, 0, a.err)) return;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int ly = threadIdx.y + k * TYT, y = y0 + ly;
        const bool valid = x < nx && y < ny;
        const T rb0 = rb0k[k], kappa = kap_k[k], theta = th_k[k];
        // the transposed derivative: Dx^T = -Dx, Dy^T = -Dy
        const T *rx = SX + (ly + oy) * WX + (lx + XS);
        const T *ry = SY + (ly + hy) * WY + (lx + ox);
        T ddx, ddy;
        if (CDM) {
            ddx = T(1.0 / 3.0) * (rx[1] - rx[-1]) +
                  T(1.0 / 12.0) * ((rx[WX + 1] + rx[-WX + 1]) - (rx[WX - 1] + rx[-WX - 1]));
            ddy = T(1.0 / 3.0) * (ry[WY] - ry[-WY]) +
                  T(1.0 / 12.0) * ((ry[WY + 1] + ry[WY - 1]) - (ry[-WY + 1] + ry[-WY - 1]));
        } else if constexpr (RECUR) {
            if (k == 0) {
                tile_hdm<false>(SX + oy * WX, WX, SY, WY, ox, DT, m, a.r, a.r5, a.r25);
                __syncthreads();
            }
            ddx = DT[ly * TX + lx];
            ddy = DT[TX * TY + ly * TX + lx];
        } else {
            ddx = stencil<T, KC, false, false>(rx, 1, m);
            ddy = stencil<T, KC, false, true>(ry, WY, m);
        }
        const T pbar = -ddx - ddy;
        const T rb = rb0 + kappa * pbar;
        if (!valid) continue;
        tacc += theta * pbar;
        const long long l0 = (long long)y * a.lpitch + a.loff;
        if (TAU1) {
            store_field<T, PAD>(a.lam_out, a.nl, l0, x, nx, rb, a.m.chk);
        } else {
            const long long d0 = (long long)y * a.dpitch + a.doff + x;
            const T jbx = ld_chk(a.aux, 4 * a.dstride + d0, a.nd, a.m.chk);
            const T jby = ld_chk(a.aux, 5 * a.dstride + d0, a.nd, a.m.chk);
            const T om1 = T(1) - m.omega;
#pragma unroll
            for (int i = 0; i < kQ; ++i) {
                const int dxs = ex(i) == 1 ? xp : (ex(i) == -1 ? xm : x);
                const int dys = ey(i) == 1 ? yp_of(y, ny) : (ey(i) == -1 ? ym_of(y, ny) : y);
                const T gi = ld_chk(a.lam, i * a.lstride + (long long)dys * a.lpitch + a.loff + dxs, a.nl, a.m.chk);
                T li = om1 * gi + rb;
                if (ex(i) == 1) li += jbx;
                if (ex(i) == -1) li -= jbx;
                if (ey(i) == 1) li += jby;
                if (ey(i) == -1) li -= jby;
                st_chk(a.lam_out, i * a.lstride + l0 + x, a.nl, li, a.m.chk);
            }
        }
    }
    warp_sum_into(tacc, a.Tpart + (size_t)(blockIdx.x + gridDim.x * blockIdx.y) * adj_warps<T>());
}

// lambda at the final step from dL/drho_T (rho_T = sum_i f_i): lambda_i = g
// for all i, i.e. (g, 0, 0) in the three-field form.
template <typename T, bool PAD>
__global__ void adj_seed_kernel(int nx, int ny, int nlam, const T *grad_rho, T *lam, long long lstride, int lpitch,
                                int loff, int *err) {
    const long long n = (long long)nx * ny, nl = nlam * lstride;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(c / nx), x = (int)(c - (long long)y * nx);
        const T g = grad_rho[c];
        const long long row = (long long)y * lpitch + loff;
        if (nlam == 3) {
            store_field<T, PAD>(lam, nl, row, x, nx, g, err);
            store_field<T, PAD>(lam, nl, lstride + row, x, nx, T(0), err);
            store_field<T, PAD>(lam, nl, 2 * lstride + row, x, nx, T(0), err);
        } else {
            for (int i = 0; i < kQ; ++i) st_chk(lam, i * lstride + row + x, nl, g, err);
        }
    }
}

// f_i = w_i rho0 at rest (Eq. 2): dL/drho0 = sum_i w_i lambda_i, which for
// lambda_i = rho_bar + e_i . j_bar is rho_bar (sum w_i = 1, sum w_i e_i = 0).
template <typename T>
__global__ void adj_initial_kernel(int nx, int ny, int nlam, const T *lam, long long lstride, int lpitch, int loff,
                                   T *grad_rho0, int *err) {
    const long long n = (long long)nx * ny, nl = nlam * lstride;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(c / nx), x = (int)(c - (long long)y * nx);
        const long long row = (long long)y * lpitch + loff + x;
        if (nlam == 3) {
            grad_rho0[c] = ld_chk(lam, row, nl, err);
        } else {
            T s = T(0);
#pragma unroll
            for (int i = 0; i < kQ; ++i) s += wq<T>(i) * ld_chk(lam, i * lstride + row, nl, err);
            grad_rho0[c] = s;
        }
    }
}

// Sum of the slots in a fixed order (lane k takes slots k, k + 32, ... in
// turn, then a fixed shuffle tree): one warp, reproducible.
__global__ void sum_slots_kernel(const double *slots, int nslots, double *out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nslots; i += 32) s += slots[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
}

template <typename T>
__global__ void density_kernel(long long n, const T *f, T *rho) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        T r = T(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) r += f[i * n + c];
        rho[c] = r;
    }
}

int blocks_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

template <typename T>
dim3 adj_grid(int nx, int ny) {
    return dim3((nx + AdjTile<T>::TX - 1) / AdjTile<T>::TX, (ny + AdjTile<T>::TY - 1) / AdjTile<T>::TY);
}

// Launch with programmatic stream serialization when `pdl`: the kernel may
// start while the preceding one finishes (its griddep_wait guards every read
// of that kernel's output and every write).
template <typename K, typename A>
cudaError_t launch_pdl(bool pdl, K kern, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const A &arg) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, arg);
}

template <typename T, bool SC, bool CDM, bool TAU1, int KC, bool PAD>
cudaError_t launch_adj_t(const AdjArgs<T> &a, bool overlap_prev, cudaStream_t s) {
    constexpr int TX = AdjTile<T>::TX, TY = AdjTile<T>::TY, TYT = AdjTile<T>::TYT;
    const int hx = CDM ? 1 : (KC ? KC : a.m.kx), hy = CDM ? 1 : (KC ? KC : a.m.ky);
    const int XS = PAD ? XO : hx;
    constexpr bool RECUR = PAD && KC == 26 && !CDM;   // B: tile derivatives after the barrier
    const size_t dt = RECUR ? 2 * sizeof(T) * TX * TY : 0;
    // A: in the padded layout the lambda tile (tau = 1) and its barrier; else
    // the field with its halo and the lambda tile
    const size_t smem_a = PAD ? (TAU1 ? sizeof(T) * 3 * (TX + 2 * LO) * (TY + 2) + sizeof(uint64_t) : 0)
                              : sizeof(T) * ((size_t)(TX + 2 * hx) * (TY + 2 * hy) + (TAU1 ? 3 * (TX + 2) * (TY + 2) : 0));
    const size_t smem_b = (CDM ? sizeof(T) * 2 * (size_t)(TX + 2) * (TY + 2)
                               : sizeof(T) * ((size_t)(TX + 2 * XS) * TY + (size_t)TX * (TY + 2 * hy))) +
                          (PAD ? 2 * sizeof(uint64_t) : 0) + dt;
    void (*ka)(const AdjArgs<T>) = nullptr;
    if constexpr (PAD) ka = adj_a_rec_kernel<SC, TAU1>;   // T = float
    else ka = adj_a_kernel<T, SC, CDM, TAU1, KC>;
    auto kb = adj_b_kernel<T, SC, CDM, TAU1, KC, PAD>;
    // the shared-memory limits, set once per device and size (a driver call per
    // launch otherwise); the largest size set so far covers every smaller one
    constexpr int kDevs = 64;
    static size_t set_a[kDevs] = {}, set_b[kDevs] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool cache = dev >= 0 && dev < kDevs;
    if (!cache || smem_a > set_a[dev]) {
        e = cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a);
        if (e == cudaSuccess && cache) set_a[dev] = smem_a;
    }
    if (e == cudaSuccess && (!cache || smem_b > set_b[dev])) {
        e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b);
        if (e == cudaSuccess && cache) set_b[dev] = smem_b;
    }
    if (e != cudaSuccess) return e;
    const dim3 grid = adj_grid<T>(a.m.nx, a.m.ny), block(TX, TYT);
    // the padded FP32 kernels wait for their predecessor's output (griddep_wait),
    // so they may overlap it: A with the previous step's B unless an event wait
    // on the recompute's stream precedes it (the first step of a segment), B
    // always with its A
    e = launch_pdl(PAD && overlap_prev, ka, grid, block, smem_a, s, a);
    if (e != cudaSuccess) return e;
    AdjArgs<T> b = a;
    b.Tpart = a.Tpart + (size_t)grid.x * grid.y * adj_warps<T>();
    e = launch_pdl(PAD, kb, grid, block, smem_b, s, b);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// compile-time HDM radius of the fast variants
template <typename T>
constexpr int adj_kc() { return sizeof(T) == 4 ? 26 : 40; }

template <typename T, bool SC, bool CDM, bool TAU1>
cudaError_t launch_adj_k(const AdjArgs<T> &a, bool padded, bool overlap_prev, cudaStream_t s) {
    if constexpr (CDM) {
        return launch_adj_t<T, SC, CDM, TAU1, 0, false>(a, overlap_prev, s);
    } else {
        if constexpr (sizeof(T) == 4)
            if (padded) return launch_adj_t<T, SC, CDM, TAU1, adj_kc<T>(), true>(a, overlap_prev, s);
        if (a.m.kx <= adj_kc<T>() && a.m.ky <= adj_kc<T>())
            return launch_adj_t<T, SC, CDM, TAU1, adj_kc<T>(), false>(a, overlap_prev, s);
        return launch_adj_t<T, SC, CDM, TAU1, 0, false>(a, overlap_prev, s);
    }
}

}  // namespace

template <typename T>
int adjoint_slots(int nx, int ny) {
    const dim3 g = adj_grid<T>(nx, ny);
    return 2 * (int)(g.x * g.y) * adj_warps<T>();
}

AdjLayout adjoint_layout(int nx, int ny, bool padded, bool tau1) {
    AdjLayout l;
    const int pp = nx + 2 * kGhost;
    l.dpitch = padded ? pp : nx;
    l.doff = padded ? kGhost : 0;
    l.dstride = (long long)l.dpitch * ny;
    l.naux = tau1 ? 4 : 6;
    l.lpitch = padded && tau1 ? pp : nx;
    l.loff = padded && tau1 ? kGhost : 0;
    l.lstride = (long long)l.lpitch * ny;
    l.nlam = tau1 ? 3 : 9;
    return l;
}

template <typename T>
cudaError_t launch_adjoint_step(const Model<T> &m, T R, T aalp, bool sc, bool cdm, bool tau1, bool padded,
                                const AdjLayout &l, const T *f, const T *q, int qpitch, int qoff, const T *lam_next,
                                T *aux, T *lam_out, double *Tpart, int *err, bool overlap_prev, cudaStream_t s) {
    AdjArgs<T> a;
    a.m = m;
    a.R = R;
    a.aalp = aalp;
    a.f = f;
    a.q = q;
    a.qpitch = qpitch;
    a.qoff = qoff;
    a.lam = lam_next;
    a.lam_out = lam_out;
    a.lstride = l.lstride;
    a.lpitch = l.lpitch;
    a.loff = l.loff;
    a.aux = aux;
    a.dstride = l.dstride;
    a.dpitch = l.dpitch;
    a.doff = l.doff;
    a.Tpart = Tpart;
    a.err = err;
    const long long n = (long long)m.nx * m.ny;
    a.nf = (padded && !cdm ? 5 : kQ) * n;   // the single-pass record or the state
    a.nq = (long long)qpitch * m.ny;
    a.nl = l.nlam * l.lstride;
    a.nd = l.naux * l.dstride;
    const double r = 0.5 * (std::sqrt(5.0) - 3.0);   // root of r^2/3 + r + 1/3 = 0 (Eq. 20's operator)
    a.r = (T)r;
    a.r5 = (T)std::pow(r, 5);
    a.r25 = (T)std::pow(r, 25);
#define LBM_ADJ_PICK(SC, CDM)                                                                             \
    return tau1 ? launch_adj_k<T, SC, CDM, true>(a, padded, overlap_prev, s)                               \
                : launch_adj_k<T, SC, CDM, false>(a, padded, overlap_prev, s)
    if (sc) {
        if (cdm) LBM_ADJ_PICK(true, true);
        LBM_ADJ_PICK(true, false);
    }
    if (cdm) LBM_ADJ_PICK(false, true);
    LBM_ADJ_PICK(false, false);
#undef LBM_ADJ_PICK
}

template <typename T>
cudaError_t launch_adjoint_seed(int nx, int ny, bool padded, const AdjLayout &l, const T *grad_rho, T *lam,
                                int *err, cudaStream_t s) {
    const long long n = (long long)nx * ny;
    if (padded)
        adj_seed_kernel<T, true><<<blocks_for(n), 256, 0, s>>>(nx, ny, l.nlam, grad_rho, lam, l.lstride, l.lpitch, l.loff,
                                                               err);
    else
        adj_seed_kernel<T, false><<<blocks_for(n), 256, 0, s>>>(nx, ny, l.nlam, grad_rho, lam, l.lstride, l.lpitch,
                                                                l.loff, err);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_initial(int nx, int ny, const AdjLayout &l, const T *lam, T *grad_rho0, int *err,
                                  cudaStream_t s) {
    const long long n = (long long)nx * ny;
    adj_initial_kernel<T><<<blocks_for(n), 256, 0, s>>>(nx, ny, l.nlam, lam, l.lstride, l.lpitch, l.loff, grad_rho0,
                                                        err);
    return cudaGetLastError();
}

cudaError_t launch_sum_slots(const double *slots, int nslots, double *out, cudaStream_t s) {
    sum_slots_kernel<<<1, 32, 0, s>>>(slots, nslots, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_density(long long n, const T *f, T *rho, cudaStream_t s) {
    density_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, f, rho);
    return cudaGetLastError();
}

#define LBM_ADJ_INST(T)                                                                                      \
    template int adjoint_slots<T>(int, int);                                                                \
    template cudaError_t launch_adjoint_step<T>(const Model<T> &, T, T, bool, bool, bool, bool, const AdjLayout &, \
                                                const T *, const T *, int, int, const T *, T *, T *, double *, int *, \
                                                bool, cudaStream_t);                                        \
    template cudaError_t launch_adjoint_seed<T>(int, int, bool, const AdjLayout &, const T *, T *, int *,         \
                                                cudaStream_t);                                                   \
    template cudaError_t launch_adjoint_initial<T>(int, int, const AdjLayout &, const T *, T *, int *, cudaStream_t); \
    template cudaError_t launch_density<T>(long long, const T *, T *, cudaStream_t);
LBM_ADJ_INST(float)
LBM_ADJ_INST(double)

}  // namespace lbm
