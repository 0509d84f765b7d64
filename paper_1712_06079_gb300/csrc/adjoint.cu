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
// (pass 1), then, because the periodic derivative is an antisymmetric
// circulant (its transpose is its negative),
//   Phi_bar = Phi_bar_centre - Dx[Dx_bar] - Dy[Dy_bar]
//   U_bar = Phi_bar sign(U) / (2 Phi) (SC) or Phi_bar (ZC)
//   rho_bar += U_bar (k dp/drho - 1/3),  T_bar += U_bar k dp/dT
//   lambda_i(t) = (1 - omega) g_i + rho_bar + e_i . j_bar
// (pass 2).  T_bar is accumulated in FP64 (block reduction, one atomic per block).
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {
namespace {

// dp_EOS/drho and dp_EOS/dT at the model temperature (Eq. 24, 27-29);
// m.RT = R T, m.aal = a alpha(T), aalp = a dalpha/dT, R the gas constant.
template <typename T>
__device__ __forceinline__ void p_derivs(const Model<T> &m, T R, T aalp, T rho, T &dpdr, T &dpdT) {
    if (m.eos == LBM_EOS_CS) {
        const T e = m.b * rho * T(0.25);
        const T om = T(1) - e;
        const T num = T(1) + e + e * e - e * e * e;
        const T Z = num / (om * om * om);
        const T dZ = ((T(1) + T(2) * e - T(3) * e * e) * om + T(3) * num) / (om * om * om * om);
        dpdr = m.RT * (Z + e * dZ) - T(2) * m.a * rho;
        dpdT = R * rho * Z;
        return;
    }
    const T om = T(1) - m.b * rho;
    const T drep_dr = m.RT / (om * om), drep_dT = R * rho / om;
    if (m.eos == LBM_EOS_VDW) {
        dpdr = drep_dr - T(2) * m.a * rho;
        dpdT = drep_dT;
    } else if (m.eos == LBM_EOS_PR) {
        const T den = T(1) + T(2) * m.b * rho - m.b * m.b * rho * rho;
        dpdr = drep_dr - m.aal * T(2) * rho * (T(1) + m.b * rho) / (den * den);
        dpdT = drep_dT - aalp * rho * rho / den;
    } else {  // RK, RKS
        const T den = T(1) + m.b * rho;
        dpdr = drep_dr - m.aal * rho * (T(2) + m.b * rho) / (den * den);
        dpdT = drep_dT - aalp * rho * rho / den;
    }
}

template <typename T>
struct AdjArgs {
    Model<T> m;
    T R;          // gas constant
    T aalp;       // a dalpha/dT
    const T *f;   // state at t
    const T *q;   // potential field of f: s Phi (SC) or U (ZC)
    const T *lam; // adjoint at t+1
    T *aux;       // 6 fields: rho_bar, jx_bar, jy_bar, Dx_bar, Dy_bar, Phi_bar_centre
    T *lam_out;   // adjoint at t
    double *Tbar; // FP64 accumulator of dL/dT
};

template <typename T, bool SC>
__device__ __forceinline__ T st(T v) {
    return SC ? fabs(v) : v;
}

// Periodic derivative of a field at (x, y) of an nx x ny lattice.
template <typename T, bool SC, bool CDM>
__device__ __forceinline__ void deriv(const Model<T> &m, const T *__restrict__ q, int x, int y, T &dx, T &dy) {
    const int nx = m.nx, ny = m.ny;
    if (CDM) {
        const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
        const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
        auto at = [&](int yy, int xx) { return st<T, SC>(q[(long long)yy * nx + xx]); };
        const T e = at(y, xp), w = at(y, xm), nn = at(yp, x), s = at(ym, x);
        const T ne = at(yp, xp), nw = at(yp, xm), se = at(ym, xp), sw = at(ym, xm);
        dx = T(1.0 / 3.0) * (e - w) + T(1.0 / 12.0) * ((ne + se) - (nw + sw));
        dy = T(1.0 / 3.0) * (nn - s) + T(1.0 / 12.0) * ((ne + nw) - (se + sw));
        return;
    }
    const T *row = q + (long long)y * nx;
    T ax = T(0), ay = T(0);
    for (int j = 1; j <= m.kx; ++j) {
        int xp = x + j, xm = x - j;
        if (xp >= nx) xp -= nx;
        if (xm < 0) xm += nx;
        ax += m.wx[j] * (st<T, SC>(row[xp]) - st<T, SC>(row[xm]));
    }
    for (int j = 1; j <= m.ky; ++j) {
        int yp = y + j, ym = y - j;
        if (yp >= ny) yp -= ny;
        if (ym < 0) ym += ny;
        ay += m.wy[j] * (st<T, SC>(q[(long long)yp * nx + x]) - st<T, SC>(q[(long long)ym * nx + x]));
    }
    dx = ax;
    dy = ay;
}

template <typename T, bool SC, bool CDM>
__global__ void adj_local_kernel(const AdjArgs<T> a) {
    const Model<T> &m = a.m;
    const long long n = (long long)m.nx * m.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(c / m.nx), x = (int)(c - (long long)y * m.nx);
        T fi[kQ], g[kQ];
        T r = T(0), jx = T(0), jy = T(0);
        const int xp = x + 1 == m.nx ? 0 : x + 1, xm = x == 0 ? m.nx - 1 : x - 1;
        const int yp = y + 1 == m.ny ? 0 : y + 1, ym = y == 0 ? m.ny - 1 : y - 1;
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            fi[i] = a.f[i * n + c];
            r += fi[i];
            jx += T(ex(i)) * fi[i];
            jy += T(ey(i)) * fi[i];
            const int dxs = ex(i) == 1 ? xp : (ex(i) == -1 ? xm : x);
            const int dys = ey(i) == 1 ? yp : (ey(i) == -1 ? ym : y);
            g[i] = a.lam[i * n + (long long)dys * m.nx + dxs];  // lambda_i(x + e_i)
        }
        T Dx, Dy;
        deriv<T, SC, CDM>(m, a.q, x, y, Dx, Dy);
        const T qc = a.q[c];
        T Fx, Fy;
        if (SC) { Fx = T(-2) * qc * Dx; Fy = T(-2) * qc * Dy; }
        else { Fx = -Dx; Fy = -Dy; }
        const T inv = T(1) / r;
        const T ux = jx * inv, uy = jy * inv, vx = ux + Fx * inv, vy = uy + Fy * inv;
        const T uu = ux * ux + uy * uy, vv = vx * vx + vy * vy;
        const T om1 = T(1) - m.omega;
        T rb = T(0), ubx = T(0), uby = T(0), vbx = T(0), vby = T(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const T exi = T(ex(i)), eyi = T(ey(i)), w = wq<T>(i);
            const T eu = exi * ux + eyi * uy, ev = exi * vx + eyi * vy;
            const T feq_u = r * w * (T(1) + T(3) * eu + T(4.5) * eu * eu - T(1.5) * uu);
            const T feq_v = r * w * (T(1) + T(3) * ev + T(4.5) * ev * ev - T(1.5) * vv);
            const T ai = -om1 * g[i], bi = g[i];
            rb += (ai * feq_u + bi * feq_v) * inv;
            const T cu = ai * r * w, cv = bi * r * w;
            ubx += cu * (T(3) * exi + T(9) * eu * exi - T(3) * ux);
            uby += cu * (T(3) * eyi + T(9) * eu * eyi - T(3) * uy);
            vbx += cv * (T(3) * exi + T(9) * ev * exi - T(3) * vx);
            vby += cv * (T(3) * eyi + T(9) * ev * eyi - T(3) * vy);
        }
        ubx += vbx;
        uby += vby;
        const T Fbx = vbx * inv, Fby = vby * inv;
        rb -= (vbx * Fx + vby * Fy) * inv * inv;
        const T jbx = ubx * inv, jby = uby * inv;
        rb -= (ubx * ux + uby * uy) * inv;
        T Dbx, Dby, Pc;
        if (SC) {
            Dbx = T(-2) * qc * Fbx;
            Dby = T(-2) * qc * Fby;
            const T s = qc >= T(0) ? T(1) : T(-1);
            Pc = T(-2) * s * (Fbx * Dx + Fby * Dy);
        } else {
            Dbx = -Fbx;
            Dby = -Fby;
            Pc = T(0);
        }
        a.aux[0 * n + c] = rb;
        a.aux[1 * n + c] = jbx;
        a.aux[2 * n + c] = jby;
        a.aux[3 * n + c] = Dbx;
        a.aux[4 * n + c] = Dby;
        a.aux[5 * n + c] = Pc;
    }
}

template <typename T, bool SC, bool CDM>
__global__ void adj_finish_kernel(const AdjArgs<T> a) {
    const Model<T> &m = a.m;
    const long long n = (long long)m.nx * m.ny;
    double tb = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(c / m.nx), x = (int)(c - (long long)y * m.nx);
        // Phi_bar = centre term - Dx[Dx_bar] - Dy[Dy_bar]  (transpose of the antisymmetric derivative)
        T ddx, ddy, tmp;
        deriv<T, false, CDM>(m, a.aux + 3 * n, x, y, ddx, tmp);
        deriv<T, false, CDM>(m, a.aux + 4 * n, x, y, tmp, ddy);
        const T pbar = a.aux[5 * n + c] - ddx - ddy;
        T r = T(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) r += a.f[i * n + c];
        const T qc = a.q[c];
        T Ubar;
        if (SC) {
            const T phi = fabs(qc);
            const T s = qc >= T(0) ? T(1) : T(-1);
            Ubar = phi > T(0) ? pbar * s / (T(2) * phi) : T(0);
        } else {
            Ubar = pbar;
        }
        T dpdr, dpdT;
        p_derivs(m, a.R, a.aalp, r, dpdr, dpdT);
        const T rb = a.aux[0 * n + c] + Ubar * (m.k * dpdr - T(1.0 / 3.0));
        tb += (double)Ubar * (double)m.k * (double)dpdT;
        const T jbx = a.aux[1 * n + c], jby = a.aux[2 * n + c];
        const T om1 = T(1) - m.omega;
        const int xp = x + 1 == m.nx ? 0 : x + 1, xm = x == 0 ? m.nx - 1 : x - 1;
        const int yp = y + 1 == m.ny ? 0 : y + 1, ym = y == 0 ? m.ny - 1 : y - 1;
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            T direct = T(0);
            if (om1 != T(0)) {
                const int dxs = ex(i) == 1 ? xp : (ex(i) == -1 ? xm : x);
                const int dys = ey(i) == 1 ? yp : (ey(i) == -1 ? ym : y);
                direct = om1 * a.lam[i * n + (long long)dys * m.nx + dxs];
            }
            a.lam_out[i * n + c] = direct + rb + T(ex(i)) * jbx + T(ey(i)) * jby;
        }
    }
    // FP64 block reduction of dL/dT
    __shared__ double sh[256];
    sh[threadIdx.x] = tb;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(a.Tbar, sh[0]);
}

template <typename T>
__global__ void adj_seed_kernel(long long n, const T *grad_rho, T *lam) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const T g = grad_rho[c];
#pragma unroll
        for (int i = 0; i < kQ; ++i) lam[i * n + c] = g;  // rho = sum_i f_i
    }
}

template <typename T>
__global__ void adj_initial_kernel(long long n, const T *lam, T *grad_rho0) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        T s = T(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) s += wq<T>(i) * lam[i * n + c];  // f_i = w_i rho0 at rest (Eq. 2)
        grad_rho0[c] = s;
    }
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

}  // namespace

template <typename T>
cudaError_t launch_adjoint_step(const Model<T> &m, T R, T aalp, bool sc, bool cdm, const T *f, const T *q,
                                const T *lam_next, T *aux, T *lam_out, double *Tbar, cudaStream_t s) {
    AdjArgs<T> a;
    a.m = m;
    a.R = R;
    a.aalp = aalp;
    a.f = f;
    a.q = q;
    a.lam = lam_next;
    a.aux = aux;
    a.lam_out = lam_out;
    a.Tbar = Tbar;
    const long long n = (long long)m.nx * m.ny;
    const int nb = blocks_for(n);
    if (sc) {
        if (cdm) { adj_local_kernel<T, true, true><<<nb, 256, 0, s>>>(a); adj_finish_kernel<T, true, true><<<nb, 256, 0, s>>>(a); }
        else { adj_local_kernel<T, true, false><<<nb, 256, 0, s>>>(a); adj_finish_kernel<T, true, false><<<nb, 256, 0, s>>>(a); }
    } else {
        if (cdm) { adj_local_kernel<T, false, true><<<nb, 256, 0, s>>>(a); adj_finish_kernel<T, false, true><<<nb, 256, 0, s>>>(a); }
        else { adj_local_kernel<T, false, false><<<nb, 256, 0, s>>>(a); adj_finish_kernel<T, false, false><<<nb, 256, 0, s>>>(a); }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_seed(long long n, const T *grad_rho, T *lam, cudaStream_t s) {
    adj_seed_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, grad_rho, lam);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_initial(long long n, const T *lam, T *grad_rho0, cudaStream_t s) {
    adj_initial_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, lam, grad_rho0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_density(long long n, const T *f, T *rho, cudaStream_t s) {
    density_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, f, rho);
    return cudaGetLastError();
}

#define LBM_ADJ_INST(T)                                                                                     \
    template cudaError_t launch_adjoint_step<T>(const Model<T> &, T, T, bool, bool, const T *, const T *,    \
                                                const T *, T *, T *, double *, cudaStream_t);                \
    template cudaError_t launch_adjoint_seed<T>(long long, const T *, T *, cudaStream_t);                  \
    template cudaError_t launch_adjoint_initial<T>(long long, const T *, T *, cudaStream_t);               \
    template cudaError_t launch_density<T>(long long, const T *, T *, cudaStream_t);
LBM_ADJ_INST(float)
LBM_ADJ_INST(double)

}  // namespace lbm
