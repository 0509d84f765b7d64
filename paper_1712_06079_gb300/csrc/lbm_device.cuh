// Device-side building blocks of the D2Q9 pseudopotential step (sm_103a).
//
// D2Q9 ordering (Eq. 2, "D2Q9 model"; the paper does not print it):
//   i : 0     1     2     3     4     5      6      7       8
//   e : (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
//   w : 4/9, 1/9 for the axes, 1/36 for the diagonals.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"

namespace lbm {

constexpr int kQ = 9;
constexpr int kMaxRadius = 48;  // largest HDM truncation radius accepted

__host__ __device__ __forceinline__ constexpr int ex(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int ey(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
template <typename T>
__host__ __device__ __forceinline__ constexpr T wq(int i) {
    return i == 0 ? T(4.0 / 9.0) : (i < 5 ? T(1.0 / 9.0) : T(1.0 / 36.0));
}

// Error word bits written by kernels (read back by lbm_sync).
constexpr int kErrUnstable = 1;  // NaN or rho <= 0 seen
constexpr int kErrTimeout = 2;   // a bounded device-side wait gave up
constexpr int kErrBounds = 4;    // a self-checked index fell outside a buffer

// Bounds self-checks of the LBM_CHECKED build: an index outside its buffer
// sets kErrBounds in the error word and the access is skipped (no fault, no
// trap); in the normal build the check is compiled away.
#ifdef LBM_CHECKED
__device__ __forceinline__ bool in_bounds(long long i, long long n, int *err) {
    if (i >= 0 && i < n) return true;
    if (err) atomicOr(err, kErrBounds);
    return false;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(long long, long long, int *) { return true; }
#endif

// Per-launch constants of the model, in the working precision.
template <typename T>
struct Model {
    int *chk;      // error word of the bounds self-checks (LBM_CHECKED builds; may be null)
    int nx, ny;
    int eos;       // lbm_eos
    int kx, ky;    // HDM stencil radius along x and y (already folded to the period)
    int walls;     // 0: periodic in y; 1: no-slip walls below row 0 and above row ny-1
    T RT;          // R * T
    T a, b;        // EOS constants; for LBM_EOS_PSI_EXP a = G/2, b = 1/rho0 (Eq. 4-5)
    T aal;         // a * alpha(T) (PR, RK, RKS)
    T k;           // Hu scaling
    T omega;       // 1 / tau
    T wx[kMaxRadius + 1];  // explicit HDM weights along x (w[0] unused)
    T wy[kMaxRadius + 1];  // ... along y
};

// p_EOS(rho) at the model's temperature (Eq. 24, 27, 28, 29); no Hu factor.
template <typename T>
__device__ __forceinline__ T p_eos(const Model<T> &m, T rho) {
    if (m.eos == LBM_EOS_CS) {
        T e = m.b * rho * T(0.25);
        T om = T(1) - e;
        return rho * m.RT * (T(1) + e + e * e - e * e * e) / (om * om * om) - m.a * rho * rho;
    }
    T rep = rho * m.RT / (T(1) - m.b * rho);
    if (m.eos == LBM_EOS_VDW) return rep - m.a * rho * rho;
    if (m.eos == LBM_EOS_PR) return rep - m.aal * rho * rho / (T(1) + T(2) * m.b * rho - m.b * m.b * rho * rho);
    return rep - m.aal * rho * rho / (T(1) + m.b * rho);  // RK, RKS
}

// Interaction potential U = k p_EOS - rho c_s^2 (Eq. 8 with Hu scaling); for
// the effective mass of Eq. 4 (a = G/2, b = 1/rho0) U = p - rho c_s^2 =
// (G/2) psi^2 (Eq. 5), so the Eq. 22 form -2 s Phi grad Phi with
// Phi = sqrt|U| is the force -G psi grad psi of Eq. 4.
template <typename T>
__device__ __forceinline__ T potential_u(const Model<T> &m, T rho) {
    if (m.eos == LBM_EOS_PSI_EXP) {
        const T psi = T(1) - exp(-rho * m.b);
        return m.a * psi * psi;
    }
    return m.k * p_eos(m, rho) - rho * T(1.0 / 3.0);
}

// Field stored for the gradient: SC (Eq. 21/22) keeps the signed root
// q = s sqrt|U| (the stencil uses |q| = Phi, the cell itself s Phi);
// ZC (Eq. 7) keeps U.
template <typename T>
__device__ __forceinline__ T potential_field(const Model<T> &m, T rho, bool sc) {
    T U = potential_u(m, rho);
    if (!sc) return U;
    return U >= T(0) ? sqrt(U) : -sqrt(-U);
}

// Row index across no-slip walls: the field's mirror image continues it
// (q(-1-j) = q(j), q(n+j) = q(n-1-j)), period 2n.
__device__ __forceinline__ int mirror_index(int i, int n) {
    const int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

// Opposite direction of population i (e_opp = -e_i).
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i < 5 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5); }

// Periodic wrap of an index that may lie several periods outside [0, n).
__device__ __forceinline__ int wrap_index(int i, int n) {
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}

// HDM derivative of four consecutive cells from a window of 60 staged values
// t[0..59], the cells at positions 28..31 (positions 2..57 are read): the
// explicit periodic operator of Eq. 20 truncated at radius 26, whose weights
// are geometric past the first, w_j = w_2 r^(j-2), run in recurrence form:
//   P_c = sum_{j=2..26} r^(j-2) t_(28+c-j),   Q_c = sum_{j=2..26} r^(j-2) t_(28+c+j),
//   D_c = w_1 (t_(29+c) - t_(27+c)) + w_2 (Q_c - P_c).
// P_0 and Q_3 are five independent 5-term Horner groups joined by r^5; the
// other cells follow by one step each (P_c = t_(26+c) + r P_(c-1) - r^25
// t_(1+c), Q mirrored), dropping the term that leaves the radius, so the
// truncation is the stencil's.  t should hold deviations from a nearby value:
// the constant part cancels between P and Q, and the sums then carry only
// local variations.
__device__ __forceinline__ void hdm_window4(const float (&t)[60], float w1, float w2, float r, float r5, float r25,
                                            float (&d)[4]) {
    float gp[5], gq[5];
#pragma unroll
    for (int g = 0; g < 5; ++g) {
        float x = t[2 + 5 * g];                 // P_0: positions 2 + 5g .. 6 + 5g, far to near
#pragma unroll
        for (int i = 1; i < 5; ++i) x = fmaf(r, x, t[2 + 5 * g + i]);
        gp[g] = x;
        float y = t[37 + 5 * g];                // Q_3: positions 37 + 5g .. 33 + 5g, far to near
#pragma unroll
        for (int i = 1; i < 5; ++i) y = fmaf(r, y, t[37 + 5 * g - i]);
        gq[g] = y;
    }
    float P[4], Q[4];
    P[0] = fmaf(fmaf(fmaf(fmaf(gp[0], r5, gp[1]), r5, gp[2]), r5, gp[3]), r5, gp[4]);
    Q[3] = fmaf(fmaf(fmaf(fmaf(gq[4], r5, gq[3]), r5, gq[2]), r5, gq[1]), r5, gq[0]);
#pragma unroll
    for (int c = 1; c < 4; ++c) P[c] = fmaf(-r25, t[1 + c], fmaf(r, P[c - 1], t[26 + c]));
#pragma unroll
    for (int c = 2; c >= 0; --c) Q[c] = fmaf(-r25, t[55 + c], fmaf(r, Q[c + 1], t[30 + c]));
#pragma unroll
    for (int c = 0; c < 4; ++c) d[c] = fmaf(w1, t[29 + c] - t[27 + c], w2 * (Q[c] - P[c]));
}

// hdm_window4 on packed FP32 pairs.  The 56 deviations arrive as the pairs
// tp[j] = (t_(2+j), t_(57-j)), j = 0..27, so that P's group g and Q's group
// 4 - g run side by side (the same positions mirrored about the window's
// centre), then the joins (P_0, Q_3) and the steps (P_c, Q_(3-c)).  Each
// component is rounded as the scalar fma, so the result equals hdm_window4's
// bit for bit with half the multiply-adds.
__device__ __forceinline__ void hdm_window4_paired(const float2 (&tp)[28], float w1, float w2, float r, float r5,
                                                   float r25, float (&d)[4]) {
    const float2 r2 = make_float2(r, r), r52 = make_float2(r5, r5), mr25 = make_float2(-r25, -r25);
    float2 G[5];
#pragma unroll
    for (int g = 0; g < 5; ++g) {
        float2 x = tp[5 * g];
#pragma unroll
        for (int i = 1; i < 5; ++i) x = __ffma2_rn(r2, x, tp[5 * g + i]);
        G[g] = x;                               // (group g of P_0, group 4 - g of Q_3)
    }
    float2 S[4];                                // S_c = (P_c, Q_(3-c))
    S[0] = G[0];
#pragma unroll
    for (int g = 1; g < 5; ++g) S[0] = __ffma2_rn(r52, S[0], G[g]);
#pragma unroll
    for (int c = 1; c < 4; ++c) S[c] = __ffma2_rn(mr25, tp[c - 1], __ffma2_rn(r2, S[c - 1], tp[24 + c]));
    auto at = [&](int p) { return p <= 29 ? tp[p - 2].x : tp[57 - p].y; };   // t_p, p = 27..32
#pragma unroll
    for (int c = 0; c < 4; ++c) d[c] = fmaf(w1, at(29 + c) - at(27 + c), w2 * (S[3 - c].y - S[c].x));
}

}  // namespace lbm
