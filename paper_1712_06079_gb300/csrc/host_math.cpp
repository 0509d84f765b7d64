// Host-side FP64 set-up math of the library: the critical point of each
// equation of state (to turn the reduced temperature T/Tc into T) and the
// weights of the explicit periodic form of the HDM operator (Eq. 20).
//
// Critical point.  Every EOS here splits as p(rho, T) = T A(rho) - beta(T) B(rho)
// with beta = 1 (VdW Eq. 24, CS Eq. 29, PR Eq. 28 and RKS at alpha(Tc) = 1)
// or beta = T^-1/2 (RK Eq. 27).  dp/drho = d2p/drho2 = 0 then gives
// A' B'' - A'' B' = 0, a one-dimensional root in rho, and T from
// T / beta(T) = B'/A'.  Derivatives come from second-order forward-mode
// automatic differentiation (a value/first/second-derivative triple).
//
// HDM weights.  On an infinite lattice the compact scheme of Eq. 20,
//   (1/3) d_{i-1} + d_i + (1/3) d_{i+1} = (1/36)(u_{i+2} - u_{i-2}) + (7/9)(u_{i+1} - u_{i-1}),
// inverts to d_i = sum_{j>=1} c_j (u_{i+j} - u_{i-j}).  The tridiagonal
// operator's Green's function is g_j = (3/sqrt 5) r^|j|, r = (sqrt 5 - 3)/2
// (the root of r^2 + 3r + 1 = 0 inside the unit circle), so
//   c_1 = (3/sqrt 5)[(7/9)(1 - r^2) + (1/36)(r - r^3)],
//   c_j = -(25/12) r^j  for j >= 2.
// On a periodic line of n points the operator is the circulant with the
// folded kernel sum_m c_{j + m n} (c_{-j} = -c_j), which is exactly the
// periodic (cyclic) tridiagonal solve.
#include <algorithm>
#include <cmath>

#include "lbm.h"

namespace {

struct Dual2 {  // value, first and second derivative w.r.t. one variable
    double v, d, dd;
};
inline Dual2 cst(double c) { return {c, 0.0, 0.0}; }
inline Dual2 operator+(Dual2 a, Dual2 b) { return {a.v + b.v, a.d + b.d, a.dd + b.dd}; }
inline Dual2 operator-(Dual2 a, Dual2 b) { return {a.v - b.v, a.d - b.d, a.dd - b.dd}; }
inline Dual2 operator*(Dual2 a, Dual2 b) {
    return {a.v * b.v, a.d * b.v + a.v * b.d, a.dd * b.v + 2.0 * a.d * b.d + a.v * b.dd};
}
inline Dual2 recip(Dual2 a) {
    double i = 1.0 / a.v;
    return {i, -a.d * i * i, (2.0 * a.d * a.d * i - a.dd) * i * i};
}
inline Dual2 operator/(Dual2 a, Dual2 b) { return a * recip(b); }

// Repulsive part A (p = T A - beta B) and attractive part B of each EOS,
// both without T; alpha enters through beta for RK and is 1 for PR/RKS at Tc.
void eos_parts(int eos, double a, double b, double R, Dual2 rho, Dual2 *A, Dual2 *B) {
    Dual2 one = cst(1.0);
    if (eos == LBM_EOS_CS) {
        Dual2 e = cst(b / 4.0) * rho;
        Dual2 om = one - e;
        *A = cst(R) * rho * (one + e + e * e - e * e * e) / (om * om * om);
        *B = cst(a) * rho * rho;
        return;
    }
    *A = cst(R) * rho / (one - cst(b) * rho);
    if (eos == LBM_EOS_VDW) *B = cst(a) * rho * rho;
    else if (eos == LBM_EOS_PR) *B = cst(a) * rho * rho / (one + cst(2.0 * b) * rho - cst(b * b) * rho * rho);
    else *B = cst(a) * rho * rho / (one + cst(b) * rho);
}

double wronskian(int eos, double a, double b, double R, double rho) {
    Dual2 A, B;
    eos_parts(eos, a, b, R, {rho, 1.0, 0.0}, &A, &B);
    return A.d * B.dd - A.dd * B.d;
}

}  // namespace

extern "C" lbm_status lbm_critical_point(int eos, double a, double b, double R, double *Tc, double *rho_c) {
    if (!Tc || !rho_c || eos < LBM_EOS_VDW || eos > LBM_EOS_RKS || !(a > 0) || !(b > 0) || !(R > 0))
        return LBM_E_INVALID;
    const double pole = (eos == LBM_EOS_CS) ? 4.0 / b : 1.0 / b;
    // scan for the first sign change of the Wronskian, then bisect
    const int N = 2000;
    double lo = -1, hi = -1, wprev = wronskian(eos, a, b, R, pole * 0.5 / N);
    for (int i = 1; i < N; ++i) {
        double r = pole * (i + 0.5) / N;
        double w = wronskian(eos, a, b, R, r);
        if ((w > 0) != (wprev > 0)) { lo = pole * (i - 0.5) / N; hi = r; break; }
        wprev = w;
    }
    if (lo < 0) return LBM_E_INVALID;
    bool lo_pos = wronskian(eos, a, b, R, lo) > 0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if ((wronskian(eos, a, b, R, mid) > 0) == lo_pos) lo = mid; else hi = mid;
    }
    double rc = 0.5 * (lo + hi);
    Dual2 A, B;
    eos_parts(eos, a, b, R, {rc, 1.0, 0.0}, &A, &B);
    double ratio = B.d / A.d;  // T / beta(T)
    *rho_c = rc;
    *Tc = (eos == LBM_EOS_RK) ? std::pow(ratio, 2.0 / 3.0) : ratio;
    return LBM_OK;
}

namespace {

// p_EOS(rho) and dp/drho at absolute temperature T with the given alpha.
void eos_p(int eos, double a, double b, double R, double T, double alpha, double rho, double *p, double *dp) {
    Dual2 A, B;
    eos_parts(eos, a, b, R, {rho, 1.0, 0.0}, &A, &B);
    *p = T * A.v - alpha * B.v;
    *dp = T * A.d - alpha * B.d;
}

struct Isotherm {
    int eos;
    double a, b, R, T, alpha;
    double G = 0, rho0 = 1;  // LBM_EOS_PSI_EXP: p = rho/3 + (G/2) psi^2, psi = 1 - exp(-rho/rho0) (Eq. 5)
    void eval(double rho, double *v, double *d) const {
        if (eos == LBM_EOS_PSI_EXP) {
            const double e = std::exp(-rho / rho0), psi = 1.0 - e;
            *v = rho / 3.0 + 0.5 * G * psi * psi;
            *d = 1.0 / 3.0 + G * psi * e / rho0;
            return;
        }
        eos_p(eos, a, b, R, T, alpha, rho, v, d);
    }
    double p(double rho) const { double v, d; eval(rho, &v, &d); return v; }
    double dp(double rho) const { double v, d; eval(rho, &v, &d); return d; }
};

// Root of dp/drho = 0 in [lo, hi] (dp changes sign there), by bisection.
double dp_root(const Isotherm &I, double lo, double hi) {
    bool lo_pos = I.dp(lo) > 0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if ((I.dp(mid) > 0) == lo_pos) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// rho in [lo, hi] with p(rho) = ps, p monotone increasing there (safeguarded Newton).
double p_root(const Isotherm &I, double ps, double lo, double hi) {
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double v = I.p(x) - ps;
        if (v > 0) hi = x; else lo = x;
        double d = I.dp(x);
        double xn = x - v / d;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (std::fabs(xn - x) <= 1e-16 * x) { x = xn; break; }
        x = xn;
    }
    return x;
}

// int_{rg}^{rl} (p - ps)/rho^2 drho, 16-point Gauss-Legendre on 64 panels in s = ln rho.
double area(const Isotherm &I, double ps, double rg, double rl) {
    static const double xg[8] = {0.0950125098376374, 0.2816035507792589, 0.4580167776572274, 0.6178762444026438,
                                 0.7554044083550030, 0.8656312023878318, 0.9445750230732326, 0.9894009349916499};
    static const double wg[8] = {0.1894506104550685, 0.1826034150449236, 0.1691565193950025, 0.1495959888165767,
                                 0.1246289712555339, 0.0951585116824928, 0.0622535239386479, 0.0271524594117541};
    const int panels = 64;
    const double s0 = std::log(rg), s1 = std::log(rl), h = (s1 - s0) / panels;
    double acc = 0.0;
    for (int k = 0; k < panels; ++k) {
        const double c = s0 + (k + 0.5) * h;
        for (int i = 0; i < 8; ++i)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                const double rho = std::exp(c + sgn * xg[i] * 0.5 * h);
                acc += wg[i] * (I.p(rho) - ps) / rho;
            }
    }
    return acc * 0.5 * h;
}

}  // namespace

extern "C" lbm_status lbm_maxwell(const lbm_params *p, double *rho_g, double *rho_l) {
    if (!p || !rho_g || !rho_l) return LBM_E_INVALID;
    Isotherm I{p->eos, p->a, p->b, p->R, 0.0, 1.0};
    double pole;
    if (p->eos == LBM_EOS_PSI_EXP) {
        if (!(p->G < 0) || !(p->rho0 > 0) || !std::isfinite(p->G)) return LBM_E_INVALID;
        I.G = p->G;
        I.rho0 = p->rho0;
        pole = 50.0 * p->rho0;  // no pole: psi saturates and p grows as rho/3
    } else {
        if (p->eos < LBM_EOS_VDW || p->eos > LBM_EOS_RKS || !(p->a > 0) || !(p->b > 0) || !(p->R > 0) ||
            !(p->Tr > 0))
            return LBM_E_INVALID;
        double Tc = p->Tc, rc = 0;
        if (!(Tc > 0) && lbm_critical_point(p->eos, p->a, p->b, p->R, &Tc, &rc) != LBM_OK) return LBM_E_INVALID;
        if (!(p->Tr < 1.0)) return LBM_E_INVALID;
        I.T = p->Tr * Tc;
        pole = (p->eos == LBM_EOS_CS) ? 4.0 / p->b : 1.0 / p->b;
    }
    if (p->eos == LBM_EOS_RK) I.alpha = 1.0 / std::sqrt(I.T);
    else if (p->eos == LBM_EOS_PR || p->eos == LBM_EOS_RKS) {
        const double w = p->omega;
        const double m = p->eos == LBM_EOS_PR ? 0.37464 + 1.54226 * w - 0.26992 * w * w : 0.480 + 1.574 * w - 0.176 * w * w;
        const double s = 1.0 + m * (1.0 - std::sqrt(p->Tr));
        I.alpha = s * s;
    }
    // the isotherm's local maximum and minimum: sign changes of dp/drho on a log grid
    const int N = 4000;
    double prev = I.dp(pole * 1e-12), lo_prev = pole * 1e-12, smax = -1, smin = -1;
    for (int i = 1; i <= N; ++i) {
        const double rho = pole * std::exp(std::log(1e-12) * (1.0 - double(i) / N)) * (1.0 - 1e-9);
        const double d = I.dp(rho);
        if (prev > 0 && d <= 0 && smax < 0) smax = dp_root(I, lo_prev, rho);
        else if (prev <= 0 && d > 0 && smax > 0) { smin = dp_root(I, lo_prev, rho); break; }
        prev = d;
        lo_prev = rho;
    }
    if (smax < 0 || smin < 0) return LBM_E_INVALID;  // no van der Waals loop
    double plo = std::max(I.p(smin), 0.0), phi = I.p(smax);
    double rg = 0, rl = 0;
    for (int it = 0; it < 200; ++it) {  // bisection on p_sat: the area decreases as p_sat rises
        const double ps = 0.5 * (plo + phi);
        if (ps <= plo || ps >= phi) break;
        rg = p_root(I, ps, 0.0, smax);
        rl = p_root(I, ps, smin, pole);
        if (area(I, ps, rg, rl) > 0) plo = ps; else phi = ps;
    }
    const double ps = 0.5 * (plo + phi);
    *rho_g = p_root(I, ps, 0.0, smax);
    *rho_l = p_root(I, ps, smin, pole);
    return LBM_OK;
}

extern "C" lbm_status lbm_hdm_weights(int n, int radius, double *w, int *k_eff) {
    if (!w || !k_eff || n < 1 || radius < 0) return LBM_E_INVALID;
    const double s5 = std::sqrt(5.0);
    const double r = (s5 - 3.0) / 2.0;
    const double c1 = (3.0 / s5) * ((7.0 / 9.0) * (1.0 - r * r) + (1.0 / 36.0) * (r - r * r * r));
    auto c = [&](long j) -> double {  // infinite-lattice kernel, antisymmetric
        if (j == 0) return 0.0;
        long aj = j < 0 ? -j : j;
        double v = (aj == 1) ? c1 : -(25.0 / 12.0) * std::pow(r, (double)aj);
        return j < 0 ? -v : v;
    };
    int ke = (n - 1) / 2;
    if (ke > radius) ke = radius;
    w[0] = 0.0;
    for (int j = 1; j <= radius; ++j) w[j] = 0.0;
    for (int j = 1; j <= ke; ++j) {
        // fold: sum over m of c_{j + m n}; terms decay as |r|^{|j + m n|}
        double acc = c(j);
        for (long m = 1;; ++m) {
            double t1 = c(j + m * (long)n), t2 = c(j - m * (long)n);
            acc += t1 + t2;
            if (std::fabs(t1) + std::fabs(t2) < 1e-300 || m * (long)n > 2000) break;
        }
        w[j] = acc;
    }
    *k_eff = ke;
    return LBM_OK;
}
