/*
 * Oracle for the pseudopotential multiphase lattice Boltzmann step with the
 * high-order-difference (HDM) interaction of Qin, Zhao, Chen, Zhang & Wen,
 * "A pseudopotential multiphase lattice Boltzmann model based on high-order
 * difference" (arXiv:1712.06079).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, FP64 CPU statement
 * of what the GPU path computes.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * Every step follows the paper's equations in the paper's order:
 *   Eq. 3   density and momentum moments
 *   Sec. 5  Hu scaling p = k p_EOS; Eq. 24, 27, 28, 29 equations of state
 *   Eq. 8   U = p - rho c_s^2;  Eq. 21  Phi = sqrt|U|
 *   Eq. 20  HDM first derivative, solved as the periodic (cyclic) tridiagonal
 *           system it is, by the chasing (Thomas) method plus a
 *           Sherman-Morrison correction for the two corner entries
 *   Eq. 15  weighted CDM (the comparison arm), scaled by 1/c_s^2
 *   Eq. 22  Shan-Chen force in Phi form;  Eq. 7  Zhang-Chen force -grad U
 *   Eq. 10  Kupershtokh exact-difference forcing;  Eq. 2 equilibrium
 *   Eq. 1   BGK collision and streaming on the periodic lattice
 *   Eq. 11  the observable half-step velocity
 * plus the Maxwell equal-area construction (Sec. 5.2), the critical point, the
 * flat-interface profile (Eq. 25-26) and a complex-step derivative of the step
 * (the same step in complex arithmetic) that checks reverse-mode gradients.
 *
 * No FMA contraction, no fast math: compile with -ffp-contract=off.
 * Threads (OpenMP) split the lattice by rows only; every cell's arithmetic and
 * every reduction order is independent of the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_VDW = 0, ORC_CS = 1, ORC_PR = 2, ORC_RK = 3, ORC_RKS = 4, ORC_PSI = 5 };
enum { ORC_SC = 0, ORC_ZC = 1 };
enum { ORC_HDM = 0, ORC_CDM = 1 };

typedef struct {
    int nx, ny;
    int eos;      /* ORC_VDW .. ORC_RKS, or ORC_PSI: the effective mass of Eq. 4 */
    int force;    /* ORC_SC (Eq. 22) or ORC_ZC (Eq. 7) */
    int grad;     /* ORC_HDM (Eq. 20) or ORC_CDM (Eq. 15) */
    int walls;    /* 0: periodic in y; 1: no-slip walls half a spacing below row 0
                     and above row ny-1 (Sec. 5.5) */
    double a, b, R, omega;
    double T;     /* absolute temperature */
    double Tc;    /* critical temperature (used by the alpha(T) of PR and RKS) */
    double k;     /* Hu scaling of the EOS, Sec. 5 */
    double tau;   /* BGK relaxation time, Eq. 1 */
    double G;     /* ORC_PSI: interaction strength of Eq. 4 */
    double rho0;  /* ORC_PSI: reference density of psi = 1 - exp(-rho/rho0) */
} orc_params;

/* D2Q9 velocity set and weights (Eq. 2 "D2Q9 model"; the paper does not print
 * them -- these are the standard 4/9, 1/9, 1/36). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const double CS2 = 1.0 / 3.0;  /* c_s^2 of D2Q9, Sec. 2 */

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* ------------------------------------------------------------------------ */
/* Equations of state (Sec. 5.2).                                            */
/* ------------------------------------------------------------------------ */

/* alpha(T) of Eq. 27 (RK: 1/sqrt(T)), Eq. 28 (PR: Soave-type with omega) and
 * the RKS form given after Eq. 27. VdW and CS have none (returned as 1). */
static double orc_alpha(int eos, double omega, double T, double Tc) {
    double m, s;
    switch (eos) {
    case ORC_PR:
        m = 0.37464 + 1.54226 * omega - 0.26992 * omega * omega;
        s = 1.0 + m * (1.0 - sqrt(T / Tc));
        return s * s;
    case ORC_RKS:
        m = 0.480 + 1.574 * omega - 0.176 * omega * omega;
        s = 1.0 + m * (1.0 - sqrt(T / Tc));
        return s * s;
    case ORC_RK:
        return 1.0 / sqrt(T);
    default:
        return 1.0;
    }
}

/* p_EOS(rho) and dp_EOS/drho at temperature T with a given alpha.
 * VdW Eq. 24; RK/RKS Eq. 27; PR Eq. 28; CS Eq. 29 with the standard
 * Carnahan-Starling denominator (1 - b rho/4)^3. */
static void eos_eval(int eos, double a, double b, double R, double T,
                     double alpha, double rho, double *p, double *dp) {
    double rep, drep, att, datt;
    if (eos == ORC_CS) {
        double e = b * rho / 4.0;
        double num = 1.0 + e + e * e - e * e * e;
        double om = 1.0 - e;
        double den = om * om * om;
        double Z = num / den;
        /* dZ/de = [(1 + 2e - 3e^2)(1-e) + 3 num] / (1-e)^4 */
        double dZ = ((1.0 + 2.0 * e - 3.0 * e * e) * om + 3.0 * num) / (den * om);
        rep = rho * R * T * Z;
        drep = R * T * (Z + e * dZ);
        att = a * rho * rho;
        datt = 2.0 * a * rho;
    } else {
        double om = 1.0 - b * rho;
        rep = rho * R * T / om;
        drep = R * T / (om * om);
        if (eos == ORC_VDW) {
            att = a * rho * rho;
            datt = 2.0 * a * rho;
        } else if (eos == ORC_PR) {
            double den = 1.0 + 2.0 * b * rho - b * b * rho * rho;
            att = a * alpha * rho * rho / den;
            datt = 2.0 * a * alpha * rho * (1.0 + b * rho) / (den * den);
        } else { /* RK, RKS */
            double den = 1.0 + b * rho;
            att = a * alpha * rho * rho / den;
            datt = a * alpha * rho * (2.0 + b * rho) / (den * den);
        }
    }
    if (p) *p = rep - att;
    if (dp) *dp = drep - datt;
}

static void eos_at(const orc_params *q, double rho, double *p, double *dp) {
    if (q->eos == ORC_PSI) {  /* Eq. 5: p = rho c_s^2 + (G/2) psi^2 */
        double e = exp(-rho / q->rho0), psi = 1.0 - e;
        if (p) *p = rho * CS2 + 0.5 * q->G * psi * psi;
        if (dp) *dp = CS2 + q->G * psi * e / q->rho0;
        return;
    }
    double al = orc_alpha(q->eos, q->omega, q->T, q->Tc);
    eos_eval(q->eos, q->a, q->b, q->R, q->T, al, rho, p, dp);
}

/* Vectorised p_EOS and dp/drho at the params' temperature (no Hu scaling). */
void orc_p_eos(const orc_params *q, const double *rho, double *p, double *dp, int n) {
    for (int i = 0; i < n; ++i) eos_at(q, rho[i], p ? &p[i] : NULL, dp ? &dp[i] : NULL);
}

/* Largest admissible density (repulsive-term pole): 1/b, or 4/b for CS. */
static double rho_pole(int eos, double b) { return eos == ORC_CS ? 4.0 / b : 1.0 / b; }

/* ------------------------------------------------------------------------ */
/* Critical point: the maximum over rho of the spinodal temperature T_sp(rho),
 * where dp/drho(rho, T_sp) = 0.  dp/drho rises with T at fixed rho for every
 * EOS here, so T_sp(rho) is a bisection in T.  For PR and RKS alpha is taken
 * as 1 (its value at T = Tc by construction); for RK alpha = 1/sqrt(T).      */
/* ------------------------------------------------------------------------ */

static double crit_alpha(int eos, double T) {
    return eos == ORC_RK ? 1.0 / sqrt(T) : 1.0;
}

static double spinodal_T(int eos, double a, double b, double R, double rho) {
    double lo = 1e-12, hi = 1.0, dp;
    /* grow hi until dp/drho > 0 */
    for (int it = 0; it < 200; ++it) {
        eos_eval(eos, a, b, R, hi, crit_alpha(eos, hi), rho, NULL, &dp);
        if (dp > 0) break;
        lo = hi;
        hi *= 2.0;
    }
    eos_eval(eos, a, b, R, lo, crit_alpha(eos, lo), rho, NULL, &dp);
    if (dp > 0) return 0.0; /* no spinodal at this density */
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        eos_eval(eos, a, b, R, mid, crit_alpha(eos, mid), rho, NULL, &dp);
        if (dp > 0) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

/* Returns 0 on success. */
int orc_critical_point(int eos, double a, double b, double R, double *Tc, double *rhoc) {
    double pole = rho_pole(eos, b);
    /* coarse scan on a fine grid, then golden-section refinement */
    int N = 4000, ibest = -1;
    double best = -1.0;
    for (int i = 1; i < N; ++i) {
        double rho = pole * i / N;
        double t = spinodal_T(eos, a, b, R, rho);
        if (t > best) { best = t; ibest = i; }
    }
    if (ibest < 0 || best <= 0) return 1;
    double lo = pole * (ibest - 1) / N, hi = pole * (ibest + 1) / N;
    const double g = 0.5 * (sqrt(5.0) - 1.0);
    double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
    double f1 = spinodal_T(eos, a, b, R, x1), f2 = spinodal_T(eos, a, b, R, x2);
    for (int it = 0; it < 200 && hi - lo > 1e-15 * pole; ++it) {
        if (f1 < f2) { lo = x1; x1 = x2; f1 = f2; x2 = lo + g * (hi - lo); f2 = spinodal_T(eos, a, b, R, x2); }
        else { hi = x2; x2 = x1; f2 = f1; x1 = hi - g * (hi - lo); f1 = spinodal_T(eos, a, b, R, x1); }
    }
    double rc = 0.5 * (lo + hi);
    *rhoc = rc;
    *Tc = spinodal_T(eos, a, b, R, rc);
    if (f1 > *Tc) *Tc = f1;
    if (f2 > *Tc) *Tc = f2;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Maxwell equal-area construction (Sec. 5.2): find p_s, rho_g < rho_l with   */
/* p(rho_g) = p(rho_l) = p_s and  int_{rho_g}^{rho_l} (p - p_s)/rho^2 drho = 0 */
/* (equal areas in the p-v plane, v = 1/rho).  The integral is taken in       */
/* s = ln(rho) by composite Simpson; p_s by bisection.                         */
/* ------------------------------------------------------------------------ */

static double p_of(const orc_params *q, double rho) {
    double p;
    eos_at(q, rho, &p, NULL);
    return p;
}

static double root_p(const orc_params *q, double ps, double lo, double hi) {
    /* p increasing on [lo, hi]; find p(rho) = ps */
    for (int it = 0; it < 300; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (p_of(q, mid) < ps) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static double area(const orc_params *q, double ps, double rg, double rl) {
    int n = 20000; /* even */
    double s0 = log(rg), s1 = log(rl), h = (s1 - s0) / n, acc = 0.0;
    for (int i = 0; i <= n; ++i) {
        double s = s0 + h * i, rho = exp(s);
        double g = (p_of(q, rho) - ps) / rho; /* (p - ps)/rho^2 * drho/ds */
        double wgt = (i == 0 || i == n) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        acc += wgt * g;
    }
    return acc * h / 3.0;
}

static double golden_extremum(const orc_params *q, double lo, double hi, int sign) {
    const double g = 0.5 * (sqrt(5.0) - 1.0);
    double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
    double f1 = sign * p_of(q, x1), f2 = sign * p_of(q, x2);
    for (int it = 0; it < 300 && hi - lo > 1e-16 * hi; ++it) {
        if (f1 < f2) { lo = x1; x1 = x2; f1 = f2; x2 = lo + g * (hi - lo); f2 = sign * p_of(q, x2); }
        else { hi = x2; x2 = x1; f2 = f1; x1 = hi - g * (hi - lo); f1 = sign * p_of(q, x1); }
    }
    return 0.5 * (lo + hi);
}

/* Returns 0 on success, 1 if the isotherm has no van der Waals loop. */
int orc_maxwell(const orc_params *q, double *rho_g, double *rho_l, double *p_sat) {
    /* Eq. 5 has no pole: p grows as rho/3 once psi saturates */
    double pole = q->eos == ORC_PSI ? 50.0 * q->rho0 : rho_pole(q->eos, q->b);
    /* locate the spinodal maximum and minimum on a log grid */
    int N = 20000;
    double lmin = log(pole * 1e-14), lmax = log(pole * (1.0 - 1e-9));
    double prev2 = 0, prev = 0;
    int imax = -1, imin = -1;
    for (int i = 0; i < N; ++i) {
        double rho = exp(lmin + (lmax - lmin) * i / (N - 1));
        double p = p_of(q, rho);
        if (i >= 2) {
            if (imax < 0 && prev > prev2 && prev >= p) imax = i - 1;
            else if (imax >= 0 && imin < 0 && prev < prev2 && prev <= p) { imin = i - 1; break; }
        }
        prev2 = prev;
        prev = p;
    }
    if (imax < 0 || imin < 0) return 1;
    double r_at = exp(lmin + (lmax - lmin) * (imax - 1) / (N - 1));
    double r_bt = exp(lmin + (lmax - lmin) * (imax + 1) / (N - 1));
    double rs1 = golden_extremum(q, r_at, r_bt, +1);
    r_at = exp(lmin + (lmax - lmin) * (imin - 1) / (N - 1));
    r_bt = exp(lmin + (lmax - lmin) * (imin + 1) / (N - 1));
    double rs2 = golden_extremum(q, r_at, r_bt, -1);
    double pmax = p_of(q, rs1), pmin = p_of(q, rs2);
    double lo = pmin > 0 ? pmin : 0.0, hi = pmax;
    double rg = 0, rl = 0;
    for (int it = 0; it < 200; ++it) {
        double ps = 0.5 * (lo + hi);
        if (ps <= lo || ps >= hi) break;
        rg = root_p(q, ps, 0.0, rs1);
        rl = root_p(q, ps, rs2, pole);
        double A = area(q, ps, rg, rl);
        if (A > 0) lo = ps; else hi = ps;
    }
    double ps = 0.5 * (lo + hi);
    *rho_g = root_p(q, ps, 0.0, rs1);
    *rho_l = root_p(q, ps, rs2, pole);
    if (p_sat) *p_sat = ps;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Flat-interface equilibrium profile (Sec. 5.1, Eq. 25-26).  For a profile  */
/* rho(y), Eq. 26 with the tensor of Eq. 25 keeps only                        */
/*   d/dy [ p(rho) - kappa rho rho'' + (kappa/2) rho'^2 ] = 0,                */
/* so the bracket equals its bulk value, the coexistence pressure p_s.        */
/* A first integral is (kappa/2) rho'^2 = W(rho) with                          */
/*   W(rho) = rho I(rho),  I(rho) = int_{rho_g}^{rho} (p(s) - p_s)/s^2 ds:     */
/* differentiating, kappa rho'' = W'(rho) = I + (p - p_s)/rho, and then       */
/* p - kappa rho rho'' + (kappa/2) rho'^2 = p - rho I - (p - p_s) + rho I =   */
/* p_s.  W has double roots at rho_g and, by the equal-area rule, at rho_l,   */
/* so the lower limit may be either bulk density; W is evaluated from the     */
/* nearer one (no cancellation in the tails) by Gauss-Legendre quadrature.    */
/* The profile rising from rho_g to rho_l is integrated in the logit          */
/*   u = ln((rho - rho_g)/(rho_l - rho)),                                      */
/*   du/dy = sqrt(2 W / kappa) (rho_l - rho_g) / ((rho - rho_g)(rho_l - rho)), */
/* which keeps rho strictly between the bulk densities and is linear in y in  */
/* the tails.  y = 0 at u = 0 (the mean density); classical Runge-Kutta (4th  */
/* order), `sub` steps per grid spacing h, outward in both directions.        */
/* ------------------------------------------------------------------------ */

#define GL_N 24
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

/* Gauss-Legendre nodes and weights on [-1, 1]: roots of P_n by Newton's      */
/* method from the guess cos(pi (i - 1/4)/(n + 1/2)), P_n and P_n' from the   */
/* three-term recurrence; w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2).                */
static void gl_init(void) {
    if (gl_ready) return;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < GL_N; ++i) {
        double x = cos(pi * (i + 0.75) / (GL_N + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= GL_N; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = GL_N * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

/* int_a^b (p(s) - ps)/s^2 ds, as int (p(e^t) - ps) e^-t dt over t = ln s,    */
/* by composite Gauss-Legendre (the integrand is smooth in t)                  */
static double area_gl(const orc_params *q, double ps, double a, double b, int panels) {
    double t0 = log(a), w = (log(b) - t0) / panels, acc = 0.0;
    for (int k = 0; k < panels; ++k) {
        double c = t0 + (k + 0.5) * w, hw = 0.5 * w;
        for (int i = 0; i < GL_N; ++i) {
            double s = exp(c + hw * gl_x[i]);
            acc += gl_w[i] * hw * (p_of(q, s) - ps) / s;
        }
    }
    return acc;
}

/* W(rho) = rho int_{rb}^{rho} (p(s) - p_s)/s^2 ds, rb the nearer bulk density */
static double profile_W(const orc_params *q, double ps, double rg, double rl, double rho) {
    double rb = (rho - rg < rl - rho) ? rg : rl;
    return rho * area_gl(q, ps, rb, rho, 4);
}

/* p(rho) = ps by Newton from rho (a stable branch, dp/drho > 0) */
static double newton_p(const orc_params *q, double ps, double rho) {
    for (int it = 0; it < 60; ++it) {
        double p, dp;
        eos_at(q, rho, &p, &dp);
        double d = (p - ps) / dp;
        rho -= d;
        if (fabs(d) <= 1e-17 * rho) break;
    }
    return rho;
}

typedef struct { const orc_params *q; double ps, rg, rl, kappa; } profile_ctx;

static void profile_at(const profile_ctx *c, double u, double *rho, double *drho, double *dudy) {
    double D = c->rl - c->rg;
    double g = D / (1.0 + exp(-u)), l = D / (1.0 + exp(u));  /* rho - rho_g, rho_l - rho */
    double r = g < l ? c->rg + g : c->rl - l;
    double W = profile_W(c->q, c->ps, c->rg, c->rl, r);
    double v = W > 0.0 ? sqrt(2.0 * W / c->kappa) : 0.0;
    *rho = r;
    *drho = v;
    *dudy = v * D / (g * l);
}

/* rho[i], drho[i] = rho'(y_i) at y_i = (i - i0) h, i = 0 .. n-1, for the     */
/* unscaled EOS of q at q->T (the Hu factor k plays no part).  Returns 0, or  */
/* 1 if the isotherm has no van der Waals loop or the arguments are invalid.  */
int orc_flat_profile(const orc_params *q, double kappa, double h, int n, int i0, int sub, double *rho, double *drho) {
    profile_ctx c;
    if (!(kappa > 0.0) || !(h > 0.0) || n < 1 || i0 < 0 || i0 >= n || sub < 1) return 1;
    if (orc_maxwell(q, &c.rg, &c.rl, &c.ps)) return 1;
    c.q = q;
    c.kappa = kappa;
    gl_init();
    /* The two branches of W meet only if the equal-area integral vanishes to  */
    /* rounding: refine p_s by Newton on A(p_s) = int_{rho_g}^{rho_l} (p -     */
    /* p_s)/s^2 ds (dA/dp_s = 1/rho_l - 1/rho_g, the limits contributing       */
    /* nothing), re-rooting the bulk densities each time.                      */
    for (int it = 0; it < 6; ++it) {
        double A = area_gl(q, c.ps, c.rg, c.rl, 32);
        double dps = A / (1.0 / c.rg - 1.0 / c.rl);
        c.ps += dps;
        c.rg = newton_p(q, c.ps, c.rg);
        c.rl = newton_p(q, c.ps, c.rl);
        if (fabs(dps) <= 1e-16 * c.ps) break;
    }
    for (int dir = -1; dir <= 1; dir += 2) {
        double u = 0.0, r, d, k1, k2, k3, k4, dy = dir * h / sub;
        for (int i = i0; i >= 0 && i < n; i += dir) {
            if (i != i0)
                for (int k = 0; k < sub; ++k) {
                    profile_at(&c, u, &r, &d, &k1);
                    profile_at(&c, u + 0.5 * dy * k1, &r, &d, &k2);
                    profile_at(&c, u + 0.5 * dy * k2, &r, &d, &k3);
                    profile_at(&c, u + dy * k3, &r, &d, &k4);
                    u += dy / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
                }
            profile_at(&c, u, &rho[i], &drho[i], &k1);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Equilibrium, Eq. 2.                                                        */
/* ------------------------------------------------------------------------ */

void orc_feq(double rho, double ux, double uy, double *feq) {
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = rho * W9[i] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* ------------------------------------------------------------------------ */
/* Derivative operators.                                                      */
/* ------------------------------------------------------------------------ */

/* Thomas ("chasing") solve of a tridiagonal system
 *   sub[i] x[i-1] + dia[i] x[i] + sup[i] x[i+1] = r[i]. */
static void thomas(int n, const double *sub, const double *dia, const double *sup,
                   const double *r, double *x, double *c) {
    double m = dia[0];
    c[0] = sup[0] / m;
    x[0] = r[0] / m;
    for (int i = 1; i < n; ++i) {
        m = dia[i] - sub[i] * c[i - 1];
        c[i] = sup[i] / m;
        x[i] = (r[i] - sub[i] * x[i - 1]) / m;
    }
    for (int i = n - 2; i >= 0; --i) x[i] -= c[i] * x[i + 1];
}

/* HDM first derivative of one periodic line u[0..n-1] (h = 1), Eq. 20:
 *   (1/3) d[i-1] + d[i] + (1/3) d[i+1]
 *        = (1/9)(u[i+2]-u[i-2])/4 + (14/9)(u[i+1]-u[i-1])/2,
 * indices taken modulo n.  The periodic system is cyclic tridiagonal; it is
 * solved by Thomas on the matrix with modified corners plus a Sherman-Morrison
 * rank-one correction.  n = 1, 2 are solved directly. */
void orc_hdm_line(const double *u, double *d, int n) {
    if (n <= 0) return;
    double *r = (double *)malloc(sizeof(double) * (size_t)n * 7);
    double *sub = r + n, *dia = sub + n, *sup = dia + n, *y = sup + n, *z = y + n, *c = z + n;
    for (int i = 0; i < n; ++i)
        r[i] = (1.0 / 9.0) * (u[wrap(i + 2, n)] - u[wrap(i - 2, n)]) / 4.0
             + (14.0 / 9.0) * (u[wrap(i + 1, n)] - u[wrap(i - 1, n)]) / 2.0;
    if (n == 1) {
        d[0] = r[0] / (1.0 + 2.0 / 3.0);
    } else if (n == 2) {
        /* both neighbours of a cell are the other cell: [[1,2/3],[2/3,1]] */
        double det = 1.0 - 4.0 / 9.0;
        d[0] = (r[0] - (2.0 / 3.0) * r[1]) / det;
        d[1] = (r[1] - (2.0 / 3.0) * r[0]) / det;
    } else {
        const double off = 1.0 / 3.0, alpha = 1.0 / 3.0, beta = 1.0 / 3.0;
        double gamma = -1.0;
        for (int i = 0; i < n; ++i) { sub[i] = off; dia[i] = 1.0; sup[i] = off; }
        dia[0] = 1.0 - gamma;
        dia[n - 1] = 1.0 - alpha * beta / gamma;
        thomas(n, sub, dia, sup, r, y, c);
        /* rank-one part u = (gamma, 0, ..., 0, alpha)^T; solve B z = u */
        for (int i = 0; i < n; ++i) r[i] = 0.0;
        r[0] = gamma;
        r[n - 1] = alpha;
        thomas(n, sub, dia, sup, r, z, c);
        double fact = (y[0] + beta * y[n - 1] / gamma) / (1.0 + z[0] + beta * z[n - 1] / gamma);
        for (int i = 0; i < n; ++i) d[i] = y[i] - fact * z[i];
    }
    free(r);
}

/* 2D HDM gradient: Eq. 20 along every row (d/dx) and every column (d/dy). */
void orc_hdm_grad(const double *q, double *gx, double *gy, int nx, int ny) {
#pragma omp parallel
    {
        int nmax = nx > ny ? nx : ny;
        double *lin = (double *)malloc(sizeof(double) * (size_t)nmax * 2);
        double *lout = lin + nmax;
#pragma omp for schedule(static)
        for (int y = 0; y < ny; ++y) orc_hdm_line(q + (size_t)y * nx, gx + (size_t)y * nx, nx);
#pragma omp for schedule(static)
        for (int x = 0; x < nx; ++x) {
            for (int y = 0; y < ny; ++y) lin[y] = q[(size_t)y * nx + x];
            orc_hdm_line(lin, lout, ny);
            for (int y = 0; y < ny; ++y) gy[(size_t)y * nx + x] = lout[y];
        }
        free(lin);
    }
}

/* 2D weighted CDM, Eq. 15, with the 1/c_s^2 factor so that a linear field has
 * unit slope: d/dx q = (1/c_s^2) sum_i w_i q(x + e_i) e_ix. */
void orc_cdm_grad(const double *q, double *gx, double *gy, int nx, int ny) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double sx = 0.0, sy = 0.0;
            for (int i = 1; i < 9; ++i) {
                double v = q[(size_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx)];
                sx += W9[i] * v * EX[i];
                sy += W9[i] * v * EY[i];
            }
            gx[(size_t)y * nx + x] = sx / CS2;
            gy[(size_t)y * nx + x] = sy / CS2;
        }
}

/* Walls (Sec. 5.5; the paper gives no closure of Eq. 20 or Eq. 15 there).    */
/* Reading: the field is continued across each wall by its mirror image,     */
/* q(-1-j) = q(j) and q(ny+j) = q(ny-1-j), i.e. zero normal gradient at the    */
/* wall (neutral wetting).  Eq. 20 along a column is then solved on the        */
/* mirrored column of period 2 ny, and Eq. 15 reads mirrored neighbours.       */
static int mirror(int i, int n) {
    int m = wrap(i, 2 * n);
    return m < n ? m : 2 * n - 1 - m;
}

static void hdm_grad_walls(const double *q, double *gx, double *gy, int nx, int ny) {
#pragma omp parallel
    {
        double *lin = (double *)malloc(sizeof(double) * (size_t)(nx > 2 * ny ? nx : 2 * ny) * 2);
        double *lout = lin + (nx > 2 * ny ? nx : 2 * ny);
#pragma omp for schedule(static)
        for (int y = 0; y < ny; ++y) orc_hdm_line(q + (size_t)y * nx, gx + (size_t)y * nx, nx);
#pragma omp for schedule(static)
        for (int x = 0; x < nx; ++x) {
            for (int y = 0; y < ny; ++y) lin[y] = lin[2 * ny - 1 - y] = q[(size_t)y * nx + x];
            orc_hdm_line(lin, lout, 2 * ny);
            for (int y = 0; y < ny; ++y) gy[(size_t)y * nx + x] = lout[y];
        }
        free(lin);
    }
}

static void cdm_grad_walls(const double *q, double *gx, double *gy, int nx, int ny) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double sx = 0.0, sy = 0.0;
            for (int i = 1; i < 9; ++i) {
                double v = q[(size_t)mirror(y + EY[i], ny) * nx + wrap(x + EX[i], nx)];
                sx += W9[i] * v * EX[i];
                sy += W9[i] * v * EY[i];
            }
            gx[(size_t)y * nx + x] = sx / CS2;
            gy[(size_t)y * nx + x] = sy / CS2;
        }
}

/* The gradient of a field as the step takes it: HDM or CDM, periodic or walled. */
void orc_grad(const orc_params *q, const double *fld, double *gx, double *gy) {
    if (q->walls) {
        if (q->grad == ORC_HDM) hdm_grad_walls(fld, gx, gy, q->nx, q->ny);
        else cdm_grad_walls(fld, gx, gy, q->nx, q->ny);
    } else {
        if (q->grad == ORC_HDM) orc_hdm_grad(fld, gx, gy, q->nx, q->ny);
        else orc_cdm_grad(fld, gx, gy, q->nx, q->ny);
    }
}

/* ------------------------------------------------------------------------ */
/* Interaction force from the density field.                                  */
/*   U = k p_EOS - rho c_s^2 (Eq. 8 with Hu's scaling, Sec. 5)                 */
/*   SC (Eq. 22): Phi = sqrt|U| (Eq. 21), F = -2 s Phi grad Phi, s = sign of U */
/*                at the cell (s = +1 for U >= 0)                             */
/*   ZC (Eq. 7):  F = -grad U                                                  */
/* With the effective mass psi = 1 - exp(-rho/rho0) (ORC_PSI):                */
/*   SC (Eq. 4):  F = -G psi grad psi                                          */
/*   ZC (Eq. 7):  F = -grad U, U = p - rho c_s^2 = (G/2) psi^2 (Eq. 5)         */
/* ------------------------------------------------------------------------ */

void orc_force(const orc_params *q, const double *rho, double *Fx, double *Fy) {
    size_t n = (size_t)q->nx * q->ny;
    double *U = (double *)malloc(sizeof(double) * n * 4);
    double *fld = U + n, *gx = fld + n, *gy = gx + n;
    const int psi_mode = q->eos == ORC_PSI;
    for (size_t c = 0; c < n; ++c) {
        if (psi_mode) {
            double psi = 1.0 - exp(-rho[c] / q->rho0);
            U[c] = 0.5 * q->G * psi * psi;
            fld[c] = (q->force == ORC_SC) ? psi : U[c];
        } else {
            double p;
            eos_at(q, rho[c], &p, NULL);
            U[c] = q->k * p - rho[c] * CS2;
            fld[c] = (q->force == ORC_SC) ? sqrt(fabs(U[c])) : U[c];
        }
    }
    orc_grad(q, fld, gx, gy);
    for (size_t c = 0; c < n; ++c) {
        if (q->force == ORC_SC && psi_mode) {
            Fx[c] = -q->G * fld[c] * gx[c];
            Fy[c] = -q->G * fld[c] * gy[c];
        } else if (q->force == ORC_SC) {
            double s = U[c] >= 0.0 ? 1.0 : -1.0;
            Fx[c] = -2.0 * s * fld[c] * gx[c];
            Fy[c] = -2.0 * s * fld[c] * gy[c];
        } else {
            Fx[c] = -gx[c];
            Fy[c] = -gy[c];
        }
    }
    free(U);
}

/* ------------------------------------------------------------------------ */
/* Lattice state: f[i * nx*ny + y*nx + x] (i = 0..8).                          */
/* ------------------------------------------------------------------------ */

/* Initial distributions f = f^eq(rho, u) (the paper is silent; standard). */
void orc_init(const orc_params *q, const double *rho, const double *ux, const double *uy, double *f) {
    size_t n = (size_t)q->nx * q->ny;
    double fe[9];
    for (size_t c = 0; c < n; ++c) {
        orc_feq(rho[c], ux ? ux[c] : 0.0, uy ? uy[c] : 0.0, fe);
        for (int i = 0; i < 9; ++i) f[i * n + c] = fe[i];
    }
}

/* Density and bare velocity, Eq. 3. */
static void moments_bare(const orc_params *q, const double *f, double *rho, double *ux, double *uy) {
    size_t n = (size_t)q->nx * q->ny;
#pragma omp parallel for schedule(static)
    for (long long cc = 0; cc < (long long)n; ++cc) {
        size_t c = (size_t)cc;
        double r = 0, jx = 0, jy = 0;
        for (int i = 0; i < 9; ++i) {
            double v = f[i * n + c];
            r += v;
            jx += EX[i] * v;
            jy += EY[i] * v;
        }
        rho[c] = r;
        ux[c] = jx / r;
        uy[c] = jy / r;
    }
}

typedef struct {
    double *rho, *ux, *uy, *Fx, *Fy;
} orc_work;

static int work_alloc(orc_work *w, size_t n) {
    w->rho = (double *)malloc(sizeof(double) * n * 5);
    if (!w->rho) return 1;
    w->ux = w->rho + n; w->uy = w->ux + n; w->Fx = w->uy + n; w->Fy = w->Fx + n;
    return 0;
}

/* One time step, Eq. 1 with Eq. 10 forcing:
 *   f_i*(x) = f_i - (f_i - f^eq(rho,u))/tau + [f^eq(rho,u+du) - f^eq(rho,u)],
 *   du = F/rho (dt = 1),  then  f_i(x + e_i, t+1) = f_i*(x).
 * With walls a population whose target row lies beyond a wall comes back to
 * the node it left, reversed: f_opp(i)(x, t+1) = f_i*(x) (half-way bounce-back,
 * the no-slip condition of Sec. 5.5; the paper does not say which form). */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static void step_with(const orc_params *q, const double *f, double *fout, orc_work *w) {
    int nx = q->nx, ny = q->ny;
    size_t n = (size_t)nx * ny;
    moments_bare(q, f, w->rho, w->ux, w->uy);
    orc_force(q, w->rho, w->Fx, w->Fy);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            double r = w->rho[c], ux = w->ux[c], uy = w->uy[c];
            double dux = w->Fx[c] / r, duy = w->Fy[c] / r;
            double fe[9], fs[9];
            orc_feq(r, ux, uy, fe);
            orc_feq(r, ux + dux, uy + duy, fs);
            for (int i = 0; i < 9; ++i) {
                double fi = f[i * n + c];
                double post = fi - (fi - fe[i]) / q->tau + (fs[i] - fe[i]);
                int yd = y + EY[i];
                if (q->walls && (yd < 0 || yd >= ny)) {
                    fout[OPP[i] * n + c] = post;
                } else {
                    size_t d = (size_t)wrap(yd, ny) * nx + wrap(x + EX[i], nx);
                    fout[i * n + d] = post;
                }
            }
        }
}

/* One step from f into fout (allocates its own work space). Returns 0 on success. */
int orc_step(const orc_params *q, const double *f, double *fout) {
    orc_work w;
    if (work_alloc(&w, (size_t)q->nx * q->ny)) return 1;
    step_with(q, f, fout, &w);
    free(w.rho);
    return 0;
}

/* nsteps steps in place on f. Returns 0 on success. */
int orc_run(const orc_params *q, double *f, int nsteps) {
    size_t n = (size_t)q->nx * q->ny;
    orc_work w;
    double *g = (double *)malloc(sizeof(double) * n * 9);
    if (!g || work_alloc(&w, n)) { free(g); return 1; }
    double *src = f, *dst = g;
    for (int s = 0; s < nsteps; ++s) {
        step_with(q, src, dst, &w);
        double *t = src; src = dst; dst = t;
    }
    if (src != f) memcpy(f, src, sizeof(double) * n * 9);
    free(g);
    free(w.rho);
    return 0;
}

/* Observable moments: rho (Eq. 3) and the half-step velocity v of Eq. 11,
 * rho v = sum_i e_i f_i + F/2. */
int orc_moments(const orc_params *q, const double *f, double *rho, double *vx, double *vy) {
    size_t n = (size_t)q->nx * q->ny;
    orc_work w;
    if (work_alloc(&w, n)) return 1;
    moments_bare(q, f, w.rho, w.ux, w.uy);
    orc_force(q, w.rho, w.Fx, w.Fy);
    for (size_t c = 0; c < n; ++c) {
        double r = w.rho[c];
        rho[c] = r;
        if (vx) vx[c] = w.ux[c] + 0.5 * w.Fx[c] / r;
        if (vy) vy[c] = w.uy[c] + 0.5 * w.Fy[c] / r;
    }
    free(w.rho);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Complex-step derivative of the discrete map (Squire & Trapp, SIAM Rev. 40, */
/* 1998; Martins, Sturdza & Alonso, ACM TOMS 29, 2003).                       */
/*                                                                            */
/* The step above, evaluated in complex arithmetic.  Give the temperature,    */
/* G and the initial density imaginary parts i h dT, i h dG, i h drho0 for a  */
/* tiny real h: after n steps the imaginary part of rho is h times the        */
/* directional derivative of rho_n along (drho0, dT, dG), free of the         */
/* cancellation of a difference quotient, and the real part is the real run   */
/* up to O(h^2).  Every operation of the step is analytic where U != 0; the   */
/* magnitude |U| of Eq. 21 continues as s U with s = sign(Re U), the branch   */
/* the real step takes.  The derivative operators (Eq. 15, Eq. 20) are real   */
/* and linear, so they act on the real and imaginary parts separately with    */
/* the real solvers above.  Serial except inside those solvers.              */
/* ------------------------------------------------------------------------ */

typedef double complex cplx;

static cplx mk_c(double re, double im) {
    cplx z;
    __real__ z = re;
    __imag__ z = im;
    return z;
}

/* alpha(T) of Eq. 27, Eq. 28 and the RKS form, at a complex temperature. */
static cplx alpha_c(int eos, double omega, cplx T, double Tc) {
    double m;
    cplx s;
    switch (eos) {
    case ORC_PR:
        m = 0.37464 + 1.54226 * omega - 0.26992 * omega * omega;
        s = 1.0 + m * (1.0 - csqrt(T / Tc));
        return s * s;
    case ORC_RKS:
        m = 0.480 + 1.574 * omega - 0.176 * omega * omega;
        s = 1.0 + m * (1.0 - csqrt(T / Tc));
        return s * s;
    case ORC_RK:
        return 1.0 / csqrt(T);
    default:
        return 1.0;
    }
}

/* p_EOS(rho) at temperature T (Eq. 24, 27, 28, 29; no Hu factor). */
static cplx p_eos_c(const orc_params *q, cplx T, cplx rho) {
    const double a = q->a, b = q->b, R = q->R;
    if (q->eos == ORC_CS) {
        cplx e = b * rho / 4.0;
        cplx num = 1.0 + e + e * e - e * e * e;
        cplx om = 1.0 - e;
        cplx Z = num / (om * om * om);
        return rho * R * T * Z - a * rho * rho;
    }
    cplx rep = rho * R * T / (1.0 - b * rho);
    if (q->eos == ORC_VDW) return rep - a * rho * rho;
    cplx al = alpha_c(q->eos, q->omega, T, q->Tc);
    if (q->eos == ORC_PR) return rep - a * al * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
    return rep - a * al * rho * rho / (1.0 + b * rho); /* RK, RKS */
}

/* Equilibrium of Eq. 2. */
static void feq_c(cplx rho, cplx ux, cplx uy, cplx *feq) {
    cplx uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        cplx eu = EX[i] * ux + EY[i] * uy;
        feq[i] = rho * W9[i] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

typedef struct {
    cplx *rho, *ux, *uy, *Fx, *Fy, *U, *fld, *gx, *gy;
    double *re, *im, *gxr, *gyr, *gxi, *gyi;
} cs_work;

/* The gradient of the step (orc_grad) applied to the real and the imaginary
 * part of a complex field. */
static void grad_c(const orc_params *q, cs_work *w, size_t n) {
    for (size_t c = 0; c < n; ++c) {
        w->re[c] = creal(w->fld[c]);
        w->im[c] = cimag(w->fld[c]);
    }
    orc_grad(q, w->re, w->gxr, w->gyr);
    orc_grad(q, w->im, w->gxi, w->gyi);
    for (size_t c = 0; c < n; ++c) {
        w->gx[c] = mk_c(w->gxr[c], w->gxi[c]);
        w->gy[c] = mk_c(w->gyr[c], w->gyi[c]);
    }
}

/* Interaction force of orc_force (Eq. 7, 22; Eq. 4-5 in psi mode). */
static void force_c(const orc_params *q, cplx T, cplx G, cs_work *w, size_t n) {
    const int psi_mode = q->eos == ORC_PSI;
    for (size_t c = 0; c < n; ++c) {
        cplx r = w->rho[c];
        if (psi_mode) {
            cplx psi = 1.0 - cexp(-r / q->rho0);
            w->U[c] = 0.5 * G * psi * psi;
            w->fld[c] = (q->force == ORC_SC) ? psi : w->U[c];
        } else {
            w->U[c] = q->k * p_eos_c(q, T, r) - r * CS2;
            double s = creal(w->U[c]) >= 0.0 ? 1.0 : -1.0;
            w->fld[c] = (q->force == ORC_SC) ? csqrt(s * w->U[c]) : w->U[c];
        }
    }
    grad_c(q, w, n);
    for (size_t c = 0; c < n; ++c) {
        if (q->force == ORC_SC && psi_mode) {
            w->Fx[c] = -G * w->fld[c] * w->gx[c];
            w->Fy[c] = -G * w->fld[c] * w->gy[c];
        } else if (q->force == ORC_SC) {
            double s = creal(w->U[c]) >= 0.0 ? 1.0 : -1.0;
            w->Fx[c] = -2.0 * s * w->fld[c] * w->gx[c];
            w->Fy[c] = -2.0 * s * w->fld[c] * w->gy[c];
        } else {
            w->Fx[c] = -w->gx[c];
            w->Fy[c] = -w->gy[c];
        }
    }
}

/* One step of step_with (Eq. 3, force, Eq. 10 forcing, Eq. 1 BGK and
 * streaming, walls by half-way bounce-back) in complex arithmetic. */
static void step_c(const orc_params *q, cplx T, cplx G, const cplx *f, cplx *fout, cs_work *w) {
    int nx = q->nx, ny = q->ny;
    size_t n = (size_t)nx * ny;
    for (size_t c = 0; c < n; ++c) {
        cplx r = 0, jx = 0, jy = 0;
        for (int i = 0; i < 9; ++i) {
            cplx v = f[i * n + c];
            r += v;
            jx += EX[i] * v;
            jy += EY[i] * v;
        }
        w->rho[c] = r;
        w->ux[c] = jx / r;
        w->uy[c] = jy / r;
    }
    force_c(q, T, G, w, n);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t c = (size_t)y * nx + x;
            cplx r = w->rho[c], ux = w->ux[c], uy = w->uy[c];
            cplx dux = w->Fx[c] / r, duy = w->Fy[c] / r;
            cplx fe[9], fs[9];
            feq_c(r, ux, uy, fe);
            feq_c(r, ux + dux, uy + duy, fs);
            for (int i = 0; i < 9; ++i) {
                cplx fi = f[i * n + c];
                cplx post = fi - (fi - fe[i]) / q->tau + (fs[i] - fe[i]);
                int yd = y + EY[i];
                if (q->walls && (yd < 0 || yd >= ny)) {
                    fout[OPP[i] * n + c] = post;
                } else {
                    size_t d = (size_t)wrap(yd, ny) * nx + wrap(x + EX[i], nx);
                    fout[i * n + d] = post;
                }
            }
        }
}

/* nsteps steps from f = f^eq(rho0 + i h drho0, 0) with the temperature
 * q->T + i h dT and the interaction strength q->G + i h dG.  Writes the
 * density after the steps (real part) to rho and its derivative along the
 * direction (drho0, dT, dG), Im(rho) / h, to drho.  drho0 may be NULL (zero).
 * Returns 0 on success, 1 on allocation failure or h <= 0. */
int orc_cs_run(const orc_params *q, const double *rho0, const double *drho0, double dT, double dG,
               double h, int nsteps, double *rho, double *drho) {
    if (!(h > 0.0)) return 1;
    size_t n = (size_t)q->nx * q->ny;
    cplx *f = (cplx *)malloc(sizeof(cplx) * n * 27);
    double *dw = (double *)malloc(sizeof(double) * n * 6);
    if (!f || !dw) { free(f); free(dw); return 1; }
    cplx *g = f + 9 * n, *cw = g + 9 * n;
    cs_work w = {cw, cw + n, cw + 2 * n, cw + 3 * n, cw + 4 * n, cw + 5 * n, cw + 6 * n, cw + 7 * n, cw + 8 * n,
                 dw, dw + n, dw + 2 * n, dw + 3 * n, dw + 4 * n, dw + 5 * n};
    const cplx T = mk_c(q->T, h * dT), G = mk_c(q->G, h * dG);
    for (size_t c = 0; c < n; ++c) {
        cplx fe[9];
        feq_c(mk_c(rho0[c], drho0 ? h * drho0[c] : 0.0), 0.0, 0.0, fe);
        for (int i = 0; i < 9; ++i) f[i * n + c] = fe[i];
    }
    cplx *src = f, *dst = g;
    for (int s = 0; s < nsteps; ++s) {
        step_c(q, T, G, src, dst, &w);
        cplx *t = src; src = dst; dst = t;
    }
    for (size_t c = 0; c < n; ++c) {
        cplx r = 0;
        for (int i = 0; i < 9; ++i) r += src[i * n + c];
        rho[c] = creal(r);
        drho[c] = cimag(r) / h;
    }
    free(f);
    free(dw);
    return 0;
}
