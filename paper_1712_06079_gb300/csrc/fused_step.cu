// Single-pass FP32 D2Q9 HDM pseudopotential step for sm_103a.
//
// One launch per time step reads f(t) and the potential field q(t) and
// writes f(t+1) and q(t+1) = potential of f(t+1), so a step moves 9 floats
// in + 9 floats out + 1 float in + 1 float out per cell (80 B) instead of
// the 116 B of the two-pass form.  The field is the signed root s Phi,
// Phi = sqrt|U| (Eq. 21), s the sign of U, for the Shan-Chen form (the
// stencils read |q| = Phi, the cell's force takes s Phi as stored) and U
// (Eq. 8) for the Zhang-Chen form.
//
// No-slip walls in y (the splash case of Sec. 5.5): the staged potential rows
// beyond a wall are the mirror images of the rows inside (zero normal
// gradient, the periodic operator of the mirrored column), the segments' halo
// rows beyond a wall send nothing, and a wall row returns the populations
// that would cross the wall to its own cells in the opposite direction
// (half-way bounce-back), the same reading as the two-pass kernels.
//
// Decomposition.  A CTA of 8 warps owns a strip of TXI = 120 columns and a
// segment of up to seg_h rows (a launch parameter: by default the tallest of
// 126, 62, 30, 14, 6 that gives every SM a CTA; the library's tuner times the
// heights on the live state).  It sweeps the segment in slabs of 8 rows, one
// warp per row and one lane per 4 consecutive cells.  Lanes 1..30 hold the
// strip's columns; lanes 0 and 31 hold the 4-column groups just outside it,
// whose collision is recomputed so that the density at t+1 of every strip
// cell can be formed on chip.  Launches use programmatic serialization: a
// grid waits for the previous step at its top (griddepcontrol.wait), before
// any read or write, so the next step's CTAs are scheduled while it drains.
// Successive steps take the strips and segments in opposite orders, so the
// first CTAs of a step read the rows the last CTAs of the previous step wrote
// while those are still in L2.
//
// f(t) of a lane's 4 cells is read with nine float4 loads into registers,
// issued during the previous slab (for tau = 1 right after its moments, which
// are the last use of f(t); otherwise after its collision) so that their
// latency hides behind the barrier and the density pass.  A slab takes the
// moments first, so f(t) is out of the registers before the derivatives
// stage their rows (the kernel runs at the 128-register limit of two CTAs
// per SM).  The potential rows arrive by the bulk-copy engine (cp.async.bulk,
// completion on mbarriers, bounded waits), issued a slab ahead by warp 0:
//  - the slab's 8 potential rows at full width (the 26-column HDM halo on
//    each side, for d/dx), double-buffered;
//  - a 48-row ring of potential rows at the lanes' 128 columns (the slab's
//    rows, the row above and the 26 rows below it, for the d/dy recurrences),
//    8 rows per chunk.
// The potential field is stored with 32 ghost columns on each side (periodic
// images), so every staged row is one contiguous 16-byte-aligned copy; rows
// wrap periodically.
//
// The derivative is the explicit periodic HDM operator (the exact solution of
// the tridiagonal system of Eq. 20, truncated at radius 26 where the
// neglected tail of the weights changes the derivative of a smooth field by
// < 3e-9).  Its weights are geometric past the first (w_j = w_2 r^(j-2)), so
// both directions run in recurrence form.  Along x each lane forms the two
// 25-term sums of its first and last cell from the staged row (five short
// Horner groups each) and steps them to its other cells.  Along y every ring
// column carries a forward sum down the segment and a 25-row backward sum per
// slab, and each row reads two values per cell; the sums of slab s+1 are
// formed at the end of slab s.  Per slab each lane forms the moments (Eq. 3),
// the force (Eq. 22 Shan-Chen or Eq. 7 Zhang-Chen) and the exact-difference
// forcing with BGK (Eq. 1, 2, 10).  It then streams (Eq. 1)
// by push: the x shift is a warp shuffle, the destination float4 of f(t+1) is
// stored straight to HBM, and the three partial sums of what lands in rows
// y-1, y, y+1 go to an 18-row shared ring.  After the slab's one barrier each
// warp sums the three partials of one finished row into rho(t+1) and writes
// the potential (Eq. 8, 21) of that row.  The rest population is formed as
// rho minus the other eight, so the FP32 collision conserves mass up to
// unbiased rounding.  For tau = 1 the BGK term vanishes exactly and the
// equilibrium at u is skipped.
//
// The CDMG variant takes the weighted central difference of Eq. 15 instead of
// the HDM operator: three ring rows and one shuffle each way give it, so it
// stages no full-width rows and runs no column recurrences.
//
// The TAPE variant (used by the reverse mode's taped and recomputed forward
// steps, never for walls or the CDM) also writes, for every cell of its own rows, the
// record of f(t) the adjoint step reads in place of f(t) and the stencil
// field: rho and j (Eq. 3) and the two HDM derivatives, five planes of nx ny.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "lbm_internal.h"
#include "ptx.cuh"

namespace lbm {
namespace {

constexpr int FK = 26;              // HDM radius of this path
constexpr int TXI = 120;            // interior columns per strip
constexpr int QG = 32;              // ghost columns on each side of a padded potential row
constexpr int WW = TXI + 2 * QG;    // floats per wide potential row (d/dx halo)
constexpr int NW = 128;             // floats per lane-column row (32 lanes x 4)
constexpr int SLAB = 8;             // rows per slab (one warp each)
constexpr int QCH = 6;              // chunks in the d/dy ring: slab s reads chunks s .. s+4, s+5 in flight
constexpr int QRING = QCH * SLAB;   // rows in the d/dy ring
constexpr int QBASE = 2;            // ring chunk 0 starts at row ys - QBASE
constexpr int QAHEAD = 4;           // slab s reads ring chunks s .. s + QAHEAD
constexpr int PROWS = 18;           // partial-density ring rows
constexpr int NTHR = 32 * SLAB;
constexpr uint64_t kWaitLimitNs = 200ull * 1000 * 1000;  // 0.2 s per wait

// shared-memory layout (bytes)
constexpr size_t kQnBytes = sizeof(float) * QRING * NW;       // d/dy ring
constexpr size_t kQwBytes = sizeof(float) * 2 * SLAB * WW;    // slab rows, full width, 2 buffers
constexpr size_t kPsBytes = sizeof(float) * 3 * PROWS * NW;   // partial densities
constexpr size_t kOffQw = kQnBytes;
constexpr size_t kAbBytes = sizeof(float) * 2 * 2 * SLAB * NW;  // P, Q of the slab rows, two slabs
constexpr size_t kOffPs = kOffQw + kQwBytes;
constexpr size_t kOffAb = kOffPs + kPsBytes;
constexpr size_t kFqBytes = sizeof(float) * NW;                 // far parts of the d/dy backward sums
constexpr size_t kOffFq = kOffAb + kAbBytes;
constexpr size_t kOffBar = kOffFq + kFqBytes;
constexpr size_t kSmemBytes = kOffBar + sizeof(uint64_t) * (QCH + 2);

struct FusedArgs {
    Model<float> m;
    const float *f;
    float *fout;
    const float *qin;   // padded field of f(t): row pitch qpitch, column x at x + QG
    float *qout;        // padded field of f(t+1)
    float *rec;         // TAPE: record of f(t), planes rho, jx, jy, Dx, Dy (nx ny each)
    int *err;
    int qpitch;         // nx + 2 * QG
    int seg_h;          // rows per CTA segment
    int n4;             // float4s per population plane (nx ny / 4)
    int rev;            // CTAs take the strips and segments in reverse order
    float w1x, w2x;     // d/dx weights w_1, w_2 (w_j = w_2 r^(j-2) for j >= 2)
    float w1y, w2y;     // d/dy weights
    float ry, ry5, ry12, ry25;  // r = (sqrt 5 - 3)/2 of Eq. 20's tridiagonal operator, and r^5, r^12, r^25
};

// f(t) is read once per step: a 16-byte load that takes no L1 line (L1 holds
// what the other loads in flight need; measured +1.5 % at 4096^2, +4 % at 2048^2)
__device__ __forceinline__ float4 ld_stream(const float4 *p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// Periodic wrap of an index at most one period outside [0, n) (every row and
// column index this file wraps lies in [-n, 2n))
__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Square root by the hardware's approximate instruction (sqrt.approx.f32, a
// PTX instruction; a few ulp against the correctly rounded root, against the
// several-instruction sequence of the IEEE sqrtf).
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Field staged for the stencil: the signed root s Phi = s sqrt|U|, s the sign
// of U (SC, Eq. 21), or U (ZC, Eq. 8).  The SC stencil reads |q| = Phi and the
// cell's own force takes s Phi as stored.
__device__ __forceinline__ float stencil_field(const Model<float> &m, float rho, bool sc) {
    float U = potential_u(m, rho);
    return sc ? copysignf(sqrt_approx(fabsf(U)), U) : U;
}

// U = k p_EOS - rho/3 (Eq. 8) with the equation of state fixed at compile time
// (VdW Eq. 24, CS Eq. 29, PR Eq. 28, RK/RKS Eq. 27), or (G/2) psi^2 for the
// effective mass of Eq. 4; quotients by the fast FP32 reciprocal (2 ulp), the
// denominators being positive and well scaled.
template <int EOS>
__device__ __forceinline__ float potential_u_t(const Model<float> &m, float rho) {
    if (EOS == LBM_EOS_PSI_EXP) {  // U = (G/2) psi^2, psi = 1 - exp(-rho/rho0) (Eq. 4-5)
        const float psi = 1.0f - expf(-rho * m.b);
        return m.a * psi * psi;
    }
    float p;
    if (EOS == LBM_EOS_CS) {
        const float e = m.b * rho * 0.25f;
        const float om = 1.0f - e;
        p = __fdividef(rho * m.RT * (1.0f + e * (1.0f + e * (1.0f - e))), om * om * om) - m.a * rho * rho;
    } else {
        const float rep = __fdividef(rho * m.RT, 1.0f - m.b * rho);
        if (EOS == LBM_EOS_VDW) p = rep - m.a * rho * rho;
        else if (EOS == LBM_EOS_PR) p = rep - __fdividef(m.aal * rho * rho, 1.0f + m.b * rho * (2.0f - m.b * rho));
        else p = rep - __fdividef(m.aal * rho * rho, 1.0f + m.b * rho);
    }
    return m.k * p - rho * (1.0f / 3.0f);
}

template <int EOS>
__device__ __forceinline__ float stencil_field_t(const Model<float> &m, float rho, bool sc) {
    const float U = potential_u_t<EOS>(m, rho);
    return sc ? copysignf(sqrt_approx(fabsf(U)), U) : U;
}

// The same potential for two cells as a packed pair: the equation of state
// in packed multiply/fma, the quotients by one fast reciprocal per cell
// (the effective mass of Eq. 4, with its exponential, cell by cell).
template <int EOS>
__device__ __forceinline__ float2 stencil_field_t2(const Model<float> &m, float2 rho, bool sc);

// f^eq_i(rho, u) of Eq. 2 for i = 1..8 with the lattice weights as FP32;
// a = 1 - 1.5 |u|^2.
__device__ __forceinline__ float feq_moving(int i, float rho, float ux, float uy, float a) {
    const float eu = float(ex(i)) * ux + float(ey(i)) * uy;
    const float w = i < 5 ? rho * (1.0f / 9.0f) : rho * (1.0f / 36.0f);
    return w * (a + eu * (3.0f + 4.5f * eu));
}

// Packed FP32 pairs (two cells per instruction; Blackwell's paired FP32
// add/multiply/fma, each component rounded as the scalar operation).
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, splat2(-1.0f), a); }   // a - b

// The bracket of f^eq_i (Eq. 2) for e_i . u = e v with e = +1 or -1 and
// a = 1 - 1.5 |u|^2:  a + (e v)(3 + 4.5 (e v)), formed as a + v (e 3 + 4.5 v),
// the same two roundings as with e v itself.
template <int E>
__device__ __forceinline__ float2 feq_bracket2(float2 v, float2 a) {
    return fma2(v, fma2(splat2(4.5f), v, splat2(3.0f * E)), a);
}

__device__ __forceinline__ float2 rcp2(float2 d) { return make_float2(__fdividef(1.0f, d.x), __fdividef(1.0f, d.y)); }

template <int EOS>
__device__ __forceinline__ float2 stencil_field_t2(const Model<float> &m, float2 rho, bool sc) {
    if (EOS == LBM_EOS_PSI_EXP)
        return make_float2(stencil_field_t<EOS>(m, rho.x, sc), stencil_field_t<EOS>(m, rho.y, sc));
    const float2 one = splat2(1.0f);
    float2 p;
    if (EOS == LBM_EOS_CS) {   // Eq. 29: rho R T (1 + e + e^2 - e^3) / (1 - e)^3 - a rho^2, e = b rho / 4
        const float2 e = mul2(mul2(splat2(m.b), rho), splat2(0.25f));
        const float2 om = sub2(one, e);
        const float2 num = mul2(mul2(rho, splat2(m.RT)), fma2(e, fma2(e, sub2(one, e), one), one));
        p = sub2(mul2(num, rcp2(mul2(mul2(om, om), om))), mul2(mul2(splat2(m.a), rho), rho));
    } else {
        const float2 rep = mul2(mul2(rho, splat2(m.RT)), rcp2(sub2(one, mul2(splat2(m.b), rho))));
        if (EOS == LBM_EOS_VDW) {          // Eq. 24
            p = sub2(rep, mul2(mul2(splat2(m.a), rho), rho));
        } else if (EOS == LBM_EOS_PR) {    // Eq. 28
            const float2 br = mul2(splat2(m.b), rho);
            const float2 den = fma2(br, sub2(splat2(2.0f), br), one);
            p = sub2(rep, mul2(mul2(mul2(splat2(m.aal), rho), rho), rcp2(den)));
        } else {                            // Eq. 27 (RK, RKS)
            const float2 den = fma2(splat2(m.b), rho, one);
            p = sub2(rep, mul2(mul2(mul2(splat2(m.aal), rho), rho), rcp2(den)));
        }
    }
    const float2 U = fma2(splat2(m.k), p, mul2(rho, splat2(-1.0f / 3.0f)));   // Eq. 8 with Hu's k
    if (!sc) return U;
    return make_float2(copysignf(sqrt_approx(fabsf(U.x)), U.x), copysignf(sqrt_approx(fabsf(U.y)), U.y));
}

// (LBM_CHECKED builds) the elements [off, off + len) lie in a buffer of n
__device__ __forceinline__ bool range_ok(long long off, long long len, long long n, int *err) {
    return in_bounds(off, n - len + 1, err);
}

template <bool SC, bool TAU1, int EOS, bool WALLS, bool TAPE = false, bool CDMG = false>
__global__ void __launch_bounds__(NTHR, 2) fused_step_kernel(const __grid_constant__ FusedArgs A) {
    static_assert(!(TAPE && WALLS), "the reverse mode takes periodic lattices");
    static_assert(!(TAPE && CDMG), "the reverse mode of CDM lattices takes the two-pass kernels");
    extern __shared__ __align__(128) unsigned char smem[];
    float *qn = reinterpret_cast<float *>(smem);               // [QRING][NW]
    float *qw = reinterpret_cast<float *>(smem + kOffQw);      // [2][SLAB][WW]
    float *ps = reinterpret_cast<float *>(smem + kOffPs);      // [3][PROWS][NW]
    float *ab = reinterpret_cast<float *>(smem + kOffAb);      // [2 slabs][2][SLAB][NW]: P_{y-1}, Q_{y+1}
    float *fq = reinterpret_cast<float *>(smem + kOffFq);      // [NW]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffBar);  // QCH chunk barriers + 2 row barriers
    uint64_t *row_bar = &bars[QCH];

    const Model<float> &m = A.m;
    const int nx = m.nx, ny = m.ny;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // reversed on alternate steps: the first CTAs of a step then read the rows
    // the last CTAs of the previous step wrote, while those are still in L2
    const int bx = A.rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    const int by = A.rev ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
    const int x0 = bx * TXI;
    const int nint = min(TXI, nx - x0);             // interior columns (multiple of 4)
    const int ys = by * A.seg_h;
    const int hseg = min(A.seg_h, ny - ys);
    const int nslab = hseg > 6 ? (hseg - 6 + SLAB - 1) / SLAB + 1 : 1;
    const int nchunks = nslab + QAHEAD;
    const int ncols = nint + 8;                     // lane columns actually staged (d/dy ring)
    const int wcols = nint + 2 * QG;                // wide-row columns actually staged
    const int glast = nint / 4 + 1;                 // right ring lane
    const bool active = lane <= glast;
    const bool interior = lane >= 1 && lane < glast;

    if (threadIdx.x == 0) {
        for (int i = 0; i < QCH + 2; ++i) ptx::mbar_init(&bars[i], 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    // Launched with programmatic serialization: the next step's grid may be
    // scheduled as soon as every CTA of this one runs, and this grid waits for
    // the previous step to complete before any read of f(t), q(t) or any write.
    ptx::griddep_launch_dependents();
    ptx::griddep_wait();

    // d/dy ring chunk c: relative rows 8c .. 8c+7 = global rows ys - QBASE + 8c + k,
    // lane columns x0 - 4 .. x0 + nint + 3 (padded x0 + QG - 4 ..), ring row (8c + k) % QRING
    auto issue_chunk = [&](int c) {  // warp 0
        uint64_t *bar = &bars[c % QCH];
        if (lane == 0) ptx::mbar_arrive_expect_tx(bar, SLAB * ncols * sizeof(float));
        __syncwarp();
        if (lane < SLAB) {
            int ry = SLAB * c + lane;
            int y = WALLS ? mirror_index(ys - QBASE + ry, ny) : wrapi(ys - QBASE + ry, ny);
            const long long src = (long long)y * A.qpitch + x0 + QG - 4;
            if (range_ok(src, ncols, (long long)A.qpitch * ny, A.err) &&
                range_ok((ry % QRING) * NW, ncols, QRING * NW, A.err))   // (else the wait times out)
                ptx::bulk_g2s(qn + (ry % QRING) * NW, A.qin + src, ncols * sizeof(float), bar);
        }
    };
    // slab s: potential rows ys - 1 + 8s + w at full width into buffer s & 1
    int rows_issued = 0;  // slab row sets issued so far (meaningful in warp 0)
    auto issue_rows = [&](int s) {  // warp 0
        uint64_t *bar = &row_bar[s & 1];
        rows_issued = s + 1;
        if (lane == 0) ptx::mbar_arrive_expect_tx(bar, SLAB * wcols * sizeof(float));
        __syncwarp();
        if (lane < SLAB) {
            int y = WALLS ? mirror_index(ys - 1 + SLAB * s + lane, ny) : wrapi(ys - 1 + SLAB * s + lane, ny);
            const long long src = (long long)y * A.qpitch + x0;
            if (range_ok(src, wcols, (long long)A.qpitch * ny, A.err) && range_ok(0, wcols, WW, A.err))
                ptx::bulk_g2s(qw + ((s & 1) * SLAB + lane) * WW, A.qin + src, wcols * sizeof(float), bar);
        }
    };
    int issued = 0;  // chunks issued so far (meaningful in warp 0)
    if (warp == 0) {
        for (; issued < min(QCH, nchunks); ++issued) issue_chunk(issued);
        if (!CDMG) issue_rows(0);
    }

    const int xg = x0 - 4 + 4 * lane;               // first of this lane's 4 columns
    const int xgw = wrapi(xg, nx);
    bool timed_out = false;
    bool unstable = false;                          // a non-positive or non-finite density

    // f(t) of row ys - 1 + 8s + warp at the lane's 4 columns
    float4 fv[9];
    auto load_f = [&](int s) {
        const float *src = A.f + (long long)wrapi(ys - 1 + SLAB * s + warp, ny) * nx + xgw;
        const float4 *p = reinterpret_cast<const float4 *>(src);
        const bool ok = range_ok(src - A.f, 4, (long long)4 * A.n4, A.err);   // the plane-0 float4 (all planes alike)
#pragma unroll
        for (int i = 0; i < 9; ++i, p += A.n4) fv[i] = ok ? ld_stream(p) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    // d/dy column recurrences: thread (warp, lane) follows ring column
    // cl = 32 (warp % 4) + lane (padded column x0 + QG - 4 + cl); warps 0..3 carry
    // the forward sum P down the segment, warps 4..7 form the backward sums.
    // P's start P_(ys-2), over rows ys - 27 .. ys - 3 above the ring, and the
    // column's reference value q(ys - 1) come from the padded field, with all
    // loads in flight while the first copies land.
    const bool fwdw = warp < SLAB / 2;
    const int cl = 32 * (warp & (SLAB / 2 - 1)) + lane;
    auto mag = [](float v) { return SC ? fabsf(v) : v; };   // the stencil's field value
    float colref = 0.f, pcarry = 0.f;
    if (!CDMG && cl < ncols) {
        const float *g = A.qin + x0 + QG - 4 + cl;
        const int yr = WALLS ? mirror_index(ys - 1, ny) : (ys - 1 < 0 ? ys - 1 + ny : ys - 1);
        colref = mag(__ldg(g + (long long)yr * A.qpitch));
        if (fwdw) {
            float v[25];
#pragma unroll
            for (int k = 0; k < 25; ++k) {
                const int y = ys - 27 + k;                  // ny >= 2 FK + 2 > 27: one wrap at most
                v[k] = __ldg(g + (long long)(WALLS ? mirror_index(y, ny) : (y < 0 ? y + ny : y)) * A.qpitch);
            }
#pragma unroll
            for (int k = 0; k < 25; ++k) pcarry = fmaf(A.ry, pcarry, mag(v[k]) - colref);
        }
    }

    // d/dy of the slab's rows in recurrence form.  The explicit periodic
    // HDM weights are w_j = w_2 r^(j-2) for j >= 2, so with t = q - q_ref along
    // a column, P_y = t_(y-1) + r P_(y-1) and Q_y = t_(y+1) + r Q_(y+1),
    //   D_y = w_1 (q_(y+1) - q_(y-1)) + w_2 (Q_(y+1) - P_(y-1)).
    // Q_(y+1) of the slab's last row sums the 25 rows below it (the same
    // truncation as the stencil): warp w + 4 takes the 12 nearest, warp w the
    // 13 farthest, which it hands over through shared memory and a two-warp
    // named barrier; then warp w steps P down the slab (carried across slabs)
    // and warp w + 4 steps Q up it.  Every ring row a step reads lies in ring
    // chunks s .. s + 4 at a compile-time offset from that chunk's slot.  Slab
    // s + 1's recurrences run at the end of slab s, so one barrier per slab
    // serves them and the partial densities (and orders the far parts' reuse).
    auto column_phase = [&](int s) {
        // row Y0 + d of the slab (Y0 its first row, -1 <= d <= 33) is row e % 8 of ring
        // chunk s + e / 8, e = d + QBASE - 1
        const float *cb[QAHEAD + 1];
        int slot = s % QCH;
#pragma unroll
        for (int j = 0; j <= QAHEAD; ++j) {
            cb[j] = qn + slot * SLAB * NW + cl;
            slot = slot == QCH - 1 ? 0 : slot + 1;
        }
        auto tq = [&](int d) { return mag(cb[(d + QBASE - 1) / SLAB][((d + QBASE - 1) % SLAB) * NW]) - colref; };
        float *buf = ab + (s & 1) * 2 * SLAB * NW + cl;
        const int bar_id = 1 + (warp & (SLAB / 2 - 1));
        if (fwdw) {
            float x = tq(33);   // the far part of Q_(Y0+8): rows Y0+33 .. Y0+21
#pragma unroll
            for (int d = 32; d >= 21; --d) x = fmaf(A.ry, x, tq(d));
            fq[cl] = x;
            __syncwarp();   // the aligned barrier instructions want the whole warp converged
            asm volatile("bar.arrive %0, %1;" ::"r"(bar_id), "r"(64) : "memory");
            float v = pcarry;   // P_(Y0-1)
#pragma unroll
            for (int k = 0; k < SLAB; ++k) {
                buf[k * NW] = v;                       // P_(Y0+k-1)
                v = fmaf(A.ry, v, tq(k - 1));          // row Y0-1+k
            }
            pcarry = v;   // P_(Y0+7) = P of the next slab's first row minus one
        } else {
            float x = tq(20);   // the near part: rows Y0+20 .. Y0+9
#pragma unroll
            for (int d = 19; d >= 9; --d) x = fmaf(A.ry, x, tq(d));
            __syncwarp();
            asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(64) : "memory");
            float v = fmaf(A.ry12, fq[cl], x);         // Q_(Y0+8)
#pragma unroll
            for (int k = 0; k < SLAB; ++k) {
                buf[(2 * SLAB - 1 - k) * NW] = v;      // Q_(Y0+8-k)
                v = fmaf(A.ry, v, tq(SLAB - k));       // row Y0+8-k
            }
        }
    };

    load_f(0);

    // slab 0's recurrences before the sweep (ring chunks 0 .. QAHEAD)
    for (int c = 0; c <= min(QAHEAD, nchunks - 1); ++c)
        if (!ptx::mbar_wait_bounded(&bars[c % QCH], (c / QCH) & 1, kWaitLimitNs)) timed_out = true;
    if (!CDMG) column_phase(0);
    bool stop = __syncthreads_or(timed_out);   // CTA-uniform

    for (int s = 0; s < nslab && !stop; ++s) {
        // copies a slab ahead: the next slab's full-width rows and the ring chunk
        // it needs last (their buffers were last read by the previous slab)
        if (warp == 0 && s >= 1) {
            ptx::fence_proxy_async_smem();
            if (s + QCH - 1 < nchunks) {
                issue_chunk(s + QCH - 1);
                issued = s + QCH;
            }
            if (!CDMG && s + 1 < nslab) issue_rows(s + 1);
        } else if (!CDMG && warp == 0 && s + 1 < nslab) {
            issue_rows(1);
        }
        const int yc = ys - 1 + SLAB * s + warp;    // collided row of this warp
        const int ryc = SLAB * s + warp + QBASE - 1;
        if (!CDMG && !ptx::mbar_wait_bounded(&row_bar[s & 1], (s >> 1) & 1, kWaitLimitNs)) timed_out = true;
        // A timed-out wait leaves stale shared rows: the slab then computes and
        // stores values of no use (in bounds), the barrier below ends the sweep
        // and the error word reports the timeout.
        // Every lane of a warp runs the collision (the shuffles need the whole
        // warp); lanes past the strip's right ring lane work on unused shared
        // columns and store nothing.
        {
            float dx[4], dy[4], qc[4];
            // moments of f(t) (Eq. 3), cells (0, 1) and (2, 3) as packed pairs, from
            // the sums over the populations moving east (1, 5, 8), west (3, 6, 7),
            // north (2, 5, 6) and south (4, 7, 8): 14 additions instead of 21
            float2 r2[2], jx2[2], jy2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                auto v = [&](int i) { return h ? make_float2(fv[i].z, fv[i].w) : make_float2(fv[i].x, fv[i].y); };
                const float2 east = add2(add2(v(1), v(5)), v(8)), west = add2(add2(v(3), v(6)), v(7));
                const float2 north = add2(add2(v(2), v(5)), v(6)), south = add2(add2(v(4), v(7)), v(8));
                r2[h] = add2(add2(add2(v(0), v(2)), v(4)), add2(east, west));
                jx2[h] = sub2(east, west);
                jy2[h] = sub2(north, south);
            }
            // for tau = 1 nothing after the moments reads f(t), so f(t) of the next
            // slab goes in flight here, across the derivatives and the collision
            if (TAU1 && s + 1 < nslab) load_f(s + 1);
            if constexpr (CDMG) {   // Eq. 15 from ring rows yc - 1, yc, yc + 1; columns +-1 by shuffles
                const float4 vm = *reinterpret_cast<const float4 *>(qn + ((ryc - 1) % QRING) * NW + 4 * lane);
                const float4 v0 = *reinterpret_cast<const float4 *>(qn + (ryc % QRING) * NW + 4 * lane);
                const float4 vp = *reinterpret_cast<const float4 *>(qn + ((ryc + 1) % QRING) * NW + 4 * lane);
                float rm[6], r0[6], rp[6];   // the field at lane columns 4 lane - 1 .. 4 lane + 4
                auto fill = [&](float (&r)[6], const float4 &v) {
                    r[0] = mag(__shfl_up_sync(0xffffffffu, v.w, 1));
                    r[1] = mag(v.x);
                    r[2] = mag(v.y);
                    r[3] = mag(v.z);
                    r[4] = mag(v.w);
                    r[5] = mag(__shfl_down_sync(0xffffffffu, v.x, 1));
                };
                fill(rm, vm);
                fill(r0, v0);
                fill(rp, vp);
                qc[0] = v0.x;
                qc[1] = v0.y;
                qc[2] = v0.z;
                qc[3] = v0.w;
#pragma unroll
                for (int c = 0; c < 4; ++c) {   // (1/cs^2) sum_i w_i q(x + e_i) e_i
                    dx[c] = fmaf(1.0f / 3.0f, r0[c + 2] - r0[c], (1.0f / 12.0f) * ((rp[c + 2] + rm[c + 2]) - (rp[c] + rm[c])));
                    dy[c] = fmaf(1.0f / 3.0f, rp[c + 1] - rm[c + 1], (1.0f / 12.0f) * ((rp[c + 2] + rp[c]) - (rm[c + 2] + rm[c])));
                }
            } else {
                {   // d/dx: wide row columns 4 lane .. 4 lane + 59; cells at window positions 28..31.
                    // The radius-26 operator in recurrence form on packed pairs
                    // (hdm_window4_paired); each staged value enters as its deviation
                    // from the lane's second cell.
                    const float *qrow = qw + ((s & 1) * SLAB + warp) * WW + 4 * lane;
                    float t[60];
    #pragma unroll
                    for (int k = 0; k < 15; ++k) {
                        const float4 v4 = *reinterpret_cast<const float4 *>(qrow + 4 * k);
                        t[4 * k] = v4.x; t[4 * k + 1] = v4.y; t[4 * k + 2] = v4.z; t[4 * k + 3] = v4.w;
                    }
    #pragma unroll
                    for (int c = 0; c < 4; ++c) qc[c] = t[28 + c];
                    const float qref = mag(t[29]);
                    float2 tp[28];   // deviations paired about the window's centre
    #pragma unroll
                    for (int j = 0; j < 28; ++j) tp[j] = make_float2(mag(t[2 + j]) - qref, mag(t[57 - j]) - qref);
                    hdm_window4_paired(tp, A.w1x, A.w2x, A.ry, A.ry5, A.ry25, dx);
                }
                {   // d/dy from the column recurrences of this row
                    const float4 qa = *reinterpret_cast<const float4 *>(qn + ((ryc + 1) % QRING) * NW + 4 * lane);
                    const float4 qb = *reinterpret_cast<const float4 *>(qn + ((ryc - 1) % QRING) * NW + 4 * lane);
                    const float *abs_ = ab + (s & 1) * 2 * SLAB * NW;
                    const float4 P = *reinterpret_cast<const float4 *>(abs_ + warp * NW + 4 * lane);
                    const float4 Q = *reinterpret_cast<const float4 *>(abs_ + (SLAB + warp) * NW + 4 * lane);
                    dy[0] = fmaf(A.w1y, mag(qa.x) - mag(qb.x), A.w2y * (Q.x - P.x));
                    dy[1] = fmaf(A.w1y, mag(qa.y) - mag(qb.y), A.w2y * (Q.y - P.y));
                    dy[2] = fmaf(A.w1y, mag(qa.z) - mag(qb.z), A.w2y * (Q.z - P.z));
                    dy[3] = fmaf(A.w1y, mag(qa.w) - mag(qb.w), A.w2y * (Q.w - P.w));
                }
            }
            if constexpr (TAPE) {   // the record of f(t) at the lane's 4 cells of an own row
                if (interior && yc >= ys && yc < ys + hseg) {
                    float4 *rp = reinterpret_cast<float4 *>(A.rec + (long long)yc * nx + xg);
                    if (range_ok(rp - reinterpret_cast<float4 *>(A.rec), 4LL * A.n4 + 1, 5LL * A.n4, A.err)) {
                        rp[0] = make_float4(r2[0].x, r2[0].y, r2[1].x, r2[1].y);
                        rp[A.n4] = make_float4(jx2[0].x, jx2[0].y, jx2[1].x, jx2[1].y);
                        rp[2 * A.n4] = make_float4(jy2[0].x, jy2[0].y, jy2[1].x, jy2[1].y);
                        rp[3 * A.n4] = make_float4(dx[0], dx[1], dx[2], dx[3]);
                        rp[4 * A.n4] = make_float4(dy[0], dy[1], dy[2], dy[3]);
                    }
                }
            }
            // force and the two velocities of the forcing (Eq. 10, 22 / 7)
            float2 ux[2], uy[2], vx[2], vy[2], au[2], av[2], moved[2];
            {   // the 4 densities positive and finite: the least above 0, the sum finite (a NaN or
                // an infinity makes it not; a sum past the FP32 range flags a blown-up state too)
                const float2 rs = add2(r2[0], r2[1]);
                const float rmin = fminf(fminf(r2[0].x, r2[0].y), fminf(r2[1].x, r2[1].y));
                unstable |= active && !(rmin > 0.f && rs.x + rs.y < INFINITY);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 gx = make_float2(dx[2 * h], dx[2 * h + 1]), gy = make_float2(dy[2 * h], dy[2 * h + 1]);
                float2 Fx, Fy;
                if (SC) {   // Eq. 22: F = -2 s Phi grad Phi, s Phi the stored field at the cell
                    const float2 m2q = mul2(splat2(-2.0f), make_float2(qc[2 * h], qc[2 * h + 1]));
                    Fx = mul2(m2q, gx);
                    Fy = mul2(m2q, gy);
                } else {    // Eq. 7: F = -grad U
                    Fx = mul2(splat2(-1.0f), gx);
                    Fy = mul2(splat2(-1.0f), gy);
                }
                const float2 inv = make_float2(__fdividef(1.0f, r2[h].x), __fdividef(1.0f, r2[h].y));
                ux[h] = mul2(jx2[h], inv);
                uy[h] = mul2(jy2[h], inv);
                vx[h] = fma2(Fx, inv, ux[h]);
                vy[h] = fma2(Fy, inv, uy[h]);
                au[h] = fma2(splat2(-1.5f), fma2(uy[h], uy[h], mul2(ux[h], ux[h])), splat2(1.0f));
                av[h] = fma2(splat2(-1.5f), fma2(vy[h], vy[h], mul2(vx[h], vx[h])), splat2(1.0f));
                moved[h] = splat2(0.f);
            }

            // post-collision populations, pushed: x shift by shuffle, store to
            // row yc + e_y if it lies in the segment, accumulate partial densities
            const int rd0 = yc - ys + 3;            // relative destination row of e_y = 0
            bool rowok[3];                          // destination row yc + k - 1 lies in the segment
#pragma unroll
            for (int k = 0; k < 3; ++k) rowok[k] = interior && yc + k - 1 >= ys && yc + k - 1 < ys + hseg;
            // with walls a collided row beyond one (the segment's halo row -1 or ny)
            // sends nothing, and a wall row returns what would cross the wall to
            // its own cells, reversed (half-way bounce-back; warp-uniform)
            const bool ghost = WALLS && (yc < 0 || yc >= ny);
            const bool wall_lo = WALLS && yc == 0, wall_hi = WALLS && yc == ny - 1;
            float4 *const dst0 = reinterpret_cast<float4 *>(A.fout + (long long)yc * nx + xg);   // plane 0, row yc
            auto store4 = [&](float4 *p, const float4 &v) {   // a streaming store of f(t+1)
                if (range_ok(p - reinterpret_cast<float4 *>(A.fout), 1, 9LL * A.n4, A.err)) __stcs(p, v);
            };
            float4 *dst = dst0;
            float4 part[3] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f),
                              make_float4(0.f, 0.f, 0.f, 0.f)};
#pragma unroll
            for (int ii = 0; ii < 9; ++ii) {
                const int i = ii == 8 ? 0 : ii + 1;     // rest population last
                float2 p2[2];
                if (i == 0) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) p2[h] = sub2(r2[h], moved[h]);
                } else if (TAU1) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        // f^eq_i(rho, v) = w_i rho (a + (e_i.v)(3 + 4.5 e_i.v)), a = 1 - 1.5 |v|^2
                        const float2 w = mul2(r2[h], splat2(i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f));
                        // e_i . v: v_x, v_y, or for the diagonals v_x + v_y (i = 5, 7), v_x - v_y (8, 6)
                        const float2 ev = i == 1 || i == 3 ? vx[h]
                                                           : (i == 2 || i == 4 ? vy[h]
                                                                               : (i == 5 || i == 7 ? add2(vx[h], vy[h])
                                                                                                   : sub2(vx[h], vy[h])));
                        const bool pos = i == 1 || i == 2 || i == 5 || i == 8;
                        p2[h] = mul2(w, pos ? feq_bracket2<1>(ev, av[h]) : feq_bracket2<-1>(ev, av[h]));
                        moved[h] = add2(moved[h], p2[h]);
                    }
                } else {   // BGK towards f^eq(u) plus the forcing difference, one cell at a time
                    const float fi[4] = {fv[i].x, fv[i].y, fv[i].z, fv[i].w};
                    float pc[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int h = c >> 1;
                        const float rc = c & 1 ? r2[h].y : r2[h].x;
                        const float eqv = feq_moving(i, rc, c & 1 ? vx[h].y : vx[h].x, c & 1 ? vy[h].y : vy[h].x,
                                                     c & 1 ? av[h].y : av[h].x);
                        const float equ = feq_moving(i, rc, c & 1 ? ux[h].y : ux[h].x, c & 1 ? uy[h].y : uy[h].x,
                                                     c & 1 ? au[h].y : au[h].x);
                        pc[c] = fmaf(1.0f - m.omega, fi[c] - equ, eqv);
                    }
                    p2[0] = make_float2(pc[0], pc[1]);
                    p2[1] = make_float2(pc[2], pc[3]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) moved[h] = add2(moved[h], p2[h]);
                }
                const float post[4] = {p2[0].x, p2[0].y, p2[1].x, p2[1].y};
                float4 d;  // values landing on this lane's 4 columns
                if (ex(i) == 1) {
                    float left = __shfl_up_sync(0xffffffffu, post[3], 1);
                    d = make_float4(left, post[0], post[1], post[2]);
                } else if (ex(i) == -1) {
                    float right = __shfl_down_sync(0xffffffffu, post[0], 1);
                    d = make_float4(post[1], post[2], post[3], right);
                } else {
                    d = make_float4(post[0], post[1], post[2], post[3]);
                }
                if (i != 0) dst += A.n4;                // plane i, stepped from plane i - 1
                auto accumulate = [](float4 &pp, const float4 &v) {
                    const float2 lo = add2(make_float2(pp.x, pp.y), make_float2(v.x, v.y));
                    const float2 hi = add2(make_float2(pp.z, pp.w), make_float2(v.z, v.w));
                    pp = make_float4(lo.x, lo.y, hi.x, hi.y);
                };
                if (!WALLS) {
                    if (rowok[ey(i) + 1]) store4((i == 0 ? dst0 : dst) + ey(i) * (nx >> 2), d);
                    accumulate(part[ey(i) + 1], d);
                } else if (!ghost) {
                    const bool bounce = (ey(i) == -1 && wall_lo) || (ey(i) == 1 && wall_hi);
                    if (bounce) {   // to the same cells, in the opposite direction, unshifted
                        const float4 b = make_float4(post[0], post[1], post[2], post[3]);
                        if (rowok[1]) store4(dst0 + opp(i) * A.n4, b);
                        accumulate(part[1], b);
                    } else {
                        if (rowok[ey(i) + 1]) store4((i == 0 ? dst0 : dst) + ey(i) * (nx >> 2), d);
                        accumulate(part[ey(i) + 1], d);
                    }
                }
            }
            if (!TAU1 && s + 1 < nslab) load_f(s + 1);   // in flight across the barrier
#pragma unroll
            for (int k = 0; k < 3; ++k) {   // component k: what row yc sends to row yc + (k - 1)
                const int slot = (rd0 + k - 1) % PROWS;
                *reinterpret_cast<float4 *>(ps + (k * PROWS + slot) * NW + 4 * lane) = part[k];
            }
        }
        if (s + 1 < nslab) {   // slab s + 1's recurrences: its last ring chunk, then the column phase
            const int c = s + 1 + QAHEAD;
            if (c < nchunks && !ptx::mbar_wait_bounded(&bars[c % QCH], (c / QCH) & 1, kWaitLimitNs)) timed_out = true;
            if (!CDMG) column_phase(s + 1);
        }
        if (__syncthreads_or(timed_out)) {
            stop = true;
            break;
        }

        // ---- rho(t+1) and the potential of row yo = ys + 8s - 2 + warp ----
        const int yo = ys + SLAB * s - 2 + warp;
        if (interior && yo >= ys && yo < ys + hseg) {
            const int slot = (yo - ys + 3) % PROWS;
            // component 0: from row yo + 1 (down-movers), 1: from row yo, 2: from row yo - 1
            const float4 a = *reinterpret_cast<const float4 *>(ps + (0 * PROWS + slot) * NW + 4 * lane);
            const float4 b = *reinterpret_cast<const float4 *>(ps + (1 * PROWS + slot) * NW + 4 * lane);
            const float4 cc = *reinterpret_cast<const float4 *>(ps + (2 * PROWS + slot) * NW + 4 * lane);
            const float2 q01 = stencil_field_t2<EOS>(
                m, add2(add2(make_float2(a.x, a.y), make_float2(b.x, b.y)), make_float2(cc.x, cc.y)), SC);
            const float2 q23 = stencil_field_t2<EOS>(
                m, add2(add2(make_float2(a.z, a.w), make_float2(b.z, b.w)), make_float2(cc.z, cc.w)), SC);
            const float4 q = make_float4(q01.x, q01.y, q23.x, q23.y);
            float *qrow = A.qout + (long long)yo * A.qpitch + QG;
            auto storeq = [&](long long x) {   // padded row offset of a float4 of q(t+1)
                if (range_ok((long long)yo * A.qpitch + QG + x, 4, (long long)A.qpitch * ny, A.err))
                    *reinterpret_cast<float4 *>(qrow + x) = q;
            };
            storeq(xg);
            if (xg < QG) storeq(xg + nx);        // right ghost image
            if (xg >= nx - QG) storeq(xg - nx);  // left ghost image
        }
    }

    if (unstable) atomicOr(A.err, kErrUnstable);
    if (stop) {   // CTA-uniform: some thread's wait timed out
        if (threadIdx.x == 0) {
            atomicOr(A.err, kErrTimeout);
            // thread 0 issued every copy: let those still in flight land before
            // the CTA's shared memory is released
            for (int c = max(0, issued - QCH); c < issued; ++c)
                (void)ptx::mbar_wait_bounded(&bars[c % QCH], (c / QCH) & 1, kWaitLimitNs);
            for (int r = max(0, rows_issued - 2); r < rows_issued; ++r)
                (void)ptx::mbar_wait_bounded(&row_bar[r & 1], (r >> 1) & 1, kWaitLimitNs);
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
    return (cdm || (radius == FK && m.kx == FK && m.ky == FK)) && m.nx % 4 == 0 && m.nx >= 2 * QG &&
           m.ny >= 2 * FK + 2;
}

int fused_q_pitch(int nx) { return nx + 2 * QG; }

// A segment of h rows collides 8 ceil((h + 2) / 8) rows (its own, the one above
// and the one below, in whole slabs) and stages h + 66 potential rows for
// d/dy, so h = 8k - 2 wastes no collided rows.  The tallest such segment that
// still gives every SM a CTA keeps the halo overhead lowest (measured on 512^2
// to 4096^2 lattices: 14, 62, 126, 126 rows); smaller grids leave SMs idle.
int fused_auto_seg_rows(int nx, int ny, int num_sms) {
    const long long strips = (nx + TXI - 1) / TXI;
    const int cand[] = {126, 62, 30, 14, 6};
    for (int h : cand)
        if (strips * ((ny + h - 1) / h) >= num_sms) return h;
    return 6;
}

cudaError_t launch_potential_padded(const Model<float> &m, bool sc, const float *f, float *qpad, int *err,
                                    cudaStream_t s) {
    const int pitch = fused_q_pitch(m.nx);
    long long total = (long long)pitch * m.ny;
    int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
    potential_pad_kernel<<<blocks, 256, 0, s>>>(m, sc, f, qpad, pitch, err);
    return cudaGetLastError();
}

cudaError_t launch_fused_step(const Model<float> &m, bool sc, bool cdm, const float *f, const float *qin,
                              float *fout, float *qout, int *err, int seg_rows, cudaStream_t s, bool pdl, float *rec,
                              bool rev) {
    if (rec && (m.walls || cdm)) return cudaErrorInvalidValue;
    FusedArgs a;
    a.m = m;
    a.f = f;
    a.fout = fout;
    a.qin = qin;
    a.qout = qout;
    a.rec = rec;
    a.err = err;
    a.qpitch = fused_q_pitch(m.nx);
    a.seg_h = seg_rows;
    a.n4 = (int)((long long)m.nx * m.ny / 4);
    a.rev = rev ? 1 : 0;
    if (seg_rows < 1) return cudaErrorInvalidValue;
    dim3 grid((m.nx + TXI - 1) / TXI, (m.ny + seg_rows - 1) / seg_rows);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    a.w1y = m.wy[1];
    a.w2y = m.wy[2];
    const double r = 0.5 * (std::sqrt(5.0) - 3.0);   // root of r^2/3 + r + 1/3 = 0 (Eq. 20's operator)
    a.w1x = m.wx[1];
    a.w2x = m.wx[2];
    a.ry = (float)r;
    a.ry5 = (float)std::pow(r, 5);
    a.ry12 = (float)std::pow(r, 12);
    a.ry25 = (float)std::pow(r, 25);
    const bool tau1 = m.omega == 1.0f;
    void (*kern)(const FusedArgs) = nullptr;
#define LBM_PICK(E)                                                                                        \
    if (cdm && m.walls)                                                                                    \
        kern = sc ? (tau1 ? fused_step_kernel<true, true, E, true, false, true>                            \
                          : fused_step_kernel<true, false, E, true, false, true>)                          \
                  : (tau1 ? fused_step_kernel<false, true, E, true, false, true>                           \
                          : fused_step_kernel<false, false, E, true, false, true>);                        \
    else if (cdm)                                                                                          \
        kern = sc ? (tau1 ? fused_step_kernel<true, true, E, false, false, true>                           \
                          : fused_step_kernel<true, false, E, false, false, true>)                         \
                  : (tau1 ? fused_step_kernel<false, true, E, false, false, true>                          \
                          : fused_step_kernel<false, false, E, false, false, true>);                       \
    else if (rec)                                                                                          \
        kern = sc ? (tau1 ? fused_step_kernel<true, true, E, false, true>                                  \
                          : fused_step_kernel<true, false, E, false, true>)                                \
                  : (tau1 ? fused_step_kernel<false, true, E, false, true>                                 \
                          : fused_step_kernel<false, false, E, false, true>);                              \
    else if (m.walls)                                                                                      \
        kern = sc ? (tau1 ? fused_step_kernel<true, true, E, true> : fused_step_kernel<true, false, E, true>) \
                  : (tau1 ? fused_step_kernel<false, true, E, true> : fused_step_kernel<false, false, E, true>); \
    else                                                                                                   \
        kern = sc ? (tau1 ? fused_step_kernel<true, true, E, false> : fused_step_kernel<true, false, E, false>) \
                  : (tau1 ? fused_step_kernel<false, true, E, false> : fused_step_kernel<false, false, E, false>)
    switch (m.eos) {
    case LBM_EOS_VDW: LBM_PICK(LBM_EOS_VDW); break;
    case LBM_EOS_CS: LBM_PICK(LBM_EOS_CS); break;
    case LBM_EOS_PR: LBM_PICK(LBM_EOS_PR); break;
    case LBM_EOS_RK: LBM_PICK(LBM_EOS_RK); break;
    case LBM_EOS_PSI_EXP: LBM_PICK(LBM_EOS_PSI_EXP); break;
    default: LBM_PICK(LBM_EOS_RKS); break;
    }
#undef LBM_PICK
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(NTHR);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace lbm
