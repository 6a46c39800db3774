// Hot-path steps a2-a6: per-event normalised PDF, -w log P, fused analytic
// adjoint and the deterministic FP64 reduction, for one fit or for many
// segments (fits) packed back to back.
//
// Sec. 3 of the paper evaluates the PDF with one thread per event, takes the
// log of the signal/background mixture in a second launch and sums the logs
// on the host.  Here one kernel does all of it.  Work is split into 512-event
// tiles owned by single warps: lane l accumulates events l, l+32, ..., l+480
// of its tile in order (coalesced 8-byte loads), the warp reduces its FP64
// accumulators with a fixed butterfly and writes one partial per tile.
// The warp that completes the last tile of a group of 32 tiles reduces the
// group, and the warp that completes a segment's last group adds its group
// partials in fixed order and writes the NLL and gradient.  No block-wide
// barrier sits in the event loop, and the result does not depend on the
// launch geometry (block size, grid, tiles taken at once).
//
// The GPU has 2 FP64 operations per clock per SM, so the per-event arithmetic
// is arranged to spend as few of them as possible:
//   * the decay-time term uses erfc(z) = 2 - exp(-z^2) erfcx(|z|) for z < 0 and
//     erfc(z) = exp(-z^2) erfcx(z) for z >= 0, with exp(-Gamma tau + Gamma^2
//     sigma^2/2) exp(-z^2) = exp(-tau^2/(2 sigma^2)): the Gaussian factor that
//     the gradient needs anyway replaces the exponential inside erfc;
//   * sin/cos, the whole angular basis and the Gaussian's exp run on the
//     integer pipe in 64-bit fixed point and are rounded once to double
//     (int_math.cuh); the decay exponential, log and erfcx are table-driven
//     FP64 (fp64_math.cuh): the split between the FP64 and the integer pipes
//     is the measured fastest one;
//   * sin(theta_K) sin(theta_mu) is one square root; the constant factors of
//     the ten angular functions are folded into the amplitude coefficients.
//
// Gradient (fused adjoint).  With r = w/P, every derivative of the NLL is a
// contraction of a few per-event sums with parameter-only factors:
//   S_k = sum r T f_k,  D_j = sum r A dT/dtheta_j (j = Gamma, sigma, mu),
//   Q = sum r,          SH = sum_k h_k S_k = sum r T A,
//   dNLL/dtime_j = -cs D_j + cs (dI_T/dtheta_j / I_T) SH,
//   dNLL/df_b    = SH / (I_T I_Omega) - Q / V,
//   dNLL/dang_j  = -cs sum_k (dh_k/dtheta_j) S_k,   cs = (1 - f_b)/(I_T I_Omega),
// so the event pass carries 15 accumulators (4D) instead of one per
// parameter and the angular derivatives cost nothing per event.
#include <math.h>

#include "fp64_math.cuh"
#include "int_math.cuh"
#include "angular.cuh"
#include "ipa_internal.cuh"
#include "tile_reduce.cuh"

namespace ipa {
namespace {

constexpr int kNllBlock = 128;                       // threads per block of the basis kernel
constexpr int kPerLane = kTile / 32;                 // events per lane per tile

// Per-warp copy of a segment's constants in shared memory, with the factors
// the event loop multiplies by folded in:
//   A' = sum_k hq_k f_k = (cs / 2) A, so that P = T2 A' + cb with T2 = 2 T,
//   hq_k = h_k c_k cs / 2 for the unscaled products f'_k (h_k cs / 2 for a
//   cached basis), aq = cs / 2 (the 1D model's A' for A = 1),
//   c2 = Gamma^2 sigma^2 / 2 + ln 2, so that exp(-Gamma tau + c2) = 2 E,
//   hcq_k = h_k c_k (cs / 2) times the power of two 2^s that brings the largest
//   into [1, 2), in Q62, so that the fixed-point sum gives A' directly.
struct WarpConsts {
    Consts c;
    double hq[10];
    double aq;
    double c2;
    double tcut;     // t above it: z < -6.25, the Gaussian-erfcx term is below 1e-17 of T
    long long hcq[10];   // h_k c_k (cs / 2) 2^s in Q62 (the fixed-point amplitude sum), with
    int hexp;            // 2 - s: A' = (sum_k hcq_k F_k in Q60) 2^-s, s making max|hcq| lie in [1, 2)
    int fixed;           // coefficients finite and s in range: the fixed-point path may be used
};

// The largest of a non-negative 64-bit value over the warp.
__device__ __forceinline__ long long max_abs_bits(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// 2^e as a double for -1022 <= e <= 1023 (built from its bit pattern).
__device__ __forceinline__ double exp2_int(int e) {
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// Decay-time events per compaction round of one lane (see nll_kernel).
constexpr int kSub = 4;
static_assert(kSub == 4, "a compaction round keeps four ballot masks");
static_assert((IPA_TILE_EVENTS / 32) % kSub == 0, "events per lane must be a multiple of kSub");

// The part of the decay-time factor that needs the Gaussian and erfcx, for an
// event with t <= tcut (z >= -6.25 up to rounding): with g = exp(-tau^2 /
// (2 sigma^2)) and X = erfcx(|z|), returns g X in .x and g in .y, the sign of
// .y carrying z >= 0 (negative) or z < 0 (positive).  Then 2 g(tau) = 2E - gX
// (z < 0) or gX (z >= 0).  Events with t > tcut have 2 g(tau) = 2E to 1e-17
// relative and a Gaussian below 1e-17; they are given (0, +0).
__device__ __forceinline__ double2 gauss_erfcx(const Consts& c, double tau, const MathTables* mt) {
    // branch-free integer exp; the argument is clamped at -705 (events more
    // than 37 sigma before mu), where the Gaussian, below 1e-306, is nothing
    // against the exponential term of 2 g(tau)
    const double gr = -(tau * tau) * c.k_g;
    const double g = exp_int_nb(below_neg(gr, -705.0) ? -705.0 : gr, mt);
    const double z = (c.Gs2 - tau) * c.k_z;
    const double x = fabs(z);
    const bool zneg = negative(z);
    double X = erfcx_poly(x, mt);
    if (above(x, 6.25)) {
        // z < 0: the erfcx term is below 1e-17 of E; z >= 0 (tau far below the
        // resolution peak, outside the usual range): exact library erfcx
        X = zneg ? 0.0 : erfcx(x);
    }
    return make_double2(g * X, zneg ? g : -g);
}

// A' = sum_k hq_k f_k in FP64 (cached basis, or angles outside basis_q62_ok).
__device__ __forceinline__ double amplitude_sum(const double* hq, const double* f) {
    double Ap = hq[0] * f[0];
#pragma unroll
    for (int k = 1; k < 10; ++k) Ap = fma(hq[k], f[k], Ap);
    return Ap;
}

// One event: the log term (w log P added to acc[0], or for w = 1 exactly, P
// folded into the lane's product) and the adjoint sums.  For the 4D model f
// holds either the unscaled products f'_k (CACHED = false) or the cached basis
// f_k (CACHED = true); Ap = (cs/2) A (wc.aq for the 1D model); ge is the
// event's gauss_erfcx value or (0, +0).
// Accumulators (kD = 12 for 4D, 3 for 1D), with r = w / P and A' = (cs/2) A:
//   acc[1] = sum r,  acc[2 + k] = sum r T2 f_k (4D) or acc[2] = sum r T2 (1D),
//   acc[kD] = sum r A' tau T2,  acc[kD + 1] = sum r A' Gx,  acc[kD + 2] = sum r A' tau Gx;
// the derivatives in Gamma, sigma and mu are linear in these (finalize).
template <int KIND, bool GRAD, bool CACHED, bool WEIGHTED>
__device__ __forceinline__ void event(const WarpConsts& wc, const MathTables* mt, double t, const double* f,
                                      double Ap, double w, double2 ge, double* acc, double* prod, int* esum) {
    const Consts& c = wc.c;
    const double tau = t - c.mu;
    const double E2 = exp_int(fma(-c.Gamma, tau, wc.c2), mt);
    const long long gb = __double_as_longlong(ge.y);
    const double T2 = gb >= 0 ? E2 - ge.x : ge.x;
    const double Gx = __longlong_as_double(gb & 0x7FFFFFFFFFFFFFFFll);
    const double P = fma(T2, Ap, c.cb);
    // events of weight exactly 1 (all events without a weight column) join the
    // lane's log product, so a column of ones gives the same bits as no column
    if (WEIGHTED && __double_as_longlong(w) != 0x3FF0000000000000ll)
        acc[0] = fma(w, log_fast(P, mt), acc[0]);
    else
        log_mul(P, prod, esum);
    if (GRAD) {
        // r = w / P feeds only the adjoint sums; its ~6e-14 relative error
        // (rcp_newton) is far inside the gradient's tolerance
        const double r = WEIGHTED ? w * rcp_newton(P) : rcp_newton(P);
        acc[1] += r;
        const double rT = r * T2;
        constexpr int kD = KIND == IPA_MODEL_ANGTIME4D ? 12 : 3;
        if (KIND == IPA_MODEL_ANGTIME4D) {
#pragma unroll
            for (int k = 0; k < 10; ++k) acc[2 + k] = fma(rT, f[k], acc[2 + k]);
        } else {
            acc[2] += rT;
        }
        const double rA = r * Ap;
        const double u = rA * tau;
        acc[kD + 0] = fma(u, T2, acc[kD + 0]);
        acc[kD + 1] = fma(rA, Gx, acc[kD + 1]);
        acc[kD + 2] = fma(u, Gx, acc[kD + 2]);
    }
}

// ---- the fast tile (4D model, angles on the integer pipe) ----
// A whole tile of the 4D model's NLL + gradient takes this path; the last,
// partial tile of a segment and the other variants take the plain loop of
// nll_kernel.
//
// On this GPU a warp FP64 instruction occupies the sub-partition's FP64 unit
// for about 64 cycles (2 FP64 operations per clock per SM).  A few FP64
// instructions spread among a warp's integer work overlap with it, but a burst
// of them does not (measured: removing the ten back-to-back DFMA of the
// angular adjoint sums saved far more time than removing isolated DMUL or DADD
// instructions, which cost about nothing).  So the ten sums S_k = sum r T f'_k
// are accumulated here on the integer pipe: r T is converted once per event to
// signed 64-bit fixed point with 40 fraction bits (rounded to nearest, for
// |r T| < 2^19), and each product with the Q62 angular product f'_k is the
// high 64 bits of the 128-bit product (Q38: the floor, corrected on average
// by half a unit per product at the end of the tile).  A lane adds its 16
// events exactly in 64-bit integers (no overflow: |r T f'_k| < 2^19) and
// converts each sum to a double once per tile, so these sums do not depend on
// the order of the events within a lane.  Error of a sum: about 2^-39 per
// event, of random sign (a sum over 1e6 events is off by ~1e-9 absolute,
// while the sums themselves are ~1e5 and the gradient tolerance is 1e-9 of
// them).  The remaining accumulators are FP64 as in the plain loop.  The
// integer work runs with the branch-free functions of int_math.cuh; lanes
// outside their ranges are fixed up with the FP64 paths of the plain loop.  A
// tile in which some P lies outside the Newton reciprocal's range (zero,
// subnormal, negative, huge, infinite or NaN) or some |r T| >= 2^19 is redone
// by the plain loop.  Either way the tile's sums depend only on its events,
// never on the launch geometry.

// The integer-pipe results of one event that its FP64 work needs.
struct RowIn {
    double tau, w, E2, Ap;
    long long F[10];   // f'_k in Q62
};

// tau, E2 = 2 e^{-Gamma tau + Gamma^2 sigma^2 / 2}, the ten f'_k and A' =
// (cs / 2) A of event e: the angular basis and A' with the branch-free
// fixed-point functions, E2 with the table-driven FP64 exp (measured 7 % faster
// here than the integer-pipe exp, whose long dependent chain sat in front of
// the event's FP64 work; the FP64 pipe has room since the adjoint sums moved to
// fixed point); false if the lane needs fix_int_phase.
template <bool WEIGHTED>
__device__ __forceinline__ bool int_phase(const WarpConsts& wc, const MathTables* mt, const Cols& cols, int64_t e,
                                          RowIn& v) {
    const double t = __ldg(cols.t + e);
    const double ck = __ldg(cols.ck + e), cl = __ldg(cols.cl + e), phi = __ldg(cols.phi + e);
    v.w = WEIGHTED ? __ldg(cols.w + e) : 1.0;
    v.tau = t - wc.c.mu;
    v.E2 = exp_fast(fma(-wc.c.Gamma, v.tau, wc.c2), mt);
    basis_q62_nb(ck, cl, phi, mt, v.F);
    long long Af = 0;
#pragma unroll
    for (int k = 0; k < 10; ++k) Af += __mul64hi(wc.hcq[k], v.F[k]);
    v.Ap = q62_to_double_nb(Af, wc.hexp);
    return wc.fixed && basis_q62_ok(ck, cl, phi);
}

// The FP64 basis of the plain loop for a lane that int_phase could not serve
// (the FP64 products, in [-1, 1] for valid angles, go to Q62).
__device__ __forceinline__ void fix_int_phase(const WarpConsts& wc, const MathTables* mt, const Cols& cols,
                                              int64_t e, RowIn& v) {
    const double ck = __ldg(cols.ck + e), cl = __ldg(cols.cl + e), phi = __ldg(cols.phi + e);
    if (!(wc.fixed && basis_q62_ok(ck, cl, phi))) {
        double f[10];
        basis_unscaled(ck, cl, phi, mt, f);
        v.Ap = amplitude_sum(wc.hq, f);
#pragma unroll
        for (int k = 0; k < 10; ++k) v.F[k] = to_q62_nb(f[k]);
    }
}

// rcp_newton and log_fast without their range branches (P in [2^-125, 2^126)).
__device__ __forceinline__ double rcp_newton_nb(double x) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned xf = ((unsigned)((unsigned long long)b >> 32) & 0x80000000u) |
                        ((unsigned)(e - 1023 + 127) << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu);
    const unsigned yf = __float_as_uint(__frcp_rn(__uint_as_float(xf)));
    const long long yb = ((long long)(yf & 0x80000000u) << 32) |
                         ((long long)(((yf >> 23) & 0xFFu) - 127 + 1023) << 52) | ((long long)(yf & 0x7FFFFFu) << 29);
    const double y = __longlong_as_double(yb);
    return fma(y, fma(-x, y, 1.0), y);
}

__device__ __forceinline__ double log_fast_nb(double x, const MathTables* t) {
    using namespace fp64tab;
    const long long b = __double_as_longlong(x);
    const int e = (int)(b >> 52) - 1023;
    const int j = (int)((b >> 45) & 127);
    const double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
    const double r = fma(m, t->linv[j], -1.0);
    double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    q = fma(q, r, 0.2);
    q = fma(q, r, -0.25);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    const double l = fma(r * r, q, r);
    const double ed = __longlong_as_double(0x4330000000000000ll + (long long)(e + 2048)) -
                      (4503599627370496.0 + 2048.0);
    return fma(ed, kLn2Hi, fma(ed, kLn2Lo, t->ltab[j] + l));
}

// log_mul for positive normal P (no branch for zero, subnormal or special P).
__device__ __forceinline__ void log_mul_nb(double P, double* prod, int* esum) {
    const long long b = __double_as_longlong(P);
    *prod *= __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
    *esum += (int)(b >> 52) - 1023;
}

// x 2^40 rounded to the nearest signed 64-bit integer (ties away from zero),
// for |x| < 2^19 (else *bad is set; NaN and infinities included).
__device__ __forceinline__ long long to_q40(double x, bool* bad) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FFull) - 1023;
    *bad |= E > 18;
    const unsigned long long M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const int sh = E - 12;
    const int s = (-sh) & 63;
    const unsigned long long dn = (M + (s ? 1ull << (s - 1) : 0ull)) >> s;
    const long long v = (long long)(sh >= 0 ? M << (sh & 63) : (sh > -64 ? dn : 0ull));
    return (b >> 63) ? -v : v;
}

// The FP64 work of one event on the fast path: event() with the exponential
// and the angular products from int_phase and the ten angular adjoint sums in
// fixed point (acci, Q38).  ge: the event's gauss_erfcx value or (0, +0).
// *bad is set when P is outside [2^-125, 2^126) or |r T| >= 2^19.
template <bool GRAD, bool WEIGHTED>
__device__ __forceinline__ void event_fast(const WarpConsts& wc, const MathTables* mt, const RowIn& v, double2 ge,
                                           double* acc, long long* acci, double* prod, int* esum, bool* bad) {
    const Consts& c = wc.c;
    const long long gb = __double_as_longlong(ge.y);
    const double T2 = gb >= 0 ? v.E2 - ge.x : ge.x;
    const double Gx = __longlong_as_double(gb & 0x7FFFFFFFFFFFFFFFll);
    const double P = fma(T2, v.Ap, c.cb);
    const long long pb = __double_as_longlong(P);
    *bad |= (unsigned long long)(pb - 0x3820000000000000ll) >= 0x0FB0000000000000ull;
    if (WEIGHTED) {
        // weight exactly 1: P joins the lane's product (as in event)
        const bool one = __double_as_longlong(v.w) == 0x3FF0000000000000ll;
        acc[0] = fma(one ? 0.0 : v.w, log_fast_nb(P, mt), acc[0]);
        log_mul_nb(one ? P : 1.0, prod, esum);
    } else {
        log_mul_nb(P, prod, esum);
    }
    if (GRAD) {
        const double r = WEIGHTED ? v.w * rcp_newton_nb(P) : rcp_newton_nb(P);
        acc[1] += r;
        const long long rq = to_q40(r * T2, bad);
#pragma unroll
        for (int k = 0; k < 10; ++k) acci[k] += __mul64hi(rq, v.F[k]);
        const double rA = r * v.Ap;
        const double u = rA * v.tau;
        acc[12] = fma(u, T2, acc[12]);
        acc[13] = fma(rA, Gx, acc[13]);
        acc[14] = fma(u, Gx, acc[14]);
    }
}

// Rows i0 .. i0 + kSub - 1 of a whole tile (lane l: events tbase + l + 32 i) of
// the 4D model on the fast path: the near-peak events of the kSub rows marked
// by ballot and their Gaussian/erfcx values evaluated packed into sbuf, then
// the events row by row into acc (FP64 sums), acci (the fixed-point S_k), the
// log product and *bad.
template <bool WEIGHTED>
__device__ __forceinline__ void block_fast(const WarpConsts& wc, const MathTables* mt, const Cols& cols,
                                           int64_t tbase, int i0, double2* sbuf, int lane, double* acc,
                                           long long* acci, double* prod, int* esum, bool* bad) {
    const unsigned below = (1u << lane) - 1u;
    unsigned m[kSub];
    int p[kSub];
#pragma unroll
    for (int q = 0; q < kSub; ++q) {
        const int64_t e = tbase + lane + 32 * (i0 + q);
        m[q] = __ballot_sync(0xffffffffu, !greater(__ldg(cols.t + e), wc.tcut));
    }
    p[0] = 0;
    p[1] = __popc(m[0]);
    p[2] = p[1] + __popc(m[1]);
    p[3] = p[2] + __popc(m[2]);
    const int n_slow = p[3] + __popc(m[3]);
    for (int j = lane; j < n_slow; j += 32) {
        const int q = (j >= p[1]) + (j >= p[2]) + (j >= p[3]);
        const unsigned mq = q == 0 ? m[0] : (q == 1 ? m[1] : (q == 2 ? m[2] : m[3]));
        const int before = q == 0 ? 0 : (q == 1 ? p[1] : (q == 2 ? p[2] : p[3]));
        const int64_t e = tbase + nth_set(mq, j - before) + 32 * (i0 + q);
        sbuf[j] = gauss_erfcx(wc.c, __ldg(cols.t + e) - wc.c.mu, mt);
    }
    __syncwarp();
#pragma unroll 1
    for (int q = 0; q < kSub; ++q) {
        const unsigned mq = q == 0 ? m[0] : (q == 1 ? m[1] : (q == 2 ? m[2] : m[3]));
        const int before = q == 0 ? 0 : (q == 1 ? p[1] : (q == 2 ? p[2] : p[3]));
        const double2 gv = sbuf[(before + __popc(mq & below)) & (kSub * 32 - 1)];
        const double2 ge = (mq >> lane) & 1u ? gv : make_double2(0.0, 0.0);
        const int64_t e = tbase + lane + 32 * (i0 + q);
        RowIn v;
        const bool ok = int_phase<WEIGHTED>(wc, mt, cols, e, v);
        if (__any_sync(0xffffffffu, !ok)) fix_int_phase(wc, mt, cols, e, v);
        event_fast<true, WEIGHTED>(wc, mt, v, ge, acc, acci, prod, esum, bad);
    }
    __syncwarp();
}

// One whole tile (kTile events from tbase) of the 4D model's NLL + gradient on
// the fast path, kSub rows at a time.  Returns false if the tile must be redone
// by the plain loop (acc, prod and esum are then meaningless).
template <bool WEIGHTED>
__device__ __forceinline__ bool tile_fast(const WarpConsts& wc, const MathTables* mt, const Cols& cols,
                                          int64_t tbase, double2* sbuf, int lane, double* acc, double* prod,
                                          int* esum) {
    bool bad = false;
    long long acci[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acci[k] = 0;
#pragma unroll 1
    for (int i0 = 0; i0 < kPerLane; i0 += kSub)
        block_fast<WEIGHTED>(wc, mt, cols, tbase, i0, sbuf, lane, acc, acci, prod, esum, &bad);
    // the lane's fixed-point sums (Q38) as doubles; each high product is the
    // floor of the exact one, half a unit low on average, so the lane's
    // kPerLane products get kPerLane / 2 units back
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[2 + k] = q62_to_double_nb(acci[k] + kPerLane / 2, 24);
    return !__any_sync(0xffffffffu, bad);
}

// Write NLL (and gradient) of one segment from its reduced accumulators.
// With S_k = sum r T f_k and SH = sum_k h_k S_k = sum r T A (A = 1 in 1D), and
// D_j = sum r A dT/dtheta_j where
//   dT/dGamma = (Gamma sigma^2 - tau) T - sigma^2 G,
//   dT/dsigma = Gamma^2 sigma T - (tau / sigma + Gamma sigma) G,
//   dT/dmu    = Gamma T - G,   G = cG Gx,
// the accumulators give cs D_Gamma = cs Gamma sigma^2 SH - Y1 - 2 sigma^2 cG Y2,
// cs D_sigma = cs Gamma^2 sigma SH - 2 cG (Y3 / sigma + Gamma sigma Y2) and
// cs D_mu = cs Gamma SH - 2 cG Y2 (Y1..Y3 = acc[kD..kD+2]).
template <int KIND, bool GRAD, bool CACHED>
__device__ void finalize(const Consts& c, const double* acc, int n_par, double* out, int lane) {
    // every lane holds acc; lane j writes component j (0: the NLL, 1 + j: the
    // derivative in parameter j), computing only what that component needs
    if (lane == 0) out[0] = -acc[0];
    if (!GRAD) return;
    const double Q = acc[1];
    constexpr int kD = KIND == IPA_MODEL_ANGTIME4D ? 12 : 3;
    double S[10];
    double SH;
    if (KIND == IPA_MODEL_ANGTIME4D) {
        SH = 0.0;
        for (int k = 0; k < 10; ++k) {
            S[k] = (CACHED ? 0.5 : 0.5 * kBasisScale[k]) * acc[2 + k];
            SH = fma(c.h[k], S[k], SH);
        }
    } else {
        SH = 0.5 * acc[2];
    }
    const double csSH = c.cs * SH;
    const double Y1 = acc[kD], Y2 = acc[kD + 1], Y3 = acc[kD + 2];
    const double tcG = 2.0 * c.cG;
    if (lane < 3) {
        double csD;
        if (lane == 0) csD = fma(c.Gs2, csSH, -fma(tcG * c.s2, Y2, Y1));
        else if (lane == 1) csD = fma(c.G2s, csSH, -tcG * fma(c.inv_s, Y3, c.Gsig * Y2));
        else csD = fma(c.Gamma, csSH, -tcG * Y2);
        out[1 + lane] = fma(c.dlnIT[lane], csSH, -csD);
    } else if (lane == IPA_FB) {
        out[1 + IPA_FB] = fma(SH, c.inv_ITIO, -Q * c.inv_V);
    } else if (KIND == IPA_MODEL_ANGTIME4D && lane < IPA_NPAR_4D) {
        const int j = lane - IPA_A0SQ;
        double s = 0.0;
        for (int k = 0; k < 10; ++k) s = fma(c.dh[k][j], S[k], s);
        out[1 + lane] = -c.cs * s;
    }
    for (int j = (KIND == IPA_MODEL_ANGTIME4D ? IPA_NPAR_4D : IPA_NPAR_1D) + lane; j < n_par; j += 32)
        out[1 + j] = 0.0;
}

// The plain loop over one tile's events [tbase, min(tbase + kTile, ev1)): lane
// l adds events l, l + 32, ... in order into acc (and the log product).  Those
// near the resolution peak are marked by ballot kSub rows at a time and their
// Gaussian/erfcx values evaluated packed, 32 per pass, into the warp's buffer.
template <int KIND, bool GRAD, bool CACHED, bool WEIGHTED>
__device__ __forceinline__ void tile_plain(const WarpConsts& wc, const MathTables* mt, const Cols& cols,
                                           int64_t tbase, int64_t ev1, double2* sbuf, int lane, double* acc,
                                           double* prod, int* esum) {
    const unsigned below = (1u << lane) - 1u;
#pragma unroll 1
    for (int i0 = 0; i0 < kPerLane; i0 += kSub) {
        unsigned m0, m1, m2, m3;
        {
            unsigned mk[kSub];
#pragma unroll
            for (int q = 0; q < kSub; ++q) {
                const int64_t e = tbase + lane + 32 * (i0 + q);
                const bool slow = e < ev1 && !greater(__ldg(cols.t + e), wc.tcut);
                mk[q] = __ballot_sync(0xffffffffu, slow);
            }
            m0 = mk[0];
            m1 = mk[1];
            m2 = mk[2];
            m3 = mk[3];
        }
        const int p1 = __popc(m0), p2 = p1 + __popc(m1), p3 = p2 + __popc(m2);
        const int n_slow = p3 + __popc(m3);
        for (int j = lane; j < n_slow; j += 32) {
            const int q = (j >= p1) + (j >= p2) + (j >= p3);
            const unsigned m = q == 0 ? m0 : (q == 1 ? m1 : (q == 2 ? m2 : m3));
            const int before = q == 0 ? 0 : (q == 1 ? p1 : (q == 2 ? p2 : p3));
            const int64_t e = tbase + nth_set(m, j - before) + 32 * (i0 + q);
            sbuf[j] = gauss_erfcx(wc.c, __ldg(cols.t + e) - wc.c.mu, mt);
        }
        __syncwarp();
#pragma unroll 1
        for (int q = 0; q < kSub; ++q) {
            const int64_t e = tbase + lane + 32 * (i0 + q);
            if (e < ev1) {
                const unsigned m = q == 0 ? m0 : (q == 1 ? m1 : (q == 2 ? m2 : m3));
                const int before = q == 0 ? 0 : (q == 1 ? p1 : (q == 2 ? p2 : p3));
                const double2 ge = (m >> lane) & 1u ? sbuf[before + __popc(m & below)]
                                                    : make_double2(0.0, 0.0);
                const double w = WEIGHTED ? __ldg(cols.w + e) : 1.0;
                double f[10];
                double Ap = wc.aq;
                if (KIND == IPA_MODEL_ANGTIME4D) {
                    if (CACHED) {
#pragma unroll
                        for (int k = 0; k < 10; ++k) f[k] = __ldg(cols.fk + k * cols.fk_stride + e);
                        Ap = amplitude_sum(wc.hq, f);
                    } else {
                        const double ck = __ldg(cols.ck + e), cl = __ldg(cols.cl + e), phi = __ldg(cols.phi + e);
                        if (wc.fixed && basis_q62_ok(ck, cl, phi)) {
                            // the angular products and A on the integer pipe
                            long long F[10];
                            basis_q62(ck, cl, phi, mt, F);
                            long long Af = 0;
#pragma unroll
                            for (int k = 0; k < 10; ++k) {
                                f[k] = q62_to_double(F[k], 0);
                                Af += __mul64hi(wc.hcq[k], F[k]);
                            }
                            Ap = q62_to_double(Af, wc.hexp);        // Af is Q60, times 2^-s
                        } else {
                            basis_unscaled(ck, cl, phi, mt, f);
                            Ap = amplitude_sum(wc.hq, f);
                        }
                    }
                }
                event<KIND, GRAD, CACHED, WEIGHTED>(wc, mt, __ldg(cols.t + e), f, Ap, w, ge, acc, prod,
                                                    esum);
            }
        }
        __syncwarp();
    }
}

// A segment's constants into the warp's copy in shared memory, with the
// factors the event loop uses (warp-collective).
template <bool CACHED>
__device__ __forceinline__ void load_warp_consts(WarpConsts& wc, const Consts* src_consts, int lane) {
    __syncwarp();
    const double* src = reinterpret_cast<const double*>(src_consts);
    double* dst = reinterpret_cast<double*>(&wc.c);
    for (int i = lane; i < kConstsDoubles; i += 32) dst[i] = __ldg(src + i);
    __syncwarp();
    const double half_cs = 0.5 * wc.c.cs;
    if (lane < 10) wc.hq[lane] = (CACHED ? wc.c.h[lane] : wc.c.h[lane] * kBasisScale[lane]) * half_cs;
    if (lane == 10) wc.aq = half_cs;
    if (lane == 11) wc.c2 = wc.c.c_exp + fp64tab::kLn2Hi;
    if (lane == 12) {
        const double tc = wc.c.mu + (wc.c.Gs2 + 6.25 / wc.c.k_z);
        wc.tcut = tc == tc ? tc : INFINITY;    // NaN constants: every event takes the full path
    }
    // h_k c_k (cs / 2) scaled by 2^s into Q62 for the fixed-point
    // amplitude sum (multiplying by a power of two is exact);
    // non-finite coefficients (non-physical theta) or a scale outside
    // [-64, 900] keep the FP64 path, which propagates NaN
    const double hca = lane < 10 ? (wc.c.h[lane] * kBasisScale[lane]) * half_cs : 0.0;
    const long long amag = __double_as_longlong(hca) & 0x7FFFFFFFFFFFFFFFll;
    const long long amax = max_abs_bits(amag);
    const int eb = (int)(amax >> 52);                 // biased exponent of max |hca|
    const int sc = amax == 0 ? 0 : 1023 - eb;         // max |hca| 2^sc in [1, 2)
    const bool sc_ok = amax < 0x7FF0000000000000ll && sc >= -64 && sc <= 900;
    if (lane < 10) wc.hcq[lane] = sc_ok ? to_q62(hca * exp2_int(sc)) : 0;
    if (lane == 0) {
        wc.hexp = 2 - sc;
        wc.fixed = sc_ok && abs_below(wc.c.cs, 1e300) ? 1 : 0;
    }
    __syncwarp();
}

// Blocks of any whole number of warps (1..kMaxWarps); each warp keeps a copy of
// its current segment's constants in dynamic shared memory.
constexpr int kMaxWarps = 8;

template <int KIND, bool GRAD, bool CACHED, bool WEIGHTED>
__global__ void __launch_bounds__(32 * kMaxWarps, 2)
nll_kernel(Cols cols, int64_t n, const int64_t* __restrict__ seg_begin,
           const int64_t* __restrict__ seg_end, const int64_t* __restrict__ seg_tiles, int n_seg,
           const Consts* __restrict__ consts,
           double* __restrict__ partials, unsigned* __restrict__ counters, unsigned* __restrict__ gcount,
           unsigned* __restrict__ work, double* __restrict__ out, int n_par, int per_take) {
    constexpr int NA = n_acc(KIND, GRAD);
    const int out_stride = GRAD ? 1 + n_par : 1;
    __shared__ MathTables mt;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n_wib = blockDim.x >> 5;
    double2* const sbuf = reinterpret_cast<double2*>(dyn_smem) + wib * (kSub * 32);
    WarpConsts& wc = reinterpret_cast<WarpConsts*>(dyn_smem + (size_t)n_wib * kSub * 32 * sizeof(double2))[wib];

    load_math_tables(&mt);
    __syncthreads();
    // Launched as a programmatic dependent of the constants kernel: the table
    // load above overlaps it; everything below waits for its results.
    asm volatile("griddepcontrol.wait;" ::: "memory");

    const bool single = seg_begin == nullptr;
    const int64_t total = single ? (n + kTile - 1) / kTile : __ldg(seg_tiles + n_seg);

    // empty segments have no tile to finalise them: block 0 writes their zeros
    if (blockIdx.x == 0) {
        for (int s = threadIdx.x; s < n_seg; s += blockDim.x) {
            const bool empty = single ? (n == 0) : (__ldg(seg_tiles + s + 1) == __ldg(seg_tiles + s));
            if (empty) {
                for (int j = 0; j < out_stride; ++j) out[(size_t)s * out_stride + j] = 0.0;
            }
        }
    }

    // Tiles are handed out dynamically, `per_take` consecutive tiles at a time
    // (work[0] counts the takes), so SMs whose warps finish early take more; a
    // tile's partial does not depend on which warp computes it.  The last warp
    // to leave resets both work counters.
    int cur = -1;
    while (true) {
        unsigned taken = 0;
        if (lane == 0) taken = atomicAdd(work, 1u);
        const int64_t first = (int64_t)__shfl_sync(0xffffffffu, taken, 0) * per_take;
        if (first >= total) break;
        const int64_t stop = first + per_take < total ? first + per_take : total;
        for (int64_t tile = first; tile < stop; ++tile) {
            int seg = 0;
            int64_t t0 = 0, t1 = total, ev0 = 0, ev1 = n;
            if (!single) {
                seg = find_segment(seg_tiles, n_seg, tile);
                t0 = __ldg(seg_tiles + seg);
                t1 = __ldg(seg_tiles + seg + 1);
                ev0 = clamp_off(__ldg(seg_begin + seg), n);
                ev1 = clamp_off(__ldg(seg_end + seg), n);
                if (ev1 < ev0) ev1 = ev0;
            }
            if (seg != cur) {
                load_warp_consts<CACHED>(wc, consts + seg, lane);
                cur = seg;
            }

            double acc[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) acc[a] = 0.0;
            double prod = 1.0;   // unweighted: product of mantissas of P ...
            int esum = 0;        // ... and sum of exponents (log_mul)

            // Events are taken kSub per lane at a time (lane l: l + 32 i).  Those
            // with t <= tcut need the Gaussian and erfcx (about a fifth of them);
            // they are listed in a ballot per i and evaluated packed, 32 per pass,
            // into the warp's buffer, so the FP64 pipe does not spend a full warp
            // instruction on lanes that would discard the result.
            const int64_t tbase = ev0 + (tile - t0) * kTile;
            bool done = false;
            if (KIND == IPA_MODEL_ANGTIME4D && GRAD && !CACHED && tbase + kTile <= ev1) {
                done = tile_fast<WEIGHTED>(wc, &mt, cols, tbase, sbuf, lane, acc, &prod, &esum);
                if (!done) {
#pragma unroll
                    for (int a = 0; a < NA; ++a) acc[a] = 0.0;
                    prod = 1.0;
                    esum = 0;
                }
            }
            if (!done)
                tile_plain<KIND, GRAD, CACHED, WEIGHTED>(wc, &mt, cols, tbase, ev1, sbuf, lane, acc, &prod, &esum);
            acc[0] += log_of(prod, esum, &mt);
            const double share = warp_butterfly<NA>(acc, lane);
            // the group and segment levels; the warp that completes the
            // segment writes its NLL and gradient
            if (!tile_commit<NA>(share, lane, tile, t0, t1, seg, partials, gcount, counters, acc)) continue;
            finalize<KIND, GRAD, CACHED>(wc.c, acc, n_par, out + (size_t)seg * out_stride, lane);
            if (lane == 0) counters[seg] = 0u;
        }
    }
    work_done(work, lane);
}

// seg_tiles[s] = sum_{r<s} tiles(r), tiles(r) = ceil(size_r / kTile) for an active
// segment (0 when active[r] == 0), one block: sequential per thread over a
// contiguous run of segments, then a block scan of the run totals.
__global__ void seg_tiles_kernel(const int64_t* __restrict__ seg_begin, const int64_t* __restrict__ seg_end,
                                 const int* __restrict__ active, int n_seg, int64_t n,
                                 int64_t* __restrict__ seg_tiles) {
    __shared__ int64_t run[1024];
    const int nt = blockDim.x;
    const int per = (n_seg + nt - 1) / nt;
    const int b = threadIdx.x * per;
    const int e = min(n_seg, b + per);
    auto tiles = [&](int s) -> int64_t {
        if (active && !active[s]) return 0;
        const int64_t lo = clamp_off(seg_begin[s], n);
        int64_t hi = clamp_off(seg_end[s], n);
        if (hi < lo) hi = lo;
        return (hi - lo + kTile - 1) / kTile;
    };
    int64_t sum = 0;
    for (int s = b; s < e; ++s) sum += tiles(s);
    run[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < nt; d <<= 1) {
        const int64_t v = threadIdx.x >= d ? run[threadIdx.x - d] : 0;
        __syncthreads();
        run[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t acc = threadIdx.x ? run[threadIdx.x - 1] : 0;
    for (int s = b; s < e; ++s) {
        seg_tiles[s] = acc;
        acc += tiles(s);
    }
    if (threadIdx.x == nt - 1) seg_tiles[n_seg] = run[nt - 1];
}

template <int KIND, bool GRAD, bool CACHED, bool WEIGHTED>
ipa_status launch_t(const Cols& cols, int64_t n, const int64_t* seg_begin, const int64_t* seg_end,
                    const int64_t* seg_tiles, int n_seg, const Consts* consts, Scratch* sc, double* out,
                    int n_par, cudaStream_t st, const LaunchCfg* force) {
    const bool single = seg_begin == nullptr;
    const int64_t tiles = tile_estimate(n, n_seg);
    const LaunchCfg cfg = force ? *force : launch_cfg(KIND, GRAD, CACHED, n_seg > 1, tiles);
    const int W = cfg.warps_per_block >= 1 && cfg.warps_per_block <= kMaxWarps ? cfg.warps_per_block : 1;
    const int K = cfg.tiles_per_take >= 1 ? cfg.tiles_per_take : 1;
    const size_t smem = (size_t)W * (sizeof(WarpConsts) + kSub * 32 * sizeof(double2));
    // resident blocks per SM for each block size (cached per device and variant)
    static int occ[64][kMaxWarps + 1] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int& per_sm = occ[dev & 63][W];
    if (per_sm == 0) {
        int v = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &v, nll_kernel<KIND, GRAD, CACHED, WEIGHTED>, 32 * W, smem);
        per_sm = e == cudaSuccess && v >= 1 ? v : 1;
    }
    const int64_t grid = launch_grid(cfg, W, K, per_sm, tiles, single);
    // programmatic dependent launch: blocks may start (and load their tables)
    // while the constants kernel that precedes every launch is still running
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(32u * W);
    lc.dynamicSmemBytes = smem;
    lc.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cuda_fail(cudaLaunchKernelEx(&lc, nll_kernel<KIND, GRAD, CACHED, WEIGHTED>, cols, n, seg_begin, seg_end,
                                        seg_tiles, n_seg, consts, sc->partials, sc->counters, sc->gcount, sc->work,
                                        out, n_par, K),
                     "likelihood kernel launch");
}

}  // namespace

ipa_status launch_seg_tiles(const int64_t* seg_begin, const int64_t* seg_end, const int* active, int n_seg,
                            int64_t n, int64_t* seg_tiles, cudaStream_t st) {
    seg_tiles_kernel<<<1, 1024, 0, st>>>(seg_begin, seg_end, active, n_seg, n, seg_tiles);
    return cuda_fail(cudaGetLastError(), "segment tiling kernel launch");
}

// Kernel variant for a launch: model, gradient, cached basis, weights.
template <int KIND, bool GRAD, bool CACHED>
ipa_status launch_w(const Cols& cols, int64_t n, const int64_t* seg_begin, const int64_t* seg_end,
                    const int64_t* seg_tiles, int n_seg, const Consts* consts, Scratch* sc, double* out,
                    int n_par, cudaStream_t st, const LaunchCfg* cfg) {
    if (cols.w)
        return launch_t<KIND, GRAD, CACHED, true>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out,
                                                  n_par, st, cfg);
    return launch_t<KIND, GRAD, CACHED, false>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out,
                                               n_par, st, cfg);
}

ipa_status launch_nll(const ModelDev& m, bool grad, const Cols& cols, int64_t n,
                      const int64_t* seg_begin, const int64_t* seg_end, const int64_t* seg_tiles, int n_seg,
                      const Consts* consts, Scratch* sc, double* out, cudaStream_t st, const LaunchCfg* cfg) {
    const int P = m.n_par;
    if (m.kind == IPA_MODEL_TAGGED1D)
        return launch_tag_nll(m, grad, cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, st, cfg);
    if (m.kind == IPA_MODEL_PHIS)
        return launch_phis_nll(m, grad, cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, st, cfg);
    if (m.kind == IPA_MODEL_TIME1D)
        return grad ? launch_w<IPA_MODEL_TIME1D, true, false>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg)
                    : launch_w<IPA_MODEL_TIME1D, false, false>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg);
    if (cols.fk)
        return grad ? launch_w<IPA_MODEL_ANGTIME4D, true, true>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg)
                    : launch_w<IPA_MODEL_ANGTIME4D, false, true>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg);
    return grad ? launch_w<IPA_MODEL_ANGTIME4D, true, false>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg)
                : launch_w<IPA_MODEL_ANGTIME4D, false, false>(cols, n, seg_begin, seg_end, seg_tiles, n_seg, consts, sc, out, P, st, cfg);
}

// f_k = c_k f'_k for every event (the cached angular basis).
__global__ void __launch_bounds__(kNllBlock)
basis_kernel(const double* __restrict__ ck, const double* __restrict__ cl, const double* __restrict__ phi,
             int64_t n, double* __restrict__ fk, int64_t stride) {
    __shared__ MathTables mt;
    load_math_tables(&mt);
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double f[10];
        basis_unscaled(__ldg(ck + e), __ldg(cl + e), __ldg(phi + e), &mt, f);
#pragma unroll
        for (int k = 0; k < 10; ++k) fk[k * stride + e] = kBasisScale[k] * f[k];
    }
}

}  // namespace ipa

extern "C" ipa_status ipa_angular_basis(const ipa_model* model, const ipa_events* ev, double* fk_dev,
                                        int64_t stride, void* stream) {
    using namespace ipa;
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if (model->kind != IPA_MODEL_ANGTIME4D && model->kind != IPA_MODEL_PHIS) {
        set_error("ipa_angular_basis: the model has no angles");
        return IPA_ERR_ARG;
    }
    ipa_events plain = *ev;
    plain.fk = nullptr;
    if ((st = check_events(model, &plain)) != IPA_OK) return st;
    if (!fk_dev || (reinterpret_cast<uintptr_t>(fk_dev) & 15u) || stride < ev->n || (stride & 1)) {
        set_error("ipa_angular_basis: 16-byte aligned output with an even stride >= n required");
        return IPA_ERR_ARG;
    }
    if (ev->n == 0) return IPA_OK;
    const int64_t blocks = (ev->n + kNllBlock - 1) / kNllBlock;
    const int grid = (int)(blocks < 4 * sm_count() * 4 ? blocks : 4 * sm_count() * 4);
    basis_kernel<<<grid, kNllBlock, 0, static_cast<cudaStream_t>(stream)>>>(ev->ck, ev->cl, ev->phi, ev->n, fk_dev,
                                                                            stride);
    return cuda_fail(cudaGetLastError(), "angular basis kernel launch");
}

namespace ipa {

namespace {

ipa_status run(const ipa_model* model, const ipa_events* ev, const int64_t* seg_off, int n_seg,
               const double* theta, double* out, bool grad, void* stream) {
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if ((st = check_events(model, ev)) != IPA_OK) return st;
    if (!theta || !out) {
        set_error("theta and out must be device pointers");
        return IPA_ERR_ARG;
    }
    if (n_seg < 1) {
        set_error("n_seg must be >= 1");
        return IPA_ERR_ARG;
    }
    if (seg_off == nullptr && n_seg != 1) {
        set_error("segment offsets are required for n_seg > 1");
        return IPA_ERR_ARG;
    }
    const int64_t tiles = (ev->n + kTile - 1) / kTile + n_seg;
    Scratch* sc = nullptr;
    if ((st = scratch_get(tiles, n_seg + 1, &sc)) != IPA_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    if ((st = launch_consts(m, theta, n_seg, sc->consts, s)) != IPA_OK) return st;
    if (seg_off) {
        if ((st = launch_seg_tiles(seg_off, seg_off + 1, nullptr, n_seg, ev->n, sc->seg_tiles, s)) != IPA_OK)
            return st;
    }
    const Cols cols{ev->t, ev->ck, ev->cl, ev->phi, ev->w, ev->fk, ev->fk_stride, ev->q};
    return launch_nll(m, grad, cols, ev->n, seg_off, seg_off ? seg_off + 1 : nullptr,
                      seg_off ? sc->seg_tiles : nullptr, n_seg, sc->consts, sc, out, s);
}

// ---- event-sharded likelihood ----
// After a single-segment launch, group g's reduced partial (the sums of its 32
// tiles) sits in the slot of its first tile, g * kGroupTiles.  Copy them out,
// n_groups x na doubles, in group order.
__global__ void group_partials_kernel(const double* __restrict__ partials, int na, int64_t n_groups,
                                      double* __restrict__ out) {
    const int64_t total = n_groups * na;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = i / na;
        out[i] = __ldcg(partials + (g * kGroupTiles) * na + (i - g * na));
    }
}

// The last level of the kernel's reduction (lane l adds groups l, l + 32, ...
// in order, then the butterfly) and the gradient contraction, over group
// partials gathered from several launches: one warp.
template <int KIND, bool CACHED>
__global__ void combine_kernel(const double* __restrict__ groups, int64_t n_groups, const Consts* __restrict__ consts,
                               int n_par, double* __restrict__ out) {
    constexpr int NA = n_acc(KIND, true);
    const int lane = threadIdx.x & 31;
    if (n_groups == 0) {
        for (int j = lane; j < 1 + n_par; j += 32) out[j] = 0.0;
        return;
    }
    double acc[NA];
    gather_butterfly<NA>(reduce_partials<NA>(groups, 0, n_groups, 1, lane), acc);
    finalize<KIND, true, CACHED>(consts[0], acc, n_par, out, lane);
}

}  // namespace
}  // namespace ipa

extern "C" ipa_status ipa_nll(const ipa_model* model, const ipa_events* ev, const double* theta_dev,
                              double* out_dev, void* stream) {
    return ipa::run(model, ev, nullptr, 1, theta_dev, out_dev, false, stream);
}

extern "C" ipa_status ipa_nll_grad(const ipa_model* model, const ipa_events* ev,
                                   const double* theta_dev, double* out_dev, void* stream) {
    return ipa::run(model, ev, nullptr, 1, theta_dev, out_dev, true, stream);
}

extern "C" ipa_status ipa_nll_grad_segmented(const ipa_model* model, const ipa_events* ev,
                                             const int64_t* seg_off_dev, int32_t n_seg,
                                             const double* theta_dev, double* out_dev,
                                             void* stream) {
    if (!seg_off_dev) {
        ipa::set_error("seg_off_dev must not be NULL");
        return IPA_ERR_ARG;
    }
    return ipa::run(model, ev, seg_off_dev, n_seg, theta_dev, out_dev, true, stream);
}


// Group partials of a single-segment call over n events: ceil(n / 16384).
static int64_t shard_groups(int64_t n) {
    const int64_t tiles = (n + ipa::kTile - 1) / ipa::kTile;
    return (tiles + ipa::kGroupTiles - 1) / ipa::kGroupTiles;
}

extern "C" ipa_status ipa_shard_width(const ipa_model* model, int32_t* width) {
    ipa_status st = ipa::check_model(model);
    if (st != IPA_OK) return st;
    if (!width) {
        ipa::set_error("ipa_shard_width: width is NULL");
        return IPA_ERR_ARG;
    }
    *width = ipa::n_acc(model->kind, true);
    return IPA_OK;
}

extern "C" ipa_status ipa_nll_grad_shard(const ipa_model* model, const ipa_events* ev, const double* theta_dev,
                                         double* out_dev, double* groups_dev, void* stream) {
    using namespace ipa;
    if (!groups_dev && ev && ev->n > 0) {
        set_error("ipa_nll_grad_shard: groups_dev is NULL");
        return IPA_ERR_ARG;
    }
    ipa_status st = run(model, ev, nullptr, 1, theta_dev, out_dev, true, stream);
    if (st != IPA_OK || ev->n == 0) return st;
    Scratch* sc = nullptr;
    if ((st = scratch_get((ev->n + kTile - 1) / kTile + 1, 2, &sc)) != IPA_OK) return st;
    const int na = n_acc(model->kind, true);
    const int64_t ng = shard_groups(ev->n);
    const int64_t blocks = (ng * na + 255) / 256;
    group_partials_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        sc->partials, na, ng, groups_dev);
    return cuda_fail(cudaGetLastError(), "group partials copy");
}

extern "C" ipa_status ipa_nll_grad_combine(const ipa_model* model, const double* theta_dev, const double* groups_dev,
                                           int64_t n_groups, int32_t cached, double* out_dev, void* stream) {
    using namespace ipa;
    ipa_status st = check_model(model);
    if (st != IPA_OK) return st;
    if (!theta_dev || !out_dev || n_groups < 0 || (n_groups > 0 && !groups_dev)) {
        set_error("ipa_nll_grad_combine: bad arguments");
        return IPA_ERR_ARG;
    }
    if (cached && model->kind != IPA_MODEL_ANGTIME4D && model->kind != IPA_MODEL_PHIS) {
        set_error("ipa_nll_grad_combine: only models with angles have a cached basis");
        return IPA_ERR_ARG;
    }
    Scratch* sc = nullptr;
    if ((st = scratch_get(1, 2, &sc)) != IPA_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ModelDev m{model->kind, model->n_par, model->t_lo, model->t_hi};
    if ((st = launch_consts(m, theta_dev, 1, sc->consts, s)) != IPA_OK) return st;
    const int P = model->n_par;
    switch (model->kind) {
    case IPA_MODEL_TIME1D:
        combine_kernel<IPA_MODEL_TIME1D, false><<<1, 32, 0, s>>>(groups_dev, n_groups, sc->consts, P, out_dev);
        break;
    case IPA_MODEL_ANGTIME4D:
        if (cached)
            combine_kernel<IPA_MODEL_ANGTIME4D, true><<<1, 32, 0, s>>>(groups_dev, n_groups, sc->consts, P, out_dev);
        else
            combine_kernel<IPA_MODEL_ANGTIME4D, false><<<1, 32, 0, s>>>(groups_dev, n_groups, sc->consts, P, out_dev);
        break;
    case IPA_MODEL_TAGGED1D:
        return launch_tag_combine(groups_dev, n_groups, sc->consts, P, out_dev, s);
    default:
        return launch_phis_combine(groups_dev, n_groups, cached != 0, sc->consts, P, out_dev, s);
    }
    return cuda_fail(cudaGetLastError(), "combine kernel launch");
}
