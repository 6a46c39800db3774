// Step a1 of the hot path: parameter-derived constants, computed on the device
// from theta once per call, so that theta can stay in device memory and calls
// can be captured in CUDA graphs.  Two layouts share every arithmetic step
// (so they give bit-identical records): one thread per fit when many fits are
// evaluated at once, one block per fit when latency matters.
//
// Time part (Sec. 3, analytic normalisation): with F(tau) = [Phi(tau/sigma) -
// g(tau)] / Gamma, dF/dtau = g, the normalisation is I_T = F(t_hi - mu) -
// F(t_lo - mu).  Its derivatives: dF/dGamma = -(F + dg/dGamma) / Gamma,
// dF/dsigma = (-(tau/sigma) G(tau) - dg/dsigma) / Gamma, dF/dmu = -g(tau),
// where dg/dGamma = (Gamma sigma^2 - tau) g - sigma^2 G and
// dg/dsigma = Gamma^2 sigma g - (Gamma sigma + tau/sigma) G.
//
// Angular part (Sec. 4, P wave + S wave): amplitude magnitudes
// |A_0|^2 = (1-F_S) A0sq, |A_perp|^2 = (1-F_S) Apesq,
// |A_par|^2 = (1-F_S)(1 - A0sq - Apesq), |A_S|^2 = F_S, delta_0 = 0, and the
// ten coefficients h_k of the helicity-basis angular functions.
//
// Latency.  For a single fit the record sits in front of every likelihood
// pass, and on this GPU a dependent FP64 operation costs of the order of a
// hundred cycles, so the 4D and 1D records are computed along short chains:
// the edges' erfc and Gaussian through exp(-x^2/2) and the table-driven erfcx
// and exp of fp64_math.cuh (as the event kernel does), every division by a
// parameter as a product with a reciprocal (recip: three FP64 operations), and
// the 70 entries of h and dh/dtheta as products of at most four factors from a
// table, one entry per lane.  The tagged and phi_s models keep the library
// functions of edge().
#pragma once

#include <math.h>

#include "fp64_math.cuh"
#include "ipa_internal.cuh"

namespace ipa {

namespace cdetail {

constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kInvSqrt2 = 0.70710678118654752440;
constexpr double kInvSqrt2Pi = 0.39894228040143267794;
constexpr double kPi = 3.14159265358979323846;

// ---- edge terms with library functions (tagged and phi_s models) ----

__device__ inline double conv_g(double tau, double Gamma, double sigma) {
    const double z = (Gamma * sigma * sigma - tau) / (kSqrt2 * sigma);
    return 0.5 * exp(-Gamma * tau + 0.5 * Gamma * Gamma * sigma * sigma) * erfc(z);
}

__device__ inline double gauss(double tau, double sigma) {
    const double x = tau / sigma;
    return kInvSqrt2Pi / sigma * exp(-0.5 * x * x);
}

// Normal CDF Phi(tau / sigma).
__device__ inline double edge_phi(double tau, double sigma) {
    return 0.5 * erfc(-tau / (kSqrt2 * sigma));
}

// F(tau) and its derivatives (Gamma, sigma, mu) at one edge of the range from
// g(tau), the Gaussian G(tau) and Phi(tau / sigma).
__device__ inline void edge_combine(double tau, double Gamma, double sigma, double g, double G, double Phi,
                                    double* F, double* dF) {
    const double dg_dG = (Gamma * sigma * sigma - tau) * g - sigma * sigma * G;
    const double dg_ds = Gamma * Gamma * sigma * g - (Gamma * sigma + tau / sigma) * G;
    *F = (Phi - g) / Gamma;
    dF[0] = -(*F + dg_dG) / Gamma;
    dF[1] = (-(tau / sigma) * G - dg_ds) / Gamma;
    dF[2] = -g;
}

// F(tau) and its derivatives (Gamma, sigma, mu) at one edge of the range.
__device__ inline void edge(double tau, double Gamma, double sigma, double* F, double* dF) {
    edge_combine(tau, Gamma, sigma, conv_g(tau, Gamma, sigma), gauss(tau, sigma), edge_phi(tau, sigma), F, dF);
}

// The six strong-phase combinations whose sine and cosine enter h_k:
// (dpe - dpa), dpa, dpe, (dpa - dS), (dpe - dS), dS.
__device__ inline double ang_arg(int i, double dpa, double dpe, double dS) {
    switch (i) {
    case 0: return dpe - dpa;
    case 1: return dpa;
    case 2: return dpe;
    case 3: return dpa - dS;
    case 4: return dpe - dS;
    default: return dS;
    }
}

// max |f_k| over the angular box
__device__ inline double basis_max(int k) {
    switch (k) {
    case 0: return 1.0;
    case 1: case 2: case 3: return 0.5;
    case 4: case 5: return kSqrt2 / 4.0;
    case 6: return 1.0 / 3.0;
    case 7: case 8: return 0.40824829046386301637;
    default: return 1.15470053837925152902;
    }
}

// Whether theta lies in the model's domain: Gamma > 0, sigma > 0, f_b in
// [0, 1] and (4D) F_S, |A_0|^2, |A_perp|^2 and |A_par|^2 = 1 - |A_0|^2 -
// |A_perp|^2 in [0, 1] (false for NaN).  Outside, the PDF is not a density.
__device__ inline bool in_domain(const double* th, bool four) {
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], fb = th[IPA_FB];
    bool ok = Gamma > 0.0 && sigma > 0.0 && fb >= 0.0 && fb <= 1.0;
    if (four) {
        const double x0 = th[IPA_A0SQ], xe = th[IPA_APESQ], F = th[IPA_FS];
        ok = ok && F >= 0.0 && F <= 1.0 && x0 >= 0.0 && xe >= 0.0 && x0 + xe <= 1.0;
    }
    return ok;
}

struct AmpParams {
    double x0, xe, xa, s, F, dpa, dpe, dS;
};

__device__ inline AmpParams amp_params(const ModelDev& m, const double* th) {
    AmpParams p{};
    if (m.kind == IPA_MODEL_ANGTIME4D) {
        p.x0 = th[IPA_A0SQ];
        p.xe = th[IPA_APESQ];
        p.dpa = th[IPA_DPA];
        p.dpe = th[IPA_DPE];
        p.F = th[IPA_FS];
        p.dS = th[IPA_DS];
    }
    p.xa = 1.0 - p.x0 - p.xe;
    p.s = 1.0 - p.F;
    return p;
}

// ---- the 4D and 1D record along short chains ----

// 1/d: the FP32 reciprocal (rcp.approx, within 1 ulp) of d's leading 24 bits,
// converted by integer operations, is a seed y with e = 1 - d y below 2^-21;
// 1/d = y (1 + e + e^2 + ...) = y + y (e + e^2) up to y e^3 < 2^-63 relative,
// so the result is within about half an ulp, from three dependent FP64
// operations instead of the seven or so of a division.  Outside 2^-125 <= |d|
// < 2^126 (0, infinities and NaN included) the division itself.
__device__ inline double recip(double d) {
    const long long b = __double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e < 1023 - 125 || e > 1023 + 125) return 1.0 / d;
    const unsigned xf = ((unsigned)((unsigned long long)b >> 32) & 0x80000000u) |
                        ((unsigned)(e - 1023 + 127) << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu);
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__uint_as_float(xf)));
    const unsigned yu = __float_as_uint(yf);
    const long long yb = ((long long)(yu & 0x80000000u) << 32) |
                         ((long long)(((yu >> 23) & 0xFFu) - 127 + 1023) << 52) | ((long long)(yu & 0x7FFFFFu) << 29);
    const double y = __longlong_as_double(yb);
    const double r = fma(-d, y, 1.0);
    return fma(y, fma(r, r, r), y);
}

// Products of theta used by the record and by the edges.
struct TimeScalars {
    double Gamma, sigma, mu, fb;
    double c_exp;            // Gamma^2 sigma^2 / 2
    double Gs2, s2, G2s, Gsig;
};

__device__ inline TimeScalars time_scalars_of(double Gamma, double sigma, double mu, double fb) {
    TimeScalars s;
    s.Gamma = Gamma;
    s.sigma = sigma;
    s.mu = mu;
    s.fb = fb;
    s.c_exp = 0.5 * s.Gamma * s.Gamma * s.sigma * s.sigma;
    s.Gs2 = s.Gamma * s.sigma * s.sigma;
    s.s2 = s.sigma * s.sigma;
    s.G2s = s.Gamma * s.Gamma * s.sigma;
    s.Gsig = s.Gamma * s.sigma;
    return s;
}

__device__ inline TimeScalars time_scalars(const double* th) {
    return time_scalars_of(th[IPA_GAMMA], th[IPA_SIGMA], th[IPA_MU], th[IPA_FB]);
}

// Edge e of the range (0: t_hi, 1: t_lo) as tau = t_e - mu.
__device__ inline double edge_tau(const ModelDev& m, double mu, int e) { return (e == 0 ? m.t_hi : m.t_lo) - mu; }

// With x = tau / sigma: the argument z = (Gamma sigma^2 - tau) / (sqrt2 sigma)
// = (Gamma sigma - x) / sqrt2 of the erfc in g(tau), the argument w =
// -x / sqrt2 of the erfc in Phi(x) = erfc(w) / 2, and the exponents of the
// Gaussian factor gq = exp(-x^2 / 2) and of E = exp(-Gamma tau + Gamma^2
// sigma^2 / 2).
__device__ inline double edge_z(const TimeScalars& s, double x) { return (s.Gsig - x) * kInvSqrt2; }
__device__ inline double edge_w(double x) { return neg_bits(x) * kInvSqrt2; }
__device__ inline double gauss_exponent(double x) { return (-0.5 * x) * x; }
__device__ inline double decay_exponent(const TimeScalars& s, double tau) { return fma(-s.Gamma, tau, s.c_exp); }

// erfcx at the argument w of one of an edge's erfc terms: erfc(w) = e^{-w^2}
// erfcx(w) for w >= 0 and 2 - e^{-w^2} erfcx(-w) for w < 0.  For w < -6.25
// the erfcx term is below 1e-18 of the term beside it (E for g, 1 for Phi)
// and leaves the sum unchanged in double precision: 0 without evaluating it.
__device__ inline double edge_erfcx(double w, const MathTables* t) {
    return below_neg(w, -6.25) ? 0.0 : erfcx_fast(abs_bits(w), t);
}

// g(tau) = E erfc(z) / 2, Phi(x) = erfc(w) / 2 and the Gaussian G(tau) = cG gq
// at one edge from gq = exp(-x^2/2) = E e^{-z^2} = e^{-w^2} and the erfcx
// values X1 (at z) and X2 (at w).
__device__ inline void edge_values(double z, double w, double gq, double E, double X1, double X2, double cG,
                                   double* g, double* Phi, double* G) {
    const double a = 0.5 * (gq * X1);
    *g = negative(z) ? E - a : a;
    const double b = 0.5 * (gq * X2);
    *Phi = negative(w) ? 1.0 - b : b;
    *G = cG * gq;
}

// F(tau) and its derivatives (Gamma, sigma, mu) at one edge (see the top of
// this file), with x = tau / sigma and rG = 1 / Gamma as factors.
__device__ inline void edge_combine_r(const TimeScalars& s, double tau, double x, double rG, double g, double G,
                                      double Phi, double* F, double* dF) {
    const double dg_dG = (s.Gs2 - tau) * g - s.s2 * G;
    const double dg_ds = s.G2s * g - (s.Gsig + x) * G;
    *F = (Phi - g) * rG;
    dF[0] = -(*F + dg_dG) * rG;
    dF[1] = (-(x * G) - dg_ds) * rG;
    dF[2] = -g;
}

// The scalars of the record that need theta only (rs = 1 / sigma, rV = 1 / V).
// For theta outside the domain cb is NaN (and cs, written with the divisions
// by I_T), so that every P, the NLL and the gradient are NaN (the fitter
// reports such a point as IPA_FIT_BAD_PDF).
__device__ inline void write_time_scalars(const TimeScalars& s, double rs, double rV, bool ok, Consts* c) {
    c->Gamma = s.Gamma;
    c->sigma = s.sigma;
    c->mu = s.mu;
    c->fb = s.fb;
    c->c_exp = s.c_exp;
    c->Gs2 = s.Gs2;
    c->k_z = rs * kInvSqrt2;
    c->k_g = 0.5 * (rs * rs);
    c->cG = kInvSqrt2Pi * rs;
    c->s2 = s.s2;
    c->G2s = s.G2s;
    c->Gsig = s.Gsig;
    c->inv_s = rs;
    c->cb = ok ? s.fb * rV : NAN;
    c->inv_V = rV;
    c->pad_ = 0.0;
}

// The range's volume V (t_hi - t_lo, times 8 pi for the angles) and the
// angular integral I_Omega of the 4D model.
__device__ inline double volume(const ModelDev& m) {
    const double span = m.t_hi - m.t_lo;
    return m.kind == IPA_MODEL_ANGTIME4D ? span * 8.0 * kPi : span;
}
__device__ inline double omega_integral(const ModelDev& m) {
    return m.kind == IPA_MODEL_ANGTIME4D ? 16.0 * kPi / 9.0 : 1.0;
}

// M_T = min(1, E) at t_lo (1 for NaN E), by a bit comparison.
__device__ inline double time_envelope(double E_lo) { return above(E_lo, 1.0) ? 1.0 : E_lo; }

// Item j of the divisions by I_T: (dI_T/dtheta_j) / I_T for j < 3 (dIT_j
// given), cs = (1 - f_b) / (I_T I_Omega) for j = 3, 1 / (I_T I_Omega) for j = 4.
__device__ inline double it_item(int j, double IT, double IO, double dIT_j, double fb) {
    const double den = j < 3 ? IT : IT * IO;
    const double num = j < 3 ? dIT_j : (j == 3 ? 1.0 - fb : 1.0);
    return num * recip(den);
}

// The factors of h_k and dh_k/dtheta_j (index: value):
//   0: 1, 1: s = 1 - F, 2: x0, 3: xa, 4: xe, 5: F, 6: sqrt xa, 7: sqrt xe,
//   8: sqrt x0, 9: sqrt F sqrt s, 10: 1/(2 sqrt xa sqrt xe), 11: 1/(2 sqrt x0
//   sqrt xa), 12: 1/(2 sqrt x0 sqrt xe), 13: 1/(2 sqrt xa), 14: 1/(2 sqrt xe),
//   15: 1/(2 sqrt x0), 16: (1 - 2F)/(2 sqrt F sqrt s), 17: xa - xe,
//   18: xa - x0, 19-24: sine and 25-30: cosine of ang_arg 0-5,
// with x0 = A0sq, xe = Apesq, xa = 1 - x0 - xe and F = F_S.
constexpr int kAngFactors = 31;

// Factors 0-5, 17 and 18 (no transcendental function).
__device__ inline double plain_factor(int i, const AmpParams& p) {
    switch (i) {
    case 0: return 1.0;
    case 1: return p.s;
    case 2: return p.x0;
    case 3: return p.xa;
    case 4: return p.xe;
    case 5: return p.F;
    case 17: return p.xa - p.xe;
    default: return p.xa - p.x0;
    }
}
__device__ inline int plain_factor_index(int i) { return i < 6 ? i : 11 + i; }   // i = 0..7
constexpr int kPlainFactors = 8;

// Square root i (0..4) is taken of x0, xa, xe, F, s.
__device__ inline double sqrt_in(int i, const AmpParams& p) {
    return i == 0 ? p.x0 : (i == 1 ? p.xa : (i == 2 ? p.xe : (i == 3 ? p.F : p.s)));
}

// Factors 9-16 as m (k (a b)): the sources of a and b (0-4: square root i,
// 5-9: its reciprocal, 10: one), k = 1 for factor 9 and 1/2 otherwise, m =
// 1 - 2F for factor 16 and 1 otherwise.
__device__ inline int combo_a(int i) {
    return i == 0 ? 3 : (i == 1 ? 6 : (i == 2 ? 5 : (i == 3 ? 5 : (i == 4 ? 6 : (i == 5 ? 7 : (i == 6 ? 5 : 8))))));
}
__device__ inline int combo_b(int i) {
    return i == 0 ? 4 : (i == 1 ? 7 : (i == 2 ? 6 : (i == 3 ? 7 : (i == 7 ? 9 : 10))));
}
__device__ inline double combo(int i, double a, double b, double omtF) {
    return (i == 7 ? omtF : 1.0) * ((i == 0 ? 1.0 : 0.5) * (a * b));
}
constexpr int kComboFactors = 8;

// Entry e of the record's h (e < 10) and dh (10 + 6k + j, j over A0sq,
// Apesq, delta_pa, delta_pe, F_S, delta_S): the product of the factors of
// its four 5-bit fields (0 in an unused field is the factor 1), negated if
// bit 30 is set, 0 if bit 31 is set.
constexpr unsigned kNeg = 1u << 30, kZero = 1u << 31;
constexpr unsigned fac(unsigned a, unsigned b = 0, unsigned c = 0, unsigned d = 0) {
    return a | b << 5 | c << 10 | d << 15;
}
constexpr int kRowEntries = 70;
__device__ const unsigned kRowSpec[kRowEntries] = {
    // h_0 .. h_9: s x0, s xa, s xe, s ra re s4, s r0 ra c5, s r0 re s6, F,
    // rFs ra c8, rFs re s9, rFs r0 c10
    fac(1, 2), fac(1, 3), fac(1, 4), fac(1, 6, 7, 19), fac(1, 8, 6, 26), fac(1, 8, 7, 21), fac(5),
    fac(9, 6, 28), fac(9, 7, 23), fac(9, 8, 30),
    // dh_0 .. dh_2
    fac(1), kZero, kZero, kZero, kNeg | fac(2), kZero,
    kNeg | fac(1), kNeg | fac(1), kZero, kZero, kNeg | fac(3), kZero,
    kZero, fac(1), kZero, kZero, kNeg | fac(4), kZero,
    // dh_3
    kNeg | fac(1, 4, 10, 19), fac(1, 17, 10, 19), kNeg | fac(1, 6, 7, 25), fac(1, 6, 7, 25),
    kNeg | fac(6, 7, 19), kZero,
    // dh_4
    fac(1, 18, 11, 26), kNeg | fac(1, 2, 11, 26), kNeg | fac(1, 8, 6, 20), kZero, kNeg | fac(8, 6, 26), kZero,
    // dh_5
    fac(1, 4, 12, 21), fac(1, 2, 12, 21), kZero, fac(1, 8, 7, 27), kNeg | fac(8, 7, 21), kZero,
    // dh_6
    kZero, kZero, kZero, kZero, fac(0), kZero,
    // dh_7
    kNeg | fac(9, 13, 28), kNeg | fac(9, 13, 28), kNeg | fac(9, 6, 22), kZero, fac(16, 6, 28), fac(9, 6, 22),
    // dh_8
    kZero, fac(9, 14, 23), kZero, fac(9, 7, 29), fac(16, 7, 23), kNeg | fac(9, 7, 29),
    // dh_9
    fac(9, 15, 30), kZero, kZero, kZero, fac(16, 8, 30), kNeg | fac(9, 8, 24),
};

__device__ inline double row_entry(unsigned spec, const double* f) {
    const double v = ((f[spec & 31u] * f[(spec >> 5) & 31u]) * f[(spec >> 10) & 31u]) * f[(spec >> 15) & 31u];
    return (spec & kZero) ? 0.0 : ((spec & kNeg) ? neg_bits(v) : v);
}

// M_Omega = sum_k |h_k| max|f_k| added pairwise in a fixed order:
// ((a_0 + a_1) + (a_2 + a_3)) + a_4 with a_i = p_2i + p_2i+1.
__device__ inline double mo_sum(const double* h) {
    double a[5];
    for (int i = 0; i < 5; ++i)
        a[i] = abs_bits(h[2 * i]) * basis_max(2 * i) + abs_bits(h[2 * i + 1]) * basis_max(2 * i + 1);
    return ((a[0] + a[1]) + (a[2] + a[3])) + a[4];
}

// The tables of exp_fast, sincos_fast and erfcx_fast into shared memory
// (block-cooperative; the caller syncs).
__device__ inline void load_consts_tables(MathTables* t) {
    using namespace fp64tab;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        t->exp2[i] = kExp2Tab[i];
        t->sn[i] = kSinTab[i];
        t->cs[i] = kCosTab[i];
    }
    for (int i = threadIdx.x; i < kErfcxPieces * kErfcxCoeffs; i += blockDim.x) t->ex[i] = kErfcxTab[i];
}

}  // namespace cdetail

// One thread computes one Consts record: used when many fits are evaluated at
// once (batched fits, the server), where lanes of a warp hold different fits
// and every FP64 instruction does useful work in all of them.  mt holds the
// tables of load_consts_tables.
__device__ inline void compute_consts_thread(const ModelDev& m, const double* th, const MathTables* mt, Consts* c) {
    using namespace cdetail;
    const bool four = m.kind == IPA_MODEL_ANGTIME4D;
    const bool ok = in_domain(th, four);
    const TimeScalars s = time_scalars(th);
    const double rs = recip(s.sigma), rG = recip(s.Gamma), rV = recip(volume(m));
    double F[2], dF[2][3];
    for (int e = 0; e < 2; ++e) {
        const double tau = edge_tau(m, s.mu, e);
        const double x = tau * rs;
        const double z = edge_z(s, x), w = edge_w(x);
        const double X1 = edge_erfcx(z, mt), X2 = edge_erfcx(w, mt);
        const double gq = exp_fast(gauss_exponent(x), mt), E = exp_fast(decay_exponent(s, tau), mt);
        double g, Phi, G;
        edge_values(z, w, gq, E, X1, X2, kInvSqrt2Pi * rs, &g, &Phi, &G);
        edge_combine_r(s, tau, x, rG, g, G, Phi, &F[e], dF[e]);
        if (e == 1) c->MT = time_envelope(E);
    }
    write_time_scalars(s, rs, rV, ok, c);
    const double IT = F[0] - F[1], IO = omega_integral(m);
    c->IT = IT;
    for (int j = 0; j < 3; ++j) c->dlnIT[j] = it_item(j, IT, IO, dF[0][j] - dF[1][j], s.fb);
    c->cs = ok ? it_item(3, IT, IO, 0.0, s.fb) : NAN;
    c->inv_ITIO = it_item(4, IT, IO, 0.0, s.fb);
    double* hd = &c->h[0];      // h[10] and dh[10][6], contiguous
    if (four) {
        const AmpParams p = amp_params(m, th);
        double f[kAngFactors];
        for (int i = 0; i < kPlainFactors; ++i) f[plain_factor_index(i)] = plain_factor(plain_factor_index(i), p);
        for (int i = 0; i < 6; ++i) sincos_fast(ang_arg(i, p.dpa, p.dpe, p.dS), mt, &f[19 + i], &f[25 + i]);
        double r[11];            // square roots, their reciprocals, one (the sources of combo)
        for (int i = 0; i < 5; ++i) {
            r[i] = sqrt(sqrt_in(i, p));
            r[5 + i] = recip(r[i]);
        }
        r[10] = 1.0;
        f[8] = r[0];
        f[6] = r[1];
        f[7] = r[2];
        const double omtF = 1.0 - 2.0 * p.F;
        for (int i = 0; i < kComboFactors; ++i) f[9 + i] = combo(i, r[combo_a(i)], r[combo_b(i)], omtF);
        for (int i = 0; i < kRowEntries; ++i) hd[i] = row_entry(kRowSpec[i], f);
        c->MO = mo_sum(c->h);
    } else {
        for (int i = 0; i < kRowEntries; ++i) hd[i] = i == 0 ? 1.0 : 0.0;
        c->MO = 1.0;
    }
}

// Exchange buffer of compute_consts_block.
struct ConstsBlockScratch {
    MathTables mt;
    double th[IPA_NPAR_4D];        // theta
    double f[32];                  // angular factors
    double X1[2], X2[2], gq[2], E[2];   // edge 0: t_hi, edge 1: t_lo
    double rG;
    double F[2], dF[2][3];
    int ok;                        // theta in the domain
    Consts c;                      // the record, copied out at the end
};
constexpr int kConstsBlock = 192;

// One block of six warps computes one Consts record: a single fit, where
// latency matters.  A warp's FP64 instruction occupies its sub-partition's
// FP64 unit for tens of cycles whatever the active lanes, and a dependent one
// waits for the one before, so independent chains go to different warps and,
// within a warp, to lanes running the same code:
//   phase 1  warp 0: erfcx at z (both edges); warp 1: erfcx at w; warp 2: the
//            Gaussian factor and E (both edges); warp 3: six sine/cosine pairs;
//            warp 4: five square roots, their reciprocals and the products
//            among them (shuffles), the plain factors; warp 5: 1/Gamma and the
//            scalars that need theta only;
//   phase 2  warp 0: g, Phi, G, F and its derivatives at both edges, M_T;
//            warps 1-3: the 70 entries of h and dh, one per lane;
//   phase 3  warp 0: I_T and the five divisions by it; warp 1: M_Omega
//            (shuffle tree);
// then every thread copies part of the record out.  Every value comes from the
// same expression as in compute_consts_thread, so both give the same bits
// (this file is compiled without FMA contraction).
__device__ inline void compute_consts_block(const ModelDev& m, const double* th, Consts* c, ConstsBlockScratch* S) {
    using namespace cdetail;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool four = m.kind == IPA_MODEL_ANGTIME4D;
    const int row = (int)threadIdx.x - 32;             // warps 1-3: entry of h / dh
    const unsigned spec = four && row >= 0 && row < kRowEntries ? kRowSpec[row] : 0u;
    // theta and the tables come from memory together; everything after the
    // barrier reads them from shared memory
    if (threadIdx.x < (four ? IPA_NPAR_4D : IPA_NPAR_1D)) S->th[threadIdx.x] = th[threadIdx.x];
    load_consts_tables(&S->mt);
    __syncthreads();
    th = S->th;

    const TimeScalars s = time_scalars(th);
    const int e = lane & 1;
    double tau = 0.0, x = 0.0, z = 0.0, rs = 0.0, X1 = 0.0;
    if (w <= 2 && lane < 4) {
        rs = recip(s.sigma);
        tau = edge_tau(m, s.mu, e);
        x = tau * rs;
    }
    if (w == 0) {
        if (lane < 2) {
            z = edge_z(s, x);
            X1 = edge_erfcx(z, &S->mt);
        }
    } else if (w == 1) {
        if (lane < 2) S->X2[e] = edge_erfcx(edge_w(x), &S->mt);
    } else if (w == 2) {
        if (lane < 4) {
            const double v = exp_fast(lane < 2 ? gauss_exponent(x) : decay_exponent(s, tau), &S->mt);
            if (lane < 2) S->gq[e] = v;
            else S->E[e] = v;
        }
    } else if (w == 3) {
        if (four && lane < 6) {
            const AmpParams p = amp_params(m, th);
            sincos_fast(ang_arg(lane, p.dpa, p.dpe, p.dS), &S->mt, &S->f[19 + lane], &S->f[25 + lane]);
        }
    } else if (w == 4) {
        if (four) {
            const AmpParams p = amp_params(m, th);
            double r = 0.0, ir = 0.0;
            if (lane < 5) {
                r = sqrt(sqrt_in(lane, p));
                ir = recip(r);
            }
            const int ia = combo_a(lane & 7), ib = combo_b(lane & 7);
            const double ra = __shfl_sync(0xffffffffu, r, ia % 5), ira = __shfl_sync(0xffffffffu, ir, ia % 5);
            const double rb = __shfl_sync(0xffffffffu, r, ib % 5), irb = __shfl_sync(0xffffffffu, ir, ib % 5);
            const double a = ia < 5 ? ra : ira;
            const double b = ib == 10 ? 1.0 : (ib < 5 ? rb : irb);
            if (lane < kComboFactors) S->f[9 + lane] = combo(lane, a, b, 1.0 - 2.0 * p.F);
            if (lane < 3) S->f[lane == 0 ? 8 : 5 + lane] = r;
            if (lane >= 16 && lane < 16 + kPlainFactors) {
                const int i = plain_factor_index(lane - 16);
                S->f[i] = plain_factor(i, p);
            }
        }
    } else if (w == 5) {
        if (lane == 0) {
            const bool ok = in_domain(th, four);
            S->ok = ok;
            S->rG = recip(s.Gamma);
            write_time_scalars(s, recip(s.sigma), recip(volume(m)), ok, &S->c);
        }
    }
    __syncthreads();

    double* hd = &S->c.h[0];   // h[10] and dh[10][6], contiguous
    if (w == 0) {
        if (lane < 2) {
            double g, Phi, G;
            edge_values(z, edge_w(x), S->gq[e], S->E[e], X1, S->X2[e], kInvSqrt2Pi * rs, &g, &Phi, &G);
            edge_combine_r(s, tau, x, S->rG, g, G, Phi, &S->F[e], S->dF[e]);
            if (e == 1) S->c.MT = time_envelope(S->E[1]);
        }
    } else if (row >= 0 && row < kRowEntries) {
        hd[row] = four ? row_entry(spec, S->f) : (row == 0 ? 1.0 : 0.0);
    }
    __syncthreads();

    if (w == 0) {
        if (lane < 5) {
            const double IT = S->F[0] - S->F[1];
            const double dIT = lane < 3 ? S->dF[0][lane] - S->dF[1][lane] : 0.0;
            const double v = it_item(lane, IT, omega_integral(m), dIT, s.fb);
            if (lane < 3) S->c.dlnIT[lane] = v;
            else if (lane == 3) S->c.cs = S->ok ? v : NAN;
            else S->c.inv_ITIO = v;
            if (lane == 0) S->c.IT = IT;
        }
    } else if (w == 1) {
        // a_i = p_2i + p_2i+1 in lane 2i, then ((a_0 + a_1) + (a_2 + a_3)) + a_4 as in mo_sum
        const double p = four && lane < 10 ? abs_bits(hd[lane]) * basis_max(lane) : 0.0;
        const double a = p + __shfl_down_sync(0xffffffffu, p, 1);
        const double b = a + __shfl_down_sync(0xffffffffu, a, 2);
        const double q = b + __shfl_down_sync(0xffffffffu, b, 4);
        const double a4 = __shfl_sync(0xffffffffu, a, 8);
        if (lane == 0) S->c.MO = four ? q + a4 : 1.0;
    }
    __syncthreads();
    const double* src = reinterpret_cast<const double*>(&S->c);
    double* dst = reinterpret_cast<double*>(c);
    for (int i = threadIdx.x; i < kConstsDoubles; i += blockDim.x) dst[i] = src[i];
}

}  // namespace ipa
