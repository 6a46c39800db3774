// The flavour-tagged decay-time model with B_s oscillation (Sec. 4, the
// B_s -> J/psi phi example; Sec. 2 for the Faddeeva function): parameter
// constants and the exact per-event signal used by the generator.
//
// Model (the paper prints no formula; the reading is stated in ipanema.h):
//   S(t, q) = aH g(tau; Gamma_H) + aL g(tau; Gamma_L) + q Ds Im g(tau; z),
//   aH = (1 - cos phi_s)/2, aL = (1 + cos phi_s)/2, Ds = (1 - 2 omega) sin phi_s,
//   Gamma_H,L = Gamma -+ DG/2, z = Gamma - i Dm, tau = t - mu,
//   g(tau; z) = int_0^inf e^{-z u} G(tau - u; sigma) du
//             = 1/2 exp(-z tau + z^2 sigma^2/2) erfc(u),  u = (z sigma^2 - tau) / (sqrt2 sigma).
// With Gx = exp(-tau^2 / (2 sigma^2)) = exp(-z tau + z^2 sigma^2/2 - u^2) and
// the Faddeeva function w (erfc(u) = e^{-u^2} w(i u)):
//   Re u >= 0:  2 g = Gx w(i u),
//   Re u <  0:  2 g = 2 exp(-z tau + z^2 sigma^2/2) - Gx w(-i u),
// where for u = a - i b (a = (Gamma sigma^2 - tau)/(sqrt2 sigma), b = Dm sigma /
// sqrt2) i u = b + i a and -i u = -b - i a: both lie in the upper half plane
// on the branch taken.  For real z, w(i a) = erfcx(a).
// Normalisation over [t_lo, t_hi] and both tags (the q term is odd in q):
//   N = (1 - c) I(Gamma_H) + (1 + c) I(Gamma_L),  I(x) = F(t_hi - mu) - F(t_lo - mu),
// with F the antiderivative of the real convolution (consts.cuh), and
//   P = (1 - f_b) S / N + f_b / (2 (t_hi - t_lo)).
#pragma once

#include <math.h>

#include "consts.cuh"
#include "faddeeva.cuh"
#include "fp64_math.cuh"
#include "int_math.cuh"
#include "ipa_internal.cuh"

namespace ipa {

// Parameter constants of the tagged model, stored in a Consts slot of the
// library scratch (one per segment).
struct TagConsts {
    double Gamma, sigma, mu, fb, DG, Dm, phi, om;   // theta
    double GH, GL;        // Gamma_H = Gamma - DG/2, Gamma_L = Gamma + DG/2
    double k_z;           // 1 / (sqrt2 sigma)
    double k_g;           // 1 / (2 sigma^2)
    double cG;            // 1 / (sqrt(2 pi) sigma): G = cG Gx
    double s2;            // sigma^2
    double inv_s;         // 1 / sigma
    double cH2, cL2, cC2; // exponent offsets: x^2 sigma^2/2 + ln2 (x = Gamma_H, Gamma_L), (Gamma^2 - Dm^2) sigma^2/2 + ln2
    double uH0, uL0, uC0; // Gamma_H sigma^2, Gamma_L sigma^2, Gamma sigma^2
    double beta;          // Dm sigma^2 k_z = Dm sigma / sqrt2 (minus the imaginary part of u)
    double ph0;           // Gamma Dm sigma^2: phase of the complex exponential = Dm tau - ph0
    double aH, aL, Ds, D, c, s;   // mixing weights; D = 1 - 2 omega, c, s = cos, sin phi_s
    double qH, qL, qD;    // aH cs/2, aL cs/2, Ds cs/2: P = qH 2gH + qL 2gL + q qD 2Im g + cb
    double cs;            // (1 - f_b) / N
    double cb;            // f_b / (2 (t_hi - t_lo))
    double inv_N, inv_V2, N;
    double dlnN[8];       // (dN / dtheta_j) / N
    double tcut;          // t above it: every erfc term of the event is below 1e-17 of its exponential
    double MS;            // generator envelope: max of S over the range and both tags (upper bound)
    double pad_;
};
static_assert(sizeof(TagConsts) <= sizeof(Consts), "TagConsts must fit a Consts slot");
static_assert(sizeof(TagConsts) % 16 == 0, "TagConsts must be a multiple of 16 bytes");
constexpr int kTagConstsDoubles = sizeof(TagConsts) / sizeof(double);

namespace tdetail {

constexpr double kLn2 = 0.69314718055994530942;

// min(1, e^{-x (t_lo - mu) + x^2 sigma^2 / 2}), in the operation order of a
// plain left-to-right evaluation.  For x >= 0 and tau >= t_lo - mu it bounds
// g(tau; x): the integrand e^{-x u} G(tau - u) is positive, so g is below its
// integral over all u, e^{-x tau + x^2 sigma^2 / 2}, and below the Gaussian's
// mass 1; |g(tau; x - i Dm)| <= g(tau; x) likewise.
__device__ inline double env_bound(double x, double t_lo, double mu, double sigma) {
    const double a = __dmul_rn(-x, __dsub_rn(t_lo, mu));
    const double b = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(0.5, x), x), sigma), sigma);
    return fmin(1.0, exp(__dadd_rn(a, b)));
}

}  // namespace tdetail

// theta (8 values) -> the record.
// The transcendental inputs of the record, independent of one another (see
// tag_piece): evaluated side by side by four warps for a few segments.
struct TagPieces {
    double F[4], dF[4][3];     // edge(): (t_hi, Gamma_H), (t_lo, Gamma_H), (t_hi, Gamma_L), (t_lo, Gamma_L)
    double sn, cn;             // sincos(phi_s)
    double M[3];               // env_bound of Gamma_H, Gamma_L, Gamma
    double tq;                 // sqrt(39.1 + beta^2)
};
constexpr int kTagPieces = 9;

// Piece k: 0-3 the edges, 4 sincos(phi_s), 5-7 the envelope bounds, 8 the cut's root.
__device__ inline void tag_piece(const ModelDev& m, const double* th, int k, TagPieces* p) {
    using namespace cdetail;
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], mu = th[IPA_MU], DG = th[IPA_DG];
    const double GH = Gamma - 0.5 * DG, GL = Gamma + 0.5 * DG;
    if (k < 4) {
        edge((k & 1) ? m.t_lo - mu : m.t_hi - mu, k < 2 ? GH : GL, sigma, &p->F[k], p->dF[k]);
    } else if (k == 4) {
        sincos(th[IPA_PHIS], &p->sn, &p->cn);
    } else if (k < 8) {
        p->M[k - 5] = tdetail::env_bound(k == 5 ? GH : (k == 6 ? GL : Gamma), m.t_lo, mu, sigma);
    } else {
        const double beta = th[IPA_DM] * sigma / kSqrt2;
        p->tq = sqrt(39.1 + beta * beta);
    }
}

__device__ inline void compute_tag_consts(const ModelDev& m, const double* th, const TagPieces* pc, TagConsts* c) {
    using namespace cdetail;
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], mu = th[IPA_MU], fb = th[IPA_FB];
    const double DG = th[IPA_DG], Dm = th[IPA_DM], phi = th[IPA_PHIS], om = th[IPA_OMEGA];
    const double GH = Gamma - 0.5 * DG, GL = Gamma + 0.5 * DG;
    const double FhH = pc->F[0], FlH = pc->F[1], FhL = pc->F[2], FlL = pc->F[3];
    const double *dFhH = pc->dF[0], *dFlH = pc->dF[1], *dFhL = pc->dF[2], *dFlL = pc->dF[3];
    const double IH = FhH - FlH, IL = FhL - FlL;
    const double sn = pc->sn, cn = pc->cn;
    const double D = 1.0 - 2.0 * om;
    const double wH = 1.0 - cn, wL = 1.0 + cn;
    const double N = wH * IH + wL * IL;
    double dN[8];
    for (int j = 0; j < 3; ++j) dN[j] = wH * (dFhH[j] - dFlH[j]) + wL * (dFhL[j] - dFlL[j]);
    dN[3] = 0.0;
    dN[4] = -0.5 * wH * (dFhH[0] - dFlH[0]) + 0.5 * wL * (dFhL[0] - dFlL[0]);
    dN[5] = 0.0;
    dN[6] = sn * IH - sn * IL;
    dN[7] = 0.0;
    const double inv_N = 1.0 / N;
    const double V2 = 2.0 * (m.t_hi - m.t_lo);
    c->Gamma = Gamma;
    c->sigma = sigma;
    c->mu = mu;
    c->fb = fb;
    c->DG = DG;
    c->Dm = Dm;
    c->phi = phi;
    c->om = om;
    c->GH = GH;
    c->GL = GL;
    c->k_z = 1.0 / (kSqrt2 * sigma);
    c->k_g = 1.0 / (2.0 * sigma * sigma);
    c->cG = kInvSqrt2Pi / sigma;
    c->s2 = sigma * sigma;
    c->inv_s = 1.0 / sigma;
    c->cH2 = 0.5 * GH * GH * sigma * sigma + tdetail::kLn2;
    c->cL2 = 0.5 * GL * GL * sigma * sigma + tdetail::kLn2;
    c->cC2 = 0.5 * (Gamma - Dm) * (Gamma + Dm) * sigma * sigma + tdetail::kLn2;
    c->uH0 = GH * sigma * sigma;
    c->uL0 = GL * sigma * sigma;
    c->uC0 = Gamma * sigma * sigma;
    c->beta = Dm * sigma / kSqrt2;
    c->ph0 = Gamma * Dm * sigma * sigma;
    c->aH = 0.5 * wH;
    c->aL = 0.5 * wL;
    c->Ds = D * sn;
    c->D = D;
    c->c = cn;
    c->s = sn;
    const double cs = (1.0 - fb) * inv_N;
    c->cs = cs;
    c->qH = 0.5 * cs * c->aH;
    c->qL = 0.5 * cs * c->aL;
    c->qD = 0.5 * cs * c->Ds;
    c->cb = fb / V2;
    c->inv_N = inv_N;
    c->inv_V2 = 1.0 / V2;
    c->N = N;
    for (int j = 0; j < 8; ++j) c->dlnN[j] = dN[j] * inv_N;
    // t > tcut: Re u <= -sqrt(39.1 + b^2) for all three rates, so |e^{-u^2} w|
    // <= e^{-39.1} ~ 1e-17 relative to the exponential, and Gx < 1e-17
    const double rmax = fmax(fmax(GH, GL), Gamma);
    const double tc = mu + (rmax * sigma * sigma + pc->tq * kSqrt2 * sigma);
    c->tcut = tc == tc ? tc : INFINITY;
    const double MH = pc->M[0], ML = pc->M[1], MC = pc->M[2];
    c->MS = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(0.5, __dsub_rn(1.0, cn)), MH),
                                __dmul_rn(__dmul_rn(0.5, __dadd_rn(1.0, cn)), ML)),
                      __dmul_rn(fabs(__dmul_rn(D, sn)), MC));
}

// The slow-branch values of one event (t <= tcut), with Gx = exp(-tau^2 /
// (2 sigma^2)):
//   xH = Gx erfcx(|uH|), xL = Gx erfcx(|uL|)  (uH,L = (Gamma_H,L sigma^2 - tau) k_z),
//   (wr, wi) = Gx w(+-beta + i |a|)          (a = (Gamma sigma^2 - tau) k_z),
//   gx = Gx.
// The sign bits of xH, xL and gx carry uH >= 0, uL >= 0 and a >= 0: then 2g is
// the stored value itself, otherwise 2 E minus it.  Events with t > tcut use
// all zeros (2g = 2E, Gaussian 0).  C is any constants record with the
// fields read below (TagConsts, PhisConsts).
struct TagSlow {
    double xH, xL, wr, wi, gx;
};

__device__ __forceinline__ double with_sign(double v, bool set) {
    return __longlong_as_double(__double_as_longlong(v) | ((long long)set << 63));
}

template <class C>
__device__ __forceinline__ TagSlow tag_slow(const C& c, double tau, const MathTables* mt) {
    // branch-free integer exp, the argument clamped at -705 (the Gaussian is then
    // below 1e-306, nothing against the exponential terms)
    const double gr = -(tau * tau) * c.k_g;
    const double gx = exp_int_nb(below_neg(gr, -705.0) ? -705.0 : gr, mt);
    const double uH = (c.uH0 - tau) * c.k_z, uL = (c.uL0 - tau) * c.k_z, a = (c.uC0 - tau) * c.k_z;
    const double XH = erfcx_fast_q(abs_bits(uH), mt), XL = erfcx_fast_q(abs_bits(uL), mt);
    const bool ap = !negative(a);
    double wr, wi;
    faddeeva_uhp(ap ? c.beta : neg_bits(c.beta), abs_bits(a), &wr, &wi);
    TagSlow s;
    s.xH = with_sign(gx * XH, !negative(uH));
    s.xL = with_sign(gx * XL, !negative(uL));
    s.wr = gx * wr;
    s.wi = gx * wi;
    s.gx = with_sign(gx, ap);
    return s;
}

// 2 g(tau; x) for real x, exact form (library exp and erfcx).  C: TagConsts or
// PhisConsts.
template <class C>
__device__ inline double conv2_real(const C& c, double tau, double x, double u0) {
    const double u = (u0 - tau) * c.k_z;
    const double Gx = exp(-(tau * tau) * c.k_g);
    if (u >= 0.0) return Gx * erfcx(u);
    return 2.0 * exp(-x * tau + 0.5 * x * x * c.s2) - Gx * erfcx(-u);
}

// 2 g(tau; Gamma - i Dm) (both parts), exact form.
template <class C>
__device__ inline void conv2_complex(const C& c, double tau, double* re, double* im) {
    const double a = (c.uC0 - tau) * c.k_z;
    const double Gx = exp(-(tau * tau) * c.k_g);
    double wr, wi;
    if (a >= 0.0) {
        faddeeva_uhp(c.beta, a, &wr, &wi);
        *re = Gx * wr;
        *im = Gx * wi;
        return;
    }
    faddeeva_uhp(-c.beta, -a, &wr, &wi);
    const double m = 2.0 * exp(-c.Gamma * tau + 0.5 * (c.Gamma - c.Dm) * (c.Gamma + c.Dm) * c.s2);
    double sn, cn;
    sincos(c.Dm * tau - c.ph0, &sn, &cn);
    *re = m * cn - Gx * wr;
    *im = m * sn - Gx * wi;
}

// 2 Im g(tau; Gamma - i Dm), exact form.
template <class C>
__device__ inline double conv2_imag(const C& c, double tau) {
    const double a = (c.uC0 - tau) * c.k_z;
    const double Gx = exp(-(tau * tau) * c.k_g);
    double wr, wi;
    if (a >= 0.0) {
        faddeeva_uhp(c.beta, a, &wr, &wi);
        return Gx * wi;
    }
    faddeeva_uhp(-c.beta, -a, &wr, &wi);
    const double m = 2.0 * exp(-c.Gamma * tau + 0.5 * (c.Gamma - c.Dm) * (c.Gamma + c.Dm) * c.s2);
    double sn, cn;
    sincos(c.Dm * tau - c.ph0, &sn, &cn);
    return m * sn - Gx * wi;
}

// The unnormalised signal S(t, q) (for the generator's accept-reject test).
__device__ inline double tag_signal(const TagConsts& c, double t, double q) {
    const double tau = t - c.mu;
    const double gH = conv2_real(c, tau, c.GH, c.uH0), gL = conv2_real(c, tau, c.GL, c.uL0);
    const double gi = conv2_imag(c, tau);
    return 0.5 * (c.aH * gH + c.aL * gL + q * c.Ds * gi);
}

}  // namespace ipa
