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

// theta (8 values) -> the record, along short chains as for the 4D record
// (consts.cuh: erfc and the Gaussian through exp(-x^2/2) and the table-driven
// erfcx and exp, products with reciprocals instead of divisions).  Edge k =
// 2r + e of the normalisation: rate r (0: Gamma_H, 1: Gamma_L) at edge e (0:
// t_hi, 1: t_lo).  One thread per segment (tag_consts_thread) and one block per
// segment (tag_consts_block) call the same functions, so both give the same bits
// (tagged.cu is compiled without FMA contraction).
namespace tdetail {

__device__ inline double rate_H(const double* th) { return th[IPA_GAMMA] - 0.5 * th[IPA_DG]; }
__device__ inline double rate_L(const double* th) { return th[IPA_GAMMA] + 0.5 * th[IPA_DG]; }

__device__ inline cdetail::TimeScalars rate_scalars(const double* th, int r) {
    return cdetail::time_scalars_of(r == 0 ? rate_H(th) : rate_L(th), th[IPA_SIGMA], th[IPA_MU], th[IPA_FB]);
}

// Piece k of the edges: erfcx at the argument of g at edge k (k < 4) or of
// Phi at edge k - 4 (k = 4, 5); rs = 1 / sigma.
__device__ inline double edge_X(const ModelDev& m, const double* th, int k, double rs, const MathTables* mt) {
    using namespace cdetail;
    const double x = edge_tau(m, th[IPA_MU], k & 1) * rs;
    const double z = edge_z(rate_scalars(th, (k >> 1) & 1), x);
    return edge_erfcx(k < 4 ? z : edge_w(x), mt);
}

// Piece k of the edges: E = exp(-Gamma_r tau + Gamma_r^2 sigma^2 / 2) at edge
// k (k < 4) or the Gaussian factor exp(-x^2/2) at edge k - 4 (k = 4, 5).
__device__ inline double edge_exp(const ModelDev& m, const double* th, int k, double rs, const MathTables* mt) {
    using namespace cdetail;
    const double tau = edge_tau(m, th[IPA_MU], k & 1);
    const double x = tau * rs;
    return exp_fast(k < 4 ? decay_exponent(rate_scalars(th, (k >> 1) & 1), tau) : gauss_exponent(x), mt);
}

// F and its derivatives (rate, sigma, mu) at edge k < 4 from its pieces:
// X1 = edge_X(k), X2 = edge_X(4 + e), E = edge_exp(k), gq = edge_exp(4 + e),
// rs = 1 / sigma, rG = 1 / Gamma_r.
__device__ inline void edge_F(const ModelDev& m, const double* th, int k, double rs, double rG, double X1,
                              double X2, double E, double gq, double* F, double* dF) {
    using namespace cdetail;
    const double tau = edge_tau(m, th[IPA_MU], k & 1);
    const double x = tau * rs;
    const TimeScalars s = rate_scalars(th, k >> 1);
    double g, Phi, G;
    edge_values(edge_z(s, x), edge_w(x), gq, E, X1, X2, kInvSqrt2Pi * rs, &g, &Phi, &G);
    edge_combine_r(s, tau, x, rG, g, G, Phi, F, dF);
}

// The denominators that get a reciprocal: sigma, Gamma_H, Gamma_L and 2 (t_hi - t_lo).
__device__ inline double recip_arg(const ModelDev& m, const double* th, int i) {
    return i == 0 ? th[IPA_SIGMA] : (i == 1 ? rate_H(th) : (i == 2 ? rate_L(th) : 2.0 * (m.t_hi - m.t_lo)));
}

// sqrt(39.1 + beta^2), beta = Dm sigma / sqrt2 (the near-peak cut's root).
__device__ inline double cut_root(const double* th) {
    const double beta = th[IPA_DM] * th[IPA_SIGMA] * cdetail::kInvSqrt2;
    return sqrt(39.1 + beta * beta);
}

// M_x for x = Gamma_H, Gamma_L, Gamma (i = 0, 1, 2).
__device__ inline double env_piece(const ModelDev& m, const double* th, int i) {
    return env_bound(i == 0 ? rate_H(th) : (i == 1 ? rate_L(th) : th[IPA_GAMMA]), m.t_lo, th[IPA_MU], th[IPA_SIGMA]);
}

// Record fields from theta alone.
__device__ inline void theta_fields(const double* th, TagConsts* c) {
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], Dm = th[IPA_DM];
    const double GH = rate_H(th), GL = rate_L(th);
    c->Gamma = Gamma;
    c->sigma = sigma;
    c->mu = th[IPA_MU];
    c->fb = th[IPA_FB];
    c->DG = th[IPA_DG];
    c->Dm = Dm;
    c->phi = th[IPA_PHIS];
    c->om = th[IPA_OMEGA];
    c->GH = GH;
    c->GL = GL;
    c->cH2 = 0.5 * GH * GH * sigma * sigma + kLn2;
    c->cL2 = 0.5 * GL * GL * sigma * sigma + kLn2;
    c->cC2 = 0.5 * (Gamma - Dm) * (Gamma + Dm) * sigma * sigma + kLn2;
}

// Record fields from theta, rs = 1 / sigma and rV2 = 1 / (2 (t_hi - t_lo)).
__device__ inline void scale_fields(const double* th, double rs, double rV2, TagConsts* c) {
    using namespace cdetail;
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], Dm = th[IPA_DM];
    c->k_z = rs * kInvSqrt2;
    c->k_g = 0.5 * (rs * rs);
    c->cG = kInvSqrt2Pi * rs;
    c->s2 = sigma * sigma;
    c->inv_s = rs;
    c->uH0 = rate_H(th) * sigma * sigma;
    c->uL0 = rate_L(th) * sigma * sigma;
    c->uC0 = Gamma * sigma * sigma;
    c->beta = Dm * sigma * kInvSqrt2;
    c->ph0 = Gamma * Dm * sigma * sigma;
    c->D = 1.0 - 2.0 * th[IPA_OMEGA];
    c->cb = th[IPA_FB] * rV2;
    c->inv_V2 = rV2;
    c->pad_ = 0.0;
}

// Record fields from sin/cos phi_s (sn, cn), the cut's root tq and the envelope bounds M.
__device__ inline void phase_fields(const double* th, double sn, double cn, double tq, const double* M, TagConsts* c) {
    using namespace cdetail;
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], mu = th[IPA_MU];
    const double D = 1.0 - 2.0 * th[IPA_OMEGA];
    c->aH = 0.5 * (1.0 - cn);
    c->aL = 0.5 * (1.0 + cn);
    c->Ds = D * sn;
    c->c = cn;
    c->s = sn;
    // t > tcut: Re u <= -sqrt(39.1 + b^2) for all three rates, so |e^{-u^2} w|
    // <= e^{-39.1} ~ 1e-17 relative to the exponential, and Gx < 1e-17
    const double rmax = fmax(fmax(rate_H(th), rate_L(th)), Gamma);
    const double tc = mu + (rmax * sigma * sigma + tq * kSqrt2 * sigma);
    c->tcut = tc == tc ? tc : INFINITY;
    c->MS = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(0.5, __dsub_rn(1.0, cn)), M[0]),
                                __dmul_rn(__dmul_rn(0.5, __dadd_rn(1.0, cn)), M[1])),
                      __dmul_rn(fabs(__dmul_rn(D, sn)), M[2]));
}

// N = (1 - cos phi_s) I(Gamma_H) + (1 + cos phi_s) I(Gamma_L), I = F(t_hi) - F(t_lo).
__device__ inline double norm_N(const double* F, double cn) {
    return (1.0 - cn) * (F[0] - F[1]) + (1.0 + cn) * (F[2] - F[3]);
}

// dN/dtheta_j as a (P - Q) + b (R - S): j < 3 (Gamma, sigma, mu) the edges'
// derivatives weighted by 1 -+ cos phi_s, j = 4 (DG) their rate derivatives
// weighted by -+(1 -+ cos phi_s)/2, j = 6 (phi_s) the integrals weighted by
// +-sin phi_s; 0 for mu's neighbours f_b, Dm and omega.
__device__ inline double norm_dN(int j, const double* F, const double (*dF)[3], double sn, double cn) {
    const double wH = 1.0 - cn, wL = 1.0 + cn;
    const int jj = j < 3 ? j : 0;
    const double a = j < 3 ? wH : (j == 4 ? -0.5 * wH : sn);
    const double b = j < 3 ? wL : (j == 4 ? 0.5 * wL : neg_bits(sn));
    const bool val = j == 6;
    const double P = val ? F[0] : dF[0][jj], Q = val ? F[1] : dF[1][jj];
    const double R = val ? F[2] : dF[2][jj], S = val ? F[3] : dF[3][jj];
    const double v = a * (P - Q) + b * (R - S);
    return (j == 3 || j == 5 || j == 7) ? 0.0 : v;
}

// cs, qH, qL, qD, N and 1/N from N and the phase fields.
__device__ inline void norm_fields(const double* th, double N, double inv_N, double sn, double cn, TagConsts* c) {
    const double cs = (1.0 - th[IPA_FB]) * inv_N;
    const double D = 1.0 - 2.0 * th[IPA_OMEGA];
    c->cs = cs;
    c->qH = 0.5 * cs * (0.5 * (1.0 - cn));
    c->qL = 0.5 * cs * (0.5 * (1.0 + cn));
    c->qD = 0.5 * cs * (D * sn);
    c->inv_N = inv_N;
    c->N = N;
}

}  // namespace tdetail

// One thread computes the record (many segments: lanes hold different fits).
__device__ inline void tag_consts_thread(const ModelDev& m, const double* th, const MathTables* mt, TagConsts* c) {
    using namespace tdetail;
    double r[4], X[6], Ex[6], M[3], F[4], dF[4][3];
    for (int i = 0; i < 4; ++i) r[i] = cdetail::recip(recip_arg(m, th, i));
    for (int k = 0; k < 6; ++k) {
        X[k] = edge_X(m, th, k, r[0], mt);
        Ex[k] = edge_exp(m, th, k, r[0], mt);
    }
    for (int i = 0; i < 3; ++i) M[i] = env_piece(m, th, i);
    double sn, cn;
    sincos_fast(th[IPA_PHIS], mt, &sn, &cn);
    theta_fields(th, c);
    scale_fields(th, r[0], r[3], c);
    phase_fields(th, sn, cn, cut_root(th), M, c);
    for (int k = 0; k < 4; ++k)
        edge_F(m, th, k, r[0], r[1 + (k >> 1)], X[k], X[4 + (k & 1)], Ex[k], Ex[4 + (k & 1)], &F[k], dF[k]);
    const double N = norm_N(F, cn), inv_N = cdetail::recip(N);
    for (int j = 0; j < 8; ++j) c->dlnN[j] = norm_dN(j, F, dF, sn, cn) * inv_N;
    norm_fields(th, N, inv_N, sn, cn, c);
}

// Exchange buffer of tag_consts_block.
struct TagBlockScratch {
    MathTables mt;
    double th[IPA_NPAR_TAGGED];
    double r[4];                  // 1/sigma, 1/Gamma_H, 1/Gamma_L, 1/(2 (t_hi - t_lo))
    double X[6], Ex[6];           // edge pieces (edge_X, edge_exp)
    double M[3], sn, cn, tq;
    double F[4], dF[4][3];
    TagConsts c;
};
constexpr int kTagConstsBlock = 256;

// One block of eight warps computes the record (few segments: latency).  A
// warp's FP64 instructions do not overlap one another, different warps' do,
// so independent pieces go to different warps and, within a warp, to lanes
// running the same code:
//   phase 1  warp 0: the six erfcx; warp 1: the six exponentials; warp 2: the
//            three envelope bounds; warp 3: sin/cos phi_s; warp 4: the four
//            reciprocals and the cut's root; warp 5: the fields of theta alone;
//   phase 2  warp 0: F and its derivatives at the four edges; warp 1: the
//            phase fields; warp 2: the fields that need 1/sigma;
//   phase 3  warp 0: N, 1/N, dN/dtheta_j / N (lane j) and the fields of 1/N;
// then every thread copies part of the record out.
__device__ inline void tag_consts_block(const ModelDev& m, const double* th, TagConsts* c, TagBlockScratch* S) {
    using namespace tdetail;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < IPA_NPAR_TAGGED) S->th[threadIdx.x] = th[threadIdx.x];
    cdetail::load_consts_tables(&S->mt);
    __syncthreads();
    th = S->th;

    if (w == 0) {
        if (lane < 6) S->X[lane] = edge_X(m, th, lane, cdetail::recip(th[IPA_SIGMA]), &S->mt);
    } else if (w == 1) {
        if (lane < 6) S->Ex[lane] = edge_exp(m, th, lane, cdetail::recip(th[IPA_SIGMA]), &S->mt);
    } else if (w == 2) {
        if (lane < 3) S->M[lane] = env_piece(m, th, lane);
    } else if (w == 3) {
        if (lane == 0) sincos_fast(th[IPA_PHIS], &S->mt, &S->sn, &S->cn);
    } else if (w == 4) {
        if (lane < 4) S->r[lane] = cdetail::recip(recip_arg(m, th, lane));
        else if (lane == 4) S->tq = cut_root(th);
    } else if (w == 5) {
        if (lane == 0) theta_fields(th, &S->c);
    }
    __syncthreads();

    if (w == 0) {
        if (lane < 4)
            edge_F(m, th, lane, S->r[0], S->r[1 + (lane >> 1)], S->X[lane], S->X[4 + (lane & 1)], S->Ex[lane],
                   S->Ex[4 + (lane & 1)], &S->F[lane], S->dF[lane]);
    } else if (w == 1) {
        if (lane == 0) phase_fields(th, S->sn, S->cn, S->tq, S->M, &S->c);
    } else if (w == 2) {
        if (lane == 0) scale_fields(th, S->r[0], S->r[3], &S->c);
    }
    __syncthreads();

    if (w == 0 && lane < 9) {
        const double N = norm_N(S->F, S->cn), inv_N = cdetail::recip(N);
        if (lane < 8) S->c.dlnN[lane] = norm_dN(lane, S->F, S->dF, S->sn, S->cn) * inv_N;
        else norm_fields(th, N, inv_N, S->sn, S->cn, &S->c);
    }
    __syncthreads();
    const double* src = reinterpret_cast<const double*>(&S->c);
    double* dst = reinterpret_cast<double*>(c);
    for (int i = threadIdx.x; i < kTagConstsDoubles; i += blockDim.x) dst[i] = src[i];
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
