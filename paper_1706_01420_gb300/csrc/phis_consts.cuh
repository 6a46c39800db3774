// The phi_s model's parameter record (Sec. 4, the B_s -> J/psi phi fit):
// the fields the likelihood kernel and the generator read (phis.cu), and
// its computation from theta along short chains, as for the 4D record
// (consts.cuh: the real edges' erfc and Gaussian through exp(-x^2/2) and
// the table-driven erfcx and exp, products with reciprocals instead of
// divisions, independent pieces in different warps).  The normalisation
// over one tag (qsel != 0) adds the two complex edges of the oscillating
// time function (cedge_F: the Faddeeva function, the table erfcx, exp and
// sin/cos).
//
// Normalisation (both tags, the interference terms integrate to zero over
// the angles): N = (16 pi / 9) (wL I_L + wH I_H), I_x = F(t_hi) - F(t_lo)
// of the real convolution with rate Gamma_x, wL = Pe (1 + c) + Po (1 - c),
// wH = Pe (1 - c) + Po (1 + c), Pe = |A_0|^2 + |A_par|^2, Po = |A_perp|^2 +
// |A_S|^2, c = cos phi_s.  Over one tag Q: N_Q = N / 2 + Q (16 pi / 9) D
// sin phi_s (Pe - Po) Im I_c, I_c the integral of g(t - mu; Gamma - i Dm).
#pragma once

#include <math.h>

#include "consts.cuh"
#include "faddeeva.cuh"
#include "fp64_math.cuh"
#include "ipa_internal.cuh"

namespace ipa {

// Constants of one fit (a Consts slot).
struct PhisConsts {
    // time part: the fields tag_slow reads, named as in TagConsts
    double Gamma, sigma, mu, fb, DG, Dm;
    double GH, GL, k_z, k_g, cG, s2, inv_s;
    double cH2, cL2, cC2, uH0, uL0, uC0, beta, ph0, tcut;
    // normalisation
    double cs, cb, inv_N, inv_V, N;
    double dlnN[IPA_NPAR_PHIS];
    // phase, mistag dilution, amplitudes
    double c, s, D;
    double x0, xe, xa, F;           // A0sq, Apesq, 1 - A0sq - Apesq, F_S
    double r0, ra, re, rF, rs;      // sqrt of x0, xa, xe, F, 1 - F
    double cw[6], sw[6];            // cos, sin of (dpe - dpa), dpa, dpe, (dpa - dS), (dpe - dS), dS
    double br[10], bi[10];          // Re, Im of b_k
    double csp;                     // C_SP: factor of the S-P interference terms k = 7, 8, 9
    double qsel;                    // normalisation over both tags (0) or over the tag +1 / -1
    double pad_;
};
static_assert(sizeof(PhisConsts) <= sizeof(Consts), "PhisConsts must fit a Consts slot");
static_assert(sizeof(PhisConsts) % 16 == 0, "PhisConsts must be a multiple of 16 bytes");
constexpr int kPhisDoubles = sizeof(PhisConsts) / sizeof(double);

namespace pdetail {

constexpr double kLn2 = 0.69314718055994530942;

// The rates Gamma_L (r = 0) and Gamma_H (r = 1); edge k = 2r + e of the
// normalisation (e = 0: t_hi, 1: t_lo).
__device__ inline double rate_L(const double* th) { return th[IPA_GAMMA] + 0.5 * th[IPA_PHIS_DG]; }
__device__ inline double rate_H(const double* th) { return th[IPA_GAMMA] - 0.5 * th[IPA_PHIS_DG]; }

__device__ inline cdetail::TimeScalars rate_scalars(const double* th, int r) {
    return cdetail::time_scalars_of(r == 0 ? rate_L(th) : rate_H(th), th[IPA_SIGMA], th[IPA_MU], th[IPA_FB]);
}

// Piece k of the real edges: erfcx at the argument of g at edge k (k < 4) or
// of Phi at edge k - 4 (k = 4, 5); rs = 1 / sigma.
__device__ inline double edge_X(const ModelDev& m, const double* th, int k, double rs, const MathTables* mt) {
    using namespace cdetail;
    const double x = edge_tau(m, th[IPA_MU], k & 1) * rs;
    const double z = edge_z(rate_scalars(th, (k >> 1) & 1), x);
    return edge_erfcx(k < 4 ? z : edge_w(x), mt);
}

// Piece k of the real edges: E = exp(-Gamma_r tau + Gamma_r^2 sigma^2 / 2) at
// edge k (k < 4) or the Gaussian factor exp(-x^2/2) at edge k - 4 (k = 4, 5).
__device__ inline double edge_exp(const ModelDev& m, const double* th, int k, double rs, const MathTables* mt) {
    using namespace cdetail;
    const double tau = edge_tau(m, th[IPA_MU], k & 1);
    const double x = tau * rs;
    return exp_fast(k < 4 ? decay_exponent(rate_scalars(th, (k >> 1) & 1), tau) : gauss_exponent(x), mt);
}

// F and its derivatives (rate, sigma, mu) at edge k < 4 from its pieces
// (X1 = edge_X(k), X2 = edge_X(4 + e), E = edge_exp(k), gq = edge_exp(4 + e)),
// rs = 1 / sigma and rG = 1 / Gamma_r.
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

// The range's volume (twice the span for the tags, 8 pi for the angles),
// halved for the normalisation over one tag.
__device__ inline double volume(const ModelDev& m, const double* th) {
    const double V = 2.0 * (m.t_hi - m.t_lo) * 8.0 * cdetail::kPi;
    return th[IPA_PHIS_QNORM] != 0.0 ? 0.5 * V : V;
}

// The denominators that get a reciprocal: sigma, Gamma_L, Gamma_H and the volume.
__device__ inline double recip_arg(const ModelDev& m, const double* th, int i) {
    return i == 0 ? th[IPA_SIGMA] : (i == 1 ? rate_L(th) : (i == 2 ? rate_H(th) : volume(m, th)));
}

struct Amp {
    double x0, xe, xa, F, sF;     // A0sq, Apesq, 1 - A0sq - Apesq, F_S, 1 - F_S
};
__device__ inline Amp amp(const double* th) {
    Amp a;
    a.x0 = th[IPA_A0SQ];
    a.xe = th[IPA_APESQ];
    a.F = th[IPA_FS];
    a.xa = 1.0 - a.x0 - a.xe;
    a.sF = 1.0 - a.F;
    return a;
}

// Square root i: of x0, xa, xe, F, 1 - F (i < 5), or the near-peak cut's root
// sqrt(39.1 + beta^2), beta = Dm sigma / sqrt2 (i = 5).
__device__ inline double root_arg(const double* th, int i) {
    const Amp a = amp(th);
    if (i < 5) return i == 0 ? a.x0 : (i == 1 ? a.xa : (i == 2 ? a.xe : (i == 3 ? a.F : a.sF)));
    const double beta = th[IPA_PHIS_DM] * th[IPA_SIGMA] * cdetail::kInvSqrt2;
    return 39.1 + beta * beta;
}

// Sine and cosine i: of the strong-phase combination i (i < 6), of phi_s (i = 6).
__device__ inline double phase_arg(const double* th, int i) {
    return i < 6 ? cdetail::ang_arg(i, th[IPA_DPA], th[IPA_DPE], th[IPA_DS]) : th[IPA_PHIS_PHIS];
}

// Record fields from theta alone.
__device__ inline void theta_fields(const double* th, PhisConsts* c) {
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], Dm = th[IPA_PHIS_DM];
    const double GH = rate_H(th), GL = rate_L(th);
    c->Gamma = Gamma;
    c->sigma = sigma;
    c->mu = th[IPA_MU];
    c->fb = th[IPA_FB];
    c->DG = th[IPA_PHIS_DG];
    c->Dm = Dm;
    c->GH = GH;
    c->GL = GL;
    c->s2 = sigma * sigma;
    c->cH2 = 0.5 * GH * GH * sigma * sigma + kLn2;
    c->cL2 = 0.5 * GL * GL * sigma * sigma + kLn2;
    c->cC2 = 0.5 * (Gamma - Dm) * (Gamma + Dm) * sigma * sigma + kLn2;
    c->uH0 = GH * sigma * sigma;
    c->uL0 = GL * sigma * sigma;
    c->uC0 = Gamma * sigma * sigma;
    c->beta = Dm * sigma * cdetail::kInvSqrt2;
    c->ph0 = Gamma * Dm * sigma * sigma;
}

// Record fields from rs = 1 / sigma and the cut's root tq.
__device__ inline void scale_fields(const double* th, double rs, double tq, PhisConsts* c) {
    using namespace cdetail;
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA];
    c->k_z = rs * kInvSqrt2;
    c->k_g = 0.5 * (rs * rs);
    c->cG = kInvSqrt2Pi * rs;
    c->inv_s = rs;
    // t > tcut: Re u <= -sqrt(39.1 + b^2) for all three rates, so |e^{-u^2} w|
    // <= e^{-39.1} ~ 1e-17 relative to the exponential, and Gx < 1e-17
    const double rmax = fmax(fmax(rate_H(th), rate_L(th)), Gamma);
    const double tc = th[IPA_MU] + (rmax * sigma * sigma + tq * kSqrt2 * sigma);
    c->tcut = tc == tc ? tc : INFINITY;
}

// Record fields of the amplitudes, phases and tags (r: the five square roots;
// sw, cw: the strong-phase sines and cosines; sn, cn: of phi_s).
__device__ inline void amp_fields(const double* th, const double* r, const double* sw, const double* cw, double sn,
                                  double cn, PhisConsts* c) {
    const Amp a = amp(th);
    c->x0 = a.x0;
    c->xe = a.xe;
    c->xa = a.xa;
    c->F = a.F;
    c->r0 = r[0];
    c->ra = r[1];
    c->re = r[2];
    c->rF = r[3];
    c->rs = r[4];
    for (int i = 0; i < 6; ++i) {
        c->sw[i] = sw[i];
        c->cw[i] = cw[i];
    }
    c->c = cn;
    c->s = sn;
    c->D = 1.0 - 2.0 * th[IPA_PHIS_OMEGA];
    const double qsel = th[IPA_PHIS_QNORM];
    c->csp = th[IPA_PHIS_CSP];
    c->qsel = qsel > 0.0 ? 1.0 : (qsel < 0.0 ? -1.0 : 0.0);
    c->pad_ = 0.0;
}

// b_k = m_k e^{i psi_k} (the P-wave magnitudes carry 1 - F_S): m_k = (f1 f2) f3,
// psi_k the strong phase of term k (none for k = 0, 1, 2, 6; minus delta_S for k = 9).
__device__ inline void b_entry(int k, const double* th, const double* r, const double* sw, const double* cw,
                               double* br, double* bi) {
    const Amp a = amp(th);
    const double rFs = r[3] * r[4];
    const double f1 = k < 6 ? a.sF : (k == 6 ? a.F : rFs);
    const double f2 = k == 0 ? a.x0
                    : k == 1 ? a.xa
                    : k == 2 ? a.xe
                    : k == 3 ? r[1]
                    : k == 4 || k == 5 ? r[0]
                    : k == 6 ? 1.0
                    : k == 7 ? r[1]
                    : k == 8 ? r[2] : r[0];
    const double f3 = k == 3 ? r[2] : (k == 4 ? r[1] : (k == 5 ? r[2] : 1.0));
    const double mag = (f1 * f2) * f3;
    const bool ph = k == 3 || k == 4 || k == 5 || k >= 7;
    const int p = !ph ? 0 : (k < 6 ? k - 3 : k - 4);
    const double cp = ph ? cw[p] : 1.0;
    const double sp = ph ? (k == 9 ? neg_bits(sw[p]) : sw[p]) : 0.0;
    *br = mag * cp;
    *bi = mag * sp;
}

// The complex antiderivative of the oscillating time function (the
// normalisation over one tag): F(tau) with dF/dtau = g(tau; z), z = zr + i zi
// = Gamma - i Dm, F = (Phi(tau / sigma) - g) / z (from g' = G - z g), and
// dF/dz, dF/dsigma, dF/dmu = -(F + dg/dz) / z, (-(tau / sigma) G - dg/dsigma)
// / z, -g with dg/dz = (z s^2 - tau) g - s^2 G and dg/dsigma = z^2 sigma g -
// (z sigma + tau / sigma) G.  g through the Faddeeva function: 1/2 gx w(x + i
// y) for y >= 0, else e^{-z tau + z^2 s^2 / 2} - 1/2 gx w(-x - i y), with gx =
// exp(-tau^2 / 2 s^2) and x + i y = i (z s^2 - tau) / (sqrt2 s).  Two halves
// of independent pieces (cedge_fad, cedge_exp) and their combination
// (cedge_F); rs = 1 / sigma, edge e = 0 (t_hi) or 1 (t_lo).
struct CEdgeArg {
    double tau, xt, y, x;        // tau, tau / sigma, and x + i y above
};
__device__ inline CEdgeArg cedge_arg(const ModelDev& m, const double* th, int e, double rs) {
    using namespace cdetail;
    const double sigma = th[IPA_SIGMA], zr = th[IPA_GAMMA], zi = -th[IPA_PHIS_DM];
    CEdgeArg a;
    a.tau = edge_tau(m, th[IPA_MU], e);
    a.xt = a.tau * rs;
    a.y = (zr * sigma - a.xt) * kInvSqrt2;
    a.x = -zi * sigma * kInvSqrt2;
    return a;
}

// (Re w, Im w, gx): w at x + i y (y >= 0) or at -x - i y (y < 0).
__device__ inline void cedge_fad(const ModelDev& m, const double* th, int e, double rs, const MathTables* mt,
                                 double* out) {
    const CEdgeArg a = cedge_arg(m, th, e, rs);
    const bool up = a.y >= 0.0;
    faddeeva_uhp(up ? a.x : neg_bits(a.x), up ? a.y : neg_bits(a.y), &out[0], &out[1]);
    out[2] = exp_fast(cdetail::gauss_exponent(a.xt), mt);
}

// (erfcx for Phi, e^{Re(-z tau + z^2 s^2 / 2)}, sin and cos of its imaginary part).
__device__ inline void cedge_exp(const ModelDev& m, const double* th, int e, double rs, const MathTables* mt,
                                 double* out) {
    using namespace cdetail;
    const CEdgeArg a = cedge_arg(m, th, e, rs);
    const double sigma = th[IPA_SIGMA], zr = th[IPA_GAMMA], zi = -th[IPA_PHIS_DM];
    const double s2 = sigma * sigma;
    out[0] = edge_erfcx(edge_w(a.xt), mt);
    const double er = -zr * a.tau + 0.5 * s2 * (zr * zr - zi * zi), ei = -zi * a.tau + zr * zi * s2;
    out[1] = exp_fast(er, mt);
    sincos_fast(ei, mt, &out[2], &out[3]);
}

// F, dF/dz, dF/dsigma, dF/dmu as (re, im) pairs at edge e from fa = cedge_fad
// and ex = cedge_exp.
__device__ inline void cedge_F(const ModelDev& m, const double* th, int e, double rs, const double* fa,
                               const double* ex, double* out) {
    using namespace cdetail;
    const CEdgeArg a = cedge_arg(m, th, e, rs);
    const double sigma = th[IPA_SIGMA], zr = th[IPA_GAMMA], zi = -th[IPA_PHIS_DM];
    const double s2 = sigma * sigma, tau = a.tau, xt = a.xt, gx = fa[2];
    double gr, gi;
    if (a.y >= 0.0) {
        gr = 0.5 * gx * fa[0];
        gi = 0.5 * gx * fa[1];
    } else {
        gr = ex[1] * ex[3] - 0.5 * gx * fa[0];
        gi = ex[1] * ex[2] - 0.5 * gx * fa[1];
    }
    const double G = gx * (kInvSqrt2Pi * rs);
    const double b2 = 0.5 * (gx * ex[0]);
    const double Phi = negative(edge_w(xt)) ? 1.0 - b2 : b2;
    const double rn = recip(zr * zr + zi * zi), ir = zr * rn, ii = -zi * rn;    // 1/z
    // F = (Phi - g) / z
    const double nr = Phi - gr, ni = -gi;
    const double Fr = nr * ir - ni * ii, Fi = nr * ii + ni * ir;
    // dg/dz = (z s^2 - tau) g - s^2 G
    const double pr = zr * s2 - tau, pi = zi * s2;
    const double dzr = pr * gr - pi * gi - s2 * G, dzi = pr * gi + pi * gr;
    // dF/dz = -(F + dg/dz) / z
    const double ar = -(Fr + dzr), ai = -(Fi + dzi);
    out[2] = ar * ir - ai * ii;
    out[3] = ar * ii + ai * ir;
    // dg/dsigma = z^2 sigma g - (z sigma + tau / sigma) G
    const double z2r = (zr * zr - zi * zi) * sigma, z2i = 2.0 * zr * zi * sigma;
    const double dsr = z2r * gr - z2i * gi - (zr * sigma + xt) * G;
    const double dsi = z2r * gi + z2i * gr - zi * sigma * G;
    // dF/dsigma = (-(tau / sigma) G - dg/dsigma) / z
    const double br = -xt * G - dsr, bi = -dsi;
    out[4] = br * ir - bi * ii;
    out[5] = br * ii + bi * ir;
    out[0] = Fr;
    out[1] = Fi;
    out[6] = -gr;
    out[7] = -gi;
}

// N over both tags, or over the tag qsel (ec: the complex edges at t_hi, t_lo).
__device__ inline double norm_N(const double* th, const double* F, const double* ec, double sn, double cn) {
    const Amp a = amp(th);
    const double IL = F[0] - F[1], IH = F[2] - F[3];
    const double Pe = a.sF * (1.0 - a.xe), Po = a.sF * a.xe + a.F;
    const double wL = Pe * (1.0 + cn) + Po * (1.0 - cn), wH = Pe * (1.0 - cn) + Po * (1.0 + cn);
    const double K = 16.0 * cdetail::kPi / 9.0;
    double N = K * (wL * IL + wH * IH);
    const double qsel = th[IPA_PHIS_QNORM];
    if (qsel != 0.0) {
        const double Q = qsel > 0.0 ? 1.0 : -1.0;
        const double Ii = ec[1] - ec[8 + 1];
        const double W = Pe - Po, D = 1.0 - 2.0 * th[IPA_PHIS_OMEGA];
        const double odd = Q * K * D * sn * W;
        N = 0.5 * N + odd * Ii;
    }
    return N;
}

// dN/dtheta_j (the amplitude parameters through Pe and Po; the phases, f_b,
// C_SP and the selector do not enter N; over one tag Dm, phi_s and omega
// also enter through the oscillating term).
__device__ inline double norm_dN(int j, const double* th, const double* F, const double (*dF)[3], const double* ec,
                                 double sn, double cn) {
    const Amp a = amp(th);
    const double IL = F[0] - F[1], IH = F[2] - F[3];
    const double Pe = a.sF * (1.0 - a.xe), Po = a.sF * a.xe + a.F;
    const double wL = Pe * (1.0 + cn) + Po * (1.0 - cn), wH = Pe * (1.0 - cn) + Po * (1.0 + cn);
    const double K = 16.0 * cdetail::kPi / 9.0;
    const bool ampj = j >= IPA_A0SQ && j < IPA_A0SQ + 6;
    const int aa = ampj ? j - IPA_A0SQ : 0;
    const double dPe = aa == 1 ? -a.sF : (aa == 4 ? -(1.0 - a.xe) : 0.0);
    const double dPo = aa == 1 ? a.sF : (aa == 4 ? 1.0 - a.xe : 0.0);
    double v = 0.0;
    if (j < 3)
        v = K * (wL * (dF[0][j] - dF[1][j]) + wH * (dF[2][j] - dF[3][j]));
    else if (ampj)
        v = K * ((dPe * (1.0 + cn) + dPo * (1.0 - cn)) * IL + (dPe * (1.0 - cn) + dPo * (1.0 + cn)) * IH);
    else if (j == IPA_PHIS_DG)
        v = K * (0.5 * wL * (dF[0][0] - dF[1][0]) - 0.5 * wH * (dF[2][0] - dF[3][0]));
    else if (j == IPA_PHIS_PHIS)
        v = K * ((-Pe * sn + Po * sn) * IL + (Pe * sn - Po * sn) * IH);
    const double qsel = th[IPA_PHIS_QNORM];
    if (qsel != 0.0) {
        const double Q = qsel > 0.0 ? 1.0 : -1.0;
        const double* eh = ec;
        const double* el = ec + 8;
        const double Ii = eh[1] - el[1];
        const double W = Pe - Po, D = 1.0 - 2.0 * th[IPA_PHIS_OMEGA];
        const double odd = Q * K * D * sn * W;
        v *= 0.5;
        if (j == IPA_GAMMA) v += odd * (eh[3] - el[3]);                     // d/dGamma = d/dz
        else if (j == IPA_SIGMA) v += odd * (eh[5] - el[5]);
        else if (j == IPA_MU) v += odd * (eh[7] - el[7]);
        else if (j == IPA_PHIS_DM) v += odd * (-(eh[2] - el[2]));          // d/dDm = -i d/dz
        else if (j == IPA_PHIS_PHIS) v += Q * K * D * cn * W * Ii;
        else if (j == IPA_PHIS_OMEGA) v += Q * K * (-2.0) * sn * W * Ii;
        else if (ampj) v += Q * K * D * sn * (dPe - dPo) * Ii;
    }
    return v;
}

}  // namespace pdetail

// One thread computes the record (many segments: lanes hold different fits).
__device__ inline void phis_consts_thread(const ModelDev& m, const double* th, const MathTables* mt, PhisConsts* c) {
    using namespace pdetail;
    double rc[4], X[6], Ex[6], r[6], sw[7], cw[7], F[4], dF[4][3], ec[16];
    for (int i = 0; i < 4; ++i) rc[i] = cdetail::recip(recip_arg(m, th, i));
    for (int k = 0; k < 6; ++k) {
        X[k] = edge_X(m, th, k, rc[0], mt);
        Ex[k] = edge_exp(m, th, k, rc[0], mt);
        r[k] = sqrt(root_arg(th, k));
    }
    for (int i = 0; i < 7; ++i) sincos_fast(phase_arg(th, i), mt, &sw[i], &cw[i]);
    for (int e = 0; e < 2; ++e) {
        if (th[IPA_PHIS_QNORM] != 0.0) {
            double fa[3], ex[4];
            cedge_fad(m, th, e, rc[0], mt, fa);
            cedge_exp(m, th, e, rc[0], mt, ex);
            cedge_F(m, th, e, rc[0], fa, ex, ec + 8 * e);
        } else {
            for (int i = 0; i < 8; ++i) ec[8 * e + i] = 0.0;
        }
    }
    theta_fields(th, c);
    scale_fields(th, rc[0], r[5], c);
    amp_fields(th, r, sw, cw, sw[6], cw[6], c);
    for (int k = 0; k < 10; ++k) b_entry(k, th, r, sw, cw, &c->br[k], &c->bi[k]);
    for (int k = 0; k < 4; ++k)
        edge_F(m, th, k, rc[0], rc[1 + (k >> 1)], X[k], X[4 + (k & 1)], Ex[k], Ex[4 + (k & 1)], &F[k], dF[k]);
    const double N = norm_N(th, F, ec, sw[6], cw[6]), inv_N = cdetail::recip(N);
    for (int j = 0; j < IPA_NPAR_PHIS; ++j) c->dlnN[j] = norm_dN(j, th, F, dF, ec, sw[6], cw[6]) * inv_N;
    c->N = N;
    c->inv_N = inv_N;
    c->cs = (1.0 - th[IPA_FB]) * inv_N;
    c->cb = th[IPA_FB] * rc[3];
    c->inv_V = rc[3];
}

// Exchange buffer of phis_consts_block.
struct PhisBlockScratch {
    MathTables mt;
    double th[IPA_NPAR_PHIS];
    double rc[4];                 // 1/sigma, 1/Gamma_L, 1/Gamma_H, 1/V
    double X[6], Ex[6];           // real-edge pieces (edge_X, edge_exp)
    double r[6];                  // sqrt of x0, xa, xe, F, 1 - F; the cut's root
    double sw[7], cw[7];          // sin, cos of the strong phases and of phi_s
    double cf[2][3], cx[2][4];    // complex-edge pieces (cedge_fad, cedge_exp) at t_hi, t_lo
    double ec[16];                // complex edges at t_hi and t_lo (one-tag normalisation)
    double F[4], dF[4][3];
    PhisConsts c;
};
constexpr int kPhisConstsBlock = 256;

// One block of eight warps computes the record (few segments: latency), with
// independent pieces in different warps and, within a warp, in lanes running
// the same code:
//   phase 1  warp 0: the six erfcx of the real edges; warp 1: their six
//            exponentials; warp 2: seven sine/cosine pairs; warp 3: six square
//            roots; warp 4: four reciprocals; warps 5 and 7: the two halves of
//            the complex edges' pieces (one tag only); warp 6: the fields of
//            theta alone;
//   phase 2  warp 0: F and its derivatives at the four real edges; warp 1: the
//            fields of 1/sigma; warp 2: b_k (lane k) and the amplitude fields;
//            warp 5: the complex edges;
//   phase 3  warps 0-2: dN/dtheta_j / N (a parameter per lane) and the fields of 1/N;
// then every thread copies part of the record out.
__device__ inline void phis_consts_block(const ModelDev& m, const double* th, PhisConsts* c, PhisBlockScratch* S) {
    using namespace pdetail;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < IPA_NPAR_PHIS) S->th[threadIdx.x] = th[threadIdx.x];
    cdetail::load_consts_tables(&S->mt);
    __syncthreads();
    th = S->th;

    if (w == 0) {
        if (lane < 6) S->X[lane] = edge_X(m, th, lane, cdetail::recip(th[IPA_SIGMA]), &S->mt);
    } else if (w == 1) {
        if (lane < 6) S->Ex[lane] = edge_exp(m, th, lane, cdetail::recip(th[IPA_SIGMA]), &S->mt);
    } else if (w == 2) {
        if (lane < 7) sincos_fast(phase_arg(th, lane), &S->mt, &S->sw[lane], &S->cw[lane]);
    } else if (w == 3) {
        if (lane < 6) S->r[lane] = sqrt(root_arg(th, lane));
    } else if (w == 4) {
        if (lane < 4) S->rc[lane] = cdetail::recip(recip_arg(m, th, lane));
    } else if (w == 5) {
        if (lane < 2 && th[IPA_PHIS_QNORM] != 0.0)
            cedge_fad(m, th, lane, cdetail::recip(th[IPA_SIGMA]), &S->mt, S->cf[lane]);
    } else if (w == 6) {
        if (lane == 0) theta_fields(th, &S->c);
    } else if (w == 7) {
        if (lane < 2 && th[IPA_PHIS_QNORM] != 0.0)
            cedge_exp(m, th, lane, cdetail::recip(th[IPA_SIGMA]), &S->mt, S->cx[lane]);
    }
    __syncthreads();

    if (w == 0) {
        if (lane < 4)
            edge_F(m, th, lane, S->rc[0], S->rc[1 + (lane >> 1)], S->X[lane], S->X[4 + (lane & 1)], S->Ex[lane],
                   S->Ex[4 + (lane & 1)], &S->F[lane], S->dF[lane]);
    } else if (w == 1) {
        if (lane == 0) scale_fields(th, S->rc[0], S->r[5], &S->c);
    } else if (w == 2) {
        if (lane < 10) b_entry(lane, th, S->r, S->sw, S->cw, &S->c.br[lane], &S->c.bi[lane]);
        else if (lane == 10) amp_fields(th, S->r, S->sw, S->cw, S->sw[6], S->cw[6], &S->c);
    } else if (w == 5) {
        if (lane < 2) {
            if (th[IPA_PHIS_QNORM] != 0.0)
                cedge_F(m, th, lane, S->rc[0], S->cf[lane], S->cx[lane], S->ec + 8 * lane);
            else
                for (int i = 0; i < 8; ++i) S->ec[8 * lane + i] = 0.0;
        }
    }
    __syncthreads();

    // parameters per lane: warp 0 the time ones, warp 1 the amplitudes and
    // phi_s, warp 2 the rest and (lane 5) the fields of 1/N
    int j = -1;
    if (w == 0) j = lane < 3 ? lane : (lane == 3 ? IPA_PHIS_DG : -1);
    else if (w == 1) j = lane < 6 ? IPA_A0SQ + lane : (lane == 6 ? IPA_PHIS_PHIS : -1);
    else if (w == 2) {
        const int rest[5] = {IPA_FB, IPA_PHIS_DM, IPA_PHIS_OMEGA, IPA_PHIS_CSP, IPA_PHIS_QNORM};
        j = lane < 5 ? rest[lane] : (lane == 5 ? IPA_NPAR_PHIS : -1);
    }
    if (j >= 0) {
        const double N = norm_N(th, S->F, S->ec, S->sw[6], S->cw[6]), inv_N = cdetail::recip(N);
        if (j < IPA_NPAR_PHIS) {
            S->c.dlnN[j] = norm_dN(j, th, S->F, S->dF, S->ec, S->sw[6], S->cw[6]) * inv_N;
        } else {
            S->c.N = N;
            S->c.inv_N = inv_N;
            S->c.cs = (1.0 - th[IPA_FB]) * inv_N;
            S->c.cb = th[IPA_FB] * S->rc[3];
            S->c.inv_V = S->rc[3];
        }
    }
    __syncthreads();
    const double* src = reinterpret_cast<const double*>(&S->c);
    double* dst = reinterpret_cast<double*>(c);
    for (int i = threadIdx.x; i < kPhisDoubles; i += blockDim.x) dst[i] = src[i];
}

}  // namespace ipa
