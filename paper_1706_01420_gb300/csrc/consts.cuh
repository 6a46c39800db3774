// Step a1 of the hot path: parameter-derived constants, computed on the device
// from theta once per call (one thread per fit), so that theta can stay in
// device memory and calls can be captured in CUDA graphs.
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
#pragma once

#include <math.h>

#include "ipa_internal.cuh"

namespace ipa {

namespace cdetail {

constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kInvSqrt2Pi = 0.39894228040143267794;
constexpr double kPi = 3.14159265358979323846;

__device__ inline double conv_g(double tau, double Gamma, double sigma) {
    const double z = (Gamma * sigma * sigma - tau) / (kSqrt2 * sigma);
    return 0.5 * exp(-Gamma * tau + 0.5 * Gamma * Gamma * sigma * sigma) * erfc(z);
}

__device__ inline double gauss(double tau, double sigma) {
    const double x = tau / sigma;
    return kInvSqrt2Pi / sigma * exp(-0.5 * x * x);
}

// F(tau) and its derivatives (Gamma, sigma, mu) at one edge of the range.
__device__ inline void edge(double tau, double Gamma, double sigma, double* F, double* dF) {
    const double g = conv_g(tau, Gamma, sigma);
    const double G = gauss(tau, sigma);
    const double Phi = 0.5 * erfc(-tau / (kSqrt2 * sigma));
    const double dg_dG = (Gamma * sigma * sigma - tau) * g - sigma * sigma * G;
    const double dg_ds = Gamma * Gamma * sigma * g - (Gamma * sigma + tau / sigma) * G;
    *F = (Phi - g) / Gamma;
    dF[0] = -(*F + dg_dG) / Gamma;
    dF[1] = (-(tau / sigma) * G - dg_ds) / Gamma;
    dF[2] = -g;
}

}  // namespace cdetail

__device__ inline void compute_consts(const ModelDev& m, const double* th, Consts* c) {
    using namespace cdetail;
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], mu = th[IPA_MU], fb = th[IPA_FB];
    c->Gamma = Gamma;
    c->sigma = sigma;
    c->mu = mu;
    c->fb = fb;
    c->c_exp = 0.5 * Gamma * Gamma * sigma * sigma;
    c->Gs2 = Gamma * sigma * sigma;
    c->k_z = 1.0 / (kSqrt2 * sigma);
    c->k_g = 1.0 / (2.0 * sigma * sigma);
    c->cG = kInvSqrt2Pi / sigma;
    c->s2 = sigma * sigma;
    c->G2s = Gamma * Gamma * sigma;
    c->Gsig = Gamma * sigma;
    c->inv_s = 1.0 / sigma;

    double Fh, Fl, dFh[3], dFl[3];
    edge(m.t_hi - mu, Gamma, sigma, &Fh, dFh);
    edge(m.t_lo - mu, Gamma, sigma, &Fl, dFl);
    const double IT = Fh - Fl;
    c->IT = IT;
    for (int j = 0; j < 3; ++j) c->dlnIT[j] = (dFh[j] - dFl[j]) / IT;
    c->MT = fmin(1.0, exp(-Gamma * (m.t_lo - mu) + 0.5 * Gamma * Gamma * sigma * sigma));

    const double span = m.t_hi - m.t_lo;
    double IO, V;
    for (int k = 0; k < 10; ++k) {
        c->h[k] = 0.0;
        for (int j = 0; j < 6; ++j) c->dh[k][j] = 0.0;
    }
    if (m.kind == IPA_MODEL_TIME1D) {
        IO = 1.0;
        V = span;
        c->h[0] = 1.0;
        c->MO = 1.0;
    } else {
        IO = 16.0 * kPi / 9.0;
        V = span * 8.0 * kPi;
        const double x0 = th[IPA_A0SQ], xe = th[IPA_APESQ], dpa = th[IPA_DPA], dpe = th[IPA_DPE];
        const double F = th[IPA_FS], dS = th[IPA_DS];
        const double xa = 1.0 - x0 - xe, s = 1.0 - F;
        const double r0 = sqrt(x0), ra = sqrt(xa), re = sqrt(xe), rF = sqrt(F), rs = sqrt(s);
        const double rFs = rF * rs;
        const double s4 = sin(dpe - dpa), c4 = cos(dpe - dpa);
        const double c5 = cos(dpa), s5 = sin(dpa);
        const double s6 = sin(dpe), c6 = cos(dpe);
        const double c8 = cos(dpa - dS), s8 = sin(dpa - dS);
        const double s9 = sin(dpe - dS), c9 = cos(dpe - dS);
        const double c10 = cos(dS), s10 = sin(dS);
        double* h = c->h;
        h[0] = s * x0;
        h[1] = s * xa;
        h[2] = s * xe;
        h[3] = s * ra * re * s4;
        h[4] = s * r0 * ra * c5;
        h[5] = s * r0 * re * s6;
        h[6] = F;
        h[7] = rFs * ra * c8;
        h[8] = rFs * re * s9;
        h[9] = rFs * r0 * c10;
        // columns: 0 A0sq, 1 Apesq, 2 delta_pa, 3 delta_pe, 4 F_S, 5 delta_S
        double(*d)[6] = c->dh;
        d[0][0] = s;   d[1][0] = -s;  d[2][0] = 0.0;
        d[3][0] = s * (-xe) / (2.0 * ra * re) * s4;
        d[4][0] = s * (xa - x0) / (2.0 * r0 * ra) * c5;
        d[5][0] = s * xe / (2.0 * r0 * re) * s6;
        d[7][0] = -rFs / (2.0 * ra) * c8;
        d[9][0] = rFs / (2.0 * r0) * c10;

        d[1][1] = -s;  d[2][1] = s;
        d[3][1] = s * (xa - xe) / (2.0 * ra * re) * s4;
        d[4][1] = s * (-x0) / (2.0 * r0 * ra) * c5;
        d[5][1] = s * x0 / (2.0 * r0 * re) * s6;
        d[7][1] = -rFs / (2.0 * ra) * c8;
        d[8][1] = rFs / (2.0 * re) * s9;

        d[3][2] = -s * ra * re * c4;
        d[4][2] = -s * r0 * ra * s5;
        d[7][2] = -rFs * ra * s8;

        d[3][3] = s * ra * re * c4;
        d[5][3] = s * r0 * re * c6;
        d[8][3] = rFs * re * c9;

        const double dFs = (1.0 - 2.0 * F) / (2.0 * rFs);
        d[0][4] = -x0; d[1][4] = -xa; d[2][4] = -xe;
        d[3][4] = -ra * re * s4;
        d[4][4] = -r0 * ra * c5;
        d[5][4] = -r0 * re * s6;
        d[6][4] = 1.0;
        d[7][4] = dFs * ra * c8;
        d[8][4] = dFs * re * s9;
        d[9][4] = dFs * r0 * c10;

        d[7][5] = rFs * ra * s8;
        d[8][5] = -rFs * re * c9;
        d[9][5] = -rFs * r0 * s10;

        const double fmax[10] = {1.0, 0.5, 0.5, 0.5, kSqrt2 / 4.0, kSqrt2 / 4.0, 1.0 / 3.0,
                                 0.40824829046386301637, 0.40824829046386301637,
                                 1.15470053837925152902};
        double MO = 0.0;
        for (int k = 0; k < 10; ++k) MO += fabs(h[k]) * fmax[k];
        c->MO = MO;
    }
    c->cs = (1.0 - fb) / (IT * IO);
    c->cb = fb / V;
    c->inv_ITIO = 1.0 / (IT * IO);
    c->inv_V = 1.0 / V;
    c->pad_ = 0.0;
}


}  // namespace ipa
