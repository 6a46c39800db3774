// Step a1 of the hot path: parameter-derived constants, computed on the device
// from theta once per call (one warp per fit), so that theta can stay in
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

// One warp computes one Consts record: the transcendental pieces (the two
// range edges of I_T, the envelope, six sine/cosine pairs, five square roots)
// go to different lanes, are shared by shuffles, and lane k < 10 then builds
// h_k and row k of dh.  Every lane of the warp must call this.
__device__ inline void compute_consts_warp(const ModelDev& m, const double* th, Consts* c) {
    using namespace cdetail;
    const int lane = threadIdx.x & 31;
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], mu = th[IPA_MU], fb = th[IPA_FB];
    const bool four = m.kind == IPA_MODEL_ANGTIME4D;
    double x0 = 0.0, xe = 0.0, dpa = 0.0, dpe = 0.0, F = 0.0, dS = 0.0;
    if (four) {
        x0 = th[IPA_A0SQ];
        xe = th[IPA_APESQ];
        dpa = th[IPA_DPA];
        dpe = th[IPA_DPE];
        F = th[IPA_FS];
        dS = th[IPA_DS];
    }
    const double xa = 1.0 - x0 - xe, s = 1.0 - F;

    // per-lane transcendental work
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    if (lane < 2) {
        double dF[3];
        edge((lane == 0 ? m.t_hi : m.t_lo) - mu, Gamma, sigma, &v0, dF);
        v1 = dF[0];
        v2 = dF[1];
        v3 = dF[2];
    } else if (lane == 2) {
        v0 = fmin(1.0, exp(-Gamma * (m.t_lo - mu) + 0.5 * Gamma * Gamma * sigma * sigma));
    } else if (four && lane >= 3 && lane <= 8) {
        const double ang[6] = {dpe - dpa, dpa, dpe, dpa - dS, dpe - dS, dS};
        sincos(ang[lane - 3], &v0, &v1);
    } else if (four && lane >= 9 && lane <= 13) {
        const double arg[5] = {x0, xa, xe, F, s};
        v0 = sqrt(arg[lane - 9]);
    }
    const unsigned all = 0xffffffffu;
    const double Fh = __shfl_sync(all, v0, 0), Fl = __shfl_sync(all, v0, 1);
    double dIT[3];
    dIT[0] = __shfl_sync(all, v1, 0) - __shfl_sync(all, v1, 1);
    dIT[1] = __shfl_sync(all, v2, 0) - __shfl_sync(all, v2, 1);
    dIT[2] = __shfl_sync(all, v3, 0) - __shfl_sync(all, v3, 1);
    const double MT = __shfl_sync(all, v0, 2);
    const double s4 = __shfl_sync(all, v0, 3), c4 = __shfl_sync(all, v1, 3);
    const double s5 = __shfl_sync(all, v0, 4), c5 = __shfl_sync(all, v1, 4);
    const double s6 = __shfl_sync(all, v0, 5), c6 = __shfl_sync(all, v1, 5);
    const double s8 = __shfl_sync(all, v0, 6), c8 = __shfl_sync(all, v1, 6);
    const double s9 = __shfl_sync(all, v0, 7), c9 = __shfl_sync(all, v1, 7);
    const double s10 = __shfl_sync(all, v0, 8), c10 = __shfl_sync(all, v1, 8);
    const double r0 = __shfl_sync(all, v0, 9), ra = __shfl_sync(all, v0, 10), re = __shfl_sync(all, v0, 11);
    const double rF = __shfl_sync(all, v0, 12), rs = __shfl_sync(all, v0, 13);
    const double rFs = rF * rs;

    const double IT = Fh - Fl;
    const double span = m.t_hi - m.t_lo;
    const double IO = four ? 16.0 * kPi / 9.0 : 1.0;
    const double V = four ? span * 8.0 * kPi : span;

    // lane k < 10: h_k and dh_k / d(A0sq, Apesq, delta_pa, delta_pe, F_S, delta_S)
    double h = 0.0, d[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const double dFs = (1.0 - 2.0 * F) / (2.0 * rFs);
    if (!four) {
        h = lane == 0 ? 1.0 : 0.0;
    } else {
        switch (lane) {
        case 0: h = s * x0; d[0] = s; d[4] = -x0; break;
        case 1: h = s * xa; d[0] = -s; d[1] = -s; d[4] = -xa; break;
        case 2: h = s * xe; d[1] = s; d[4] = -xe; break;
        case 3:
            h = s * ra * re * s4;
            d[0] = s * (-xe) / (2.0 * ra * re) * s4;
            d[1] = s * (xa - xe) / (2.0 * ra * re) * s4;
            d[2] = -s * ra * re * c4;
            d[3] = s * ra * re * c4;
            d[4] = -ra * re * s4;
            break;
        case 4:
            h = s * r0 * ra * c5;
            d[0] = s * (xa - x0) / (2.0 * r0 * ra) * c5;
            d[1] = s * (-x0) / (2.0 * r0 * ra) * c5;
            d[2] = -s * r0 * ra * s5;
            d[4] = -r0 * ra * c5;
            break;
        case 5:
            h = s * r0 * re * s6;
            d[0] = s * xe / (2.0 * r0 * re) * s6;
            d[1] = s * x0 / (2.0 * r0 * re) * s6;
            d[3] = s * r0 * re * c6;
            d[4] = -r0 * re * s6;
            break;
        case 6: h = F; d[4] = 1.0; break;
        case 7:
            h = rFs * ra * c8;
            d[0] = -rFs / (2.0 * ra) * c8;
            d[1] = -rFs / (2.0 * ra) * c8;
            d[2] = -rFs * ra * s8;
            d[4] = dFs * ra * c8;
            d[5] = rFs * ra * s8;
            break;
        case 8:
            h = rFs * re * s9;
            d[1] = rFs / (2.0 * re) * s9;
            d[3] = rFs * re * c9;
            d[4] = dFs * re * s9;
            d[5] = -rFs * re * c9;
            break;
        case 9:
            h = rFs * r0 * c10;
            d[0] = rFs / (2.0 * r0) * c10;
            d[4] = dFs * r0 * c10;
            d[5] = -rFs * r0 * s10;
            break;
        default: break;
        }
    }
    // M_Omega = sum_k |h_k| max|f_k|
    const double fmax[10] = {1.0, 0.5, 0.5, 0.5, kSqrt2 / 4.0, kSqrt2 / 4.0, 1.0 / 3.0,
                             0.40824829046386301637, 0.40824829046386301637, 1.15470053837925152902};
    double mo = lane < 10 ? fabs(h) * fmax[lane] : 0.0;
    // fixed-order sum over lanes 0..9 (lane 0 ends with the total)
    for (int k = 1; k < 10; ++k) {
        const double v = __shfl_sync(all, mo, k);
        if (lane == 0) mo += v;
    }
    if (lane < 10) {
        c->h[lane] = h;
        for (int j = 0; j < 6; ++j) c->dh[lane][j] = d[j];
    }
    if (lane == 0) {
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
        c->IT = IT;
        for (int j = 0; j < 3; ++j) c->dlnIT[j] = dIT[j] / IT;
        c->MT = MT;
        c->MO = four ? mo : 1.0;
        c->cs = (1.0 - fb) / (IT * IO);
        c->cb = fb / V;
        c->inv_ITIO = 1.0 / (IT * IO);
        c->inv_V = 1.0 / V;
        c->pad_ = 0.0;
    }
}

}  // namespace ipa
