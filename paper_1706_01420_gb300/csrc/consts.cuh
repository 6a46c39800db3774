// Step a1 of the hot path: parameter-derived constants, computed on the device
// from theta once per call, so that theta can stay in device memory and calls
// can be captured in CUDA graphs.  Two layouts share every arithmetic step
// (so they give bit-identical records): one thread per fit when many fits are
// evaluated at once, one warp per fit when latency matters.
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


// The transcendental inputs of the angular coefficients.
struct AngPieces {
    double sn[6], cs[6];   // sin/cos of (dpe - dpa), dpa, dpe, (dpa - dS), (dpe - dS), dS
    double rt[5];          // sqrt of x0, xa, xe, F, s
};

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

__device__ inline double sqrt_arg(int i, double x0, double xa, double xe, double F, double s) {
    switch (i) {
    case 0: return x0;
    case 1: return xa;
    case 2: return xe;
    case 3: return F;
    default: return s;
    }
}

// h_k and dh_k / d(A0sq, Apesq, delta_pa, delta_pe, F_S, delta_S) for row k.
__device__ inline void h_row(int k, const AngPieces& a, double x0, double xe, double xa, double s, double F,
                             double* h, double* d) {
    const double s4 = a.sn[0], c4 = a.cs[0], s5 = a.sn[1], c5 = a.cs[1], s6 = a.sn[2], c6 = a.cs[2];
    const double s8 = a.sn[3], c8 = a.cs[3], s9 = a.sn[4], c9 = a.cs[4], s10 = a.sn[5], c10 = a.cs[5];
    const double r0 = a.rt[0], ra = a.rt[1], re = a.rt[2], rF = a.rt[3], rs = a.rt[4];
    const double rFs = rF * rs;
    const double dFs = (1.0 - 2.0 * F) / (2.0 * rFs);
    for (int j = 0; j < 6; ++j) d[j] = 0.0;
    switch (k) {
    case 0: *h = s * x0; d[0] = s; d[4] = -x0; break;
    case 1: *h = s * xa; d[0] = -s; d[1] = -s; d[4] = -xa; break;
    case 2: *h = s * xe; d[1] = s; d[4] = -xe; break;
    case 3:
        *h = s * ra * re * s4;
        d[0] = s * (-xe) / (2.0 * ra * re) * s4;
        d[1] = s * (xa - xe) / (2.0 * ra * re) * s4;
        d[2] = -s * ra * re * c4;
        d[3] = s * ra * re * c4;
        d[4] = -ra * re * s4;
        break;
    case 4:
        *h = s * r0 * ra * c5;
        d[0] = s * (xa - x0) / (2.0 * r0 * ra) * c5;
        d[1] = s * (-x0) / (2.0 * r0 * ra) * c5;
        d[2] = -s * r0 * ra * s5;
        d[4] = -r0 * ra * c5;
        break;
    case 5:
        *h = s * r0 * re * s6;
        d[0] = s * xe / (2.0 * r0 * re) * s6;
        d[1] = s * x0 / (2.0 * r0 * re) * s6;
        d[3] = s * r0 * re * c6;
        d[4] = -r0 * re * s6;
        break;
    case 6: *h = F; d[4] = 1.0; break;
    case 7:
        *h = rFs * ra * c8;
        d[0] = -rFs / (2.0 * ra) * c8;
        d[1] = -rFs / (2.0 * ra) * c8;
        d[2] = -rFs * ra * s8;
        d[4] = dFs * ra * c8;
        d[5] = rFs * ra * s8;
        break;
    case 8:
        *h = rFs * re * s9;
        d[1] = rFs / (2.0 * re) * s9;
        d[3] = rFs * re * c9;
        d[4] = dFs * re * s9;
        d[5] = -rFs * re * c9;
        break;
    default:
        *h = rFs * r0 * c10;
        d[0] = rFs / (2.0 * r0) * c10;
        d[4] = dFs * r0 * c10;
        d[5] = -rFs * r0 * s10;
        break;
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

__device__ inline double time_envelope(const ModelDev& m, double Gamma, double sigma, double mu) {
    return fmin(1.0, exp(-Gamma * (m.t_lo - mu) + 0.5 * Gamma * Gamma * sigma * sigma));
}

// Scalars of the record from I_T pieces and the envelopes.
__device__ inline void write_scalars(const ModelDev& m, const double* th, double Fh, double Fl,
                                     const double* dIT, double MT, double MO, Consts* c) {
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], mu = th[IPA_MU], fb = th[IPA_FB];
    const bool four = m.kind == IPA_MODEL_ANGTIME4D;
    const double IT = Fh - Fl;
    const double span = m.t_hi - m.t_lo;
    const double IO = four ? 16.0 * kPi / 9.0 : 1.0;
    const double V = four ? span * 8.0 * kPi : span;
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
    c->MO = four ? MO : 1.0;
    c->cs = (1.0 - fb) / (IT * IO);
    c->cb = fb / V;
    c->inv_ITIO = 1.0 / (IT * IO);
    c->inv_V = 1.0 / V;
    c->pad_ = 0.0;
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

}  // namespace cdetail

// One thread computes one Consts record: used when many fits are evaluated at
// once (batched fits, the server), where lanes of a warp hold different fits
// and every FP64 instruction does useful work in all of them.
__device__ inline void compute_consts_thread(const ModelDev& m, const double* th, Consts* c) {
    using namespace cdetail;
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], mu = th[IPA_MU];
    double Fh, Fl, dFh[3], dFl[3];
    edge(m.t_hi - mu, Gamma, sigma, &Fh, dFh);
    edge(m.t_lo - mu, Gamma, sigma, &Fl, dFl);
    double dIT[3];
    for (int j = 0; j < 3; ++j) dIT[j] = dFh[j] - dFl[j];
    const double MT = time_envelope(m, Gamma, sigma, mu);
    const AmpParams p = amp_params(m, th);
    double MO = 0.0;
    if (m.kind == IPA_MODEL_ANGTIME4D) {
        AngPieces a;
        for (int i = 0; i < 6; ++i) sincos(ang_arg(i, p.dpa, p.dpe, p.dS), &a.sn[i], &a.cs[i]);
        for (int i = 0; i < 5; ++i) a.rt[i] = sqrt(sqrt_arg(i, p.x0, p.xa, p.xe, p.F, p.s));
        for (int k = 0; k < 10; ++k) {
            double h, d[6];
            h_row(k, a, p.x0, p.xe, p.xa, p.s, p.F, &h, d);
            c->h[k] = h;
            for (int j = 0; j < 6; ++j) c->dh[k][j] = d[j];
            MO = k ? MO + fabs(h) * basis_max(k) : fabs(h) * basis_max(k);
        }
    } else {
        for (int k = 0; k < 10; ++k) {
            c->h[k] = k == 0 ? 1.0 : 0.0;
            for (int j = 0; j < 6; ++j) c->dh[k][j] = 0.0;
        }
    }
    write_scalars(m, th, Fh, Fl, dIT, MT, MO, c);
}

// One warp computes one Consts record (a single fit, where latency matters):
// the transcendental pieces (both range edges of I_T, the envelope, six
// sine/cosine pairs, five square roots) go to different lanes and are shared
// by shuffles; lane k < 10 then builds h_k and row k of dh.  Every lane of
// the warp must call this.
__device__ inline void compute_consts_warp(const ModelDev& m, const double* th, Consts* c) {
    using namespace cdetail;
    const int lane = threadIdx.x & 31;
    const unsigned all = 0xffffffffu;
    const double Gamma = th[IPA_GAMMA], sigma = th[IPA_SIGMA], mu = th[IPA_MU];
    const bool four = m.kind == IPA_MODEL_ANGTIME4D;
    const AmpParams p = amp_params(m, th);
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    if (lane < 2) {
        double dF[3];
        edge((lane == 0 ? m.t_hi : m.t_lo) - mu, Gamma, sigma, &v0, dF);
        v1 = dF[0];
        v2 = dF[1];
        v3 = dF[2];
    } else if (lane == 2) {
        v0 = time_envelope(m, Gamma, sigma, mu);
    } else if (four && lane >= 3 && lane <= 8) {
        sincos(ang_arg(lane - 3, p.dpa, p.dpe, p.dS), &v0, &v1);
    } else if (four && lane >= 9 && lane <= 13) {
        v0 = sqrt(sqrt_arg(lane - 9, p.x0, p.xa, p.xe, p.F, p.s));
    }
    const double Fh = __shfl_sync(all, v0, 0), Fl = __shfl_sync(all, v0, 1);
    double dIT[3];
    dIT[0] = __shfl_sync(all, v1, 0) - __shfl_sync(all, v1, 1);
    dIT[1] = __shfl_sync(all, v2, 0) - __shfl_sync(all, v2, 1);
    dIT[2] = __shfl_sync(all, v3, 0) - __shfl_sync(all, v3, 1);
    const double MT = __shfl_sync(all, v0, 2);
    AngPieces a;
    for (int i = 0; i < 6; ++i) {
        a.sn[i] = __shfl_sync(all, v0, 3 + i);
        a.cs[i] = __shfl_sync(all, v1, 3 + i);
    }
    for (int i = 0; i < 5; ++i) a.rt[i] = __shfl_sync(all, v0, 9 + i);
    double h = 0.0, d[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (four && lane < 10) h_row(lane, a, p.x0, p.xe, p.xa, p.s, p.F, &h, d);
    if (!four) h = lane == 0 ? 1.0 : 0.0;
    // M_Omega = sum_k |h_k| max|f_k| in k order (lane 0 ends with the total)
    double mo = lane < 10 ? fabs(h) * basis_max(lane) : 0.0;
    for (int k = 1; k < 10; ++k) {
        const double v = __shfl_sync(all, mo, k);
        if (lane == 0) mo += v;
    }
    if (lane < 10) {
        c->h[lane] = h;
        for (int j = 0; j < 6; ++j) c->dh[lane][j] = d[j];
    }
    if (lane == 0) write_scalars(m, th, Fh, Fl, dIT, MT, mo, c);
}

}  // namespace ipa
